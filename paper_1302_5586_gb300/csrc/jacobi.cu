// jacobi.cu -- 5-point Jacobi sweeps and the FP64 residual norm for sm_103a.
//
// Sweep (the data-parallel body of the sequential `untilconverged` loop,
// Sec. 3.2; its points are independent, Sec. 2.2.3):
//   v[i][j] = 0.25f * ((u[i-1][j] + u[i+1][j]) + (u[i][j-1] + u[i][j+1]))
// on the interior, in FP32 and in exactly this order, boundary ring copied.
//
// Residual (the `reduction` directive, Sec. 2.2.3):
//   sqrt(sum_interior r^2),  r = 4u[i][j] - ((up + down) + (left + right)),
// r in FP32 (one rounding: 4u is exact, so fma(4, u, -s) is 4u - s rounded
// once), r^2 rounded to FP32 and added per thread into a compensated FP32
// pair (Knuth's TwoSum), which holds the sum of the rounded squares to about
// 2^-44 of it; the per-thread pairs are then added in FP64: warp butterfly,
// block, and one fixed-order pass over the per-block partials.  The order depends only on the grid
// shape, so the same iterate always gives the same residual bits.
//
// Layout: a thread owns 4 adjacent columns (one float4) and JR rows of a
// column strip; it streams the strip top to bottom keeping (up, cur, down)
// in registers, takes the left/right neighbours from adjacent lanes with
// shuffles (lanes 0 and 31 read one extra scalar), and writes one float4
// per row.  Each u element comes from HBM once per sweep; v is written once.
// Grids whose width is not a multiple of 4 (or unaligned buffers) take a
// scalar kernel with the same arithmetic.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <utility>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "jacobi_tile.cuh"

namespace pencil {
namespace {

constexpr int JT = 128;  // threads per block
constexpr int JR = 16;   // rows per thread
// Sum one double per thread over the block in a fixed order; thread 0 writes it.
__device__ __forceinline__ void block_sum_store(double d, double *dst) {
    __shared__ double wsum[JT / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(FULL, d, off);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = wsum[0];
#pragma unroll
        for (int k = 1; k < JT / 32; ++k) t += wsum[k];
        *dst = t;
    }
}

// Sum one double per thread over an NT-thread block in a fixed order; thread 0
// writes it.  Ends with a barrier, so it can be called repeatedly.
template <int NT>
__device__ __forceinline__ void block_sum_store_n(double d, double *dst) {
    __shared__ double wsum[NT / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(FULL, d, off);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = wsum[0];
#pragma unroll
        for (int k = 1; k < NT / 32; ++k) t += wsum[k];
        *dst = t;
    }
    __syncthreads();
}

template <bool RESID, bool STORE>
__global__ void __launch_bounds__(JT)
    jacobi_v4_kernel(const float *__restrict__ u, float *__restrict__ v, int h, int w,
                     double *__restrict__ partials) {
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * JT + threadIdx.x;  // float4 column
    const int j0 = q * 4;
    const bool colok = j0 < w;
    const int w4 = w >> 2;
    const int i0 = blockIdx.y * JR;
    const float4 *U = reinterpret_cast<const float4 *>(u);
    float4 *V = reinterpret_cast<float4 *>(v);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);

    float hi = 0.f, lo = 0.f;
    // All JR + 2 rows of the strip are loaded before any is used, so a warp has
    // them all in flight at once (the sweep is bound by memory latency, not by
    // the few flops per point); row o + 1 of `x` is grid row i0 + o.
    // Lanes 0 and 31 also load the column beyond the warp's edge for every row.
    float4 x[JR + 2];
    float edge[JR];
#pragma unroll
    for (int o = 0; o < JR + 2; ++o) {
        const int i = i0 - 1 + o;
        x[o] = (colok && i >= 0 && i < h) ? __ldg(U + (size_t)i * w4 + q) : z4;
    }
    const int ec = lane == 0 ? j0 - 1 : j0 + 4;  // edge column of lanes 0 and 31
    const bool eok = colok && (lane == 0 || lane == 31) && ec >= 0 && ec < w;
#pragma unroll
    for (int o = 0; o < JR; ++o) {
        const int i = i0 + o;
        edge[o] = (eok && i < h) ? __ldg(u + (size_t)i * w + ec) : 0.f;
    }
    float4 up = x[0], cur = x[1];
#pragma unroll
    for (int o = 0; o < JR; ++o) {
        const int i = i0 + o;
        if (i >= h) break;
        const float4 dn = x[o + 2];
        float lf = __shfl_up_sync(FULL, cur.w, 1);
        float rt = __shfl_down_sync(FULL, cur.x, 1);
        if (lane == 0) lf = edge[o];
        if (lane == 31) rt = edge[o];
        if (i > 0 && i < h - 1) {
            const float sx = nsum(up.x, dn.x, lf, cur.y);
            const float sy = nsum(up.y, dn.y, cur.x, cur.z);
            const float sz = nsum(up.z, dn.z, cur.y, cur.w);
            const float sw = nsum(up.w, dn.w, cur.z, rt);
            if (STORE && colok) {
                float4 n;
                n.x = (j0 == 0) ? cur.x : __fmul_rn(0.25f, sx);
                n.y = __fmul_rn(0.25f, sy);
                n.z = __fmul_rn(0.25f, sz);
                n.w = (j0 + 3 == w - 1) ? cur.w : __fmul_rn(0.25f, sw);
                V[(size_t)i * w4 + q] = n;
            }
            if (RESID && colok) {
                if (j0 > 0) acc_sq(__fmaf_rn(4.f, cur.x, -sx), hi, lo);
                acc_sq(__fmaf_rn(4.f, cur.y, -sy), hi, lo);
                acc_sq(__fmaf_rn(4.f, cur.z, -sz), hi, lo);
                if (j0 + 3 < w - 1) acc_sq(__fmaf_rn(4.f, cur.w, -sw), hi, lo);
            }
        } else if (STORE && colok) {
            V[(size_t)i * w4 + q] = cur;  // boundary row
        }
        up = cur;
        cur = dn;
    }
    if (RESID)
        block_sum_store((double)hi + (double)lo, partials + (size_t)blockIdx.y * gridDim.x + blockIdx.x);
}

// Scalar variant: one column per thread, neighbours read through L1.
template <bool RESID, bool STORE>
__global__ void __launch_bounds__(JT)
    jacobi_s_kernel(const float *__restrict__ u, float *__restrict__ v, int h, int w,
                    double *__restrict__ partials) {
    const int j = blockIdx.x * JT + threadIdx.x;
    const bool colok = j < w;
    const int i0 = blockIdx.y * JR;
    float hi = 0.f, lo = 0.f;
    for (int o = 0; o < JR; ++o) {
        const int i = i0 + o;
        if (i >= h) break;
        if (!colok) continue;
        const size_t p = (size_t)i * w + j;
        const float c = __ldg(u + p);
        if (i > 0 && i < h - 1 && j > 0 && j < w - 1) {
            const float s = nsum(__ldg(u + p - w), __ldg(u + p + w), __ldg(u + p - 1), __ldg(u + p + 1));
            if (STORE) v[p] = __fmul_rn(0.25f, s);
            if (RESID) acc_sq(__fmaf_rn(4.f, c, -s), hi, lo);
        } else if (STORE) {
            v[p] = c;
        }
    }
    if (RESID)
        block_sum_store((double)hi + (double)lo, partials + (size_t)blockIdx.y * gridDim.x + blockIdx.x);
}

// ------------------------------------------------- red-black SOR sweeps
// One colour pass, in place: interior points with (i + j) % 2 == color become
// u + omega * (0.25f * ((up + down) + (left + right)) - u)   [fma(omega, d, u)]
// in FP32 in exactly that order.  A point's four neighbours have the other
// colour and are not written in this pass, so the pass has no read-after-write
// dependence.  This scalar kernel serves grids whose rows are not 16-byte
// aligned; aligned grids take the register tiles below.
template <int COLOR>
__global__ void __launch_bounds__(JT) rbsor_s_kernel(float *__restrict__ u, int h, int w, float omega) {
    const int j = blockIdx.x * JT + threadIdx.x;
    const int i0 = blockIdx.y * JR;
    if (j < 1 || j >= w - 1) return;
    for (int o = 0; o < JR; ++o) {
        const int i = i0 + o;
        if (i >= h - 1) break;
        if (i < 1 || ((i + j) & 1) != COLOR) continue;
        const size_t p = (size_t)i * w + j;
        const float s = nsum(u[p - w], u[p + w], u[p - 1], u[p + 1]);
        u[p] = __fmaf_rn(omega, __fsub_rn(__fmul_rn(0.25f, s), u[p]), u[p]);
    }
}

// res = sqrt(sum of n partials), one block, fixed order.
__global__ void __launch_bounds__(256) residual_finish_kernel(const double *__restrict__ partials,
                                                              int n, double *__restrict__ res) {
    __shared__ double wsum[8];
    double t = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) t += partials[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(FULL, t, off);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = wsum[0];
#pragma unroll
        for (int k = 1; k < 8; ++k) s += wsum[k];
        *res = sqrt(s);
    }
}

template <typename Cfg, bool EDGE>
__device__ __forceinline__ void jacobi_reg_body(const float *__restrict__ u, float *__restrict__ v, int h, int w,
                                                int n, int gy0, int gx0, int iter0, int check_every,
                                                float4 *xch, double *wres) {
    constexpr int RS = Cfg::RS;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const RegGeom<Cfg> q(h, w, gy0, gx0);
    const bool chunk_in = q.gc0 >= 0 && q.gc0 < w;  // w % 4 == 0: a chunk is wholly in or out
    float4 y[RS + 1];  // row r in y[1 + r] between pairs of sweeps
    y[0] = z4;
#pragma unroll
    for (int r = 0; r < RS; ++r) {
        const int g = q.g_first + r;
        y[1 + r] = (g >= 0 && g < h && chunk_in)
                       ? __ldg(reinterpret_cast<const float4 *>(u + (size_t)g * w + q.gc0))
                       : z4;
    }
    reg_sweeps_store<Cfg, EDGE>(y, v, h, w, n, q, iter0, check_every, xch, wres);
}

// MINB: CTAs per SM the register budget is sized for.
template <typename Cfg, int MINB>
__global__ void __launch_bounds__(Cfg::NT, MINB)
    jacobi_reg_kernel(const float *__restrict__ u, float *__restrict__ v, int h, int w, int n, int iter0,
                      int check_every, double *__restrict__ partials, int nblk) {
    constexpr int T = Cfg::T;
    __shared__ float4 xch[2 * Cfg::NW * 2 * 32];
    __shared__ double wres[T * Cfg::NW];
    const int gy0 = blockIdx.y * Cfg::BH - T;       // global row of window row 0
    const int gx0 = blockIdx.x * Cfg::BW - Cfg::P;  // global column of window column 0 (multiple of 4)
    if (gy0 <= 0 || gy0 + Cfg::SH - 1 >= h - 1 || gx0 <= 0 || gx0 + Cfg::W - 1 >= w - 1)
        jacobi_reg_body<Cfg, true>(u, v, h, w, n, gy0, gx0, iter0, check_every, xch, wres);
    else
        jacobi_reg_body<Cfg, false>(u, v, h, w, n, gy0, gx0, iter0, check_every, xch, wres);
    __syncthreads();
    if (threadIdx.x == 0 && check_every > 0) {
        const int bid = blockIdx.y * gridDim.x + blockIdx.x;
        int slot = 0;
        for (int t = 0; t < n; ++t) {
            const int it = iter0 + t;
            if (it > 0 && it % check_every == 0) {
                double sum = wres[slot * Cfg::NW];
                for (int k = 1; k < Cfg::NW; ++k) sum += wres[slot * Cfg::NW + k];
                partials[(size_t)slot * nblk + bid] = sum;
                ++slot;
            }
        }
    }
}

// Red-black SOR passes with the tile in registers: the same 128 x 128
// window of 8 warps x 16 rows as the Jacobi tiles.  A sweep is two colour
// phases; in each, the points of one colour ((i + j) even first) take
// u <- fma(omega, 0.25*s - u, u), s = (up + down) + (left + right), in place:
// their neighbours all have the other colour, so the phase reads none of its
// own results.  Band edge rows are exchanged through shared memory before
// every phase.  Wrong values at the window edges move inward two points per
// sweep, so the core is the window minus 2T rows and P columns (P = 2T
// rounded up to 4) on each side.  Reads u, writes the core to v.
template <int T>
struct SorCfg {
    static constexpr int NW = 8, RS = 16, NT = 32 * NW, W = 128, SH = NW * RS;
    static constexpr int P = round_up(2 * T, 4);
    static constexpr int BW = W - 2 * P;
    static constexpr int BH = SH - 4 * T;
};

template <int RS, bool EDGE>
__device__ __forceinline__ void sor_phase(float4 (&x)[RS], const float4 above, const float4 below, int color,
                                          int g_first, int h, const bool (&cint)[4], float omega) {
#pragma unroll
    for (int r = 0; r < RS; ++r) {
        const float4 cur = x[r];
        const float4 up = r > 0 ? x[r - 1] : above;
        const float4 dn = r + 1 < RS ? x[r + 1] : below;
        const int g = g_first + r;
        // columns of this lane are 4-aligned, so the colour's points are
        // e = a and e = a + 2 with a = (colour + g) & 1
        const int a = (color + g) & 1;
        const bool rint = !EDGE || (g >= 1 && g <= h - 2);
        if (a == 0) {
            const float lf = __shfl_up_sync(FULL, cur.w, 1);  // lane 0: its own value (window edge)
            const float s0 = nsum(up.x, dn.x, lf, cur.y);
            const float s2 = nsum(up.z, dn.z, cur.y, cur.w);
            if (rint && (!EDGE || cint[0])) x[r].x = __fmaf_rn(omega, __fsub_rn(__fmul_rn(0.25f, s0), cur.x), cur.x);
            if (rint && (!EDGE || cint[2])) x[r].z = __fmaf_rn(omega, __fsub_rn(__fmul_rn(0.25f, s2), cur.z), cur.z);
        } else {
            const float rt = __shfl_down_sync(FULL, cur.x, 1);  // lane 31: its own value (window edge)
            const float s1 = nsum(up.y, dn.y, cur.x, cur.z);
            const float s3 = nsum(up.w, dn.w, cur.z, rt);
            if (rint && (!EDGE || cint[1])) x[r].y = __fmaf_rn(omega, __fsub_rn(__fmul_rn(0.25f, s1), cur.y), cur.y);
            if (rint && (!EDGE || cint[3])) x[r].w = __fmaf_rn(omega, __fsub_rn(__fmul_rn(0.25f, s3), cur.w), cur.w);
        }
    }
}

template <int T, bool EDGE>
__device__ __forceinline__ void rbsor_reg_body(const float *__restrict__ u, float *__restrict__ v, int h, int w,
                                               int n, float omega, int gy0, int gx0, float4 *xch) {
    using Cfg = SorCfg<T>;
    constexpr int RS = Cfg::RS, NW = Cfg::NW, P = Cfg::P, BW = Cfg::BW;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int gc0 = gx0 + 4 * lane;
    const bool chunk_in = gc0 >= 0 && gc0 < w;  // w % 4 == 0: a chunk is wholly in or out
    const bool core_cols = 4 * lane >= P && 4 * lane < P + BW && gc0 < w;
    bool cint[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) cint[e] = gc0 + e >= 1 && gc0 + e <= w - 2;
    const int g_first = gy0 + wp * RS;
    const int core_lo = gy0 + 2 * T, core_hi = min(h, gy0 + 2 * T + Cfg::BH);
    float4 x[RS];
#pragma unroll
    for (int r = 0; r < RS; ++r) {
        const int g = g_first + r;
        x[r] = (g >= 0 && g < h && chunk_in) ? __ldg(reinterpret_cast<const float4 *>(u + (size_t)g * w + gc0)) : z4;
    }
#pragma unroll 1
    for (int k = 0; k < 2 * n; ++k) {  // phase k: colour k & 1
        float4 *xb = xch + (k & 1) * (NW * 2 * 32);
        xb[(wp * 2 + 0) * 32 + lane] = x[0];
        xb[(wp * 2 + 1) * 32 + lane] = x[RS - 1];
        __syncthreads();
        const float4 above = wp > 0 ? xb[((wp - 1) * 2 + 1) * 32 + lane] : x[0];
        const float4 below = wp < NW - 1 ? xb[((wp + 1) * 2 + 0) * 32 + lane] : x[RS - 1];
        sor_phase<RS, EDGE>(x, above, below, k & 1, g_first, h, cint, omega);
    }
    if (core_cols) {
#pragma unroll
        for (int r = 0; r < RS; ++r) {
            const int g = g_first + r;
            if (g >= core_lo && g < core_hi) *reinterpret_cast<float4 *>(v + (size_t)g * w + gc0) = x[r];
        }
    }
}

template <int T>
__global__ void __launch_bounds__(SorCfg<T>::NT, 2)
    rbsor_reg_kernel(const float *__restrict__ u, float *__restrict__ v, int h, int w, int n, float omega) {
    using Cfg = SorCfg<T>;
    __shared__ float4 xch[2 * Cfg::NW * 2 * 32];
    const int gy0 = blockIdx.y * Cfg::BH - 2 * T;   // global row of window row 0
    const int gx0 = blockIdx.x * Cfg::BW - Cfg::P;  // global column of window column 0 (multiple of 4)
    if (gy0 <= 0 || gy0 + Cfg::SH - 1 >= h - 1 || gx0 <= 0 || gx0 + Cfg::W - 1 >= w - 1)
        rbsor_reg_body<T, true>(u, v, h, w, n, omega, gy0, gx0, xch);
    else
        rbsor_reg_body<T, false>(u, v, h, w, n, omega, gy0, gx0, xch);
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Plan {
    bool vec;
    dim3 grid;
    int nblocks;
};

Plan make_plan(int h, int w, const float *a, const float *b) {
    Plan p;
    p.vec = (w % 4 == 0) && ((uintptr_t)a % 16 == 0) && (b == nullptr || (uintptr_t)b % 16 == 0);
    const int cols = p.vec ? (w / 4) : w;
    p.grid = dim3((cols + JT - 1) / JT, (h + JR - 1) / JR);
    p.nblocks = (int)(p.grid.x * p.grid.y);
    return p;
}

template <bool RESID, bool STORE>
cudaError_t sweep(const Plan &p, const float *u, float *v, int h, int w, double *partials,
                  cudaStream_t s) {
    if (p.vec)
        jacobi_v4_kernel<RESID, STORE><<<p.grid, JT, 0, s>>>(u, v, h, w, partials);
    else
        jacobi_s_kernel<RESID, STORE><<<p.grid, JT, 0, s>>>(u, v, h, w, partials);
    return cudaGetLastError();
}

cudaError_t finish(const double *partials, int n, double *res, cudaStream_t s) {
    residual_finish_kernel<<<1, 256, 0, s>>>(partials, n, res);
    return cudaGetLastError();
}

template <int T>
int reg_nblk(int h, int w) {
    return ((w + RegCfg<T>::BW - 1) / RegCfg<T>::BW) * ((h + RegCfg<T>::BH - 1) / RegCfg<T>::BH);
}

// Partials capacity for every supported T (T checkpoints per pass at most).
size_t tiled_partials(int h, int w) {
    size_t m = 0;
    m = std::max(m, (size_t)reg_nblk<2>(h, w) * 2);
    m = std::max(m, (size_t)reg_nblk<4>(h, w) * 4);
    m = std::max(m, (size_t)reg_nblk<5>(h, w) * 5);
    m = std::max(m, (size_t)reg_nblk<8>(h, w) * 8);
    m = std::max(m, (size_t)reg_nblk<10>(h, w) * 10);
    return m;
}

// Sweeps `iters` times from u (ping-pong with v) using passes of at most
// `per_pass` (<= T) sweeps; residuals of checkpoint iterates inside a pass go
// to res.  Returns the buffer holding the final iterate through *final.
template <int T>
cudaError_t run_tiled(int h, int w, float *u, float *v, int iters, int per_pass, int ce,
                      double *res, double *partials, cudaStream_t s, float **final) {
    using Cfg = RegCfg<T>;
    const dim3 grid((w + Cfg::BW - 1) / Cfg::BW, (h + Cfg::BH - 1) / Cfg::BH);
    const int nblk = (int)(grid.x * grid.y);
    float *cur = u, *nxt = v;
    for (int iter = 0; iter < iters;) {
        const int n = std::min(per_pass, iters - iter);
        jacobi_reg_kernel<Cfg, 2><<<grid, Cfg::NT, 0, s>>>(cur, nxt, h, w, n, iter, ce, partials, nblk);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        int slot = 0;
        for (int t = 0; t < n; ++t) {
            const int it = iter + t;
            if (ce > 0 && it > 0 && it % ce == 0) {
                e = finish(partials + (size_t)slot * nblk, nblk, res + (it / ce - 1), s);
                if (e != cudaSuccess) return e;
                ++slot;
            }
        }
        std::swap(cur, nxt);
        iter += n;
    }
    *final = cur;
    return cudaSuccess;
}

}  // namespace

size_t jacobi_workspace_bytes(int h, int w) {
    const size_t grid = align256(sizeof(float) * (size_t)h * (size_t)w);
    const size_t nb = (size_t)((w + JT - 1) / JT) * (size_t)((h + JR - 1) / JR);
    return grid + align256(sizeof(double) * std::max(nb, tiled_partials(h, w)));
}

static double *partials_of(void *ws, int h, int w) {
    return reinterpret_cast<double *>(static_cast<char *>(ws) +
                                      align256(sizeof(float) * (size_t)h * (size_t)w));
}

// Sweeps per pass actually used for a request (0 = library choice: 10 on
// grids large enough that the halo work of a 128 x 128 tile pays off, else 4;
// measured on GB300, 8192^2 x 100 sweeps: T = 4/5/8/10 take 3.8/3.6/3.3/3.2 ms).
static int choose_t(int temporal_t, bool vec, int h, int w) {
    if (!vec) return 1;
    if (temporal_t == 0) return (h >= 512 && w >= 512) ? 10 : 4;
    return std::min(temporal_t, 10);
}

cudaError_t jacobi_run(int h, int w, float *u, int iters, int check_every, double *res, void *ws,
                       size_t ws_bytes, int temporal_t, cudaStream_t s) {
    (void)ws_bytes;
    const int nres = (check_every > 0) ? iters / check_every : 0;
    if (h < 3 || w < 3 || iters == 0) {
        if (nres > 0) return cudaMemsetAsync(res, 0, sizeof(double) * (size_t)nres, s);
        return cudaSuccess;
    }
    float *v = static_cast<float *>(ws);
    double *partials = partials_of(ws, h, w);
    const Plan p = make_plan(h, w, u, v);
    const int t = choose_t(temporal_t, p.vec, h, w);
    float *cur = u;
    cudaError_t e = cudaSuccess;
    if (t >= 2) {
        if (t == 2) e = run_tiled<2>(h, w, u, v, iters, t, check_every, res, partials, s, &cur);
        else if (t <= 4) e = run_tiled<4>(h, w, u, v, iters, t, check_every, res, partials, s, &cur);
        else if (t == 5) e = run_tiled<5>(h, w, u, v, iters, t, check_every, res, partials, s, &cur);
        else if (t <= 8) e = run_tiled<8>(h, w, u, v, iters, t, check_every, res, partials, s, &cur);
        else e = run_tiled<10>(h, w, u, v, iters, t, check_every, res, partials, s, &cur);
        if (e != cudaSuccess) return e;
    } else {
        float *nxt = v;
        for (int k = 1; k <= iters; ++k) {
            const int prev = k - 1;  // iterate index held in cur
            const bool want = check_every > 0 && prev > 0 && prev % check_every == 0;
            if (want) {
                e = sweep<true, true>(p, cur, nxt, h, w, partials, s);
                if (e == cudaSuccess) e = finish(partials, p.nblocks, res + (prev / check_every - 1), s);
            } else {
                e = sweep<false, true>(p, cur, nxt, h, w, partials, s);
            }
            if (e != cudaSuccess) return e;
            std::swap(cur, nxt);
        }
    }
    if (check_every > 0 && iters % check_every == 0) {
        const Plan q = make_plan(h, w, cur, nullptr);
        e = sweep<true, false>(q, cur, nullptr, h, w, partials, s);
        if (e == cudaSuccess) e = finish(partials, q.nblocks, res + (nres - 1), s);
        if (e != cudaSuccess) return e;
    }
    if (cur != u)
        e = cudaMemcpyAsync(u, cur, sizeof(float) * (size_t)h * (size_t)w, cudaMemcpyDeviceToDevice, s);
    return e;
}

cudaError_t residual_run(int h, int w, const float *u, double *res, void *ws, cudaStream_t s) {
    if (h < 3 || w < 3) return cudaMemsetAsync(res, 0, sizeof(double), s);
    double *partials = partials_of(ws, h, w);
    const Plan p = make_plan(h, w, u, nullptr);
    cudaError_t e = sweep<true, false>(p, u, nullptr, h, w, partials, s);
    if (e == cudaSuccess) e = finish(partials, p.nblocks, res, s);
    return e;
}

}  // namespace pencil

// ------------------------------------------------ SOR and converge-to-tol
namespace pencil {

// Workspace: a second grid (the tiled passes ping-pong) and the residual partials.
size_t rbsor_workspace_bytes(int h, int w) {
    const size_t nb = (size_t)((w + JT - 1) / JT) * (size_t)((h + JR - 1) / JR);
    return align256(sizeof(float) * (size_t)h * (size_t)w) + align256(sizeof(double) * nb);
}

constexpr int kSorT = 5;  // sweeps per tiled SOR pass (halo 2T: measured best on 8192^2)

cudaError_t rbsor_run(int h, int w, float *u, int iters, float omega, int check_every, double *res,
                      void *ws, cudaStream_t s) {
    const int nres = (check_every > 0) ? iters / check_every : 0;
    if (h < 3 || w < 3 || iters == 0) {
        if (nres > 0) return cudaMemsetAsync(res, 0, sizeof(double) * (size_t)nres, s);
        return cudaSuccess;
    }
    float *v = static_cast<float *>(ws);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(ws) +
                                                  align256(sizeof(float) * (size_t)h * (size_t)w));
    const Plan p = make_plan(h, w, u, v);
    if (p.vec) {
        // tiled passes of up to kSorT sweeps, ending at every checkpoint; u/v ping-pong
        using Cfg = SorCfg<kSorT>;
        const dim3 grid((w + Cfg::BW - 1) / Cfg::BW, (h + Cfg::BH - 1) / Cfg::BH);
        float *cur = u, *nxt = v;
        for (int k = 0; k < iters;) {
            int n = std::min(kSorT, iters - k);
            if (check_every > 0) n = std::min(n, check_every - k % check_every);
            rbsor_reg_kernel<kSorT><<<grid, Cfg::NT, 0, s>>>(cur, nxt, h, w, n, omega);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            std::swap(cur, nxt);
            k += n;
            if (check_every > 0 && k % check_every == 0) {
                const Plan q = make_plan(h, w, cur, nullptr);
                e = sweep<true, false>(q, cur, nullptr, h, w, partials, s);
                if (e == cudaSuccess) e = finish(partials, q.nblocks, res + (k / check_every - 1), s);
                if (e != cudaSuccess) return e;
            }
        }
        if (cur != u) return cudaMemcpyAsync(u, cur, sizeof(float) * (size_t)h * (size_t)w,
                                             cudaMemcpyDeviceToDevice, s);
        return cudaSuccess;
    }
    for (int k = 1; k <= iters; ++k) {  // rows not 16-byte aligned: one kernel per colour
        rbsor_s_kernel<0><<<p.grid, JT, 0, s>>>(u, h, w, omega);
        rbsor_s_kernel<1><<<p.grid, JT, 0, s>>>(u, h, w, omega);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (check_every > 0 && k % check_every == 0) {
            e = sweep<true, false>(p, u, nullptr, h, w, partials, s);
            if (e == cudaSuccess) e = finish(partials, p.nblocks, res + (k / check_every - 1), s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace pencil

namespace {
// Read one residual back to the host (the stream is synchronised).
cudaError_t read_res(const double *dev, double *host, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}
}  // namespace

namespace pencil {

cudaError_t jacobi_until(int h, int w, float *u, int max_iters, int check_every, double tol,
                         double *res, int *done, void *ws, size_t ws_bytes, int temporal_t,
                         cudaStream_t s) {
    *done = 0;
    for (int m = 1; m * check_every <= max_iters; ++m) {
        cudaError_t e = jacobi_run(h, w, u, check_every, check_every, res + (m - 1), ws, ws_bytes,
                                   temporal_t, s);
        double r = 0.0;
        if (e == cudaSuccess) e = read_res(res + (m - 1), &r, s);
        if (e != cudaSuccess) return e;
        *done = m * check_every;
        if (r <= tol) break;
    }
    return cudaSuccess;
}

cudaError_t rbsor_until(int h, int w, float *u, int max_iters, float omega, int check_every,
                        double tol, double *res, int *done, void *ws, cudaStream_t s) {
    *done = 0;
    for (int m = 1; m * check_every <= max_iters; ++m) {
        cudaError_t e = rbsor_run(h, w, u, check_every, omega, check_every, res + (m - 1), ws, s);
        double r = 0.0;
        if (e == cudaSuccess) e = read_res(res + (m - 1), &r, s);
        if (e != cudaSuccess) return e;
        *done = m * check_every;
        if (r <= tol) break;
    }
    return cudaSuccess;
}

}  // namespace pencil

// ------------------------------------------------ allocation-free entry point
// Scratch of pencil_jacobi2d_noalloc: the second grid buffer and the residual
// partials, laid out exactly as a caller workspace.  In host code the name
// below is only a stand-in; the device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PENCIL_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};

// Unique id of the calling thread's current context (0 if none is current or
// the driver does not offer the query).  Ids are never reused, so a primary
// context torn down and created again (cudaDeviceReset) gets a new one.
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_ctx = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_ctx = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_ctx || !get_id || get_ctx(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the static scratch on the current device, or the failing
// CUDA status.  Looked up once per device and context: after a device reset
// the module is loaded again and the array may sit elsewhere, so a changed
// context id makes the next call look it up again.
cudaError_t noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_noalloc_ptr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = current_context_id();  // the lookup made the primary context current
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" int pencil_jacobi2d_noalloc(int h, int w, float *u, int iters, int check_every,
                                       double *res_out, int temporal_t, void *stream) {
    if (h <= 0 || w <= 0 || iters < 0 || check_every < 0 || temporal_t < 0) return PENCIL_ERR_ARG;
    if ((int64_t)h * (int64_t)w > ((int64_t)1 << 40)) return PENCIL_ERR_ARG;
    if (h > PENCIL_MAX_ROWS) return PENCIL_ERR_UNSUPPORTED;  // the row limit of every _ex call
    if (!u) return PENCIL_ERR_NULL;
    const int nres = check_every > 0 ? iters / check_every : 0;
    if (nres > 0 && !res_out) return PENCIL_ERR_NULL;
    const size_t need = pencil::jacobi_workspace_bytes(h, w);
    if (need > PENCIL_NOALLOC_SCRATCH_BYTES) return PENCIL_ERR_NOMEM;
    if (!on_device(u) || (nres > 0 && !on_device(res_out))) return PENCIL_ERR_PTR;
    const uintptr_t ub = (uintptr_t)u, rb = (uintptr_t)res_out;
    const size_t un = sizeof(float) * (size_t)h * w, rn = sizeof(double) * (size_t)nres;
    if (nres > 0 && rb < ub + un && ub < rb + rn) return PENCIL_ERR_ALIAS;
    void *ws = nullptr;
    cudaError_t e = noalloc_scratch(&ws);
    if (e != cudaSuccess) return pencil::cuda_fail(e);
    e = pencil::jacobi_run(h, w, u, iters, check_every, res_out, ws, PENCIL_NOALLOC_SCRATCH_BYTES,
                           temporal_t, (cudaStream_t)stream);
    return e == cudaSuccess ? PENCIL_OK : pencil::cuda_fail(e);
}
