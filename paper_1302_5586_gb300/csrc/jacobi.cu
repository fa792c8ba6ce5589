// jacobi.cu -- 5-point Jacobi sweeps and the FP64 residual norm for sm_103a.
//
// Sweep (the data-parallel body of the sequential `untilconverged` loop,
// Sec. 3.2; its points are independent, Sec. 2.2.3):
//   v[i][j] = 0.25f * ((u[i-1][j] + u[i+1][j]) + (u[i][j-1] + u[i][j+1]))
// on the interior, in FP32 and in exactly this order, boundary ring copied.
//
// Residual (the `reduction` directive, Sec. 2.2.3):
//   sqrt(sum_interior r^2),  r = 4u[i][j] - ((up + down) + (left + right)),
// r in FP32 (4u is exact); r^2 is split exactly into p + e (p = r*r rounded,
// e = fma(r, r, -p)) and added per thread into a compensated FP32 pair
// (Knuth's TwoSum), which is exact to about 2^-44 of the sum; the per-thread
// pairs are then added in FP64: warp butterfly, block, and one fixed-order
// pass over the per-block partials.  The order depends only on the grid
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

#include "internal.cuh"

namespace pencil {
namespace {

constexpr int JT = 128;  // threads per block
constexpr int JR = 16;   // rows per thread
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void acc_sq(float r, float &hi, float &lo) {
    const float p = __fmul_rn(r, r);
    const float e = __fmaf_rn(r, r, -p);  // p + e == r*r exactly
    const float t = __fadd_rn(hi, p);
    const float bp = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

__device__ __forceinline__ float nsum(float up, float dn, float lf, float rt) {
    return __fadd_rn(__fadd_rn(up, dn), __fadd_rn(lf, rt));
}

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
    float4 up = (colok && i0 > 0) ? __ldg(U + (size_t)(i0 - 1) * w4 + q) : z4;
    float4 cur = (colok && i0 < h) ? __ldg(U + (size_t)i0 * w4 + q) : z4;
#pragma unroll
    for (int o = 0; o < JR; ++o) {
        const int i = i0 + o;
        if (i >= h) break;
        const float4 dn = (colok && i + 1 < h) ? __ldg(U + (size_t)(i + 1) * w4 + q) : z4;
        float lf = __shfl_up_sync(FULL, cur.w, 1);
        float rt = __shfl_down_sync(FULL, cur.x, 1);
        if (lane == 0) lf = (colok && j0 > 0) ? __ldg(u + (size_t)i * w + j0 - 1) : 0.f;
        if (lane == 31) rt = (colok && j0 + 4 < w) ? __ldg(u + (size_t)i * w + j0 + 4) : 0.f;
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
                if (j0 > 0) acc_sq(__fsub_rn(__fmul_rn(4.f, cur.x), sx), hi, lo);
                acc_sq(__fsub_rn(__fmul_rn(4.f, cur.y), sy), hi, lo);
                acc_sq(__fsub_rn(__fmul_rn(4.f, cur.z), sz), hi, lo);
                if (j0 + 3 < w - 1) acc_sq(__fsub_rn(__fmul_rn(4.f, cur.w), sw), hi, lo);
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
            if (RESID) acc_sq(__fsub_rn(__fmul_rn(4.f, c), s), hi, lo);
        } else if (STORE) {
            v[p] = c;
        }
    }
    if (RESID)
        block_sum_store((double)hi + (double)lo, partials + (size_t)blockIdx.y * gridDim.x + blockIdx.x);
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

cudaError_t finish(const Plan &p, const double *partials, double *res, cudaStream_t s) {
    residual_finish_kernel<<<1, 256, 0, s>>>(partials, p.nblocks, res);
    return cudaGetLastError();
}

}  // namespace

size_t jacobi_workspace_bytes(int h, int w) {
    const size_t grid = align256(sizeof(float) * (size_t)h * (size_t)w);
    const size_t nb = (size_t)((w + JT - 1) / JT) * (size_t)((h + JR - 1) / JR);
    return grid + align256(sizeof(double) * nb);
}

static double *partials_of(void *ws, int h, int w) {
    return reinterpret_cast<double *>(static_cast<char *>(ws) +
                                      align256(sizeof(float) * (size_t)h * (size_t)w));
}

cudaError_t jacobi_run(int h, int w, float *u, int iters, int check_every, double *res, void *ws,
                       size_t ws_bytes, int temporal_t, cudaStream_t s) {
    (void)ws_bytes;
    (void)temporal_t;
    const int nres = (check_every > 0) ? iters / check_every : 0;
    if (h < 3 || w < 3 || iters == 0) {
        if (nres > 0) return cudaMemsetAsync(res, 0, sizeof(double) * (size_t)nres, s);
        return cudaSuccess;
    }
    float *v = static_cast<float *>(ws);
    double *partials = partials_of(ws, h, w);
    const Plan p = make_plan(h, w, u, v);
    float *cur = u, *nxt = v;
    cudaError_t e = cudaSuccess;
    for (int k = 1; k <= iters; ++k) {
        const int prev = k - 1;  // iterate index held in cur
        const bool want = check_every > 0 && prev > 0 && prev % check_every == 0;
        if (want) {
            e = sweep<true, true>(p, cur, nxt, h, w, partials, s);
            if (e == cudaSuccess) e = finish(p, partials, res + (prev / check_every - 1), s);
        } else {
            e = sweep<false, true>(p, cur, nxt, h, w, partials, s);
        }
        if (e != cudaSuccess) return e;
        float *t = cur;
        cur = nxt;
        nxt = t;
    }
    if (check_every > 0 && iters % check_every == 0) {
        e = sweep<true, false>(p, cur, nullptr, h, w, partials, s);
        if (e == cudaSuccess) e = finish(p, partials, res + (nres - 1), s);
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
    if (e == cudaSuccess) e = finish(p, partials, res, s);
    return e;
}

}  // namespace pencil
