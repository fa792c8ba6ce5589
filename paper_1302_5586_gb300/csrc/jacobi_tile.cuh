// jacobi_tile.cuh -- the pieces of the 5-point Jacobi sweep shared by the
// Jacobi kernels (jacobi.cu) and the fused conv -> Jacobi kernel
// (conv_jacobi.cu): the per-point expression, the residual accumulation and
// the register-tiled multi-sweep window.  Internal linkage: each translation
// unit instantiates what it launches.
#pragma once

#include "internal.cuh"

namespace pencil {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// Add r^2, rounded to FP32, to the compensated pair (hi, lo): Knuth's TwoSum
// keeps the rounding error of each addition in lo, so hi + lo holds the sum
// of the rounded squares to about 2^-44 of it.
__device__ __forceinline__ void acc_sq(float r, float &hi, float &lo) {
    const float p = __fmul_rn(r, r);  // r^2 rounded to FP32
    const float t = __fadd_rn(hi, p);
    const float bp = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    hi = t;
    lo = __fadd_rn(lo, err);
}

__device__ __forceinline__ float nsum(float up, float dn, float lf, float rt) {
    return __fadd_rn(__fadd_rn(up, dn), __fadd_rn(lf, rt));
}


// ------------------------------------------------------ temporal tiling
// Up to T sweeps per HBM round trip with the tile held in registers.  A CTA
// owns a window of NW*RS rows x 128 columns (lane l: columns 4l .. 4l+3; warp
// k: rows k*RS .. k*RS+RS-1) and its core, rows [T, NW*RS-T) x columns
// [P, 128-P) with P = T rounded up to 4.  It loads the window once, runs the
// sweeps on registers -- each warp updates its rows top to bottom, taking
// left/right neighbours from adjacent lanes (shuffles) and the rows just
// outside its band from the neighbouring warps through shared memory (one
// barrier per sweep) -- and writes the core back.  Window rows 0 and NW*RS-1
// and columns 0 and 127 have no neighbours and take their own values in
// their place; the wrong values this makes move inward one point per sweep,
// like stale halo data, so after T sweeps the core is exact.  Grid boundary
// points keep their values.  Per point the update is the same FP32
// expression as the one-sweep kernel, so the iterate is the same bits for
// every T.  Residuals of iterates inside the pass are accumulated, over core
// points, during the sweep that updates them.
// NW warps of RS rows each; the library runs NW = 8, RS = 16 (two 256-thread
// CTAs per SM).
template <int T_, int NW_ = 8, int RS_ = 16>
struct RegCfg {
    static constexpr int T = T_;              // sweeps per pass (the halo width)
    static constexpr int NW = NW_;            // warps
    static constexpr int RS = RS_;            // rows per warp
    static constexpr int NT = 32 * NW;
    static constexpr int W = 128;             // window columns: 32 lanes x 4
    static constexpr int SH = NW * RS;        // window rows
    static constexpr int P = round_up(T, 4);  // core starts at window column P (16-byte aligned)
    static constexpr int BW = W - 2 * P;      // core columns
    static constexpr int BH = SH - 2 * T;     // core rows
};

// One sweep over a warp's RS rows, row r held in y[OFF + r].  DOWN: rows
// are updated top to bottom and new row r goes to y[OFF + r - 1] (the slot of
// old row r-1, dead once row r is done); otherwise bottom to top into
// y[OFF + r + 1].  A DOWN sweep from OFF = 1 and an up sweep from OFF = 0
// bring the band back to its slots without a register copy.  above/below:
// the rows just outside the band (old values).  EDGE: the window reaches the
// grid boundary, so points there (and outside the grid) keep their values.
template <int RS, bool DOWN, int OFF, bool EDGE, bool RESID>
__device__ __forceinline__ void reg_sweep(float4 (&y)[RS + 1], const float4 above, const float4 below, int g_first,
                                          int h, const bool (&cint)[4], bool core_cols, int core_lo, int core_hi,
                                          float &hi, float &lo) {
#pragma unroll
    for (int k = 0; k < RS; ++k) {
        const int r = DOWN ? k : RS - 1 - k;
        const float4 cur = y[OFF + r];
        const float4 upv = r > 0 ? y[OFF + r - 1] : above;
        const float4 dn = r + 1 < RS ? y[OFF + r + 1] : below;
        const float lf = __shfl_up_sync(FULL, cur.w, 1);    // lane 0: its own value (window column 0)
        const float rt = __shfl_down_sync(FULL, cur.x, 1);  // lane 31: its own value (window column 127)
        const float sx = nsum(upv.x, dn.x, lf, cur.y);
        const float sy = nsum(upv.y, dn.y, cur.x, cur.z);
        const float sz = nsum(upv.z, dn.z, cur.y, cur.w);
        const float sw = nsum(upv.w, dn.w, cur.z, rt);
        float4 nv = make_float4(__fmul_rn(0.25f, sx), __fmul_rn(0.25f, sy), __fmul_rn(0.25f, sz),
                                __fmul_rn(0.25f, sw));
        const int g = g_first + r;
        if (EDGE) {
            const bool rint = g >= 1 && g <= h - 2;
            nv.x = (rint && cint[0]) ? nv.x : cur.x;
            nv.y = (rint && cint[1]) ? nv.y : cur.y;
            nv.z = (rint && cint[2]) ? nv.z : cur.z;
            nv.w = (rint && cint[3]) ? nv.w : cur.w;
        }
        if (RESID && core_cols && g >= core_lo && g < core_hi && g >= 1 && g <= h - 2) {
            if (cint[0]) acc_sq(__fmaf_rn(4.f, cur.x, -sx), hi, lo);
            if (cint[1]) acc_sq(__fmaf_rn(4.f, cur.y, -sy), hi, lo);
            if (cint[2]) acc_sq(__fmaf_rn(4.f, cur.z, -sz), hi, lo);
            if (cint[3]) acc_sq(__fmaf_rn(4.f, cur.w, -sw), hi, lo);
        }
        y[DOWN ? OFF + r - 1 : OFF + r + 1] = nv;
    }
}

// One sweep (DOWN from slots 1..RS, or up from slots 0..RS-1), with the band
// edge rows exchanged first and, on checkpoint iterates, the residual partial
// of the warp recorded in wres.
template <int RS, int NW, bool DOWN, bool EDGE>
__device__ __forceinline__ void reg_step(float4 (&y)[RS + 1], int t, int iter0, int check_every, float4 *xch,
                                         double *wres, int &slot, int g_first, int h, const bool (&cint)[4],
                                         bool core_cols, int core_lo, int core_hi) {
    constexpr int OFF = DOWN ? 1 : 0;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int it = iter0 + t;
    const bool resid = check_every > 0 && it > 0 && it % check_every == 0;
    // band edge rows to the neighbours (double-buffered by sweep parity)
    float4 *xb = xch + (t & 1) * (NW * 2 * 32);
    xb[(wp * 2 + 0) * 32 + lane] = y[OFF];
    xb[(wp * 2 + 1) * 32 + lane] = y[OFF + RS - 1];
    __syncthreads();
    const float4 above = wp > 0 ? xb[((wp - 1) * 2 + 1) * 32 + lane] : y[OFF];
    const float4 below = wp < NW - 1 ? xb[((wp + 1) * 2 + 0) * 32 + lane] : y[OFF + RS - 1];
    if (resid) {
        float hi = 0.f, lo = 0.f;
        reg_sweep<RS, DOWN, OFF, EDGE, true>(y, above, below, g_first, h, cint, core_cols, core_lo, core_hi, hi, lo);
        // this iterate's partial: fixed butterfly per warp, warps in order later
        double d = (double)hi + (double)lo;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(FULL, d, off);
        if (lane == 0) wres[slot * NW + wp] = d;
        ++slot;
    } else {
        float hi = 0.f, lo = 0.f;
        reg_sweep<RS, DOWN, OFF, EDGE, false>(y, above, below, g_first, h, cint, core_cols, core_lo, core_hi, hi,
                                              lo);
    }
}

// Where a thread of a window with origin (gy0, gx0) sits: its first column
// gc0, its first row g_first, whether its columns are core columns and which
// of its four columns are interior, and the core's rows [core_lo, core_hi).
template <typename Cfg>
struct RegGeom {
    int gc0, g_first, core_lo, core_hi;
    bool core_cols;
    bool cint[4];
    __device__ __forceinline__ RegGeom(int h, int w, int gy0, int gx0) {
        constexpr int T = Cfg::T;
        const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
        gc0 = gx0 + 4 * lane;
        core_cols = 4 * lane >= Cfg::P && 4 * lane < Cfg::P + Cfg::BW && gc0 < w;
#pragma unroll
        for (int e = 0; e < 4; ++e) cint[e] = gc0 + e >= 1 && gc0 + e <= w - 2;
        g_first = gy0 + wp * Cfg::RS;
        core_lo = gy0 + T;
        core_hi = min(h, gy0 + T + Cfg::BH);
    }
};

// n <= T sweeps of a loaded window (row r of warp wp in y[1 + r]; y[0] is
// scratch) and the core written to v: sweeps in pairs (down, then up, which
// brings the band back to its slots), an odd count ending with one more down
// sweep.  Residuals of checkpoint iterates go to wres as reg_step records them.
template <typename Cfg, bool EDGE>
__device__ __forceinline__ void reg_sweeps_store(float4 (&y)[Cfg::RS + 1], float *__restrict__ v, int h, int w,
                                                 int n, const RegGeom<Cfg> &q, int iter0, int check_every,
                                                 float4 *xch, double *wres) {
    constexpr int RS = Cfg::RS, NW = Cfg::NW;
    const int gc0 = q.gc0, g_first = q.g_first, core_lo = q.core_lo, core_hi = q.core_hi;
    const bool core_cols = q.core_cols;
    const bool(&cint)[4] = q.cint;
    int slot = 0;
    int t = 0;
#pragma unroll 1
    for (; t + 1 < n; t += 2) {
        reg_step<RS, NW, true, EDGE>(y, t, iter0, check_every, xch, wres, slot, g_first, h, cint, core_cols,
                                     core_lo, core_hi);
        reg_step<RS, NW, false, EDGE>(y, t + 1, iter0, check_every, xch, wres, slot, g_first, h, cint, core_cols,
                                      core_lo, core_hi);
    }
    const int base = (t < n) ? 0 : 1;  // an odd count ends with one more DOWN sweep
    if (t < n)
        reg_step<RS, NW, true, EDGE>(y, t, iter0, check_every, xch, wres, slot, g_first, h, cint, core_cols,
                                     core_lo, core_hi);
    // the core back to HBM
    if (core_cols) {
#pragma unroll
        for (int r = 0; r < RS; ++r) {
            const int g = g_first + r;
            if (g >= core_lo && g < core_hi)
                *reinterpret_cast<float4 *>(v + (size_t)g * w + gc0) = base ? y[1 + r] : y[r];
        }
    }
}

}  // namespace
}  // namespace pencil
