// conv_kernels.cuh -- the conv2d kernels for sm_103a and their launch
// helpers, included by the planar (conv2d.cu) and interleaved (conv2d_hwc.cu)
// translation units; every definition has internal linkage, so each unit
// instantiates what it launches (and has its own wait-timeout counter).
//
// out[i][j] = sum_a sum_b k[a][b] * in[clamp(i+a-kh/2)][clamp(j+b-kw/2)]
// (the independent pixel loops of Sec. 2.2.3; a map over output pixels,
// Sec. 3.2).  Every kernel here accumulates one output pixel in the same FP32
// order: for each filter row a, s = k[a][0]*x0 then s = fma(k[a][b], xb, s)
// for b = 1..kw-1, and acc = acc + s with acc starting at +0 -- so the direct,
// generic and batched kernels return identical bits for the same pixel.
#pragma once

#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>

#include "conv_tile.cuh"
#include "tma.cuh"

namespace pencil {
namespace {

using namespace tile;

// Per-lane operations on a pair of FP32 values (fma.rn.f32x2, mul.rn.f32x2),
// each lane rounded to nearest even exactly like the scalar operation.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// VMODE: how rows that are not 16-byte aligned are handled.  0: vec_ok at
// run time, such rows staged in 4-byte copies and stored with scalar stores
// (the least code around the FMA loop); 1: every row aligned (compile-time);
// 2: rows not aligned (compile-time), each chunk copied and stored with the
// widest accesses its address allows; 3: rows not aligned (compile-time),
// 4-byte copies and scalar stores.
// CS > 1: one interleaved image of CS channels, w = pixels * CS elements per
// row (grid.z = 1).
template <typename T, int KH, int KW, int TX, int TY, int R, int G, int MINB, bool ANYB, bool HALFW, int VMODE,
          int CS = 1, int C = 4>
__global__ void __launch_bounds__(TX *TY, MINB)
    conv2d_direct_kernel(const T *__restrict__ in, const float *__restrict__ k, T *__restrict__ out,
                         int h, int w, bool vec_ok, int border) {
    using Cfg = DirectCfg<KH, KW, TX, TY, R, G, CS, C>;
    extern __shared__ __align__(128) float smem[];
    const size_t plane = (size_t)h * (size_t)w * blockIdx.z;
    const bool vok = VMODE == 0 ? vec_ok : VMODE == 1;
    direct_tile<T, KH, KW, TX, TY, R, G, ANYB, HALFW, VMODE == 2, CS, C>(in + plane, k, out + plane, h, w, vok,
                                                   blockIdx.y * Cfg::TH, blockIdx.x * Cfg::TW, smem, border);
}

// ---------------------------------------------------------- TMA-staged kernel
// Tile loads that did not complete within their bounded wait (each such CTA
// skipped its tile); read and cleared by pencil_device_status.
__device__ unsigned int g_wait_timeouts;

// This translation unit's count of tile loads that gave up their wait (each
// skipped its tile); clear resets it.
inline cudaError_t read_wait_counter(unsigned *n, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(n, g_wait_timeouts, sizeof(unsigned));
    if (e == cudaSuccess && clear && *n) {
        const unsigned zero = 0;
        e = cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(unsigned));
    }
    return e;
}

// Clamp-to-edge on a staged tile that holds zeros outside the image (a TMA
// load fills out-of-range elements with zeros): rows above or below the
// image take the nearest edge row, then columns left or right of it the
// nearest edge column, so corners get both clamps.  (gy0, gx0): global
// position of t[0][0].  CS > 1 (interleaved, w elements = pixels * CS): an
// element outside takes the same channel of the nearest edge pixel.
// Block-uniform; ends with a barrier when it writes.
template <typename S, int SH, int SW, int NT, int CS = 1>
__device__ __forceinline__ void clamp_fixup(S *__restrict__ t, int h, int w, int gy0, int gx0) {
    const int top = -gy0, bot = h - gy0;  // staged rows [top, bot) are inside the image
    if (top > 0 || bot < SH) {
        for (int idx = threadIdx.x; idx < SH * SW; idx += NT) {
            const int r = idx / SW, c = idx - r * SW;
            const int src = r < top ? top : (r >= bot ? bot - 1 : r);
            if (src != r) t[idx] = t[src * SW + c];
        }
        __syncthreads();
    }
    const int left = -gx0, right = w - gx0;  // staged columns [left, right) are inside
    if (left > 0 || right < SW) {
        for (int idx = threadIdx.x; idx < SH * SW; idx += NT) {
            const int r = idx / SW, c = idx - r * SW;
            int src = c;
            if (c < left)
                src = left + ((c - left) % CS + CS) % CS;
            else if (c >= right)
                src = right - CS + (c - right) % CS;
            if (src != c) t[idx] = t[r * SW + src];
        }
        __syncthreads();
    }
}

// The direct kernel with its halo tile loaded by the tensor memory
// accelerator: one thread arms an mbarrier and issues a single
// cp.async.bulk.tensor copy of the (TH+kh-1) x (TW+2P) box of plane
// blockIdx.z (rows 16-byte aligned, which the tensor map requires); the other
// threads stage the filter meanwhile.  Out-of-image elements arrive as zeros:
// the zero border as it is, clamp-to-edge after clamp_fixup.  The compute is
// the shared tile body, so the bits are those of the cp.async kernel.
// Shared memory: the staged tile (type T, first, 128-byte aligned), the FP32
// copy of a binary16 tile unless HALFW, the filter rows.
template <typename T, int KH, int KW, int TX, int TY, int R, int G, int MINB, bool HALFW, bool CLAMP, int CS = 1,
          int C = 4>
__global__ void __launch_bounds__(TX *TY, MINB)
    conv2d_direct_tma_kernel(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ k,
                             T *__restrict__ out, int h, int w) {
    using Cfg = DirectCfg<KH, KW, TX, TY, R, G, CS, C>;
    constexpr int SW = Cfg::SW, SH = Cfg::SH, KWP = Cfg::KWP, NT = Cfg::NT;
    constexpr bool F16 = sizeof(T) == 2;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar;
    T *s_t = reinterpret_cast<T *>(smem);                                           // the TMA box
    float *s_in = F16 ? reinterpret_cast<float *>(s_t + SH * SW) : smem;            // FP32 tile
    float *s_k = F16 && HALFW ? s_in : s_in + SH * SW;                              // filter rows
    const int y0 = blockIdx.y * Cfg::TH, x0 = blockIdx.x * Cfg::TW;
    const int gy0 = y0 - Cfg::AH, gx0 = x0 - Cfg::P;
    if ((tma::smem_addr(s_t) & 127u) != 0) {  // a TMA box needs a 128-byte aligned destination
        if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);
        return;
    }

    if (threadIdx.x == 0) tma::mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        tma::mbar_arrive_expect_tx(&bar, (unsigned)(sizeof(T) * SH * SW));
        tma::load_3d(s_t, &tmap, gx0, gy0, (int)blockIdx.z, &bar);
    }
    stage_filter<KH, KW, KWP, NT>(k, s_k);
    const bool ok = __syncthreads_and(tma::mbar_wait(&bar, 0, tma::kLoadWaitNs));
    if (!ok) {  // the copy did not complete in time: report, let it land, skip the tile
        if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);
        tma::mbar_wait(&bar, 0, tma::kLoadWaitNs);
        return;
    }
    if (CLAMP) clamp_fixup<T, SH, SW, NT, CS>(s_t, h, w, gy0, gx0);
    T *dst = out + (size_t)h * (size_t)w * blockIdx.z;
    if constexpr (F16 && HALFW) {
        direct_compute<T, KH, KW, TX, TY, R, G, T, false, CS, C>(s_t, s_k, dst, h, w, true, y0, x0);
    } else {
        stage_widen<T, SH, SW, NT>(s_in, s_t);
        direct_compute<T, KH, KW, TX, TY, R, G, float, false, CS, C>(s_in, s_k, dst, h, w, true, y0, x0);
    }
}

// Planar images whose rows are not 16-byte aligned, clamp (CLAMP) or zero
// border: the tile staged by row-wise TMA boxes of the flat image (tile's
// RowStage), then realigned -- in place for FP32 (the tile is the landing
// area, row stride LP), into a binary16 tile for HALFW, widened into an FP32
// tile for other binary16 images (each measured faster than the other
// choices) -- and the same compute as the other direct kernels.  Stores take
// the widest access each address allows.  Shared memory: landing rows
// (128-byte aligned, first), the separate tile, the filter rows.
template <typename T, int KH, int KW, int TX, int TY, int R, int G, int MINB, bool HALFW, bool CLAMP, int C = 4>
struct DirectRows {
    using Cfg = DirectCfg<KH, KW, TX, TY, R, G, 1, C>;
    using RS = RowStage<T, Cfg::SH, Cfg::SW>;
    static constexpr bool INPLACE = sizeof(T) == 4;
    static constexpr size_t tile_bytes = INPLACE ? 0 : (HALFW ? 2 : 4) * (size_t)Cfg::SH * Cfg::SW;
    static constexpr size_t smem = RS::bytes + tile_bytes + sizeof(float) * KH * Cfg::KWP;
};

template <typename T, int KH, int KW, int TX, int TY, int R, int G, int MINB, bool HALFW, bool CLAMP, int C = 4>
__global__ void __launch_bounds__(TX *TY, MINB)
    conv2d_direct_rows_kernel(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ k,
                              T *__restrict__ out, int h, int w) {
    using DR = DirectRows<T, KH, KW, TX, TY, R, G, MINB, HALFW, CLAMP, C>;
    using Cfg = typename DR::Cfg;
    using RS = typename DR::RS;
    constexpr int SW = Cfg::SW, SH = Cfg::SH, KWP = Cfg::KWP, NT = Cfg::NT;
    static_assert(!HALFW || sizeof(T) == 2, "HALFW reads a binary16 tile");
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_shift[SH];
    T *land = reinterpret_cast<T *>(smem);
    float *s_in = smem + RS::bytes / sizeof(float);  // the separate tile (FP32, or HALFW binary16)
    T *s16 = reinterpret_cast<T *>(s_in);
    float *s_k = s_in + DR::tile_bytes / sizeof(float);
    const int y0 = blockIdx.y * Cfg::TH, x0 = blockIdx.x * Cfg::TW;
    const int gy0 = y0 - Cfg::AH, gx0 = x0 - Cfg::P;
    if ((tma::smem_addr(land) & 127u) != 0) {  // a TMA box needs a 128-byte aligned destination
        if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);
        return;
    }
    if (threadIdx.x == 0) tma::mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x < 32)
        rows_issue<T, SH, SW, CLAMP>(&tmap, (long long)h * w * blockIdx.z, h, w, gy0, gx0, land, s_shift, &bar);
    stage_filter<KH, KW, KWP, NT>(k, s_k);
    const bool ok = __syncthreads_and(tma::mbar_wait(&bar, 0, tma::kLoadWaitNs));
    if (!ok) {  // the copies did not complete in time: report, let them land, skip the tile
        if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);
        tma::mbar_wait(&bar, 0, tma::kLoadWaitNs);
        return;
    }
    T *dst = out + (size_t)h * (size_t)w * blockIdx.z;
    if constexpr (DR::INPLACE) {
        rows_realign_inplace<T, SH, SW, NT, CLAMP>(land, s_shift, w, gx0);
        __syncthreads();
        direct_compute<T, KH, KW, TX, TY, R, G, T, true, 1, C, RS::LP>(land, s_k, dst, h, w, false, y0, x0);
    } else if constexpr (HALFW) {
        rows_realign<T, T, SH, SW, NT, CLAMP>(land, s_shift, s16, w, gx0);
        __syncthreads();
        direct_compute<T, KH, KW, TX, TY, R, G, T, true, 1, C>(s16, s_k, dst, h, w, false, y0, x0);
    } else {
        rows_realign<T, float, SH, SW, NT, CLAMP>(land, s_shift, s_in, w, gx0);
        __syncthreads();
        direct_compute<T, KH, KW, TX, TY, R, G, float, true, 1, C>(s_in, s_k, dst, h, w, false, y0, x0);
    }
}

// ------------------------------------------------------------ generic kernel
// Any kh, kw: one output per thread, reads straight from global memory with
// clamped indices (L1/L2 serve the reuse).  Same per-pixel order as above.
// Pixel (i, j) of channel z = blockIdx.z is element z*h*w + i*w + j of a
// planar image (cs = 0), or (i*w + j)*cs + z of an interleaved one of cs
// channels.
template <typename T>
__global__ void __launch_bounds__(256)
    conv2d_generic_kernel(const T *__restrict__ in, const float *__restrict__ k, T *__restrict__ out,
                          int h, int w, int kh, int kw, int border, int cs) {
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    const int i = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (i >= h || j >= w) return;
    const size_t base = cs ? (size_t)blockIdx.z : (size_t)h * (size_t)w * blockIdx.z;
    const size_t px_stride = cs ? (size_t)cs : 1;
    const T *src = in + base;
    const int ah = kh / 2, aw = kw / 2;
    float acc = 0.0f;
    for (int a = 0; a < kh; ++a) {
        const int r = border_index(i + a - ah, h, border);
        const T *row = src + (size_t)max(r, 0) * (size_t)w * px_stride;
        const float *kr = k + (size_t)a * kw;
        auto px = [&](int b) {
            const int c = border_index(j + b - aw, w, border);
            return (r < 0 || c < 0) ? 0.0f : Io<T>::ld(row + (size_t)c * px_stride);
        };
        float s = __fmul_rn(__ldg(kr), px(0));
        for (int b = 1; b < kw; ++b) s = __fmaf_rn(__ldg(kr + b), px(b), s);
        acc = __fadd_rn(acc, s);
    }
    Io<T>::st(out + base + ((size_t)i * w + j) * px_stride, acc);
}

// --------------------------------------------------------- separable kernel
// Row pass (kx taps) of the staged halo tile into shared memory, then the
// column pass (ky taps) from it; nothing intermediate goes to HBM.  PAIR bit 1
// runs the row pass, bit 2 the column pass, on packed FP32 pairs (two adjacent
// columns per instruction, the same bits as the scalar form; on GB300 a pair
// instruction costs the issue slots of two scalar ones, so it pays only where
// it shortens the schedule: measured per side, see sep_pair).
// CS > 1: interleaved images of CS channels (row-pass taps CS elements apart).
// HALFR (binary16 images): the row pass reads the staged binary16 tile and
// widens each window in registers, so no FP32 copy of the tile exists; its
// results go to their own FP32 buffer (INPLACE must be false).
// CR: columns per row-pass item (a multiple of 4 dividing the tile width);
// the column pass always takes 4.  Wider items share one tap window among
// more outputs, which pays where the taps are CS apart.
template <int KX, int KY, int TX, int TY, int R, bool INPLACE = false, int CS = 1, bool HALFR = false,
          int CR_ = 4>
struct SepCfg {
    static constexpr int C = 4, CR = CR_;
    static constexpr int AX = KX / 2, AY = KY / 2;
    static constexpr int AXE = AX * CS;       // row-pass halo in elements
    static constexpr int NT = TX * TY;
    static constexpr int TW = TX * C, TH = TY * R;
    static constexpr int P = round_up(AXE, 8);
    static constexpr int SW = TW + 2 * P;
    static constexpr int SH = TH + KY - 1;
    static constexpr int M0 = (P - AXE) & ~3;  // first 16-byte chunk a row pass reads
    static constexpr int NX = round_up(P - AXE - M0 + CR + (KX - 1) * CS, 4);
    static_assert(CR % 4 == 0 && TW % CR == 0, "row-pass items of whole 16-byte chunks tile a row");
    // in place: the row-pass results overwrite the staged tile (row stride SW);
    // HALFR: only the row-pass results are FP32
    static_assert(!(HALFR && INPLACE), "a binary16 tile read directly cannot take the row-pass results");
    static constexpr size_t smem_f32 =
        sizeof(float) * (size_t)(HALFR ? SH * TW : SH * SW + (INPLACE ? 0 : SH * TW));
    // the binary16 staging area follows, 128-byte aligned (a TMA box destination)
    static constexpr size_t off16 = (smem_f32 + 127) / 128 * 128;
    static constexpr size_t smem(size_t esz) { return esz == 2 ? off16 + 2 * (size_t)SH * SW : smem_f32; }
};

// VMODE 0-2 as for the direct kernel (cp.async staging); 3: rows 16-byte
// aligned, clamp (border 0) or zero (border 1) border, the halo tile loaded
// as one TMA box of `tmap` (unused by the other modes), as the direct TMA
// kernel does.
template <typename T, int KX, int KY, int TX, int TY, int R, int MINB, bool INPLACE, bool ANYB, int PAIR,
          int VMODE, int CS = 1, bool HALFR = false, int CR = 4>
__global__ void __launch_bounds__(TX *TY, MINB)
    conv2d_sep_kernel(const __grid_constant__ CUtensorMap tmap, const T *__restrict__ in,
                      const float *__restrict__ gx, const float *__restrict__ gy, T *__restrict__ out, int h,
                      int w, bool vec_ok_, int border) {
    constexpr bool ADAPT = VMODE == 2, TMA = VMODE == 3;
    static_assert(!HALFR || sizeof(T) == 2, "HALFR reads a binary16 tile");
    const bool vec_ok = VMODE == 0 ? vec_ok_ : VMODE != 2;
    using Cfg = SepCfg<KX, KY, TX, TY, R, INPLACE, CS, HALFR, CR>;
    constexpr int C = Cfg::C, P = Cfg::P, SW = Cfg::SW, SH = Cfg::SH, TW = Cfg::TW,
                  NX = Cfg::NX, AY = Cfg::AY, NT = Cfg::NT;
    constexpr int TS = INPLACE ? SW : TW;  // row stride of the row-pass results
    extern __shared__ __align__(128) float smem[];
    float *s_in = smem;
    float *s_t = INPLACE || HALFR ? smem : smem + SH * SW;
    T *s16 = reinterpret_cast<T *>(smem + Cfg::off16 / sizeof(float));

    const size_t plane = (size_t)h * (size_t)w * blockIdx.z;
    const T *src = in + plane;
    T *dst = out + plane;
    const int x0 = blockIdx.x * TW;
    const int y0 = blockIdx.y * Cfg::TH;
    if constexpr (TMA) {
        __shared__ __align__(8) uint64_t bar;
        T *s_box = sizeof(T) == 2 ? s16 : reinterpret_cast<T *>(s_in);
        if ((tma::smem_addr(s_box) & 127u) != 0) {  // a TMA box needs a 128-byte aligned destination
            if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);
            return;
        }
        if (threadIdx.x == 0) tma::mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            tma::mbar_arrive_expect_tx(&bar, (unsigned)(sizeof(T) * SH * SW));
            tma::load_3d(s_box, &tmap, x0 - P, y0 - AY, (int)blockIdx.z, &bar);
        }
        if (!__syncthreads_and(tma::mbar_wait(&bar, 0, tma::kLoadWaitNs))) {
            if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);
            tma::mbar_wait(&bar, 0, tma::kLoadWaitNs);
            return;
        }
        if (border == 0) clamp_fixup<T, SH, SW, NT, CS>(s_box, h, w, y0 - AY, x0 - P);
        if constexpr (!HALFR) stage_widen<T, SH, SW, NT>(s_in, s16);
    } else if constexpr (HALFR) {
        stage_issue<T, SH, SW, NT, ANYB, ADAPT, CS>(src, h, w, y0 - AY, x0 - P, vec_ok, nullptr, s16, border);
        cp_async_wait_all();
        __syncthreads();
    } else {
        stage_tile<T, SH, SW, NT, ANYB, ADAPT, CS>(src, h, w, y0 - AY, x0 - P, vec_ok, s_in, s16, border);
    }

    // row pass: t[r][q*CR + c] = sum_b gx[b] * in[r][q*CR + c + b - AX]
    {
        float fx[KX];
#pragma unroll
        for (int b = 0; b < KX; ++b) fx[b] = __ldg(gx + b);
        constexpr int X0 = P - Cfg::AXE - Cfg::M0;  // window index of tap 0 of column 0
        constexpr int QPR = TW / CR;
        constexpr int ITEMS = SH * QPR;
        constexpr int PER = (ITEMS + NT - 1) / NT;  // items per thread
        constexpr int NQ = CR / 4;                  // 16-byte chunks per item
        float4 res[INPLACE ? PER : 1][NQ];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int idx = threadIdx.x + k * NT;
            if (idx < ITEMS) {
                const int r = idx / QPR, q = idx - r * QPR;
                float x[NX];
                if constexpr (HALFR) {
                    const T *sp = s16 + r * SW + q * CR + Cfg::M0;
#pragma unroll
                    for (int m = 0; m < NX; m += 4) ld4s(sp + m, &x[m]);
                } else {
                    const float *sp = s_in + r * SW + q * CR + Cfg::M0;
#pragma unroll
                    for (int m = 0; m < NX; m += 4) ld4s(sp + m, &x[m]);
                }
                float tv[CR];
                if constexpr ((PAIR & 1) != 0) {
#pragma unroll
                    for (int c = 0; c < CR; c += 2) {
                        float2 sum = mul2(make_float2(fx[0], fx[0]), make_float2(x[X0 + c], x[X0 + c + 1]));
#pragma unroll
                        for (int b = 1; b < KX; ++b)
                            sum = fma2(make_float2(fx[b], fx[b]),
                                       make_float2(x[X0 + c + b * CS], x[X0 + c + b * CS + 1]), sum);
                        tv[c] = sum.x;
                        tv[c + 1] = sum.y;
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < CR; ++c) {
                        float sum = __fmul_rn(fx[0], x[X0 + c]);
#pragma unroll
                        for (int b = 1; b < KX; ++b) sum = __fmaf_rn(fx[b], x[X0 + c + b * CS], sum);
                        tv[c] = sum;
                    }
                }
#pragma unroll
                for (int j = 0; j < NQ; ++j) {
                    const float4 t4 = make_float4(tv[4 * j], tv[4 * j + 1], tv[4 * j + 2], tv[4 * j + 3]);
                    if (INPLACE)
                        res[k][j] = t4;
                    else
                        *reinterpret_cast<float4 *>(s_t + r * TS + q * CR + 4 * j) = t4;
                }
            }
        }
        if (INPLACE) {
            __syncthreads();  // every read of the staged tile is done
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int idx = threadIdx.x + k * NT;
                if (idx < ITEMS) {
                    const int r = idx / QPR, q = idx - r * QPR;
#pragma unroll
                    for (int j = 0; j < NQ; ++j) *reinterpret_cast<float4 *>(s_t + r * TS + q * CR + 4 * j) = res[k][j];
                }
            }
        }
    }
    __syncthreads();

    // column pass: out[o][c] = sum_a gy[a] * t[o + a][c]
    float fy[KY];
#pragma unroll
    for (int a = 0; a < KY; ++a) fy[a] = __ldg(gy + a);
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    float acc[R][C];
    if constexpr ((PAIR & 2) != 0) {
        float2 acc2[R][C / 2];
#pragma unroll
        for (int r = 0; r < R + KY - 1; ++r) {
            const float4 v = *reinterpret_cast<const float4 *>(s_t + (ty * R + r) * TS + tx * C);
            const float2 tv[C / 2] = {make_float2(v.x, v.y), make_float2(v.z, v.w)};
#pragma unroll
            for (int o = 0; o < R; ++o) {
                const int a = r - o;
                if (a == 0) {
#pragma unroll
                    for (int q = 0; q < C / 2; ++q) acc2[o][q] = mul2(make_float2(fy[0], fy[0]), tv[q]);
                } else if (a > 0 && a < KY) {
#pragma unroll
                    for (int q = 0; q < C / 2; ++q) acc2[o][q] = fma2(make_float2(fy[a], fy[a]), tv[q], acc2[o][q]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < R; ++o)
#pragma unroll
            for (int q = 0; q < C / 2; ++q) {
                acc[o][2 * q] = acc2[o][q].x;
                acc[o][2 * q + 1] = acc2[o][q].y;
            }
    } else {
#pragma unroll
        for (int r = 0; r < R + KY - 1; ++r) {
            const float4 v = *reinterpret_cast<const float4 *>(s_t + (ty * R + r) * TS + tx * C);
            const float tv[C] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int o = 0; o < R; ++o) {
                const int a = r - o;
                if (a == 0) {
#pragma unroll
                    for (int c = 0; c < C; ++c) acc[o][c] = __fmul_rn(fy[0], tv[c]);
                } else if (a > 0 && a < KY) {
#pragma unroll
                    for (int c = 0; c < C; ++c) acc[o][c] = __fmaf_rn(fy[a], tv[c], acc[o][c]);
                }
            }
        }
    }
    store_block<T, R, ADAPT>(dst, h, w, y0 + ty * R, x0 + tx * C, vec_ok, acc);
}

// Separable with runtime tap counts (fallback for sides without a
// specialisation): same order, taps read from shared memory.
// Addressing as for the generic direct kernel (cs = 0 planar, else interleaved).
template <typename T>
__global__ void __launch_bounds__(256)
    conv2d_sep_generic_kernel(const T *__restrict__ in, const float *__restrict__ gx,
                              const float *__restrict__ gy, T *__restrict__ out, int h, int w,
                              int kx, int ky, int border, int cs) {
    // tile 32 x 32 outputs, 256 threads
    extern __shared__ __align__(128) float smem[];
    const int SH = 32 + ky - 1;
    float *s_t = smem;                  // SH x 32
    const size_t plane = cs ? (size_t)blockIdx.z : (size_t)h * (size_t)w * blockIdx.z;
    const size_t px_stride = cs ? (size_t)cs : 1;
    const T *src = in + plane;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    const int ax = kx / 2, ay = ky / 2;
    for (int idx = threadIdx.x; idx < SH * 32; idx += 256) {
        const int r = idx / 32, c = idx % 32;
        const int gr = border_index(y0 + r - ay, h, border);
        const T *row = src + (size_t)max(gr, 0) * (size_t)w * px_stride;
        const int j = x0 + c;
        auto px = [&](int b) {
            const int gc = border_index(j + b - ax, w, border);
            return (gr < 0 || gc < 0) ? 0.0f : Io<T>::ld(row + (size_t)gc * px_stride);
        };
        float s = __fmul_rn(__ldg(gx), px(0));
        for (int b = 1; b < kx; ++b) s = __fmaf_rn(__ldg(gx + b), px(b), s);
        s_t[idx] = s;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * 32; idx += 256) {
        const int r = idx / 32, c = idx % 32;
        const int i = y0 + r, j = x0 + c;
        if (i >= h || j >= w) continue;
        float acc = __fmul_rn(__ldg(gy), s_t[r * 32 + c]);
        for (int a = 1; a < ky; ++a) acc = __fmaf_rn(__ldg(gy + a), s_t[(r + a) * 32 + c], acc);
        Io<T>::st(out + plane + ((size_t)i * w + j) * px_stride, acc);
    }
}

// ------------------------------------------------------------------ launch
template <typename Kern>
cudaError_t set_smem(Kern kern, size_t bytes) {
    // without the attribute, static and dynamic shared memory share 48 KB;
    // the kernels' static part stays under 1 KB
    if (bytes + 1024 <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on it),
// or null where the driver does not offer it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// Tensor map of a [c][h][w] image with rows 16-byte aligned, box (bw, bh, 1);
// false if it cannot be made (the caller then stages with cp.async).
template <typename T>
bool image_tensor_map(CUtensorMap *m, const T *base, int c, int h, int w, int bw, int bh) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)c};
    const cuuint64_t strides[2] = {(cuuint64_t)w * sizeof(T), (cuuint64_t)h * (cuuint64_t)w * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1u};
    const cuuint32_t elem[3] = {1u, 1u, 1u};
    return enc(m, sizeof(T) == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
               const_cast<T *>(base), dims, strides, box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 1-D tensor map over the n elements of an image (box of `box` elements);
// false if it cannot be made: base not 16-byte aligned, or n too large for
// the 32-bit box coordinates.
template <typename T>
bool flat_tensor_map(CUtensorMap *m, const T *base, long long n, int box) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || n <= 0 || n > 0x7fffff00ll || ((uintptr_t)base & 15u) != 0) return false;
    const cuuint64_t dims[1] = {(cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(T)};  // unused for one dimension
    const cuuint32_t boxd[1] = {(cuuint32_t)box};
    const cuuint32_t elem[1] = {1u};
    return enc(m, sizeof(T) == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 1,
               const_cast<T *>(base), dims, strides, boxd, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The row-staged launch for planar images whose rows are not 16-byte aligned
// (clamp or zero border); false, with nothing launched, where it does not
// apply.
template <typename T, int K, int TX, int TY, int R, int G, int MINB, bool HALFW, int C = 4>
bool try_direct_rows(int c, int h, int w, const T *in, const float *k, T *out, int border, cudaStream_t s,
                     cudaError_t *err) {
    using DR = DirectRows<T, K, K, TX, TY, R, G, MINB, HALFW, true, C>;
    using Cfg = typename DR::Cfg;
    CUtensorMap tmap;
    const long long n = (long long)c * h * w;
    if ((border != 0 && border != 1) || n < DR::RS::LB || !flat_tensor_map<T>(&tmap, in, n, DR::RS::LB))
        return false;
    auto kern = border == 0 ? conv2d_direct_rows_kernel<T, K, K, TX, TY, R, G, MINB, HALFW, true, C>
                            : conv2d_direct_rows_kernel<T, K, K, TX, TY, R, G, MINB, HALFW, false, C>;
    const size_t smem = DR::smem;
    *err = set_smem(kern, smem);
    if (*err == cudaSuccess) {
        dim3 grid((w + Cfg::TW - 1) / Cfg::TW, (h + Cfg::TH - 1) / Cfg::TH, c);
        kern<<<grid, Cfg::NT, smem, s>>>(tmap, k, out, h, w);
        *err = cudaGetLastError();
    }
    return true;
}

// The TMA-staged launch for aligned rows with the clamp or zero border (a box
// side is at most 256 elements); false, with nothing launched, where it does
// not apply.
// CS > 1: w is the element width of one interleaved image (pixels * CS), c = 1.
template <typename T, int K, int TX, int TY, int R, int G, int MINB, bool HALFW, int CS = 1, int C = 4>
bool try_direct_tma(int c, int h, int w, const T *in, const float *k, T *out, bool vec_ok, int border,
                    cudaStream_t s, cudaError_t *err) {
    using Cfg = DirectCfg<K, K, TX, TY, R, G, CS, C>;
    static_assert(Cfg::SW <= 256 && Cfg::SH <= 256, "a TMA box side is at most 256 elements");
    CUtensorMap tmap;
    if (!vec_ok || (border != 0 && border != 1) || !image_tensor_map<T>(&tmap, in, c, h, w, Cfg::SW, Cfg::SH))
        return false;
    auto kern = border == 0 ? conv2d_direct_tma_kernel<T, K, K, TX, TY, R, G, MINB, HALFW, true, CS, C>
                            : conv2d_direct_tma_kernel<T, K, K, TX, TY, R, G, MINB, HALFW, false, CS, C>;
    const size_t smem = HALFW ? Cfg::smem_half : Cfg::smem(sizeof(T));
    *err = set_smem(kern, smem);
    if (*err == cudaSuccess) {
        dim3 grid((w + Cfg::TW - 1) / Cfg::TW, (h + Cfg::TH - 1) / Cfg::TH, c);
        kern<<<grid, Cfg::NT, smem, s>>>(tmap, k, out, h, w);
        *err = cudaGetLastError();
    }
    return true;
}

// Planar rows that are not 16-byte aligned take the row staging on images
// of at least 2^20 elements (smaller ones are latency-bound, and there the
// cp.async staging measured faster) at sides up to 5, when the rows are not
// even 8-byte (FP32) or 4-byte (binary16) aligned: odd widths.  Elsewhere the
// cp.async kernel compiled for unaligned rows, with the widest copies each
// row allows, measured faster (3 x 4096 x 4094: FP32 3x3 0.083 -> 0.078 ms,
// 5x5 0.101 -> 0.095, 7x7 0.140 -> 0.130; binary16 3x3 0.071 -> 0.060, 7x7
// 0.143 -> 0.125, 11x11 0.292 -> 0.260, 15x15 0.476 -> 0.461, and more at
// 3 x 4096 x 4092; odd widths, 3 x 4096 x 4095: FP32 7x7 0.141 -> 0.137,
// binary16 7x7 0.142 -> 0.140, 11x11 0.295 -> 0.280, 15x15 0.523 -> 0.515).
constexpr long long kRowsMin = 1ll << 20;
template <typename T, int K>
constexpr bool rows_pay() {
    return K <= 5;
}

template <typename T, int K, int TX, int TY, int R, int G = 1, int MINB = 1, bool HALFW = false, int CS = 1,
          int C = 4>
cudaError_t run_direct(int c, int h, int w, const T *in, const float *k, T *out, bool vec_ok,
                       int border, cudaStream_t s) {
    using Cfg = DirectCfg<K, K, TX, TY, R, G, CS, C>;
    cudaError_t err = cudaSuccess;
    if (try_direct_tma<T, K, TX, TY, R, G, MINB, HALFW, CS, C>(c, h, w, in, k, out, vec_ok, border, s, &err))
        return err;
    if constexpr (CS == 1 && rows_pay<T, K>()) {
        // rows at least 8-byte (FP32) or 4-byte (binary16) aligned
        const unsigned a = sizeof(T) == 4 ? 8u : 4u;
        const bool wide = w % 2 == 0 && (uintptr_t)in % a == 0 && (uintptr_t)out % a == 0;
        if (!vec_ok && !wide && (long long)c * h * w >= kRowsMin &&
            try_direct_rows<T, K, TX, TY, R, G, MINB, HALFW, C>(c, h, w, in, k, out, border, s, &err))
            return err;
    }
    // sides up to 5 (memory-bound): an aligned-row kernel and an adaptive
    // any-row kernel; larger sides: one kernel with vec_ok at run time, and
    // for rows that are not aligned (clamp border) a kernel compiled for them:
    // adaptive copies and stores, but 4-byte ones at FP32 side 9 (3 x 4096 x
    // 4095 / 4094: 2-12% faster than the run-time kernel, the same bits)
    using Kern = void (*)(const T *, const float *, T *, int, int, bool, int);
    Kern kern;
    if constexpr (K <= 5 && CS == 1)
        kern = border != 0 ? conv2d_direct_kernel<T, K, K, TX, TY, R, G, MINB, true, HALFW, 2, 1, C>
               : vec_ok    ? conv2d_direct_kernel<T, K, K, TX, TY, R, G, MINB, false, HALFW, 1, 1, C>
                           : conv2d_direct_kernel<T, K, K, TX, TY, R, G, MINB, false, HALFW, 2, 1, C>;
    else if constexpr (K >= 7 && CS == 1)
        kern = border != 0 ? conv2d_direct_kernel<T, K, K, TX, TY, R, G, MINB, true, HALFW, 0, 1, C>
               : vec_ok    ? conv2d_direct_kernel<T, K, K, TX, TY, R, G, MINB, false, HALFW, 0, 1, C>
                           : conv2d_direct_kernel<T, K, K, TX, TY, R, G, MINB, false, HALFW,
                                                  sizeof(T) == 4 && K == 9 ? 3 : 2, 1, C>;
    else  // interleaved images keep to one kernel per border class (their aligned rows take TMA)
        kern = border != 0 ? conv2d_direct_kernel<T, K, K, TX, TY, R, G, MINB, true, HALFW, 0, CS, C>
                           : conv2d_direct_kernel<T, K, K, TX, TY, R, G, MINB, false, HALFW, 0, CS, C>;
    const size_t smem = HALFW ? Cfg::smem_half : Cfg::smem(sizeof(T));
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((w + Cfg::TW - 1) / Cfg::TW, (h + Cfg::TH - 1) / Cfg::TH, c);
    kern<<<grid, Cfg::NT, smem, s>>>(in, k, out, h, w, vec_ok, border);
    return cudaGetLastError();
}

// cs = 0: c planar channels of h x w pixels; cs > 0: one interleaved image of
// c = cs channels, w pixels per row.
template <typename T>
cudaError_t run_generic(int c, int h, int w, const T *in, int kh, int kw, const float *k, T *out,
                        int border, cudaStream_t s, int cs = 0) {
    dim3 grid((w + 31) / 32, (h + 7) / 8, c);
    conv2d_generic_kernel<T><<<grid, 256, 0, s>>>(in, k, out, h, w, kh, kw, border, cs);
    return cudaGetLastError();
}

template <typename T>
cudaError_t run_sep_generic(int c, int h, int w, const T *in, int kx, const float *gx, int ky, const float *gy,
                            T *out, int border, cudaStream_t s, int cs = 0) {
    const size_t smem = sizeof(float) * (size_t)(32 + ky - 1) * 32;
    dim3 grid((w + 31) / 32, (h + 31) / 32, c);
    conv2d_sep_generic_kernel<T><<<grid, 256, smem, s>>>(in, gx, gy, out, h, w, kx, ky, border, cs);
    return cudaGetLastError();
}

// CS > 1: w is the element width of one interleaved image (pixels * CS), c = 1.
// CR: columns per row-pass item (SepCfg).
template <typename T, int K, int TX, int TY, int R, int MINB = 1, bool INPLACE = false, int PAIR = 0, int CS = 1,
          bool HALFR = false, int CR = 4>
cudaError_t run_sep(int c, int h, int w, const T *in, const float *gx, const float *gy, T *out,
                    bool vec_ok, int border, cudaStream_t s) {
    using Cfg = SepCfg<K, K, TX, TY, R, INPLACE, CS, HALFR, CR>;
    using Kern = void (*)(const CUtensorMap, const T *, const float *, const float *, T *, int, int, bool, int);
    Kern kern;
    CUtensorMap tmap = {};
    static_assert(Cfg::SW <= 256 && Cfg::SH <= 256, "a TMA box side is at most 256 elements");
    if (vec_ok && (border == 0 || border == 1) && image_tensor_map<T>(&tmap, in, c, h, w, Cfg::SW, Cfg::SH)) {
        kern = conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, false, PAIR, 3, CS, HALFR, CR>;  // TMA staging
    } else if constexpr (K <= 5 && CS == 1) {  // as for the direct kernels
        kern = border != 0 ? conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, true, PAIR, 2, 1, HALFR, CR>
               : vec_ok    ? conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, false, PAIR, 1, 1, HALFR, CR>
                           : conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, false, PAIR, 2, 1, HALFR, CR>;
    } else {
        kern = border != 0 ? conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, true, PAIR, 0, CS, HALFR, CR>
                           : conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, false, PAIR, 0, CS, HALFR, CR>;
        if constexpr (CS == 1) {
            // planar rows that are not aligned (clamp border): the kernel
            // compiled for them, with the widest copies each row allows, except
            // FP32 rows not even 8-byte aligned from side 9 (3 x 4096 x 4094:
            // FP32 7x7 0.124 -> 0.092 ms, 15x15 0.142 -> 0.128, binary16 15x15
            // 0.124 -> 0.107; odd width 4095: FP32 7x7 0.122 -> 0.110 but 15x15
            // 0.141 -> 0.149, binary16 15x15 0.142 -> 0.132)
            const bool rows8 = w % 2 == 0 && (uintptr_t)in % 8 == 0 && (uintptr_t)out % 8 == 0;
            if (border == 0 && !vec_ok && (sizeof(T) == 2 || K == 7 || rows8))
                kern = conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, false, PAIR, 2, 1, HALFR, CR>;
        }
    }
    const size_t smem = Cfg::smem(sizeof(T));
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((w + Cfg::TW - 1) / Cfg::TW, (h + Cfg::TH - 1) / Cfg::TH, c);
    kern<<<grid, Cfg::NT, smem, s>>>(tmap, in, gx, gy, out, h, w, vec_ok, border);
    return cudaGetLastError();
}

// Packed pair arithmetic in the separable passes (bit 1: row pass, bit 2:
// column pass), where it measured faster on GB300 at 8192 x 8192 x 3.
template <typename T>
constexpr int sep_pair(int k) {
    if (sizeof(T) == 4) return k == 15 ? 2 : 0;
    return k == 5 || k == 9 ? 3 : (k >= 7 ? 2 : 0);
}

}  // namespace
}  // namespace pencil
