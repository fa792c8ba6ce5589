// chain.cu -- two clamp-to-edge correlations in one pass over HBM:
// out = conv(conv(in, k1), k2), the intermediate y = conv(in, k1) kept in
// shared memory (the cross-kernel fusion of dependent stencils, Sec. 2.2.3).
//
// Bits: every value is what two separate conv2d calls give.  The intermediate
// is rounded to the storage type exactly as the first call would store it
// (FP32, or binary16 round-to-nearest-even), and the second stencil reads it at
// clamped positions: y at a row or column outside the image is y at the
// nearest edge -- not a value computed from further-out input.  Each output
// pixel and each intermediate value accumulate in the documented order (per
// filter row a, s = k[a][0]*x0 then fmas over b, acc = acc + s from +0).
//
// Specialised kernel (square odd k1, k2 in {3, 5, 7}), one CTA per
// 32 x 128 output tile, 256 threads:
//   1. stage the input rows and columns the tile's intermediate region needs:
//      FP32 images with 16-byte aligned rows as one TMA box (the clamp
//      rebuilt in shared memory on edge tiles, as the direct TMA kernel does),
//      others clamped with cp.async;
//   2. compute the intermediate region (32 + k2 - 1 rows, 128 + k2 - 1
//      columns) into shared memory: up to 7 warps each own a band of R1 rows,
//      one lane per 4 columns, and the last warp takes the columns beyond 128;
//   3. on tiles that touch the image border, copy the edge rows and columns
//      of the intermediate outward (the clamp of the second stencil);
//   4. the second stencil from shared memory with the direct kernel's
//      register blocking (4 rows x 4 columns per thread), stored to HBM.
// Any other pair of sizes takes a generic fused kernel (runtime sizes; the
// intermediate computed at clamped positions from global memory).
#include "conv_kernels.cuh"

#ifndef PENCIL_CHAIN_MINB
#define PENCIL_CHAIN_MINB 4  // CTAs per SM the register budget is sized for
#endif

namespace pencil {
namespace {

using namespace tile;

template <int K1, int K2>
struct ChainCfg {
    static constexpr int TX = 32, TY = 8, R = 4, G = 1;
    using Out = DirectCfg<K2, K2, TX, TY, R, G>;
    static constexpr int NT = Out::NT, TW = Out::TW, TH = Out::TH;
    static constexpr int A1 = K1 / 2, A2 = K2 / 2;
    static constexpr int P1 = round_up(A1, 8), P2 = Out::P;
    static constexpr int SWY = Out::SW;      // intermediate row stride; column 0 = x0 - P2
    static constexpr int YH = Out::SH;       // intermediate rows; row 0 = y0 - A2
    static constexpr int YC0 = P2 - A2;      // first intermediate column the second stencil reads
    static constexpr int NYC = TW + K2 - 1;  // intermediate columns it reads
    static constexpr int LO = YC0 & ~3, HI = round_up(YC0 + NYC, 4);
    static constexpr int NBX = (HI - LO) / 4;  // 4-column blocks of the intermediate
    // row bands of R1 rows, one warp each, at most NT/32 - 1 of them (the last
    // warp takes the columns beyond 32 blocks): of the two smallest band
    // heights, the one that computes fewer rows beyond YH
    static constexpr int RMIN = (YH + NT / 32 - 2) / (NT / 32 - 1);
    static constexpr int R1 = ((YH + RMIN - 1) / RMIN) * RMIN <= ((YH + RMIN) / (RMIN + 1)) * (RMIN + 1)
                                  ? RMIN
                                  : RMIN + 1;
    static constexpr int RG = (YH + R1 - 1) / R1;  // bands
    static constexpr int EXTRA = NBX - 32;     // blocks per band left to the last warp
    static constexpr int KWP1 = round_up(K1, 4), KWP2 = round_up(K2, 4);
    static constexpr int NX1 = round_up(P1 - A1 + 4 + K1 - 1, 4);
    static constexpr int XH = RG * R1 + K1 - 1;              // staged input rows; row 0 = y0 - A2 - A1
    static constexpr int SWX = round_up(HI - 4 + NX1, 8);    // column 0 = x0 - P2 - P1
    // shared memory (floats): staged input, intermediate, filters, binary16 staging
    static constexpr int OFF_Y = XH * SWX, OFF_K1 = OFF_Y + YH * SWY, OFF_K2 = OFF_K1 + K1 * KWP1,
                         OFF_16 = OFF_K2 + K2 * KWP2;
    static constexpr size_t smem(size_t esz) {
        return sizeof(float) * (size_t)OFF_16 + (esz == 2 ? 2 * (size_t)XH * SWX : 0);
    }
    static_assert(EXTRA >= 0 && RG * EXTRA <= 32 && RG <= NT / 32 - 1, "intermediate does not fit the warp layout");
    static_assert(HI <= SWY, "intermediate block beyond its row");
    static_assert(OFF_Y % 4 == 0 && OFF_K1 % 4 == 0 && OFF_K2 % 4 == 0 && OFF_16 % 4 == 0 && (XH * SWX) % 8 == 0,
                  "alignment");
    static_assert(XH <= 256 && SWX <= 256, "a TMA box side is at most 256 elements");
};

template <typename T>
__device__ __forceinline__ float storage_round(float v) {
    if constexpr (sizeof(T) == 2)
        return __half2float(__float2half_rn(v));
    else
        return v;
}

// TMA: the input region arrives as one box of `tmap` (FP32 images whose rows
// are 16-byte aligned); otherwise it is staged with cp.async from `in`.
template <typename T, int K1, int K2, int MINB, bool TMA>
__global__ void __launch_bounds__(256, MINB)
    conv2d_chain_kernel(const __grid_constant__ CUtensorMap tmap, const T *__restrict__ in,
                        const float *__restrict__ k1, const float *__restrict__ k2, T *__restrict__ out, int h,
                        int w, bool vec_ok) {
    using Cfg = ChainCfg<K1, K2>;
    constexpr int NT = Cfg::NT, SWX = Cfg::SWX, SWY = Cfg::SWY, YH = Cfg::YH, R1 = Cfg::R1;
    extern __shared__ __align__(128) float smem[];
    float *s_x = smem;
    float *s_y = smem + Cfg::OFF_Y;
    float *s_k1 = smem + Cfg::OFF_K1;
    float *s_k2 = smem + Cfg::OFF_K2;
    T *s16 = reinterpret_cast<T *>(smem + Cfg::OFF_16);

    const size_t plane = (size_t)h * (size_t)w * blockIdx.z;
    const int y0 = blockIdx.y * Cfg::TH, x0 = blockIdx.x * Cfg::TW;
    const int yr0 = y0 - Cfg::A2, yc0 = x0 - Cfg::P2;  // global position of s_y[0][0]

    // 1. filters and the input region (clamped)
    if constexpr (TMA) {
        static_assert(sizeof(T) == 4, "the TMA path stages FP32 images");
        __shared__ __align__(8) uint64_t bar;
        if ((tma::smem_addr(s_x) & 127u) != 0) {  // a TMA box needs a 128-byte aligned destination
            if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);
            return;
        }
        if (threadIdx.x == 0) tma::mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            tma::mbar_arrive_expect_tx(&bar, (unsigned)(sizeof(float) * Cfg::XH * SWX));
            tma::load_3d(s_x, &tmap, yc0 - Cfg::P1, yr0 - Cfg::A1, (int)blockIdx.z, &bar);
        }
        stage_filter<K1, K1, Cfg::KWP1, NT>(k1, s_k1);
        stage_filter<K2, K2, Cfg::KWP2, NT>(k2, s_k2);
        if (!__syncthreads_and(tma::mbar_wait(&bar, 0, tma::kLoadWaitNs))) {
            if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);  // skip the tile; let the copy land
            tma::mbar_wait(&bar, 0, tma::kLoadWaitNs);
            return;
        }
        clamp_fixup<float, Cfg::XH, SWX, NT>(s_x, h, w, yr0 - Cfg::A1, yc0 - Cfg::P1);
    } else {
        stage_filter_async<K1, K1, Cfg::KWP1, NT>(k1, s_k1);
        stage_filter_async<K2, K2, Cfg::KWP2, NT>(k2, s_k2);
        stage_issue<T, Cfg::XH, SWX, NT, false, false>(in + plane, h, w, yr0 - Cfg::A1, yc0 - Cfg::P1, vec_ok, s_x,
                                                     s16);
        stage_finish<T, Cfg::XH, SWX, NT>(s_x, s16);
    }

    // 2. the intermediate region
    {
        constexpr int EX = Cfg::EXTRA > 0 ? Cfg::EXTRA : 1;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        int band = warp, bx = lane;
        bool active = true;
        if (warp >= Cfg::RG) {  // the last warp: the columns beyond the first 32 blocks of every band
            active = warp == NT / 32 - 1 && Cfg::EXTRA > 0 && lane < Cfg::RG * Cfg::EXTRA;
            band = lane / EX;
            bx = 32 + lane % EX;
        }
        if (active) {
            const int c = Cfg::LO + 4 * bx;
            float acc[R1][4];
            direct_accumulate<K1, K1, R1, 1, 4, SWX, Cfg::KWP1, Cfg::P1 - Cfg::A1>(s_x + (band * R1) * SWX + c,
                                                                                   s_k1, acc);
#pragma unroll
            for (int o = 0; o < R1; ++o) {
                const int r = band * R1 + o;
                if (r < YH)
                    *reinterpret_cast<float4 *>(s_y + r * SWY + c) =
                        make_float4(storage_round<T>(acc[o][0]), storage_round<T>(acc[o][1]),
                                    storage_round<T>(acc[o][2]), storage_round<T>(acc[o][3]));
            }
        }
    }
    __syncthreads();

    // 3. the clamp of the second stencil: positions outside the image take the
    // intermediate value at the nearest edge (rows first, then columns)
    constexpr int NC = Cfg::NYC;
    if (yr0 < 0 || yr0 + YH > h) {
        for (int idx = threadIdx.x; idx < YH * NC; idx += NT) {
            const int r = idx / NC, c = Cfg::YC0 + (idx - r * NC);
            const int gr = yr0 + r;
            if (gr < 0 || gr >= h) s_y[r * SWY + c] = s_y[(clampi(gr, 0, h - 1) - yr0) * SWY + c];
        }
        __syncthreads();
    }
    if (yc0 + Cfg::YC0 < 0 || yc0 + Cfg::YC0 + NC > w) {
        for (int idx = threadIdx.x; idx < YH * NC; idx += NT) {
            const int r = idx / NC, c = Cfg::YC0 + (idx - r * NC);
            const int gc = yc0 + c;
            if (gc < 0 || gc >= w) s_y[r * SWY + c] = s_y[r * SWY + (clampi(gc, 0, w - 1) - yc0)];
        }
        __syncthreads();
    }

    // 4. the second stencil
    direct_compute<T, K2, K2, Cfg::TX, Cfg::TY, Cfg::R, Cfg::G, float, false>(s_y, s_k2, out + plane, h, w, vec_ok,
                                                                              y0, x0);
}

// Generic fused chain: any sizes.  A 256-thread CTA owns a 16 x 32 output
// tile; the intermediate region (16 + kh2 - 1) x (32 + kw2 - 1) is computed at
// clamped positions straight from global memory into shared memory, then
// every thread computes two outputs from it.
constexpr int GTW = 32, GTH = 16;

template <typename T>
__global__ void __launch_bounds__(256)
    conv2d_chain_generic_kernel(const T *__restrict__ in, const float *__restrict__ k1, int kh1, int kw1,
                                const float *__restrict__ k2, int kh2, int kw2, T *__restrict__ out,
                                int h, int w) {
    extern __shared__ __align__(16) float s_y[];
    const int yh = GTH + kh2 - 1, yw = GTW + kw2 - 1;
    const int a1h = kh1 / 2, a1w = kw1 / 2, a2h = kh2 / 2, a2w = kw2 / 2;
    const size_t plane = (size_t)h * (size_t)w * blockIdx.z;
    const T *src = in + plane;
    const int y0 = blockIdx.y * GTH, x0 = blockIdx.x * GTW;
    for (int idx = threadIdx.x; idx < yh * yw; idx += blockDim.x) {
        const int r = idx / yw, c = idx - r * yw;
        const int i = clampi(y0 - a2h + r, 0, h - 1), j = clampi(x0 - a2w + c, 0, w - 1);
        float acc = 0.0f;
        for (int a = 0; a < kh1; ++a) {
            const T *row = src + (size_t)clampi(i + a - a1h, 0, h - 1) * (size_t)w;
            const float *kr = k1 + (size_t)a * kw1;
            float s = __fmul_rn(__ldg(kr), Io<T>::ld(row + clampi(j - a1w, 0, w - 1)));
            for (int b = 1; b < kw1; ++b)
                s = __fmaf_rn(__ldg(kr + b), Io<T>::ld(row + clampi(j + b - a1w, 0, w - 1)), s);
            acc = __fadd_rn(acc, s);
        }
        s_y[idx] = storage_round<T>(acc);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < GTH * GTW; o += blockDim.x) {
        const int r = o / GTW, c = o - r * GTW;
        const int i = y0 + r, j = x0 + c;
        if (i >= h || j >= w) continue;
        float acc = 0.0f;
        for (int a = 0; a < kh2; ++a) {
            const float *yr = s_y + (r + a) * yw + c;
            const float *kr = k2 + (size_t)a * kw2;
            float s = __fmul_rn(__ldg(kr), yr[0]);
            for (int b = 1; b < kw2; ++b) s = __fmaf_rn(__ldg(kr + b), yr[b], s);
            acc = __fadd_rn(acc, s);
        }
        Io<T>::st(out + plane + (size_t)i * w + j, acc);
    }
}

template <typename T, int K1, int K2>
cudaError_t run_chain(int c, int h, int w, const T *in, const float *k1, const float *k2, T *out,
                      bool vec_ok, cudaStream_t s) {
    using Cfg = ChainCfg<K1, K2>;
    // a 7-tap first filter needs more than 64 registers a thread
    constexpr int MINB = K1 >= 7 ? PENCIL_CHAIN_MINB - 1 : PENCIL_CHAIN_MINB;
    CUtensorMap tmap = {};
    auto kern = conv2d_chain_kernel<T, K1, K2, MINB, false>;
    if constexpr (sizeof(T) == 4) {
        if (vec_ok && image_tensor_map<T>(&tmap, in, c, h, w, Cfg::SWX, Cfg::XH))
            kern = conv2d_chain_kernel<T, K1, K2, MINB, true>;
    }
    const size_t smem = Cfg::smem(sizeof(T));
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((w + Cfg::TW - 1) / Cfg::TW, (h + Cfg::TH - 1) / Cfg::TH, c);
    kern<<<grid, Cfg::NT, smem, s>>>(tmap, in, k1, k2, out, h, w, vec_ok);
    return cudaGetLastError();
}

template <typename T, int K1>
cudaError_t run_chain_k2(int k2s, int c, int h, int w, const T *in, const float *k1, const float *k2,
                         T *out, bool vec_ok, cudaStream_t s) {
    switch (k2s) {
        case 3: return run_chain<T, K1, 3>(c, h, w, in, k1, k2, out, vec_ok, s);
        case 5: return run_chain<T, K1, 5>(c, h, w, in, k1, k2, out, vec_ok, s);
        case 7: return run_chain<T, K1, 7>(c, h, w, in, k1, k2, out, vec_ok, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t run_chain_any(int c, int h, int w, const T *in, int kh1, int kw1, const float *k1, int kh2,
                          int kw2, const float *k2, T *out, bool vec_ok, bool generic, cudaStream_t s) {
    auto spec = [](int a, int b) { return a == b && (a == 3 || a == 5 || a == 7); };
    if (!generic && spec(kh1, kw1) && spec(kh2, kw2)) {
        switch (kh1) {
            case 3: return run_chain_k2<T, 3>(kh2, c, h, w, in, k1, k2, out, vec_ok, s);
            case 5: return run_chain_k2<T, 5>(kh2, c, h, w, in, k1, k2, out, vec_ok, s);
            case 7: return run_chain_k2<T, 7>(kh2, c, h, w, in, k1, k2, out, vec_ok, s);
        }
    }
    const size_t smem = sizeof(float) * (size_t)(GTH + kh2 - 1) * (GTW + kw2 - 1);
    cudaError_t e = set_smem(conv2d_chain_generic_kernel<T>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((w + GTW - 1) / GTW, (h + GTH - 1) / GTH, c);
    conv2d_chain_generic_kernel<T><<<grid, 256, smem, s>>>(in, k1, kh1, kw1, k2, kh2, kw2, out, h, w);
    return cudaGetLastError();
}

bool rows_aligned(const void *p, int w, int vec) { return (w % vec == 0) && ((uintptr_t)p % 16 == 0); }

}  // namespace

size_t chain_generic_smem(int kh2, int kw2) {
    return sizeof(float) * (size_t)(GTH + kh2 - 1) * (size_t)(GTW + kw2 - 1);
}

cudaError_t wait_timeouts_chain(unsigned *n, bool clear) { return read_wait_counter(n, clear); }

cudaError_t launch_conv2d_chain(int dtype, int c, int h, int w, const void *in, int kh1, int kw1,
                                const float *k1, int kh2, int kw2, const float *k2, void *out,
                                bool generic, cudaStream_t s) {
    if (dtype == PENCIL_F32) {
        const bool v = rows_aligned(in, w, 4) && rows_aligned(out, w, 4);
        return run_chain_any<float>(c, h, w, static_cast<const float *>(in), kh1, kw1, k1, kh2, kw2, k2,
                                    static_cast<float *>(out), v, generic, s);
    }
    const bool v = rows_aligned(in, w, 8) && rows_aligned(out, w, 8);
    return run_chain_any<__half>(c, h, w, static_cast<const __half *>(in), kh1, kw1, k1, kh2, kw2, k2,
                                 static_cast<__half *>(out), v, generic, s);
}

}  // namespace pencil
