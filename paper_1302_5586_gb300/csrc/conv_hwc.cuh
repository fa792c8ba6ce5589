// conv_hwc.cuh -- tiled conv2d kernels for interleaved [h][w][c] images of
// c = 3 or 4 channels (the pixel layout image DSLs hand over, Sec. 1):
// channel ch of pixel (i, j) is element (i*w + j)*c + ch, and every channel
// is correlated with the same filter on its own.
//
// The image is treated as ONE plane of h rows of w*c elements: an output
// element depends on the elements kw/2*c to either side of it in steps of c
// (the same channel of the neighbouring pixels), so the planar tile body runs
// unchanged on element columns with its taps c elements apart (DirectCfg's
// CS).  Tiles, TMA boxes and stores cover consecutive elements, so loads and
// stores stay as wide and coalesced as for a planar image; the clamp acts on
// pixels (an element outside the image takes the same channel of the nearest
// edge pixel).  Per element the FP32 operation order is the planar one, so
// each channel's result is the same bits as the planar kernels give for that
// channel alone.  One translation unit per (storage type, channel count)
// instantiates these, so they compile in parallel.
#pragma once

#include "conv_kernels.cuh"

namespace pencil {
namespace {

using namespace tile;

// Element tiles of TY*R rows x TX*C elements, C consecutive elements per
// thread: C = 12 (three 16-byte chunks) for sides from 5 up, so one tap
// window of (kw-1)*CS + C elements feeds 12 outputs instead of 4 -- with taps
// CS elements apart, a 4-element group re-reads most of its window from
// shared memory for every 4 outputs, and that traffic, not the FMAs, bounded
// the 4-wide tiles.  Binary16 images up to side 7 read their staged tile as
// binary16, as the planar kernels do.  Rows that are 16-byte aligned (clamp or
// zero border) load by TMA; every other case takes one cp.async kernel per
// side that handles all border modes.
template <typename T, int K, int TX, int TY, int R, int MINB, bool HW, int CS, int C = 4>
cudaError_t run_direct_hwc_k(int h, int we, const T *in, const float *k, T *out, bool vec_ok, int border,
                             cudaStream_t s) {
    using Cfg = DirectCfg<K, K, TX, TY, R, 1, CS, C>;
    cudaError_t err = cudaSuccess;
    if (try_direct_tma<T, K, TX, TY, R, 1, MINB, HW, CS, C>(1, h, we, in, k, out, vec_ok, border, s, &err))
        return err;
    auto kern = conv2d_direct_kernel<T, K, K, TX, TY, R, 1, MINB, true, HW, 0, CS, C>;
    const size_t smem = HW ? Cfg::smem_half : Cfg::smem(sizeof(T));
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((we + Cfg::TW - 1) / Cfg::TW, (h + Cfg::TH - 1) / Cfg::TH, 1);
    kern<<<grid, Cfg::NT, smem, s>>>(in, k, out, h, we, vec_ok, border);
    return cudaGetLastError();
}

template <typename T, int CS>
cudaError_t run_direct_hwc(int K, int h, int we, const T *in, const float *k, T *out, bool vec_ok, int border,
                           cudaStream_t s) {
    constexpr bool F16 = sizeof(T) == 2;
#define PENCIL_HWC_RUN(K_, TX, TY, R, MINB, HW, C) \
    return run_direct_hwc_k<T, K_, TX, TY, R, MINB, HW, CS, C>(h, we, in, k, out, vec_ok, border, s)
    switch (K) {
        case 1: PENCIL_HWC_RUN(1, 32, 8, 4, 8, F16, 4);
        case 3:
            if constexpr (F16) PENCIL_HWC_RUN(3, 16, 8, 2, 8, true, 12);
            else PENCIL_HWC_RUN(3, 32, 8, 4, 8, false, 4);
        case 5:
            if constexpr (F16) PENCIL_HWC_RUN(5, 16, 8, 4, 4, true, 12);
            else PENCIL_HWC_RUN(5, 16, 8, 2, 6, false, 12);
        case 7:
            if constexpr (F16) PENCIL_HWC_RUN(7, 16, 8, 4, 3, true, 12);
            else PENCIL_HWC_RUN(7, 16, 8, 2, CS == 3 ? 6 : 5, false, 12);
        case 9: PENCIL_HWC_RUN(9, 16, 8, 2, 3, false, 12);
        case 11: PENCIL_HWC_RUN(11, 16, 8, 2, 3, false, 12);
        case 13: PENCIL_HWC_RUN(13, 16, 8, 2, 3, false, 12);
        case 15:
            if constexpr (F16) PENCIL_HWC_RUN(15, 16, 16, 2, 2, false, 12);
            else PENCIL_HWC_RUN(15, 16, 8, 2, 4, false, 12);
        default: return cudaErrorInvalidValue;
    }
#undef PENCIL_HWC_RUN
}

// Separable: the planar tiles, row-pass taps CS elements apart, row-pass
// items of 12 elements (three chunks share one tap window; the column pass
// keeps 4-column items); TMA for aligned rows (clamp or zero border), one
// cp.async kernel otherwise.
template <typename T, int K, int TX, int TY, int R, int MINB, bool INPLACE, int CS, int CR = 4>
cudaError_t run_sep_hwc_k(int h, int we, const T *in, const float *gx, const float *gy, T *out, bool vec_ok,
                          int border, cudaStream_t s) {
    using Cfg = SepCfg<K, K, TX, TY, R, INPLACE, CS, false, CR>;
    using Kern = void (*)(const CUtensorMap, const T *, const float *, const float *, T *, int, int, bool, int);
    static_assert(Cfg::SW <= 256 && Cfg::SH <= 256, "a TMA box side is at most 256 elements");
    constexpr int PAIR = sep_pair<T>(K);
    CUtensorMap tmap = {};
    Kern kern = conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, true, PAIR, 0, CS, false, CR>;
    if (vec_ok && (border == 0 || border == 1) && image_tensor_map<T>(&tmap, in, 1, h, we, Cfg::SW, Cfg::SH))
        kern = conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, false, PAIR, 3, CS, false, CR>;
    const size_t smem = Cfg::smem(sizeof(T));
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((we + Cfg::TW - 1) / Cfg::TW, (h + Cfg::TH - 1) / Cfg::TH, 1);
    kern<<<grid, Cfg::NT, smem, s>>>(tmap, in, gx, gy, out, h, we, vec_ok, border);
    return cudaGetLastError();
}

template <typename T, int CS>
cudaError_t run_sep_hwc(int K, int h, int we, const T *in, const float *gx, const float *gy, T *out, bool vec_ok,
                        int border, cudaStream_t s) {
#define PENCIL_HWC_SEP(K_, TX, TY, R, MINB, IP) \
    return run_sep_hwc_k<T, K_, TX, TY, R, MINB, IP, CS, 12>(h, we, in, gx, gy, out, vec_ok, border, s)
    switch (K) {
        case 3: PENCIL_HWC_SEP(3, 48, 4, 4, 2, false);
        case 5: PENCIL_HWC_SEP(5, 24, 8, 4, 2, false);
        case 7: PENCIL_HWC_SEP(7, 24, 8, 4, 2, false);
        case 9: PENCIL_HWC_SEP(9, 24, 8, 8, 2, true);
        case 11: PENCIL_HWC_SEP(11, 24, 8, 8, 2, true);
        case 13: PENCIL_HWC_SEP(13, 24, 8, 8, 2, true);
        case 15:
            if constexpr (sizeof(T) == 2) PENCIL_HWC_SEP(15, 24, 8, 8, 2, true);
            else PENCIL_HWC_SEP(15, 24, 8, 16, 1, true);
        default: return cudaErrorInvalidValue;
    }
#undef PENCIL_HWC_SEP
}

}  // namespace
}  // namespace pencil

// The entry points of one (storage type, channel count) unit:
//   hwc_direct_<NAME>(K, h, we, in, k, out, vec_ok, border, s)
//   hwc_sep_<NAME>(K, h, we, in, gx, gy, out, vec_ok, border, s)
//   wait_timeouts_<NAME>(n, clear)  -- this unit's wait-timeout counter
#define PENCIL_HWC_UNIT(T, CS, NAME)                                                                          \
    namespace pencil {                                                                                        \
    cudaError_t hwc_direct_##NAME(int K, int h, int we, const void *in, const float *k, void *out,            \
                                  bool vec_ok, int border, cudaStream_t s) {                                  \
        return run_direct_hwc<T, CS>(K, h, we, static_cast<const T *>(in), k, static_cast<T *>(out), vec_ok, \
                                     border, s);                                                              \
    }                                                                                                         \
    cudaError_t hwc_sep_##NAME(int K, int h, int we, const void *in, const float *gx, const float *gy,        \
                               void *out, bool vec_ok, int border, cudaStream_t s) {                          \
        return run_sep_hwc<T, CS>(K, h, we, static_cast<const T *>(in), gx, gy, static_cast<T *>(out), vec_ok, \
                                  border, s);                                                                 \
    }                                                                                                         \
    cudaError_t wait_timeouts_##NAME(unsigned *n, bool clear) { return read_wait_counter(n, clear); }        \
    }
