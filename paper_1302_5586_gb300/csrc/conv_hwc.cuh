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

// Element tiles of 32 rows x 128 elements, one 4-element group per thread
// (the tap window of a group is (kw-1)*CS + 4 elements wide).  Binary16
// images up to side 7 read their staged tile as binary16, as the planar
// kernels do.  Rows that are 16-byte aligned (clamp or zero border) load by
// TMA; every other case takes one cp.async kernel per side that handles all
// border modes.
template <typename T, int K, int TX, int TY, int R, int MINB, bool HW, int CS>
cudaError_t run_direct_hwc_k(int h, int we, const T *in, const float *k, T *out, bool vec_ok, int border,
                             cudaStream_t s) {
    using Cfg = DirectCfg<K, K, TX, TY, R, 1, CS>;
    cudaError_t err = cudaSuccess;
    if (try_direct_tma<T, K, TX, TY, R, 1, MINB, HW, CS>(1, h, we, in, k, out, vec_ok, border, s, &err)) return err;
    auto kern = conv2d_direct_kernel<T, K, K, TX, TY, R, 1, MINB, true, HW, 0, CS>;
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
    constexpr bool HW = sizeof(T) == 2;
    switch (K) {
        case 1: return run_direct_hwc_k<T, 1, 32, 8, 4, 8, HW, CS>(h, we, in, k, out, vec_ok, border, s);
        case 3: return run_direct_hwc_k<T, 3, 32, 8, 4, 8, HW, CS>(h, we, in, k, out, vec_ok, border, s);
        case 5: return run_direct_hwc_k<T, 5, 32, 8, 4, 6, HW, CS>(h, we, in, k, out, vec_ok, border, s);
        case 7: return run_direct_hwc_k<T, 7, 32, 8, 4, 4, HW, CS>(h, we, in, k, out, vec_ok, border, s);
        case 9: return run_direct_hwc_k<T, 9, 32, 8, 4, 2, false, CS>(h, we, in, k, out, vec_ok, border, s);
        case 11: return run_direct_hwc_k<T, 11, 32, 8, 4, 2, false, CS>(h, we, in, k, out, vec_ok, border, s);
        case 13: return run_direct_hwc_k<T, 13, 32, 8, 4, 2, false, CS>(h, we, in, k, out, vec_ok, border, s);
        case 15: return run_direct_hwc_k<T, 15, 32, 8, 4, 2, false, CS>(h, we, in, k, out, vec_ok, border, s);
        default: return cudaErrorInvalidValue;
    }
}

// Separable: the planar tiles, row-pass taps CS elements apart; TMA for
// aligned rows (clamp or zero border), one cp.async kernel otherwise.
template <typename T, int K, int TX, int TY, int R, int MINB, bool INPLACE, int CS>
cudaError_t run_sep_hwc_k(int h, int we, const T *in, const float *gx, const float *gy, T *out, bool vec_ok,
                          int border, cudaStream_t s) {
    using Cfg = SepCfg<K, K, TX, TY, R, INPLACE, CS>;
    using Kern = void (*)(const CUtensorMap, const T *, const float *, const float *, T *, int, int, bool, int);
    static_assert(Cfg::SW <= 256 && Cfg::SH <= 256, "a TMA box side is at most 256 elements");
    constexpr int PAIR = sep_pair<T>(K);
    CUtensorMap tmap = {};
    Kern kern = conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, true, PAIR, 0, CS>;
    if (vec_ok && (border == 0 || border == 1) && image_tensor_map<T>(&tmap, in, 1, h, we, Cfg::SW, Cfg::SH))
        kern = conv2d_sep_kernel<T, K, K, TX, TY, R, MINB, INPLACE, false, PAIR, 3, CS>;
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
    switch (K) {
        case 3: return run_sep_hwc_k<T, 3, 32, 8, 4, 1, false, CS>(h, we, in, gx, gy, out, vec_ok, border, s);
        case 5: return run_sep_hwc_k<T, 5, 32, 8, 4, 1, false, CS>(h, we, in, gx, gy, out, vec_ok, border, s);
        case 7: return run_sep_hwc_k<T, 7, 32, 8, 4, 1, false, CS>(h, we, in, gx, gy, out, vec_ok, border, s);
        case 9: return run_sep_hwc_k<T, 9, 16, 8, 8, 2, true, CS>(h, we, in, gx, gy, out, vec_ok, border, s);
        case 11: return run_sep_hwc_k<T, 11, 16, 8, 8, 2, true, CS>(h, we, in, gx, gy, out, vec_ok, border, s);
        case 13: return run_sep_hwc_k<T, 13, 16, 8, 8, 2, true, CS>(h, we, in, gx, gy, out, vec_ok, border, s);
        case 15: return run_sep_hwc_k<T, 15, 16, 8, 16, 2, true, CS>(h, we, in, gx, gy, out, vec_ok, border, s);
        default: return cudaErrorInvalidValue;
    }
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
