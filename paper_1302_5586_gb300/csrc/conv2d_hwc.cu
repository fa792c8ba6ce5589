// conv2d_hwc.cu -- dispatch of conv2d on interleaved [h][w][c] images (c > 1):
// 3 and 4 channels with square odd filters up to 15 run the tiled kernels of
// conv_hwc.cuh (one translation unit per channel count and storage type),
// everything else the generic kernels with strided addressing.  Channel ch of
// pixel (i, j) is element (i*w + j)*c + ch.
#include "internal.cuh"

namespace pencil {
namespace {

bool rows_aligned(const void *p, long long we, int vec) { return (we % vec == 0) && ((uintptr_t)p % 16 == 0); }

}  // namespace

cudaError_t launch_conv2d_hwc(int dtype, int c, int h, int w, const void *in, int kh, int kw, const float *k,
                              void *out, cudaStream_t s, int border) {
    const bool special = (kh == kw) && (kh % 2 == 1) && kh <= PENCIL_MAX_SPECIALISED_K && (c == 3 || c == 4);
    if (!special) return launch_conv2d_generic(dtype, c, h, w, in, kh, kw, k, out, s, border, c);
    const int we = w * c, vec = dtype == PENCIL_F16 ? 8 : 4;
    const bool v = rows_aligned(in, we, vec) && rows_aligned(out, we, vec);
    if (dtype == PENCIL_F32)
        return c == 3 ? hwc_direct_hwc3_f32(kh, h, we, in, k, out, v, border, s)
                      : hwc_direct_hwc4_f32(kh, h, we, in, k, out, v, border, s);
    return c == 3 ? hwc_direct_hwc3_f16(kh, h, we, in, k, out, v, border, s)
                  : hwc_direct_hwc4_f16(kh, h, we, in, k, out, v, border, s);
}

cudaError_t launch_conv2d_hwc_generic(int dtype, int c, int h, int w, const void *in, int kh, int kw,
                                      const float *k, void *out, cudaStream_t s, int border) {
    return launch_conv2d_generic(dtype, c, h, w, in, kh, kw, k, out, s, border, c);
}

cudaError_t launch_conv2d_sep_hwc(int dtype, int c, int h, int w, const void *in, int kx, const float *gx, int ky,
                                  const float *gy, void *out, cudaStream_t s, int border) {
    const bool special = kx == ky && (kx & 1) && kx >= 3 && kx <= PENCIL_MAX_SPECIALISED_K && (c == 3 || c == 4);
    if (!special) return launch_conv2d_sep_generic(dtype, c, h, w, in, kx, gx, ky, gy, out, s, border, c);
    const int we = w * c, vec = dtype == PENCIL_F16 ? 8 : 4;
    const bool v = rows_aligned(in, we, vec) && rows_aligned(out, we, vec);
    if (dtype == PENCIL_F32)
        return c == 3 ? hwc_sep_hwc3_f32(kx, h, we, in, gx, gy, out, v, border, s)
                      : hwc_sep_hwc4_f32(kx, h, we, in, gx, gy, out, v, border, s);
    return c == 3 ? hwc_sep_hwc3_f16(kx, h, we, in, gx, gy, out, v, border, s)
                  : hwc_sep_hwc4_f16(kx, h, we, in, gx, gy, out, v, border, s);
}

cudaError_t wait_timeouts_hwc(unsigned *n, bool clear) {
    unsigned total = 0;
    cudaError_t (*const units[4])(unsigned *, bool) = {wait_timeouts_hwc3_f32, wait_timeouts_hwc3_f16,
                                                       wait_timeouts_hwc4_f32, wait_timeouts_hwc4_f16};
    for (auto f : units) {
        unsigned m = 0;
        const cudaError_t e = f(&m, clear);
        if (e != cudaSuccess) return e;
        total += m;
    }
    *n = total;
    return cudaSuccess;
}

}  // namespace pencil
