// internal.cuh -- declarations shared by the library's translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "pencil.h"

namespace pencil {

// Record `e` as the calling thread's last CUDA error and return PENCIL_ERR_CUDA.
int cuda_fail(cudaError_t e);

#define PENCIL_CUDA_TRY(expr)                                      \
    do {                                                           \
        cudaError_t _pe = (expr);                                  \
        if (_pe != cudaSuccess) return ::pencil::cuda_fail(_pe);   \
    } while (0)

// Round x up to a multiple of a (a > 0).
__host__ __device__ constexpr int round_up(int x, int a) { return (x + a - 1) / a * a; }

// ------------------------------------------------------- async copies
// 16-byte global -> shared copy that bypasses registers and L1
// (cp.async.cg); both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
// 8-byte global -> shared copy (cp.async.ca); both addresses 8-byte aligned.
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
// 4-byte global -> shared copy (cp.async.ca); both addresses 4-byte aligned.
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Wait until at most one committed group of this thread is still in flight.
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ----------------------------------------------------------------- conv2d
// All launchers queue work on `s` and return the launch status.
// Arrays are device memory; the host layer has validated sizes and pointers.
// border: 0 clamp-to-edge, 1 zero, 2 reflect, 3 mirror, 4 wrap.
cudaError_t launch_conv2d(int dtype, int c, int h, int w, const void *in, int kh, int kw,
                          const float *k, void *out, cudaStream_t s, int border = 0);
// Binary16 on the tensor cores (conv_tc.cu): queued only where it applies
// (odd square side 7..15, rows and pointers 16-byte aligned, clamp or zero
// border); *done says whether it was.
cudaError_t launch_conv2d_tc(int c, int h, int w, const void *in, int ks, const float *k, void *out, int border,
                             cudaStream_t s, bool *done);
cudaError_t wait_timeouts_tc(unsigned *n, bool clear);
// Force the generic (any-size) kernel; used by tests of the fixed-order rule.
// cs = 0: c planar channels; cs = c > 1: one interleaved [h][w][c] image.
cudaError_t launch_conv2d_generic(int dtype, int c, int h, int w, const void *in, int kh, int kw,
                                  const float *k, void *out, cudaStream_t s, int border = 0, int cs = 0);
cudaError_t launch_conv2d_sep_generic(int dtype, int c, int h, int w, const void *in, int kx, const float *gx,
                                      int ky, const float *gy, void *out, cudaStream_t s, int border = 0,
                                      int cs = 0);
cudaError_t launch_conv2d_sep(int dtype, int c, int h, int w, const void *in, int kx,
                              const float *gx, int ky, const float *gy, void *out,
                              cudaStream_t s, int border = 0);

// Interleaved [h][w][c] images (c > 1): the same operations per channel.
cudaError_t launch_conv2d_hwc(int dtype, int c, int h, int w, const void *in, int kh, int kw,
                              const float *k, void *out, cudaStream_t s, int border = 0);
cudaError_t launch_conv2d_hwc_generic(int dtype, int c, int h, int w, const void *in, int kh, int kw,
                                      const float *k, void *out, cudaStream_t s, int border = 0);
cudaError_t launch_conv2d_sep_hwc(int dtype, int c, int h, int w, const void *in, int kx,
                                  const float *gx, int ky, const float *gy, void *out,
                                  cudaStream_t s, int border = 0);

// The tiled interleaved kernels, one translation unit per (channels, dtype);
// we = w * channels elements per row.
#define PENCIL_HWC_DECL(NAME)                                                                           \
    cudaError_t hwc_direct_##NAME(int K, int h, int we, const void *in, const float *k, void *out,      \
                                  bool vec_ok, int border, cudaStream_t s);                             \
    cudaError_t hwc_sep_##NAME(int K, int h, int we, const void *in, const float *gx, const float *gy,  \
                               void *out, bool vec_ok, int border, cudaStream_t s);                     \
    cudaError_t wait_timeouts_##NAME(unsigned *n, bool clear);
PENCIL_HWC_DECL(hwc3_f32)
PENCIL_HWC_DECL(hwc3_f16)
PENCIL_HWC_DECL(hwc4_f32)
PENCIL_HWC_DECL(hwc4_f16)
#undef PENCIL_HWC_DECL

// Tile loads whose bounded wait ran out since the last clear (each skipped its
// tile); clear resets the count.  Each translation unit of kernels keeps its
// own counter: wait_timeouts reads the planar unit's, wait_timeouts_hwc the sum
// of the interleaved units'.
cudaError_t wait_timeouts(unsigned *n, bool clear);
cudaError_t wait_timeouts_hwc(unsigned *n, bool clear);
cudaError_t wait_timeouts_chain(unsigned *n, bool clear);
// Run the bounded mbarrier wait against a barrier that never completes, for
// limit_ns; *completed = 1 if it completed (it should not), 0 if it ran out.
cudaError_t wait_selftest(uint64_t limit_ns, int *completed);

// out = conv(conv(in, k1), k2) in one kernel, clamp-to-edge, the intermediate
// rounded to the storage type; generic forces the runtime-size kernel.
cudaError_t launch_conv2d_chain(int dtype, int c, int h, int w, const void *in, int kh1, int kw1,
                                const float *k1, int kh2, int kw2, const float *k2, void *out,
                                bool generic, cudaStream_t s);
// Shared memory the generic chain kernel needs for a second filter of kh2 x kw2.
size_t chain_generic_smem(int kh2, int kw2);

// conv -> Jacobi fused (conv_jacobi.cu): square odd filters up to
// kConvJacobiMaxK, rows of w % 4 == 0 floats, 16-byte aligned buffers, at most
// kConvJacobiMaxSweeps sweeps per launch.
constexpr int kConvJacobiMaxK = 7;
constexpr int kConvJacobiMaxSweeps = 10;
bool conv_jacobi_fusable(int h, int w, int kh, int kw, const void *in, const void *out);
cudaError_t launch_conv_jacobi_fused(int c, int h, int w, const float *in, int ks, const float *k, int n,
                                     float *out, cudaStream_t s);
cudaError_t wait_timeouts_cj(unsigned *n, bool clear);

// ----------------------------------------------------------------- jacobi
size_t jacobi_workspace_bytes(int h, int w);
cudaError_t jacobi_run(int h, int w, float *u, int iters, int check_every, double *res,
                       void *ws, size_t ws_bytes, int temporal_t, cudaStream_t s);
cudaError_t residual_run(int h, int w, const float *u, double *res, void *ws, cudaStream_t s);
// Sweeps in chunks of check_every until the chunk's residual <= tol or
// max_iters; *done = sweeps performed (the stream is synchronised per chunk).
cudaError_t jacobi_until(int h, int w, float *u, int max_iters, int check_every, double tol,
                         double *res, int *done, void *ws, size_t ws_bytes, int temporal_t,
                         cudaStream_t s);
size_t rbsor_workspace_bytes(int h, int w);
cudaError_t rbsor_run(int h, int w, float *u, int iters, float omega, int check_every, double *res,
                      void *ws, cudaStream_t s);
cudaError_t rbsor_until(int h, int w, float *u, int max_iters, float omega, int check_every,
                        double tol, double *res, int *done, void *ws, cudaStream_t s);

}  // namespace pencil
