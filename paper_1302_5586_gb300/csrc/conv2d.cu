// conv2d.cu -- clamp-to-edge 2-D correlation kernels for sm_103a.
//
// out[i][j] = sum_a sum_b k[a][b] * in[clamp(i+a-kh/2)][clamp(j+b-kw/2)]
// (the independent pixel loops of Sec. 2.2.3; a map over output pixels,
// Sec. 3.2).  Every kernel here accumulates one output pixel in the same FP32
// order: for each filter row a, s = k[a][0]*x0 then s = fma(k[a][b], xb, s)
// for b = 1..kw-1, and acc = acc + s with acc starting at +0 -- so the direct,
// generic and batched kernels return identical bits for the same pixel.
//
// Design (one GPU, HBM-streaming):
//   * a CTA owns a TH x TW output tile and stages its halo tile
//     (TH+kh-1) x (TW+2P) in shared memory.  Images whose rows are 16-byte
//     aligned (clamp or zero border) are staged by the tensor memory
//     accelerator: one cp.async.bulk.tensor box per CTA, completion on an
//     mbarrier with a bounded wait, the clamp rebuilt in shared memory on
//     edge tiles.  Other images use cp.async copies (16 bytes where the
//     address allows), clamping rows per row and columns only in the chunks
//     that cross an edge;
//   * each thread computes R rows x C=4 columns in registers; for every
//     staged input row it loads its (C+kw-1)-wide window once (LDS.128) and
//     applies it to every output row that uses it (register blocking along
//     rows), with the filter row fetched by a broadcast LDS.128;
//   * the output is written with one 16-byte (FP32) or 8-byte (FP16) store per
//     thread and row.
#include "conv_kernels.cuh"

namespace pencil {
namespace {

using namespace tile;

// The bounded wait on its own: an mbarrier that expects 16 bytes no copy
// delivers, waited on for limit_ns; a wait that runs out is counted like a
// tile load's.  result: 1 if the wait completed, 0 if it ran out.
__global__ void wait_selftest_kernel(uint64_t limit_ns, int *result) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) tma::mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) tma::mbar_arrive_expect_tx(&bar, 16u);
    const bool ok = __syncthreads_and(tma::mbar_wait(&bar, 0, limit_ns));
    if (threadIdx.x == 0) {
        if (!ok) atomicAdd(&g_wait_timeouts, 1u);
        *result = ok ? 1 : 0;
    }
}

// SMs of the current device (cached per device; 152 if the query fails).
int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// Images with fewer 32 x 128 tiles than two per SM (a small image leaves most
// SMs idle): 8-row tiles (sides up to 7) or 16-row tiles (larger sides), TMA
// staging.  512 x 512 with a 5 x 5 filter: 5.3 -> 3.2 us on GB300.  False if
// it does not apply (then the default tiling runs).
template <typename T>
bool try_direct_small(int K, int c, int h, int w, const T *in, const float *k, T *out, bool vec_ok, int border,
                      cudaStream_t s, cudaError_t *err) {
    const long long tiles = (long long)c * ((h + 31) / 32) * ((w + 127) / 128);
    if (!vec_ok || tiles >= 2ll * sm_count()) return false;
    constexpr bool HW = sizeof(T) == 2;  // binary16 tiles of sides up to 7 stay binary16
    switch (K) {
        case 1: return try_direct_tma<T, 1, 32, 8, 1, 1, 8, HW>(c, h, w, in, k, out, vec_ok, border, s, err);
        case 3: return try_direct_tma<T, 3, 32, 8, 1, 1, 8, HW>(c, h, w, in, k, out, vec_ok, border, s, err);
        case 5: return try_direct_tma<T, 5, 32, 8, 1, 1, 8, HW>(c, h, w, in, k, out, vec_ok, border, s, err);
        case 7: return try_direct_tma<T, 7, 32, 8, 1, 1, 8, HW>(c, h, w, in, k, out, vec_ok, border, s, err);
        case 9: return try_direct_tma<T, 9, 16, 8, 2, 2, 3, false>(c, h, w, in, k, out, vec_ok, border, s, err);
        case 11: return try_direct_tma<T, 11, 16, 8, 2, 2, 3, false>(c, h, w, in, k, out, vec_ok, border, s, err);
        case 13: return try_direct_tma<T, 13, 16, 8, 2, 2, 3, false>(c, h, w, in, k, out, vec_ok, border, s, err);
        case 15: return try_direct_tma<T, 15, 16, 8, 2, 2, 3, false>(c, h, w, in, k, out, vec_ok, border, s, err);
        default: return false;
    }
}

template <typename T>
cudaError_t run_direct_k(int K, int c, int h, int w, const T *in, const float *k, T *out,
                         bool vec_ok, int border, cudaStream_t s) {
    cudaError_t err = cudaSuccess;
    if (try_direct_small<T>(K, c, h, w, in, k, out, vec_ok, border, s, &err)) return err;
    // Tile shapes and register caps per side, from timing sweeps on GB300 at
    // 8192 x 8192 x 3 (small sides: occupancy for HBM streaming; side 9: two
    // 4-column groups so each filter-row load feeds eight FMA chains; sides
    // 11..15: one 12-column group over 2 rows, 192-column tiles, 1-3% faster
    // than the two groups).  The staged box (at most 208 columns) fits one
    // TMA load.
    // Binary16 images up to side 7 keep the tile binary16 in shared memory
    // (HALFW): those kernels are bound by shared-memory traffic, which the
    // FP32 copy doubles; from side 9 the widening in the inner loop costs more
    // issue slots than it saves.
    if constexpr (sizeof(T) == 2) {
        switch (K) {
            case 1: return run_direct<T, 1, 32, 4, 8, 1, 8, true>(c, h, w, in, k, out, vec_ok, border, s);
            case 3: return run_direct<T, 3, 32, 4, 8, 1, 8, true>(c, h, w, in, k, out, vec_ok, border, s);
            case 5: return run_direct<T, 5, 32, 4, 8, 1, 8, true>(c, h, w, in, k, out, vec_ok, border, s);
            // 256-thread CTAs (64-row tiles): 0.418 -> 0.394 ms on 3 x 8192^2
            case 7: return run_direct<T, 7, 32, 8, 8, 1, 4, true>(c, h, w, in, k, out, vec_ok, border, s);
            default: break;
        }
    } else {
        switch (K) {
            case 1: return run_direct<T, 1, 32, 8, 4, 1, 8>(c, h, w, in, k, out, vec_ok, border, s);
            case 3: return run_direct<T, 3, 32, 8, 4, 1, 8>(c, h, w, in, k, out, vec_ok, border, s);
            case 5: return run_direct<T, 5, 32, 4, 8, 1, 8>(c, h, w, in, k, out, vec_ok, border, s);
            case 7: return run_direct<T, 7, 32, 4, 8, 1, 8>(c, h, w, in, k, out, vec_ok, border, s);
            default: break;
        }
    }
    constexpr bool F16 = sizeof(T) == 2;
    switch (K) {
        case 9: return run_direct<T, 9, 16, 8, 4, 2, 3>(c, h, w, in, k, out, vec_ok, border, s);
        case 11:
            if constexpr (F16) return run_direct<T, 11, 16, 8, 4, 2, 3>(c, h, w, in, k, out, vec_ok, border, s);
            else return run_direct<T, 11, 16, 8, 2, 1, 3, false, 1, 12>(c, h, w, in, k, out, vec_ok, border, s);
        case 13: return run_direct<T, 13, 16, 8, 2, 1, 3, false, 1, 12>(c, h, w, in, k, out, vec_ok, border, s);
        case 15:
            if constexpr (F16) return run_direct<T, 15, 16, 16, 2, 1, 2, false, 1, 12>(c, h, w, in, k, out, vec_ok, border, s);
            else return run_direct<T, 15, 16, 8, 2, 1, 3, false, 1, 12>(c, h, w, in, k, out, vec_ok, border, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t run_sep_any(int c, int h, int w, const T *in, int kx, const float *gx, int ky,
                        const float *gy, T *out, bool vec_ok, int border, cudaStream_t s) {
    // Tiles from timing sweeps at 8192 x 8192 x 3; the 15-tap tiles are 128
    // rows tall (the row pass recomputes 14 halo rows per tile, 11% extra).
    // Binary16 images: the row pass reads the staged binary16 tile directly
    // (no FP32 copy, no widening pass), 256-thread CTAs of 8 rows per thread;
    // that measured 17-40% faster than widening the tile first on every side
    // (15 taps: 0.375 -> 0.299 ms, 3 taps: 0.257 -> 0.156 ms).  Row-pass
    // items of 8 columns (sides 11..15) or 12 (side 3) widen each binary16
    // window once for more outputs: 3-5% more.
    if constexpr (sizeof(T) == 2) {
        if (kx == ky) {
            switch (kx) {
                case 3: return run_sep<T, 3, 48, 4, 8, 3, false, sep_pair<T>(3), 1, true, 12>(c, h, w, in, gx, gy, out, vec_ok, border, s);
                case 5: return run_sep<T, 5, 32, 8, 8, 3, false, sep_pair<T>(5), 1, true>(c, h, w, in, gx, gy, out, vec_ok, border, s);
                case 7: return run_sep<T, 7, 32, 8, 8, 3, false, sep_pair<T>(7), 1, true>(c, h, w, in, gx, gy, out, vec_ok, border, s);
                case 9: return run_sep<T, 9, 32, 8, 8, 3, false, sep_pair<T>(9), 1, true>(c, h, w, in, gx, gy, out, vec_ok, border, s);
                case 11: return run_sep<T, 11, 16, 16, 8, 3, false, sep_pair<T>(11), 1, true, 8>(c, h, w, in, gx, gy, out, vec_ok, border, s);
                case 13: return run_sep<T, 13, 16, 16, 8, 3, false, sep_pair<T>(13), 1, true, 8>(c, h, w, in, gx, gy, out, vec_ok, border, s);
                case 15: return run_sep<T, 15, 16, 16, 8, 3, false, sep_pair<T>(15), 1, true, 8>(c, h, w, in, gx, gy, out, vec_ok, border, s);
                default: break;
            }
        }
        return run_sep_generic<T>(c, h, w, in, kx, gx, ky, gy, out, border, s);
    }
    // FP32 sides 3..9: in-place tiles of 8 or 16 rows per thread measured 3-12%
    // faster than the 4-row tiles with a separate row-pass buffer.
    if (kx == ky) {
        switch (kx) {
            case 3: return run_sep<T, 3, 32, 4, 8, 4, true, sep_pair<T>(3)>(c, h, w, in, gx, gy, out, vec_ok, border, s);
            case 5: return run_sep<T, 5, 16, 8, 16, 4, true, sep_pair<T>(5)>(c, h, w, in, gx, gy, out, vec_ok, border, s);
            case 7: return run_sep<T, 7, 32, 4, 8, 4, true, sep_pair<T>(7)>(c, h, w, in, gx, gy, out, vec_ok, border, s);
            case 9: return run_sep<T, 9, 16, 8, 16, 4, true, sep_pair<T>(9)>(c, h, w, in, gx, gy, out, vec_ok, border, s);
            case 11: return run_sep<T, 11, 16, 8, 8, 4, true, sep_pair<T>(11)>(c, h, w, in, gx, gy, out, vec_ok, border, s);
            case 13: return run_sep<T, 13, 16, 8, 8, 4, true, sep_pair<T>(13)>(c, h, w, in, gx, gy, out, vec_ok, border, s);
            case 15: return run_sep<T, 15, 16, 8, 16, 4, true, sep_pair<T>(15)>(c, h, w, in, gx, gy, out, vec_ok, border, s);
            default: break;
        }
    }
    return run_sep_generic<T>(c, h, w, in, kx, gx, ky, gy, out, border, s);
}

}  // namespace

cudaError_t wait_selftest(uint64_t limit_ns, int *completed) {
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e != cudaSuccess) return e;
    wait_selftest_kernel<<<1, 64>>>(limit_ns, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(completed, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e;
}

cudaError_t wait_timeouts(unsigned *n, bool clear) { return read_wait_counter(n, clear); }

namespace {

bool rows_aligned(const void *p, int w, int vec) {
    return (w % vec == 0) && ((uintptr_t)p % 16 == 0);
}

}  // namespace

cudaError_t launch_conv2d(int dtype, int c, int h, int w, const void *in, int kh, int kw,
                          const float *k, void *out, cudaStream_t s, int border) {
    const bool special = (kh == kw) && (kh % 2 == 1) && kh <= PENCIL_MAX_SPECIALISED_K;
    if (dtype == PENCIL_F32) {
        const float *i = static_cast<const float *>(in);
        float *o = static_cast<float *>(out);
        const bool v = rows_aligned(in, w, 4) && rows_aligned(out, w, 4);
        if (special) return run_direct_k<float>(kh, c, h, w, i, k, o, v, border, s);
        return run_generic<float>(c, h, w, i, kh, kw, k, o, border, s);
    }
    const __half *i = static_cast<const __half *>(in);
    __half *o = static_cast<__half *>(out);
    const bool v = rows_aligned(in, w, 8) && rows_aligned(out, w, 8);
    if (special) return run_direct_k<__half>(kh, c, h, w, i, k, o, v, border, s);
    return run_generic<__half>(c, h, w, i, kh, kw, k, o, border, s);
}

cudaError_t launch_conv2d_generic(int dtype, int c, int h, int w, const void *in, int kh, int kw,
                                  const float *k, void *out, cudaStream_t s, int border, int cs) {
    if (dtype == PENCIL_F32)
        return run_generic<float>(c, h, w, static_cast<const float *>(in), kh, kw, k,
                                  static_cast<float *>(out), border, s, cs);
    return run_generic<__half>(c, h, w, static_cast<const __half *>(in), kh, kw, k,
                               static_cast<__half *>(out), border, s, cs);
}

cudaError_t launch_conv2d_sep_generic(int dtype, int c, int h, int w, const void *in, int kx, const float *gx,
                                      int ky, const float *gy, void *out, cudaStream_t s, int border, int cs) {
    if (dtype == PENCIL_F32)
        return run_sep_generic<float>(c, h, w, static_cast<const float *>(in), kx, gx, ky, gy,
                                      static_cast<float *>(out), border, s, cs);
    return run_sep_generic<__half>(c, h, w, static_cast<const __half *>(in), kx, gx, ky, gy,
                                   static_cast<__half *>(out), border, s, cs);
}

cudaError_t launch_conv2d_sep(int dtype, int c, int h, int w, const void *in, int kx,
                              const float *gx, int ky, const float *gy, void *out,
                              cudaStream_t s, int border) {
    if (dtype == PENCIL_F32) {
        const bool v = rows_aligned(in, w, 4) && rows_aligned(out, w, 4);
        return run_sep_any<float>(c, h, w, static_cast<const float *>(in), kx, gx, ky, gy,
                                  static_cast<float *>(out), v, border, s);
    }
    const bool v = rows_aligned(in, w, 8) && rows_aligned(out, w, 8);
    return run_sep_any<__half>(c, h, w, static_cast<const __half *>(in), kx, gx, ky, gy,
                               static_cast<__half *>(out), v, border, s);
}

}  // namespace pencil
