// conv_jacobi.cu -- a filter pass followed by Jacobi smoothing sweeps, fused
// into one kernel: out = J^n(conv(in, k)) per planar channel, where conv is
// the clamp-to-edge correlation of conv2d.cu and J the 5-point Jacobi sweep of
// jacobi.cu (boundary ring fixed).  This is the cross-component fusion of a
// stencil chain (Sec. 2.2.3: the filtered image goes straight into the
// sweeps instead of making a round trip through HBM).
//
// A CTA owns the 128 x 128 window of the register-tiled Jacobi kernel (8 warps
// x 16 rows, lane l: columns 4l .. 4l+3) and its core.  Instead of loading
// the window from HBM it computes it: one TMA box of the input, (128 + k - 1)
// rows x (128 + 2P) columns, is staged in shared memory (clamp rebuilt on edge
// tiles), and every thread runs the direct tile body for its own 16 rows x 4
// columns -- exactly the window positions it holds for the sweeps -- so the
// filter results land in the registers the sweeps start from.  The sweeps
// and the core store are the Jacobi kernel's.  Per pixel the filter sum and
// per point the sweep are the same FP32 expressions as the separate kernels,
// so the result is the same bits as pencil_conv2d_ex followed by
// pencil_jacobi2d_ex on each channel.
#include "conv_kernels.cuh"
#include "jacobi_tile.cuh"

namespace pencil {
namespace {

using namespace tile;

template <int K, int T>
struct CJCfg {
    using J = RegCfg<T>;
    static constexpr int A = K / 2;
    static constexpr int PC = round_up(A, 8);    // input columns staged left of the window (16-byte aligned x)
    static constexpr int SW = J::W + 2 * PC;     // staged box width
    static constexpr int SH = J::SH + K - 1;     // staged box rows
    static constexpr int KWP = round_up(K, 4);
    static constexpr size_t smem = sizeof(float) * ((size_t)SH * SW + (size_t)K * KWP);
    static_assert(SW <= 256 && SH <= 256, "a TMA box side is at most 256 elements");
};

template <int K, int T>
__global__ void __launch_bounds__(RegCfg<T>::NT, 2)
    conv_jacobi_kernel(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ k,
                       float *__restrict__ out, int h, int w, int n) {
    using Cfg = CJCfg<K, T>;
    using J = RegCfg<T>;
    constexpr int RS = J::RS, NW = J::NW, SW = Cfg::SW, SH = Cfg::SH;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float4 xch[2 * NW * 2 * 32];
    float *s_in = smem;
    float *s_k = smem + SH * SW;
    const int gy0 = blockIdx.y * J::BH - T;   // global row of window row 0
    const int gx0 = blockIdx.x * J::BW - J::P;  // global column of window column 0 (multiple of 4)
    if ((tma::smem_addr(s_in) & 127u) != 0) {  // a TMA box needs a 128-byte aligned destination
        if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);
        return;
    }
    if (threadIdx.x == 0) tma::mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        tma::mbar_arrive_expect_tx(&bar, (unsigned)(sizeof(float) * SH * SW));
        tma::load_3d(s_in, &tmap, gx0 - Cfg::PC, gy0 - Cfg::A, (int)blockIdx.z, &bar);
    }
    stage_filter<K, K, Cfg::KWP, J::NT>(k, s_k);
    if (!__syncthreads_and(tma::mbar_wait(&bar, 0, tma::kLoadWaitNs))) {
        if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1u);  // the copy did not land in time: skip the tile
        tma::mbar_wait(&bar, 0, tma::kLoadWaitNs);
        return;
    }
    clamp_fixup<float, SH, SW, J::NT>(s_in, h, w, gy0 - Cfg::A, gx0 - Cfg::PC);

    // the filter over this thread's window positions: rows wp*16 .. +15, columns 4*lane .. +3
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    float acc[RS][4];
    direct_accumulate<K, K, RS, 1, 4 * 32, SW, Cfg::KWP, Cfg::PC - Cfg::A>(s_in + (wp * RS) * SW + 4 * lane, s_k,
                                                                             acc);
    float4 y[RS + 1];
    y[0] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < RS; ++r) y[1 + r] = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    float *dst = out + (size_t)h * (size_t)w * blockIdx.z;
    const RegGeom<J> q(h, w, gy0, gx0);
    if (gy0 <= 0 || gy0 + J::SH - 1 >= h - 1 || gx0 <= 0 || gx0 + J::W - 1 >= w - 1)
        reg_sweeps_store<J, true>(y, dst, h, w, n, q, 0, 0, xch, nullptr);
    else
        reg_sweeps_store<J, false>(y, dst, h, w, n, q, 0, 0, xch, nullptr);
}

template <int K, int T>
cudaError_t run_fused(int c, int h, int w, const float *in, const float *k, float *out, int n, cudaStream_t s) {
    using Cfg = CJCfg<K, T>;
    using J = RegCfg<T>;
    CUtensorMap tmap;
    if (!image_tensor_map<float>(&tmap, in, c, h, w, Cfg::SW, Cfg::SH)) return cudaErrorNotSupported;
    auto kern = conv_jacobi_kernel<K, T>;
    cudaError_t e = set_smem(kern, Cfg::smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((w + J::BW - 1) / J::BW, (h + J::BH - 1) / J::BH, c);
    kern<<<grid, J::NT, Cfg::smem, s>>>(tmap, k, out, h, w, n);
    return cudaGetLastError();
}

template <int T>
cudaError_t run_fused_t(int K, int c, int h, int w, const float *in, const float *k, float *out, int n,
                        cudaStream_t s) {
    switch (K) {
        case 1: return run_fused<1, T>(c, h, w, in, k, out, n, s);
        case 3: return run_fused<3, T>(c, h, w, in, k, out, n, s);
        case 5: return run_fused<5, T>(c, h, w, in, k, out, n, s);
        case 7: return run_fused<7, T>(c, h, w, in, k, out, n, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool conv_jacobi_fusable(int h, int w, int kh, int kw, const void *in, const void *out) {
    return kh == kw && (kh & 1) && kh <= kConvJacobiMaxK && h >= 3 && w >= 3 && w % 4 == 0 &&
           (uintptr_t)in % 16 == 0 && (uintptr_t)out % 16 == 0;
}

cudaError_t launch_conv_jacobi_fused(int c, int h, int w, const float *in, int ks, const float *k, int n,
                                     float *out, cudaStream_t s) {
    if (n < 1 || n > kConvJacobiMaxSweeps) return cudaErrorInvalidValue;
    return n <= 4 ? run_fused_t<4>(ks, c, h, w, in, k, out, n, s) : run_fused_t<10>(ks, c, h, w, in, k, out, n, s);
}

cudaError_t wait_timeouts_cj(unsigned *n, bool clear) { return read_wait_counter(n, clear); }

}  // namespace pencil
