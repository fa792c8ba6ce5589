// conv_tc.cu -- binary16 images on the 5th-generation tensor cores (tcgen05):
// an opt-in alternative (PENCIL_CONV_TENSOR) to the CUDA-core kernels for
// planar binary16 images whose rows are 16-byte aligned, odd square filters
// of side 9..15 and the clamp or zero border.
//
// For one filter row a, a block of 128 output rows x 16 output columns is a
// matrix product: out[m][n] += sum_k in[y0 + m + a - kh/2][xs + k] * T_a[n][k]
// over 32 staged columns k (xs = the block's first column - 8), where
// T_a[n][k] = k[a][k - n - d] (zero off the filter row), d = 8 - kw/2, is the
// banded matrix of that row: the band holds kw of the 32 products, the rest
// are zeros.  The weights are scaled by a power of two that puts the largest
// in [0.5, 1), and each scaled weight is split into two binary16 terms (hi,
// its rounding; lo, the rounding of the rest), so a weight keeps about 22
// significant bits.  The two banded matrices of a row are stacked along N:
// one MMA of M = 128, N = 32 (16 hi + 16 lo columns), K = 16 reads each slice
// of the input once for both terms (shared-memory operand reads, not the
// tensor pipe, bound this kernel), two per filter row and block.  Both sums
// accumulate in FP32 in tensor memory (TMEM); the epilogue adds them, undoes
// the scale and rounds to binary16 once.  The result stays within the
// binary16 tolerance of the FP64 correlation but is not the same bits as the
// CUDA-core kernels (a different summation order).
//
// A CTA computes one 128 x 128 output tile: eight 16-column blocks, 32 TMEM
// columns each (hi sums, then lo sums).  Its input, (128 + kh - 1) rows x 144 columns starting 8 columns
// left of the tile, arrives as 18 TMA boxes of 8 columns x all rows; each box
// lands as rows of 16 bytes one after another, which is the no-swizzle
// K-major layout of core matrices (8 rows x 16 bytes), so the A operand of
// filter row a is the same data a rows further down: its descriptor start
// moves by 16 a bytes.  The CTA builds the banded matrices (kh rows x 32 x 32
// binary16, hi rows then lo rows) from the filter, staged once in shared
// memory, while the boxes are in flight; one thread then issues the kh x 8 x 2
// MMAs and commits them to an
// mbarrier, and the four warps read the accumulators back (warp w: rows
// 32 w .. 32 w + 31, the TMEM lanes it may access), scale, round and store.
#include "conv_kernels.cuh"
#include "umma.cuh"

namespace pencil {
namespace {

constexpr int kTcM = 128;              // output rows per tile (the MMA's M)
constexpr int kTcBlocks = 8;           // 16-column blocks per tile
constexpr int kTcW = 16 * kTcBlocks;   // output columns per tile
constexpr int kTcChunks = 2 * kTcBlocks + 2;  // staged 8-column chunks (144 columns)
constexpr int kTcThreads = 128;
constexpr unsigned kTcTmemCols = 32 * kTcBlocks;  // per block: 16 hi + 16 lo sums

template <int K>
struct TcCfg {
    static constexpr int A = K / 2;
    static constexpr int SH = kTcM + K - 1;                       // staged rows
    static constexpr int CHB = round_up(SH * 16, 128);            // bytes per staged chunk (TMA destinations 128-byte aligned)
    static constexpr int A_BYTES = kTcChunks * CHB;
    static constexpr int B_BYTES = K * 2048;                      // banded matrices: K rows x 32 (hi, lo) x 32 binary16
    static constexpr size_t smem = (size_t)A_BYTES + B_BYTES;
    static constexpr int D = 8 - A;                               // window offset inside the 32 staged columns
    static_assert(15 + D + K - 1 < 32, "a block's window fits two K-steps");
};

// Binary16 element (r, c) of the staged tile (chunk-major).
template <int K>
__device__ __forceinline__ __half &staged(unsigned char *sa, int r, int c) {
    return *reinterpret_cast<__half *>(sa + (c >> 3) * TcCfg<K>::CHB + r * 16 + (c & 7) * 2);
}

template <int K, bool CLAMP>
__global__ void __launch_bounds__(kTcThreads, 1)
    conv2d_tc_kernel(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ k,
                     __half *__restrict__ out, int h, int w) {
    using Cfg = TcCfg<K>;
    constexpr int SH = Cfg::SH, SWC = 8 * kTcChunks;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar_a, bar_d;
    __shared__ unsigned s_tmem;
    __shared__ float s_max[kTcThreads / 32];
    __shared__ float s_w[K * K];
    unsigned char *sa = tc_smem, *sb = tc_smem + Cfg::A_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int y0 = blockIdx.y * kTcM, x0 = blockIdx.x * kTcW;
    const int gy0 = y0 - Cfg::A, gx0 = x0 - 8;
    if ((tma::smem_addr(sa) & 127u) != 0) {  // TMA destinations need 128-byte alignment
        if (tid == 0) atomicAdd(&g_wait_timeouts, 1u);
        return;
    }
    if (warp == 0) umma::tmem_alloc(&s_tmem, kTcTmemCols);
    if (tid == 0) {
        tma::mbar_init(&bar_a, 1);
        tma::mbar_init(&bar_d, 1);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const unsigned tmem = s_tmem;
    if (tid == 0) {
        tma::mbar_arrive_expect_tx(&bar_a, (unsigned)(kTcChunks * SH * 16));
        for (int i = 0; i < kTcChunks; ++i)
            tma::load_3d(sa + i * Cfg::CHB, &tmap, gx0 + 8 * i, gy0, (int)blockIdx.z, &bar_a);
    }

    // the scale 2^-e that puts the largest |weight| in [0.5, 1)
    float m = 0.0f;
    for (int i = tid; i < K * K; i += kTcThreads) {
        const float v = __ldg(k + i);
        s_w[i] = v;
        m = fmaxf(m, fabsf(v));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) s_max[warp] = m;
    __syncthreads();
    m = fmaxf(fmaxf(s_max[0], s_max[1]), fmaxf(s_max[2], s_max[3]));
    int e = 0;
    if (m > 0.0f && m <= 3.0e38f) frexpf(m, &e);
    e = max(-126, min(126, e));
    const float scale = ldexpf(1.0f, -e), unscale = ldexpf(1.0f, e);

    // banded matrices: row a at 2a KB; element (n, k) at (k / 8) * 512 +
    // n * 16 + (k % 8) * 2, hi terms in rows n < 16, lo terms in rows 16 + n;
    // one 16-byte chunk row of both per item
    for (int it = tid; it < K * 16 * 4; it += kTcThreads) {
        const int a = it / 64, n = (it >> 2) & 15, kc = it & 3;
        uint32_t hi2[4], lo2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __half hv[2], lv[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int b = kc * 8 + 2 * q + t - n - Cfg::D;
                const float v = (b >= 0 && b < K) ? s_w[a * K + b] * scale : 0.0f;
                hv[t] = __float2half_rn(v);
                lv[t] = __float2half_rn(v - __half2float(hv[t]));
            }
            hi2[q] = (uint32_t)__half_as_ushort(hv[0]) | ((uint32_t)__half_as_ushort(hv[1]) << 16);
            lo2[q] = (uint32_t)__half_as_ushort(lv[0]) | ((uint32_t)__half_as_ushort(lv[1]) << 16);
        }
        unsigned char *row = sb + a * 2048 + kc * 512 + n * 16;
        *reinterpret_cast<uint4 *>(row) = make_uint4(hi2[0], hi2[1], hi2[2], hi2[3]);
        *reinterpret_cast<uint4 *>(row + 256) = make_uint4(lo2[0], lo2[1], lo2[2], lo2[3]);
    }

    if (!__syncthreads_and(tma::mbar_wait(&bar_a, 0, tma::kLoadWaitNs))) {
        if (tid == 0) atomicAdd(&g_wait_timeouts, 1u);  // the boxes did not land in time: skip the tile
        tma::mbar_wait(&bar_a, 0, tma::kLoadWaitNs);
        __syncthreads();
        if (warp == 0) umma::tmem_free(tmem, kTcTmemCols);
        return;
    }
    if (CLAMP) {  // out-of-image rows, then columns, take the nearest edge element
        const int top = -gy0, bot = h - gy0, left = -gx0, right = w - gx0;
        if (top > 0 || bot < SH) {
            for (int i = tid; i < SH * SWC; i += kTcThreads) {
                const int r = i / SWC, c = i - r * SWC;
                const int src = r < top ? top : (r >= bot ? bot - 1 : r);
                if (src != r) staged<K>(sa, r, c) = staged<K>(sa, src, c);
            }
            __syncthreads();
        }
        if (left > 0 || right < SWC) {
            for (int i = tid; i < SH * SWC; i += kTcThreads) {
                const int r = i / SWC, c = i - r * SWC;
                const int src = c < left ? left : (c >= right ? right - 1 : c);
                if (src != c) staged<K>(sa, r, c) = staged<K>(sa, r, src);
            }
        }
    }
    umma::fence_proxy_async();  // the banded matrices and the clamp, written by threads, are read by the MMAs
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();

    if (tid == 0) {
        constexpr uint32_t idesc = umma::idesc_f16_f32(kTcM, 32);
        const uint64_t a0 = umma::smem_desc(tma::smem_addr(sa), Cfg::CHB, 128);
        const uint64_t b0 = umma::smem_desc(tma::smem_addr(sb), 512, 128);
#pragma unroll 1
        for (int a = 0; a < K; ++a)
#pragma unroll
            for (int j = 0; j < kTcBlocks; ++j)
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t da = a0 + ((unsigned)((2 * j + 2 * ks) * Cfg::CHB + 16 * a) >> 4);
                    const uint64_t db = b0 + ((unsigned)(a * 2048 + 1024 * ks) >> 4);
                    umma::mma_f16(tmem + 32 * j, da, db, idesc, a > 0 || ks > 0);
                }
        umma::commit(&bar_d);
    }
    if (!__syncthreads_and(tma::mbar_wait(&bar_d, 0, tma::kLoadWaitNs))) {
        if (tid == 0) atomicAdd(&g_wait_timeouts, 1u);
        tma::mbar_wait(&bar_d, 0, tma::kLoadWaitNs);
        __syncthreads();
        if (warp == 0) umma::tmem_free(tmem, kTcTmemCols);
        return;
    }
    umma::fence_after_sync();

    // epilogue: warp w holds rows 32 w .. 32 w + 31 (TMEM lanes), a thread one row
    const int row = y0 + 32 * warp + lane;
    __half *orow = out + ((size_t)blockIdx.z * h + (size_t)min(row, h - 1)) * (size_t)w;
#pragma unroll 1
    for (int j = 0; j < kTcBlocks; ++j) {
        float v[16], lo[16];
        umma::ld16(tmem + ((unsigned)(32 * warp) << 16) + 32 * j, v);
        umma::ld16(tmem + ((unsigned)(32 * warp) << 16) + 32 * j + 16, lo);
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] += lo[q];
        const int col = x0 + 16 * j;
        if (row >= h || col >= w) continue;
        uint32_t p[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            p[q] = (uint32_t)__half_as_ushort(__float2half_rn(v[2 * q] * unscale)) |
                   ((uint32_t)__half_as_ushort(__float2half_rn(v[2 * q + 1] * unscale)) << 16);
        if (col + 16 <= w) {
            uint4 *d = reinterpret_cast<uint4 *>(orow + col);
            d[0] = make_uint4(p[0], p[1], p[2], p[3]);
            d[1] = make_uint4(p[4], p[5], p[6], p[7]);
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (col + q < w) orow[col + q] = __ushort_as_half((unsigned short)(p[q >> 1] >> (16 * (q & 1))));
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, kTcTmemCols);
}

template <int K>
cudaError_t run_tc(int c, int h, int w, const __half *in, const float *k, __half *out, int border,
                   cudaStream_t s, bool *done) {
    using Cfg = TcCfg<K>;
    CUtensorMap tmap;
    *done = false;
    if (!image_tensor_map<__half>(&tmap, in, c, h, w, 8, Cfg::SH)) return cudaSuccess;
    auto kern = border == 0 ? conv2d_tc_kernel<K, true> : conv2d_tc_kernel<K, false>;
    cudaError_t e = set_smem(kern, Cfg::smem);
    if (e != cudaSuccess) return e;
    dim3 grid((w + kTcW - 1) / kTcW, (h + kTcM - 1) / kTcM, c);
    kern<<<grid, kTcThreads, Cfg::smem, s>>>(tmap, k, out, h, w);
    *done = true;
    return cudaGetLastError();
}

}  // namespace

// Queue the tensor-core correlation if it applies (binary16, odd side 9..15,
// rows of in and out 16-byte aligned, clamp or zero border); *done says
// whether it was queued.  On 3 x 8192^2 each filter row costs ~0.037 ms of
// MMAs (bound by their shared-memory operand reads, ~84 bytes per cycle per
// SM) on top of ~0.11 ms per launch of staging, banded matrices and
// epilogue: 15x15 0.669 ms against 1.542 ms on the CUDA cores, 9x9 0.446
// against 0.642.  Sides 3..7 stay on the CUDA cores, where that fixed part
// alone is most of their time (3x3: 0.163 ms).
cudaError_t launch_conv2d_tc(int c, int h, int w, const void *in, int ks, const float *k, void *out, int border,
                             cudaStream_t s, bool *done) {
    *done = false;
    if ((border != 0 && border != 1) || (w % 8) != 0 || ((uintptr_t)in & 15u) != 0 || ((uintptr_t)out & 15u) != 0)
        return cudaSuccess;
    const __half *i = static_cast<const __half *>(in);
    __half *o = static_cast<__half *>(out);
    switch (ks) {
        case 9: return run_tc<9>(c, h, w, i, k, o, border, s, done);
        case 11: return run_tc<11>(c, h, w, i, k, o, border, s, done);
        case 13: return run_tc<13>(c, h, w, i, k, o, border, s, done);
        case 15: return run_tc<15>(c, h, w, i, k, o, border, s, done);
        default: return cudaSuccess;
    }
}

cudaError_t wait_timeouts_tc(unsigned *n, bool clear) { return read_wait_counter(n, clear); }

}  // namespace pencil
