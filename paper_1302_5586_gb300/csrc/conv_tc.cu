// conv_tc.cu -- binary16 images on the 5th-generation tensor cores (tcgen05):
// an opt-in alternative (PENCIL_CONV_TENSOR) to the CUDA-core kernels for
// planar binary16 images whose rows are 16-byte aligned, odd square filters
// of side 7..15 and the clamp or zero border.
//
// For one filter row a, a block of 128 output rows x 16 output columns is a
// matrix product: out[m][n] += sum_k in[y0 + m + a - kh/2][xs + k] * T_a[n][k]
// over 32 staged columns k (xs = the block's first column - 8), where
// T_a[n][k] = k[a][k - n - d] (zero off the filter row), d = 8 - kw/2, is the
// banded matrix of that row: the band holds kw of the 32 products, the rest
// are zeros.  The weights are scaled by a power of two that puts the largest
// in [0.5, 1), and each scaled weight is split into two binary16 terms (hi,
// its rounding; lo, the rounding of the rest), so a weight keeps about 22
// significant bits.  Shared-memory operand reads, not the tensor pipe, bound
// the MMAs, so each 16-column slice of the input is read once per filter row:
// one MMA of M = 128, N = 64, K = 16 multiplies it by the hi and lo terms of
// the first half of the band (for the block at that slice) and of the second
// half (for the block to its left).  The accumulator is cleared once per tile
// (an MMA with a zero B operand) and every product accumulates in FP32 in
// tensor memory (TMEM); the epilogue adds the hi and lo sums, undoes the
// scale and rounds to binary16 once.  The result stays within the
// binary16 tolerance of the FP64 correlation but is not the same bits as the
// CUDA-core kernels (a different summation order).
//
// The kernel is persistent and warp-specialised, one CTA per SM looping
// over 128 x 96 output tiles (six 16-column blocks, 32 TMEM columns each: hi
// sums, then lo sums; block b at column 32 (6 - b), so slice c's 64 columns
// start at 32 (6 - c)).  The CTA builds the banded matrices once (kh B
// operands of 64 x 16 binary16, from the filter staged in shared memory).
// Warp 0 streams input tiles by TMA into four stages: a tile's
// (128 + kh - 1) rows x 112 columns, starting 8 columns left of it, arrive as
// 14 boxes of 8 columns x all rows, each landing as consecutive 16-byte rows
// -- the no-swizzle K-major layout of core matrices (8 rows x 16 bytes) -- so
// the A operand of filter row a is the same data a rows further down: its
// descriptor start moves by 16 a bytes.  Warp 1 waits for a stage, rebuilds
// the clamp on edge tiles, and issues the 1 + kh x 7 MMAs of the tile into
// one of two TMEM accumulators (2 x 256 columns); its commits free the stage
// and hand the accumulator on.  Warps 2-9 read the other accumulator (warp w:
// TMEM lanes 32 (w % 4) .. + 31, its output rows), add the two sums, undo the
// scale, round and store (eight warps, two per lane quarter, each with the
// TMEM loads of its three blocks in flight), and hand it back -- so loads,
// MMAs and stores of neighbouring tiles overlap.  Every wait is bounded; a role that runs out
// stops issuing, records a timeout and lets what it has in flight finish
// before the CTA frees its TMEM.
#include "conv_kernels.cuh"
#include "umma.cuh"

namespace pencil {
namespace {

constexpr int kTcM = 128;                      // output rows per tile (the MMA's M)
constexpr int kTcBlocks = 6;                   // 16-column blocks per tile
constexpr int kTcW = 16 * kTcBlocks;           // output columns per tile
constexpr int kTcSlices = kTcBlocks + 1;       // 16-column input slices (112 staged columns)
constexpr int kTcChunks = 2 * kTcSlices;       // staged 8-column chunks
constexpr int kTcStoreWarps = 8;               // two per TMEM lane quarter, four blocks each
constexpr int kTcThreads = 32 * (2 + kTcStoreWarps);  // warp 0 loads, warp 1 MMAs, warps 2-9 store
constexpr int kTcStages = 4;                   // input tiles in flight per SM
// one accumulator: block b's 16 hi + 16 lo sums at columns 32 (blocks - b),
// plus the two 32-column ends that the first and last slice also write
constexpr unsigned kTcAccCols = 32 * (kTcBlocks + 2);
constexpr unsigned kTcTmemCols = 2 * kTcAccCols;

template <int K>
struct TcCfg {
    static constexpr int A = K / 2;
    static constexpr int SH = kTcM + K - 1;                 // staged rows
    static constexpr int CHB = round_up(SH * 16, 128);      // bytes per staged chunk (TMA destinations 128-byte aligned)
    static constexpr int A_BYTES = kTcChunks * CHB;         // one stage
    static constexpr int B_BYTES = K * 2048;                // banded matrices: K rows x 64 x 16 binary16
    static constexpr int Z_BYTES = 256 * 16 * 2;            // zeros: the B operand that clears an accumulator
    static constexpr size_t smem = kTcStages * (size_t)A_BYTES + B_BYTES + Z_BYTES;
    static constexpr int D = 8 - A;                         // window offset inside the 32 staged columns
    static_assert(15 + D + K - 1 < 32, "a block's window fits two K-steps");
};

// Binary16 element (r, c) of a staged tile (chunk-major).
template <int K>
__device__ __forceinline__ __half &staged(unsigned char *sa, int r, int c) {
    return *reinterpret_cast<__half *>(sa + (c >> 3) * TcCfg<K>::CHB + r * 16 + (c & 7) * 2);
}

struct TcTile {
    int plane, y0, x0;
};
__device__ __forceinline__ TcTile tc_tile(int t, int tiles_x, int tiles_y) {
    const int tx = t % tiles_x, r = t / tiles_x;
    return {r / tiles_y, (r % tiles_y) * kTcM, tx * kTcW};
}

template <int K, bool CLAMP>
__global__ void __launch_bounds__(kTcThreads, 1)
    conv2d_tc_kernel(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ k,
                     __half *__restrict__ out, int h, int w, int tiles_x, int tiles_y, int tiles) {
    using Cfg = TcCfg<K>;
    constexpr int SH = Cfg::SH, SWC = 8 * kTcChunks;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], acc_full[2], acc_empty[2], fin;
    __shared__ unsigned s_tmem;
    __shared__ volatile int s_abort;
    __shared__ float s_max[kTcThreads / 32];
    __shared__ float s_w[K * K];
    unsigned char *sb = tc_smem + kTcStages * Cfg::A_BYTES, *sz = sb + Cfg::B_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if ((tma::smem_addr(tc_smem) & 127u) != 0) {  // TMA destinations need 128-byte alignment
        if (tid == 0) atomicAdd(&g_wait_timeouts, 1u);
        return;
    }
    if (warp == 0) umma::tmem_alloc(&s_tmem, kTcTmemCols);
    if (tid == 0) {
        for (int i = 0; i < kTcStages; ++i) {
            tma::mbar_init(&full[i], 1);
            tma::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tma::mbar_init(&acc_full[i], 1);
            tma::mbar_init(&acc_empty[i], kTcStoreWarps);  // one arrival per storing warp
        }
        tma::mbar_init(&fin, 1);
        s_abort = 0;
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
    m = s_max[0];
#pragma unroll
    for (int i = 1; i < kTcThreads / 32; ++i) m = fmaxf(m, s_max[i]);
    int e = 0;
    if (m > 0.0f && m <= 3.0e38f) frexpf(m, &e);
    e = max(-126, min(126, e));
    const float scale = ldexpf(1.0f, -e), unscale = ldexpf(1.0f, e);

    // banded matrices, one 64 x 16 B operand per filter row a (at 2a KB),
    // element (row, k) at (k / 8) * 1024 + row * 16 + (k % 8) * 2: rows
    // 32 ks + n (hi) and 32 ks + 16 + n (lo) hold T_a[n][16 ks + k], so one
    // 16-column input slice feeds the first half (ks = 0) of the window of its
    // own block and the second half (ks = 1) of the block to its left; one
    // 8-column chunk row of both terms per item
    for (int it = tid; it < K * 64; it += kTcThreads) {
        const int a = it >> 6, n = (it >> 2) & 15, ks = (it >> 1) & 1, kc = it & 1;
        uint32_t hi2[4], lo2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __half hv[2], lv[2];
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int b = 16 * ks + kc * 8 + 2 * q + t - n - Cfg::D;
                const float v = (b >= 0 && b < K) ? s_w[a * K + b] * scale : 0.0f;
                hv[t] = __float2half_rn(v);
                lv[t] = __float2half_rn(v - __half2float(hv[t]));
            }
            hi2[q] = (uint32_t)__half_as_ushort(hv[0]) | ((uint32_t)__half_as_ushort(hv[1]) << 16);
            lo2[q] = (uint32_t)__half_as_ushort(lv[0]) | ((uint32_t)__half_as_ushort(lv[1]) << 16);
        }
        unsigned char *row = sb + a * 2048 + kc * 1024 + (32 * ks + n) * 16;
        *reinterpret_cast<uint4 *>(row) = make_uint4(hi2[0], hi2[1], hi2[2], hi2[3]);
        *reinterpret_cast<uint4 *>(row + 256) = make_uint4(lo2[0], lo2[1], lo2[2], lo2[3]);
    }
    for (int i = tid; i < Cfg::Z_BYTES / 16; i += kTcThreads)
        reinterpret_cast<uint4 *>(sz)[i] = make_uint4(0u, 0u, 0u, 0u);
    umma::fence_proxy_async();  // the banded matrices, written by threads, are read by the MMAs
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const unsigned tmem = s_tmem;
    const int nmine = tiles > (int)blockIdx.x ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 0) {
        // ---- loads: tile i into stage i % S once the MMAs of tile i - S are done
        int issued = 0;
        if (lane == 0) {
            for (int i = 0; i < nmine && !s_abort; ++i) {
                const int st = i % kTcStages;
                if (!tma::mbar_wait(&empty[st], ((i / kTcStages) & 1) ^ 1, tma::kLoadWaitNs)) {
                    s_abort = 1;
                    atomicAdd(&g_wait_timeouts, 1u);
                    break;
                }
                const TcTile tl = tc_tile((int)blockIdx.x + i * (int)gridDim.x, tiles_x, tiles_y);
                unsigned char *sa = tc_smem + st * Cfg::A_BYTES;
                tma::mbar_arrive_expect_tx(&full[st], (unsigned)(kTcChunks * SH * 16));
                for (int q = 0; q < kTcChunks; ++q)
                    tma::load_3d(sa + q * Cfg::CHB, &tmap, tl.x0 - 8 + 8 * q, tl.y0 - Cfg::A, tl.plane, &full[st]);
                issued = i + 1;
            }
            // let the last copies of each stage land before the CTA ends
            for (int i = max(0, issued - kTcStages); i < issued; ++i)
                tma::mbar_wait(&full[i % kTcStages], (i / kTcStages) & 1, tma::kLoadWaitNs);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMAs: tile i from stage i % S into accumulator i % 2
        constexpr uint32_t idesc = umma::idesc_f16_f32(kTcM, 64), idesc_z = umma::idesc_f16_f32(kTcM, 256);
        const uint64_t b0 = umma::smem_desc(tma::smem_addr(sb), 1024, 128);
        const uint64_t z0 = umma::smem_desc(tma::smem_addr(sz), 4096, 128);
        int issued = 0;
        for (int i = 0; i < nmine; ++i) {
            const int st = i % kTcStages, ab = i & 1;
            bool ok = !s_abort && tma::mbar_wait(&full[st], (i / kTcStages) & 1, tma::kLoadWaitNs);
            ok = __all_sync(0xffffffffu, ok);
            unsigned char *sa = tc_smem + st * Cfg::A_BYTES;
            const TcTile tl = tc_tile((int)blockIdx.x + i * (int)gridDim.x, tiles_x, tiles_y);
            const int gy0 = tl.y0 - Cfg::A, gx0 = tl.x0 - 8;
            if (ok && CLAMP) {
                // out-of-image rows, then columns, take the nearest edge
                // element -- only the kh/2 rows and kw/2 columns beyond each
                // edge that valid outputs reach; further out the box's zeros
                // meet zero weights of the band
                const int top = -gy0, bot = h - gy0, left = -gx0, right = w - gx0;
                const int nb = bot < SH ? min(SH, bot + Cfg::A) - bot : 0;  // rows below the image to fix
                const int nt = max(0, top);                                 // rows above it (<= kh/2)
                if (nt + nb > 0) {
                    for (int q = lane; q < (nt + nb) * SWC; q += 32) {
                        const int u = q / SWC, c = q - u * SWC;
                        const int r = u < nt ? u : bot + (u - nt);
                        staged<K>(sa, r, c) = staged<K>(sa, u < nt ? top : bot - 1, c);
                    }
                    __syncwarp();
                }
                const int c_lo = left > 0 ? left - Cfg::A : 0;              // columns [8 - kw/2, 8) left of it
                const int nl = left > 0 ? Cfg::A : 0;
                const int nr = right < SWC ? min(SWC, right + Cfg::A) - right : 0;
                if (nl + nr > 0) {
                    for (int q = lane; q < (nl + nr) * SH; q += 32) {
                        const int u = q / SH, r = q - u * SH;
                        const int c = u < nl ? c_lo + u : right + (u - nl);
                        staged<K>(sa, r, c) = staged<K>(sa, r, u < nl ? left : right - 1);
                    }
                }
                umma::fence_proxy_async();
                __syncwarp();
            }
            if (ok) ok = tma::mbar_wait(&acc_empty[ab], ((i >> 1) & 1) ^ 1, tma::kLoadWaitNs);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    s_abort = 1;
                    atomicAdd(&g_wait_timeouts, 1u);
                }
                break;
            }
            umma::fence_after_sync();
            if (lane == 0) {
                const uint64_t a0 = umma::smem_desc(tma::smem_addr(sa), Cfg::CHB, 128);
                const unsigned acc = tmem + kTcAccCols * ab;
                // clear the accumulator (A times a zero B), then every product accumulates:
                // slice c writes block c's first half and block c - 1's second half
                umma::mma_f16(acc, a0, z0, idesc_z, false);
#pragma unroll 1
                for (int a = 0; a < K; ++a) {
                    const uint64_t db = b0 + ((unsigned)(a * 2048) >> 4);
#pragma unroll
                    for (int c = 0; c < kTcSlices; ++c) {
                        const uint64_t da = a0 + ((unsigned)(2 * c * Cfg::CHB + 16 * a) >> 4);
                        umma::mma_f16(acc + 32 * (kTcBlocks - c), da, db, idesc, true);
                    }
                }
                umma::commit(&empty[st]);     // the stage may be refilled
                umma::commit(&acc_full[ab]);  // the accumulator may be read
            }
            issued = i + 1;
            __syncwarp();
        }
        if (lane == 0 && issued > 0) {  // every MMA done before the TMEM is freed
            umma::commit(&fin);
            tma::mbar_wait(&fin, 0, tma::kLoadWaitNs);
        }
        __syncwarp();
    } else {
        // ---- stores: accumulator i % 2 of tile i; warp w owns TMEM lanes
        // 32 (w % 4) .. + 31 (its output rows) and three of the six blocks
        const int quarter = warp & 3, j0 = ((warp - 2) >> 2) * (kTcBlocks / 2);
        for (int i = 0; i < nmine; ++i) {
            const int st = i & 1;
            bool ok = !s_abort && tma::mbar_wait(&acc_full[st], (i >> 1) & 1, tma::kLoadWaitNs);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) {
                    s_abort = 1;
                    atomicAdd(&g_wait_timeouts, 1u);
                }
                break;
            }
            umma::fence_after_sync();
            const TcTile tl = tc_tile((int)blockIdx.x + i * (int)gridDim.x, tiles_x, tiles_y);
            const int row = tl.y0 + 32 * quarter + lane;
            __half *orow = out + ((size_t)tl.plane * h + (size_t)min(row, h - 1)) * (size_t)w;
            const unsigned acc = tmem + kTcAccCols * st + ((unsigned)(32 * quarter) << 16);
            uint32_t r[kTcBlocks / 2][32];  // per block: 16 hi sums, then 16 lo sums
#pragma unroll
            for (int u = 0; u < kTcBlocks / 2; ++u) umma::ld32_async(acc + 32 * (kTcBlocks - (j0 + u)), r[u]);
            umma::wait_ld();
#pragma unroll
            for (int u = 0; u < kTcBlocks / 2; ++u) {
                const int col = tl.x0 + 16 * (j0 + u);
                if (row >= h || col >= w) continue;
                uint32_t p[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float a0 = __uint_as_float(r[u][2 * q]) + __uint_as_float(r[u][16 + 2 * q]);
                    const float a1 = __uint_as_float(r[u][2 * q + 1]) + __uint_as_float(r[u][17 + 2 * q]);
                    p[q] = (uint32_t)__half_as_ushort(__float2half_rn(a0 * unscale)) |
                           ((uint32_t)__half_as_ushort(__float2half_rn(a1 * unscale)) << 16);
                }
                if (col + 16 <= w) {
                    uint4 *d = reinterpret_cast<uint4 *>(orow + col);
                    d[0] = make_uint4(p[0], p[1], p[2], p[3]);
                    d[1] = make_uint4(p[4], p[5], p[6], p[7]);
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (col + q < w)
                            orow[col + q] = __ushort_as_half((unsigned short)(p[q >> 1] >> (16 * (q & 1))));
                }
            }
            umma::fence_before_sync();
            __syncwarp();
            if (lane == 0) umma::arrive(&acc_empty[st]);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        umma::fence_after_sync();
        umma::tmem_free(tmem, kTcTmemCols);
    }
}

int tc_sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

template <int K>
cudaError_t run_tc(int c, int h, int w, const __half *in, const float *k, __half *out, int border,
                   cudaStream_t s, bool *done) {
    using Cfg = TcCfg<K>;
    CUtensorMap tmap;
    *done = false;
    const long long tx = (w + kTcW - 1) / kTcW, ty = (h + kTcM - 1) / kTcM, tiles = tx * ty * c;
    if (tiles > 0x7fffffffll || !image_tensor_map<__half>(&tmap, in, c, h, w, 8, Cfg::SH)) return cudaSuccess;
    auto kern = border == 0 ? conv2d_tc_kernel<K, true> : conv2d_tc_kernel<K, false>;
    // at least 120 KB, so one CTA (and its 512 TMEM columns) per SM: a second
    // one would wait in its TMEM allocation while other SMs stay empty
    const size_t smem = std::max<size_t>(Cfg::smem, 120 * 1024);
    cudaError_t e = set_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<long long>(tiles, tc_sm_count());
    kern<<<grid, kTcThreads, smem, s>>>(tmap, k, out, h, w, (int)tx, (int)ty, (int)tiles);
    *done = true;
    return cudaGetLastError();
}

}  // namespace

// Queue the tensor-core correlation if it applies (binary16, odd side 7..15,
// rows of in and out 16-byte aligned, clamp or zero border); *done says
// whether it was queued.  On 3 x 8192^2 each filter row costs ~0.020 ms of
// MMAs (bound by their shared-memory operand reads) on top of ~0.18 ms per
// launch: 15x15 0.481 ms against 1.542 on the CUDA cores, 9x9 0.360 against
// 0.642, 7x7 0.319 against 0.396.  Sides 3 and 5 stay on the CUDA cores,
// which are faster there (3x3 0.163 ms, about the HBM time).
cudaError_t launch_conv2d_tc(int c, int h, int w, const void *in, int ks, const float *k, void *out, int border,
                             cudaStream_t s, bool *done) {
    *done = false;
    if ((border != 0 && border != 1) || (w % 8) != 0 || ((uintptr_t)in & 15u) != 0 || ((uintptr_t)out & 15u) != 0)
        return cudaSuccess;
    const __half *i = static_cast<const __half *>(in);
    __half *o = static_cast<__half *>(out);
    switch (ks) {
        case 7: return run_tc<7>(c, h, w, i, k, o, border, s, done);
        case 9: return run_tc<9>(c, h, w, i, k, o, border, s, done);
        case 11: return run_tc<11>(c, h, w, i, k, o, border, s, done);
        case 13: return run_tc<13>(c, h, w, i, k, o, border, s, done);
        case 15: return run_tc<15>(c, h, w, i, k, o, border, s, done);
        default: return cudaSuccess;
    }
}

cudaError_t wait_timeouts_tc(unsigned *n, bool clear) { return read_wait_counter(n, clear); }

}  // namespace pencil
