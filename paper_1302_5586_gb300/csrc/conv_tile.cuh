// conv_tile.cuh -- the shared tile body of the direct conv2d kernels
// (standalone and batched).  Every caller computes an output pixel with the
// same FP32 operation order: per filter row a, s = k[a][0]*x0 then
// s = fma(k[a][b], xb, s) for b = 1..kw-1, and acc = acc + s from acc = +0.
#pragma once

#include "internal.cuh"
#include "tma.cuh"

namespace pencil {
namespace tile {

template <typename T>
struct Io;

template <>
struct Io<float> {
    static constexpr int VEC = 4;  // elements per 16-byte chunk
    __device__ __forceinline__ static float ld(const float *p) { return __ldg(p); }
    __device__ __forceinline__ static void ld16(const float *p, float *d) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    }
    __device__ __forceinline__ static void st(float *p, float v) { *p = v; }
    __device__ __forceinline__ static void st4(float *p, const float *v) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    // four values at any 4-byte aligned address: the widest stores it allows
    __device__ __forceinline__ static void st4_any(float *p, const float *v) {
        const unsigned a = (unsigned)(uintptr_t)p;
        if ((a & 15) == 0) {
            st4(p, v);
        } else if ((a & 7) == 0) {
            *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
            *reinterpret_cast<float2 *>(p + 2) = make_float2(v[2], v[3]);
        } else {
            p[0] = v[0]; p[1] = v[1]; p[2] = v[2]; p[3] = v[3];
        }
    }
    __device__ __forceinline__ static void ld16s(const float *p, float *d) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    }
};

template <>
struct Io<__half> {
    static constexpr int VEC = 8;
    __device__ __forceinline__ static float ld(const __half *p) { return __half2float(__ldg(p)); }
    __device__ __forceinline__ static void ld16(const __half *p, float *d) {
        unpack(__ldg(reinterpret_cast<const uint4 *>(p)), d);
    }
    __device__ __forceinline__ static void ld16s(const __half *p, float *d) {
        unpack(*reinterpret_cast<const uint4 *>(p), d);
    }
    __device__ __forceinline__ static void unpack(const uint4 v, float *d) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __half2 hh;
            memcpy(&hh, &w[q], 4);
            const float2 f = __half22float2(hh);
            d[2 * q] = f.x;
            d[2 * q + 1] = f.y;
        }
    }
    __device__ __forceinline__ static void st(__half *p, float v) { *p = __float2half_rn(v); }
    __device__ __forceinline__ static void st4(__half *p, const float *v) {
        const __half2 a = __floats2half2_rn(v[0], v[1]);
        const __half2 b = __floats2half2_rn(v[2], v[3]);
        uint2 u;
        memcpy(&u.x, &a, 4);
        memcpy(&u.y, &b, 4);
        *reinterpret_cast<uint2 *>(p) = u;
    }
    // four values at any 2-byte aligned address: the widest stores it allows
    __device__ __forceinline__ static void st4_any(__half *p, const float *v) {
        const unsigned a = (unsigned)(uintptr_t)p;
        if ((a & 7) == 0) {
            st4(p, v);
        } else if ((a & 3) == 0) {
            *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v[0], v[1]);
            *reinterpret_cast<__half2 *>(p + 2) = __floats2half2_rn(v[2], v[3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) p[c] = __float2half_rn(v[c]);
        }
    }
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Where index i of an axis of length n lands under a border mode, or -1 for a
// zero value: 0 clamp (replicate the edge), 1 zero, 2 reflect (edge repeated,
// period 2n), 3 mirror (edge not repeated, period 2n-2), 4 wrap (period n).
// The periodic modes sit out of line: they are rare and need divisions.
static __device__ __noinline__ int border_index_periodic(int i, int n, int mode) {
    if (mode == 2) {
        const int p = 2 * n, j = ((i % p) + p) % p;
        return j < n ? j : p - 1 - j;
    }
    if (mode == 3) {
        if (n == 1) return 0;
        const int p = 2 * n - 2, j = ((i % p) + p) % p;
        return j < n ? j : p - j;
    }
    return ((i % n) + n) % n;
}

__device__ __forceinline__ int border_index(int i, int n, int mode) {
    if (i >= 0 && i < n) return i;
    if (mode == 0) return clampi(i, 0, n - 1);
    if (mode == 1) return -1;
    return border_index_periodic(i, n, mode);
}

// Stage s[r][c] = in[map(y0 + r)][map(x0 + c)] for r < SH, c < SW (as FP32),
// map = the border mode (clamp-to-edge by default; zero mode stages zeros).
// x0 is a multiple of VEC, SW a multiple of VEC.  Everything goes through
// cp.async (all of a CTA's copies in flight at once).  vec_ok: every row is
// 16-byte aligned (w % VEC == 0 and the plane base 16-byte aligned), so a
// 16-byte chunk inside its row is one 16-byte copy.  Otherwise each chunk
// inside its row takes the widest copies its own address allows (one
// 16-byte, two 8-byte, or -- FP32 -- four 4-byte copies), so rows whose pitch
// is not a multiple of 16 bytes still move mostly in wide copies.  Chunks
// across the image edge take 4-byte copies per element from the column the
// border mode selects (FP32); binary16 chunks that are not 4-byte aligned use
// scalar loads.  FP32 chunks land in s directly; binary16 chunks land in the
// staging area `s16` (widened into s afterwards, unless the caller reads
// s16).  Commits one group.  ANYB = false compiles the clamp-to-edge staging
// only (border ignored).  ADAPT = false leaves out the per-chunk alignment
// tests (rows that are not 16-byte aligned then move in 4-byte copies): for
// compute-bound kernels, where staging is a small part of the time and the
// extra code costs registers; those kernels pass vec_ok at run time.
// CS > 1: an interleaved image of CS channels, staged as one plane of rows of
// w = pixels * CS elements; element q is channel q mod CS of pixel q / CS, and
// the border mode maps the pixel, keeping the channel.
template <typename T, int SH, int SW, int NT, bool ANYB = false, bool ADAPT = true, int CS = 1>
__device__ __forceinline__ void stage_issue(const T *__restrict__ src, int h, int w, int y0, int x0,
                                            bool vec_ok, float *__restrict__ s, T *__restrict__ s16,
                                            int border = 0) {
    constexpr int V = Io<T>::VEC;
    constexpr int CPR = SW / V;
    constexpr bool F16 = sizeof(T) == 2;
    // element column of staged element q under the border mode, or -1 for a zero
    auto col = [&](int q) -> int {
        if constexpr (CS == 1) {
            if constexpr (ANYB) return border_index(q, w, border);
            return clampi(q, 0, w - 1);
        } else {
            const int p = q >= 0 ? q / CS : -((CS - 1 - q) / CS);  // floor(q / CS)
            const int ch = q - p * CS;
            int pc;
            if constexpr (ANYB) pc = border_index(p, w / CS, border);
            else pc = clampi(p, 0, w / CS - 1);
            return pc < 0 ? -1 : pc * CS + ch;
        }
    };
    // chunk q of staged row r
    auto chunk = [&](int r, int q) {
        const int gc = x0 + q * V;
        int gr;
        if constexpr (ANYB) {
            gr = border_index(y0 + r, h, border);
            if (gr < 0) {  // a row of zeros (zero border)
                if (F16) {
#pragma unroll
                    for (int e = 0; e < V; ++e) s16[r * SW + q * V + e] = static_cast<T>(0.0f);
                } else {
                    *reinterpret_cast<float4 *>(s + r * SW + q * V) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                return;
            }
        } else {
            gr = clampi(y0 + r, 0, h - 1);
        }
        const T *row = src + (size_t)gr * (size_t)w;
        const bool inside = gc >= 0 && gc + V <= w;
        const unsigned mis = (unsigned)(uintptr_t)(row + gc) & 15u;
        if (inside && (ADAPT ? (vec_ok || mis == 0) : vec_ok)) {
            if (F16)
                cp_async16(s16 + r * SW + q * V, row + gc);
            else
                cp_async16(s + r * SW + q * V, row + gc);
        } else if (ADAPT && !vec_ok && inside && (mis & 7u) == 0) {
            if (F16) {
                cp_async8(s16 + r * SW + q * V, row + gc);
                cp_async8(s16 + r * SW + q * V + V / 2, row + gc + V / 2);
            } else {
                cp_async8(s + r * SW + q * V, row + gc);
                cp_async8(s + r * SW + q * V + V / 2, row + gc + V / 2);
            }
        } else if (!F16 && inside) {
            // unaligned row, chunk inside it: one 4-byte copy per element at
            // constant offsets from one source and one destination address
            float *d = s + r * SW + q * V;
#pragma unroll
            for (int e = 0; e < V; ++e) cp_async4(d + e, row + gc + e);
        } else if (!F16) {
            // a chunk across the edge: one 4-byte copy per element, from the
            // column the border mode selects
            float *d = s + r * SW + q * V;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int c = col(gc + e);
                if (c < 0)
                    d[e] = 0.0f;
                else
                    cp_async4(d + e, row + c);
            }
        } else if (inside && (mis & 3u) == 0) {
            // binary16 row that is only 4-byte aligned: pairs of elements
            T *d16 = s16 + r * SW + q * V;
#pragma unroll
            for (int e = 0; e < V; e += 2) cp_async4(d16 + e, row + gc + e);
        } else if (inside) {
            // binary16 row aligned to 2 bytes only, chunk inside it
            T *d16 = s16 + r * SW + q * V;
#pragma unroll
            for (int e = 0; e < V; ++e) d16[e] = row[gc + e];
        } else {
            T *d16 = s16 + r * SW + q * V;  // raw binary16 values, widened below
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int c = col(gc + e);
                d16[e] = c < 0 ? static_cast<T>(0.0f) : row[c];
            }
        }
    };
    // A thread keeps one chunk column and steps down the rows (no division
    // per chunk); when a row has more chunks than the CTA has threads, the
    // chunks are dealt out in order.
    constexpr int RPP = NT / CPR;
    if constexpr (RPP >= 1) {
        const int q = threadIdx.x % CPR, r0 = threadIdx.x / CPR;
        if (r0 < RPP)
            for (int r = r0; r < SH; r += RPP) chunk(r, q);
    } else {
        for (int idx = threadIdx.x; idx < SH * CPR; idx += NT) chunk(idx / CPR, idx % CPR);
    }
    cp_async_commit();
}

// After the copies of a staged tile have landed and a barrier: widen a
// binary16 tile into s (no-op for FP32).  Ends with a barrier for binary16.
template <typename T, int SH, int SW, int NT>
__device__ __forceinline__ void stage_widen(float *__restrict__ s, const T *__restrict__ s16) {
    constexpr int V = Io<T>::VEC;
    constexpr int CPR = SW / V;
    if (sizeof(T) == 2) {
        for (int idx = threadIdx.x; idx < SH * CPR; idx += NT) {
            float v[V];
            Io<T>::ld16s(s16 + idx * V, v);
            float *d = s + idx * V;
#pragma unroll
            for (int e = 0; e < V; e += 4)
                *reinterpret_cast<float4 *>(d + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        }
        __syncthreads();
    }
}

// Second half of staging: wait for this thread's copies, then (binary16)
// widen the staged tile into s.  Ends with a barrier.
template <typename T, int SH, int SW, int NT>
__device__ __forceinline__ void stage_finish(float *__restrict__ s, const T *__restrict__ s16) {
    constexpr int V = Io<T>::VEC;
    constexpr int CPR = SW / V;
    cp_async_wait_all();
    if (sizeof(T) == 2) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < SH * CPR; idx += NT) {
            float v[V];
            Io<T>::ld16s(s16 + idx * V, v);
            float *d = s + idx * V;
#pragma unroll
            for (int e = 0; e < V; e += 4)
                *reinterpret_cast<float4 *>(d + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        }
    }
    __syncthreads();
}

// stage_issue followed by stage_finish: the staged tile in s (as FP32), ready
// after the closing barrier.
template <typename T, int SH, int SW, int NT, bool ANYB = false, bool ADAPT = true, int CS = 1>
__device__ __forceinline__ void stage_tile(const T *__restrict__ src, int h, int w, int y0, int x0,
                                           bool vec_ok, float *__restrict__ s, T *__restrict__ s16,
                                           int border = 0) {
    stage_issue<T, SH, SW, NT, ANYB, ADAPT, CS>(src, h, w, y0, x0, vec_ok, s, s16, border);
    stage_finish<T, SH, SW, NT>(s, s16);
}

// ------------------------------------------------------------ row staging
// TMA staging for images whose rows are not 16-byte aligned (a TMA box must
// start on a 16-byte boundary, and a 2-D tensor map needs a row pitch that
// is a multiple of 16 bytes).  The image is seen as one flat array (a 1-D
// tensor map over all its elements) and each staged row is one box of
// LB = SW + V elements, started at the 16-byte boundary at or below the
// row's first staged element: the row lands in a landing row of LP elements
// shifted by its misalignment s (0 <= s < V), which is recorded.  Rows
// outside the image take the edge row (clamp) or none (zero border).  The
// realign pass then moves each landing row into its place in the tile,
// taking the clamp (or zero) for columns outside the image: the tile always
// overlaps the image, so the edge column a clamp reads lies inside the box.
// Elements past either end of the array read as zeros, so no copy leaves the
// allocation.  Planar images (CS = 1) only.
template <typename T, int SH, int SW>
struct RowStage {
    static constexpr int V = 16 / (int)sizeof(T);                 // elements per 16 bytes
    static constexpr int LB = SW + V;                             // box elements
    static constexpr int LP = round_up(LB, 128 / (int)sizeof(T));  // landing row pitch: 128-byte rows
    static constexpr size_t bytes = sizeof(T) * (size_t)SH * LP;
    static_assert(LB <= 256, "a TMA box side is at most 256 elements");
    static_assert(sizeof(T) * (size_t)SH * LB < (1u << 20), "an mbarrier counts fewer than 2^20 bytes");
};

// Issue the boxes of the SH staged rows of a tile whose top-left staged
// element is (gy0, gx0) in plane `plane` (its first flat element), all
// completing `bar`; shift[r] gets row r's misalignment, or -1 for a zero
// row.  Called by the 32 threads of one warp, after `bar` is initialised and
// visible.
template <typename T, int SH, int SW, bool CLAMP>
__device__ __forceinline__ void rows_issue(const CUtensorMap *map, long long plane, int h, int w, int gy0,
                                           int gx0, T *__restrict__ land, int *__restrict__ shift,
                                           uint64_t *bar) {
    using RS = RowStage<T, SH, SW>;
    const int lane = threadIdx.x & 31;
    const int lo = CLAMP ? 0 : max(0, -gy0), hi = CLAMP ? SH : min(SH, h - gy0);
    const int n = max(0, hi - lo);  // boxes issued
    if (lane == 0) tma::mbar_arrive_expect_tx(bar, (unsigned)(n * RS::LB * (int)sizeof(T)));
    __syncwarp();
    for (int r = lane; r < SH; r += 32) {
        int gr = gy0 + r;
        if (CLAMP) {
            gr = clampi(gr, 0, h - 1);
        } else if (gr < 0 || gr >= h) {
            shift[r] = -1;
            continue;
        }
        const long long f = plane + (long long)gr * w + gx0;  // flat index of staged column 0
        const int s = (int)(((f % RS::V) + RS::V) % RS::V);   // floor remainder (f may be negative)
        shift[r] = s;
        tma::load_1d(land + r * RS::LP, map, (int)(f - s), bar);
    }
}

template <typename D, typename T>
__device__ __forceinline__ D row_elem(T v) {
    if constexpr (sizeof(D) == sizeof(T)) return v;
    else return __half2float(v);
}

// After the boxes have landed and a barrier: every landing row into its
// place in the tile (row stride SW), as D (float: widened; T: as stored).
// One warp per row, lanes on consecutive columns (conflict-free).
template <typename T, typename D, int SH, int SW, int NT, bool CLAMP>
__device__ __forceinline__ void rows_realign(const T *__restrict__ land, const int *__restrict__ shift,
                                             D *__restrict__ tile, int w, int gx0) {
    using RS = RowStage<T, SH, SW>;
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const bool inside = gx0 >= 0 && gx0 + SW <= w;  // no staged column outside the image
    for (int r = wp; r < SH; r += NW) {
        const int s = shift[r];
        D *dr = tile + r * SW;
        if (s < 0) {
#pragma unroll
            for (int t = lane; t < SW; t += 32) dr[t] = static_cast<D>(0.0f);
            continue;
        }
        const T *lr = land + r * RS::LP + s;  // lr[t]: the element of staged column t
        if (inside) {
#pragma unroll
            for (int t = lane; t < SW; t += 32) dr[t] = row_elem<D>(lr[t]);
        } else {
#pragma unroll
            for (int t = lane; t < SW; t += 32) {
                const int c = gx0 + t;
                if (CLAMP)
                    dr[t] = row_elem<D>(lr[clampi(c, 0, w - 1) - gx0]);
                else
                    dr[t] = c >= 0 && c < w ? row_elem<D>(lr[t]) : static_cast<D>(0.0f);
            }
        }
    }
}

// The same in place: each landing row shifted to its start, so the tile is
// the landing area with row stride LP.  A warp reads its whole row into
// registers before writing it back.
template <typename T, int SH, int SW, int NT, bool CLAMP>
__device__ __forceinline__ void rows_realign_inplace(T *__restrict__ land, const int *__restrict__ shift, int w,
                                                     int gx0) {
    using RS = RowStage<T, SH, SW>;
    constexpr int NW = NT / 32, NR = (SW + 31) / 32;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const bool inside = gx0 >= 0 && gx0 + SW <= w;
    for (int r = wp; r < SH; r += NW) {
        const int s = shift[r];
        T *lr = land + r * RS::LP;
        T v[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const int t = lane + 32 * j;
            v[j] = static_cast<T>(0.0f);
            if (t < SW && s >= 0) {
                const int c = gx0 + t;
                if (inside)
                    v[j] = lr[s + t];
                else if (CLAMP)
                    v[j] = lr[s + clampi(c, 0, w - 1) - gx0];
                else if (c >= 0 && c < w)
                    v[j] = lr[s + t];
            }
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const int t = lane + 32 * j;
            if (t < SW) lr[t] = v[j];
        }
    }
}

// Write a thread's R x 4 block (rows y, cols x..x+3), bounds-checked.  Rows
// that are not 16-byte aligned: the widest stores each address allows
// (ADAPT), or scalar stores.
template <typename T, int R, bool ADAPT = true>
__device__ __forceinline__ void store_block(T *__restrict__ dst, int h, int w, int y, int x,
                                            bool vec_ok, const float (&acc)[R][4]) {
#pragma unroll
    for (int o = 0; o < R; ++o) {
        const int i = y + o;
        if (i >= h) break;
        T *row = dst + (size_t)i * (size_t)w;
        if (vec_ok && x + 4 <= w) {
            Io<T>::st4(row + x, acc[o]);
        } else if (ADAPT && x + 4 <= w) {
            Io<T>::st4_any(row + x, acc[o]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (x + c < w) Io<T>::st(row + x + c, acc[o][c]);
        }
    }
}

// ------------------------------------------------------------ direct kernel
// Tile: TH = TY*R output rows by TW = G*TX*4 columns.  A thread owns R rows and
// G groups of 4 adjacent columns; group g starts TX*4*g columns after group 0,
// so the loads of a warp stay contiguous (conflict-free LDS.128) in every group.
// CS > 1: columns are elements of an interleaved image of CS channels; tap b
// of an element lies b*CS elements further, so the halo is AW*CS elements.
// C_: adjacent columns per group (a multiple of 4): wider groups share one
// window load among more outputs, which pays where the taps are CS apart.
template <int KH, int KW, int TX, int TY, int R, int G, int CS_ = 1, int C_ = 4>
struct DirectCfg {
    static constexpr int C = C_;
    static_assert(C_ % 4 == 0, "groups of whole 16-byte chunks");
    static constexpr int CS = CS_;
    static constexpr int AH = KH / 2, AW = KW / 2;
    static constexpr int AWE = AW * CS;             // left halo in elements
    static constexpr int NT = TX * TY;
    static constexpr int GS = TX * C;               // column stride between groups
    static constexpr int TW = G * GS, TH = TY * R;
    static constexpr int P = round_up(AWE, 8);      // left halo, 16-byte aligned for f32 and f16
    static constexpr int SW = TW + 2 * P;
    static constexpr int SH = TH + KH - 1;
    static constexpr int KWP = round_up(KW, 4);     // filter row padded to LDS.128
    static constexpr size_t smem_f32 = sizeof(float) * (size_t)(SH * SW + KH * KWP);
    // binary16 staging area appended for FP16 images
    static constexpr size_t smem(size_t esz) { return smem_f32 + (esz == 2 ? 2 * (size_t)SH * SW : 0); }
    // binary16 tile read as staged (no FP32 copy): filter rows, then the tile
    static constexpr size_t smem_half = sizeof(float) * (size_t)(KH * KWP) + 2 * (size_t)SH * SW;
};

// Four consecutive staged values as FP32: one LDS.128 from an FP32 tile, or
// one LDS.64 from a binary16 tile widened in registers (exact).  p is 16-byte
// (FP32) or 8-byte (binary16) aligned.
__device__ __forceinline__ void ld4s(const float *p, float *d) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
}
__device__ __forceinline__ void ld4s(const __half *p, float *d) {
    const uint2 v = *reinterpret_cast<const uint2 *>(p);
    __half2 lo, hi;
    memcpy(&lo, &v.x, 4);
    memcpy(&hi, &v.y, 4);
    const float2 a = __half22float2(lo), b = __half22float2(hi);
    d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
}

// One staged input row r applied to every output row o that uses it (filter
// row a = r - o).  CHECK tests a against [0, KH); for a compile-time r the test
// folds away.
template <bool CHECK, int R, int G, int GS, int KH, int KW, int KWP, int NX, int B0, typename S, int CS = 1,
          int C = 4>
__device__ __forceinline__ void direct_row(int r, const S *__restrict__ xrow,
                                           const float *__restrict__ s_k, float (&acc)[R][G * C]) {
    float x[G][NX];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int m = 0; m < NX; m += 4) ld4s(xrow + g * GS + m, &x[g][m]);
#pragma unroll
    for (int o = 0; o < R; ++o) {
        const int a = r - o;
        if (!CHECK || (a >= 0 && a < KH)) {
            float kr[KWP];
#pragma unroll
            for (int m = 0; m < KWP; m += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(s_k + a * KWP + m);
                kr[m] = v.x; kr[m + 1] = v.y; kr[m + 2] = v.z; kr[m + 3] = v.w;
            }
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    float sum = __fmul_rn(kr[0], x[g][B0 + c]);
#pragma unroll
                    for (int b = 1; b < KW; ++b) sum = __fmaf_rn(kr[b], x[g][B0 + c + b * CS], sum);
                    acc[o][g * C + c] = __fadd_rn(acc[o][g * C + c], sum);
                }
        }
    }
}

// The R x (G*4) block of output sums whose taps start at srow (row stride SW;
// tap (a, b) of column c of group g is srow[a * SW + g * GS + B0 + c + b]),
// from zero, in the documented order.  Each staged row is read from the
// aligned group of four values that holds tap 0 of column 0 onwards, only as
// far as the taps of column 3 reach.  S: the staged type (FP32, or binary16
// widened as it is read).  CS: element distance between taps (the channels
// of an interleaved image).
template <int KH, int KW, int R, int G, int GS, int SW, int KWP, int B0_, typename S = float, int CS = 1,
          int C = 4>
__device__ __forceinline__ void direct_accumulate(const S *__restrict__ srow_,
                                                  const float *__restrict__ s_k, float (&acc)[R][G * C]) {
    constexpr int M0 = B0_ & ~3, B0 = B0_ - M0;
    constexpr int NX = round_up(B0 + C + (KW - 1) * CS, 4);
    const S *srow = srow_ + M0;
#pragma unroll
    for (int o = 0; o < R; ++o)
#pragma unroll
        for (int c = 0; c < G * C; ++c) acc[o][c] = 0.0f;

    // Rows r < R-1 and r >= KH feed only some output rows: fully unrolled, so
    // the validity tests are resolved at compile time.  Rows R-1 <= r <= KH-1
    // feed every output row: that loop has no branches.
    constexpr int NR = R + KH - 1;
    constexpr int PRO = (R - 1 < NR) ? R - 1 : NR;
    constexpr int EPI = (KH > PRO) ? KH : PRO;
#pragma unroll
    for (int r = 0; r < PRO; ++r)
        direct_row<true, R, G, GS, KH, KW, KWP, NX, B0, S, CS, C>(r, srow + r * SW, s_k, acc);
#pragma unroll 1
    for (int r = PRO; r < EPI; ++r)
        direct_row<false, R, G, GS, KH, KW, KWP, NX, B0, S, CS, C>(r, srow + r * SW, s_k, acc);
#pragma unroll
    for (int r = EPI; r < NR; ++r)
        direct_row<true, R, G, GS, KH, KW, KWP, NX, B0, S, CS, C>(r, srow + r * SW, s_k, acc);
}

// Compute and store one TH x TW output tile with origin (y0, x0) from a
// staged tile s_in (see stage_tile; FP32, or the binary16 staging area read
// directly) and staged filter rows s_k.
// PITCH: the staged tile's row stride, when it is wider than SW.
template <typename T, int KH, int KW, int TX, int TY, int R, int G, typename S = float, bool ADAPT = true,
          int CS = 1, int C_ = 4, int PITCH = 0>
__device__ __forceinline__ void direct_compute(const S *__restrict__ s_in,
                                               const float *__restrict__ s_k, T *__restrict__ dst,
                                               int h, int w, bool vec_ok, int y0, int x0) {
    using Cfg = DirectCfg<KH, KW, TX, TY, R, G, CS, C_>;
    constexpr int C = Cfg::C, P = Cfg::P, SW = PITCH ? PITCH : Cfg::SW, KWP = Cfg::KWP, GS = Cfg::GS;
    constexpr int B0 = P - Cfg::AWE;  // x index of tap 0 for column 0
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    float acc[R][G * C];
    direct_accumulate<KH, KW, R, G, GS, SW, KWP, B0, S, CS, C>(s_in + (ty * R) * SW + tx * C, s_k, acc);

#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
            float blk[R][4];
#pragma unroll
            for (int o = 0; o < R; ++o)
#pragma unroll
                for (int c = 0; c < 4; ++c) blk[o][c] = acc[o][g * C + q * 4 + c];
            store_block<T, R, ADAPT>(dst, h, w, y0 + ty * R, x0 + g * GS + tx * C + q * 4, vec_ok, blk);
        }
}

// Filter rows into shared memory with 4-byte cp.async (part of the caller's
// next commit group), each padded with zeros to KWP.
template <int KH, int KW, int KWP, int NT>
__device__ __forceinline__ void stage_filter_async(const float *__restrict__ k, float *__restrict__ s_k) {
    for (int t = threadIdx.x; t < KH * KWP; t += NT) {
        const int a = t / KWP, b = t - a * KWP;
        if (b < KW)
            cp_async4(s_k + t, k + a * KW + b);
        else
            s_k[t] = 0.0f;
    }
}

// Filter rows into shared memory, each padded with zeros to KWP.
template <int KH, int KW, int KWP, int NT>
__device__ __forceinline__ void stage_filter(const float *__restrict__ k, float *__restrict__ s_k) {
    for (int t = threadIdx.x; t < KH * KWP; t += NT) {
        const int a = t / KWP, b = t - a * KWP;
        s_k[t] = b < KW ? __ldg(k + a * KW + b) : 0.0f;
    }
}

// One TH x TW output tile with origin (y0, x0) of one plane: stage, compute,
// store.  Called by every thread of an NT-thread block (it contains barriers);
// `smem` must hold DirectCfg::smem(sizeof(T)) bytes, or DirectCfg::smem_half
// for HALFW.  HALFW (binary16 images): the tile stays binary16 in shared
// memory and is widened as the windows are read -- half the shared-memory
// traffic of an FP32 copy, for sides where that traffic is the limit.
template <typename T, int KH, int KW, int TX, int TY, int R, int G, bool ANYB = false, bool HALFW = false,
          bool ADAPT = true, int CS = 1, int C = 4>
__device__ __forceinline__ void direct_tile(const T *__restrict__ src, const float *__restrict__ k,
                                            T *__restrict__ dst, int h, int w, bool vec_ok, int y0,
                                            int x0, float *__restrict__ smem, int border = 0) {
    using Cfg = DirectCfg<KH, KW, TX, TY, R, G, CS, C>;
    constexpr int SW = Cfg::SW, SH = Cfg::SH, KWP = Cfg::KWP, AH = Cfg::AH, P = Cfg::P;
    if constexpr (HALFW) {
        static_assert(sizeof(T) == 2, "HALFW reads a binary16 tile");
        float *s_k = smem;
        T *s16 = reinterpret_cast<T *>(smem + KH * KWP);
        stage_filter<KH, KW, KWP, Cfg::NT>(k, s_k);
        stage_issue<T, SH, SW, Cfg::NT, ANYB, ADAPT, CS>(src, h, w, y0 - AH, x0 - P, vec_ok, nullptr, s16, border);
        cp_async_wait_all();
        __syncthreads();
        direct_compute<T, KH, KW, TX, TY, R, G, T, ADAPT, CS, C>(s16, s_k, dst, h, w, vec_ok, y0, x0);
    } else {
        float *s_in = smem;
        float *s_k = smem + SH * SW;
        T *s16 = reinterpret_cast<T *>(smem + SH * SW + KH * KWP);
        stage_filter<KH, KW, KWP, Cfg::NT>(k, s_k);
        stage_tile<T, SH, SW, Cfg::NT, ANYB, ADAPT, CS>(src, h, w, y0 - AH, x0 - P, vec_ok, s_in, s16, border);
        direct_compute<T, KH, KW, TX, TY, R, G, float, ADAPT, CS, C>(s_in, s_k, dst, h, w, vec_ok, y0, x0);
    }
}

}  // namespace tile
}  // namespace pencil
