// batch.cu -- many images, each with its own size and filter side, convolved
// by one graph launch, one kernel per filter side.
//
// The host builds a tile table grouped by filter side (within a side, images
// with more tiles first) and a queue header {next, total, start} per side;
// every tile of image i gets the entry i.  Header, image descriptors and
// table are copied to a device buffer owned by the plan.  The graph holds,
// for every side present in the batch, one node of that side's kernel, as
// independent nodes that may run side by side.  Under a persistent variant
// the node is a resident grid (SMs x CTAs per SM) whose CTAs take tile
// indices from the side's `next` with one atomicAdd per tile; under a
// one-tile variant it has one CTA per tile of the side.  Either way a CTA
// looks the image up and runs the same tile body as the standalone direct
// kernel, so every batched pixel is the same bits as pencil_conv2d_ex on that
// image alone.  One kernel per side and tile variant keeps each kernel's code
// small (one tile body) and gives it its own register budget and
// shared-memory slot size, so small filters run more CTAs per SM.  Each side
// of a persistent variant has one or two staging slots (two: the copies of a
// CTA's next tile run while the current one is computed), chosen per side by
// measurement, as is its CTA count per SM.  Kernels read the tile counts
// from the device headers, so the graph captured for a set of sides serves
// every batch with that set (a one-tile node's grid is reset to the run's
// tile count of its side when that changes).
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "conv_tile.cuh"

namespace pencil {
namespace {

using namespace tile;

struct BatchHeader {
    int next;   // next tile of this side's segment to hand out
    int total;  // tiles of this side in the batch
    int start;  // first table entry of the segment
    int pad;
};

struct BatchImage {
    const void *in;
    void *out;
    const float *k;
    int h, w, ks, var;
    int tiles_x, tile_base;
    int vec_ok, pad;
};

constexpr int kSides = 8;   // filter sides 1, 3, ..., 15; side index = ks / 2

// Tile variants, all 128 columns wide; each is its own kernel per side, so
// the tuner chooses tile height, rows per thread, CTA size and schedule per
// side:
//   0: 32-row tiles, 128 threads     2: 64-row tiles, 256 threads
//   1: 16-row tiles, 128 threads     3: 32-row tiles, 256 threads
//   4: as 0, one tile per CTA        5: as 3, one tile per CTA
// Variants 0-3 run a resident grid whose CTAs take tiles from the side's
// queue; 4 and 5 launch one CTA per tile of the side (the grid is set on the
// graph node before each run), so the block scheduler hands out the tiles
// and neighbouring tiles of an image run together, as in the standalone
// kernels.  Sides up to 7 give a thread one 4-column group (32 threads
// across a row), larger sides two groups (16 threads across); the rows per
// thread follow.
__host__ __device__ constexpr int var_th(int v) { return v == 1 ? 16 : (v == 2 ? 64 : 32); }
__host__ __device__ constexpr int var_nt(int v) { return (v == 2 || v == 3 || v == 5) ? 256 : 128; }
__host__ __device__ constexpr bool var_onetile(int v) { return v >= 4; }
constexpr int kTileW = 128;
__host__ __device__ constexpr int btx(int k) { return k <= 7 ? 32 : 16; }
__host__ __device__ constexpr int bg(int k) { return k <= 7 ? 1 : 2; }
__host__ __device__ constexpr int bty(int k, int v) { return var_nt(v) / btx(k); }
__host__ __device__ constexpr int brows(int k, int v) { return var_th(v) / bty(k, v); }
template <int K, int V>
using BCfg = DirectCfg<K, K, btx(K), bty(K, V), brows(K, V), bg(K)>;

// Binary16 sides up to 7 compute from the staged binary16 tile (no FP32 copy;
// the standalone kernels do the same).
__host__ __device__ constexpr bool bhalfw(int k, size_t esz) { return esz == 2 && k <= 7; }
// Rows that are not 16-byte aligned move in the widest copies and stores each
// address allows, except on the FP32 sides from 11, where 4-byte copies and
// scalar stores measured 0.5-2% faster on the 512-image batch (less code
// around their FMA loop).
__host__ __device__ constexpr bool badapt(int k, size_t esz) { return esz == 2 || k <= 9; }

// A staging slot of side K, variant V: filter rows | FP32 tile | binary16
// tile; without the FP32 tile where the binary16 tile is read directly.
template <int K, int V>
struct Slot {
    static constexpr int KF = K * BCfg<K, V>::KWP;  // a multiple of 4 floats
    static constexpr int IN = BCfg<K, V>::SH * BCfg<K, V>::SW;
    __host__ __device__ static constexpr int f16_off(int esz) { return KF + (bhalfw(K, esz) ? 0 : IN); }
    __host__ __device__ static constexpr int floats(int esz) {
        return bhalfw(K, esz) ? KF + IN / 2 : KF + IN + (esz == 2 ? IN / 2 : 0);
    }
};
// Staging slots and CTAs per SM (the register budget, for 128-thread CTAs;
// halved for 256-thread ones) per side, from sweeps on GB300 over the
// 512-image benchmark batch.  Two slots let a CTA's next tile copy while it
// computes the current one; where one slot wins, more resident CTAs hide the
// copies better than the prefetch does.  (A timing sweep may build other
// tables by defining the macros in a header it force-includes.)
#ifndef PENCIL_BATCH_NSLOT
#define PENCIL_BATCH_NSLOT {{2, 1, 1, 1, 1, 1, 2, 1}, {2, 2, 1, 1, 1, 1, 1, 1}}  // FP32, binary16; sides 1..15
#endif
#ifndef PENCIL_BATCH_REGCAP
#define PENCIL_BATCH_REGCAP {{8, 8, 8, 8, 5, 4, 4, 4}, {8, 8, 8, 8, 6, 4, 4, 4}}
#endif
constexpr int kNslot[2][kSides] = PENCIL_BATCH_NSLOT;
constexpr int kRegCap[2][kSides] = PENCIL_BATCH_REGCAP;
template <int K, int V>
constexpr int nslot(size_t esz) { return var_onetile(V) ? 1 : kNslot[esz == 2][K / 2]; }
template <int K, int V>
constexpr size_t batch_smem(size_t esz) {
    return nslot<K, V>(esz) * sizeof(float) * (size_t)Slot<K, V>::floats((int)esz);
}
// CTAs per SM the register budget is sized for: the table's (in 128-thread
// CTAs), or fewer where the shared memory holds fewer.
template <int K, int V>
constexpr int batch_minb(size_t esz) {
    return std::max<int>(1, std::min<int>(kRegCap[esz == 2][K / 2] * 128 / var_nt(V),
                                          (int)((228 * 1024) / (batch_smem<K, V>(esz) + 1024))));
}

// Issue the copies of one tile (filter and halo tile) into a slot; one commit group.
template <typename T, int K, int V>
__device__ __forceinline__ void issue_tile(const BatchImage &d, int y0, int x0, float *slot) {
    using Cfg = BCfg<K, V>;
    stage_filter_async<K, K, Cfg::KWP, Cfg::NT>(d.k, slot);
    stage_issue<T, Cfg::SH, Cfg::SW, Cfg::NT, false, badapt(K, sizeof(T))>(
        static_cast<const T *>(d.in), d.h, d.w, y0 - Cfg::AH, x0 - Cfg::P, d.vec_ok, slot + Slot<K, V>::KF,
        reinterpret_cast<T *>(slot + Slot<K, V>::f16_off(sizeof(T))));
}

// Widen (binary16, unless read directly) and compute one staged tile.
template <typename T, int K, int V>
__device__ __forceinline__ void compute_tile(const BatchImage &d, int y0, int x0, float *slot) {
    using Cfg = BCfg<K, V>;
    const T *s16 = reinterpret_cast<const T *>(slot + Slot<K, V>::f16_off(sizeof(T)));
    if constexpr (bhalfw(K, sizeof(T))) {
        direct_compute<T, K, K, btx(K), bty(K, V), brows(K, V), bg(K), T, badapt(K, sizeof(T))>(
            s16, slot, static_cast<T *>(d.out), d.h, d.w, d.vec_ok, y0, x0);
    } else {
        stage_widen<T, Cfg::SH, Cfg::SW, Cfg::NT>(slot + Slot<K, V>::KF, s16);
        direct_compute<T, K, K, btx(K), bty(K, V), brows(K, V), bg(K), float, badapt(K, sizeof(T))>(
            slot + Slot<K, V>::KF, slot, static_cast<T *>(d.out), d.h, d.w, d.vec_ok, y0, x0);
    }
}

template <int V>
__device__ __forceinline__ void tile_origin(const BatchImage &d, int t, int &y0, int &x0) {
    const int local = t - d.tile_base;
    const int ty = local / d.tiles_x, tx = local - ty * d.tiles_x;
    y0 = ty * var_th(V);
    x0 = tx * kTileW;
}

// The tiles of one filter side under one tile variant.  NSLOT = 2: while
// tile i is computed from one staging slot, the copies of tile i+1 are
// already in flight into the other.  NSLOT = 1: the next tile's copies are
// issued after the compute.
template <typename T, int K, int V, int NSLOT, int MINB>
__global__ void __launch_bounds__(var_nt(V), MINB)
    conv2d_batch_kernel(BatchHeader *__restrict__ hdr, const BatchImage *__restrict__ imgs,
                        const int *__restrict__ tile_img) {
    extern __shared__ __align__(16) float smem[];
    __shared__ int s_next;
    constexpr int SLOT = Slot<K, V>::floats(sizeof(T));
    const int total = hdr->total, start = hdr->start;
    if (threadIdx.x == 0) s_next = atomicAdd(&hdr->next, 1);
    __syncthreads();
    int t = s_next;
    if (t >= total) return;
    __syncthreads();
    if (threadIdx.x == 0) s_next = atomicAdd(&hdr->next, 1);
    BatchImage d = imgs[__ldg(tile_img + start + t)];
    int y0, x0;
    tile_origin<V>(d, start + t, y0, x0);
    issue_tile<T, K, V>(d, y0, x0, smem);
    __syncthreads();
    int tn = s_next;
    for (int i = 0; t < total; ++i) {
        float *cur = smem + (NSLOT == 2 ? (i & 1) * SLOT : 0);
        float *nxt = smem + (NSLOT == 2 ? ((i + 1) & 1) * SLOT : 0);
        BatchImage dn;
        int yn = 0, xn = 0;
        if (tn < total) {
            dn = imgs[__ldg(tile_img + start + tn)];
            tile_origin<V>(dn, start + tn, yn, xn);
        }
        if (NSLOT == 2 && tn < total) {
            issue_tile<T, K, V>(dn, yn, xn, nxt);
            cp_async_wait_prev();  // the current tile's group has landed
        } else {
            cp_async_wait_all();
        }
        __syncthreads();  // every thread has read s_next (end of the previous iteration)
        if (threadIdx.x == 0) s_next = atomicAdd(&hdr->next, 1);
        compute_tile<T, K, V>(d, y0, x0, cur);
        __syncthreads();  // `cur` is free; s_next is visible
        if (NSLOT == 1 && tn < total) issue_tile<T, K, V>(dn, yn, xn, nxt);
        t = tn;
        d = dn;
        y0 = yn;
        x0 = xn;
        tn = s_next;
    }
}

// One tile per CTA: block t of the side's grid computes the side's tile t
// (the grid is exactly the side's tile count).  Same staging and tile body
// as the resident kernel, so the same bits.
template <typename T, int K, int V, int MINB>
__global__ void __launch_bounds__(var_nt(V), MINB)
    conv2d_batch_tile_kernel(BatchHeader *__restrict__ hdr, const BatchImage *__restrict__ imgs,
                             const int *__restrict__ tile_img) {
    extern __shared__ __align__(16) float smem[];
    const int t = blockIdx.x;
    if (t >= hdr->total) return;
    const int start = hdr->start;
    const BatchImage d = imgs[__ldg(tile_img + start + t)];
    int y0, x0;
    tile_origin<V>(d, start + t, y0, x0);
    issue_tile<T, K, V>(d, y0, x0, smem);
    cp_async_wait_all();
    __syncthreads();
    compute_tile<T, K, V>(d, y0, x0, smem);
}

using BatchKernel = void (*)(BatchHeader *, const BatchImage *, const int *);

struct SideKernel {
    BatchKernel fn;
    size_t smem;
    int nt;  // threads per CTA
};

template <typename T, int K, int V>
SideKernel side_kernel() {
    constexpr size_t esz = sizeof(T);
    if constexpr (var_onetile(V))
        return {conv2d_batch_tile_kernel<T, K, V, batch_minb<K, V>(esz)>, batch_smem<K, V>(esz), var_nt(V)};
    else
        return {conv2d_batch_kernel<T, K, V, nslot<K, V>(esz), batch_minb<K, V>(esz)>, batch_smem<K, V>(esz),
                var_nt(V)};
}

template <typename T, int K>
SideKernel side_kernel_v(int v) {
    switch (v) {
        case 0: return side_kernel<T, K, 0>();
        case 1: return side_kernel<T, K, 1>();
        case 2: return side_kernel<T, K, 2>();
        case 3: return side_kernel<T, K, 3>();
        case 4: return side_kernel<T, K, 4>();
        default: return side_kernel<T, K, 5>();
    }
}

template <typename T>
SideKernel side_kernel(int idx, int v) {
    switch (idx) {
        case 0: return side_kernel_v<T, 1>(v);
        case 1: return side_kernel_v<T, 3>(v);
        case 2: return side_kernel_v<T, 5>(v);
        case 3: return side_kernel_v<T, 7>(v);
        case 4: return side_kernel_v<T, 9>(v);
        case 5: return side_kernel_v<T, 11>(v);
        case 6: return side_kernel_v<T, 13>(v);
        default: return side_kernel_v<T, 15>(v);
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace pencil

using namespace pencil;

struct pencil_batch {
    int dtype = PENCIL_F32;
    int max_images = 0;
    long long max_tiles = 0;
    unsigned char var_of_k[16] = {};
    size_t bytes = 0;          // table bytes (device and each host copy)
    void *dbuf = nullptr;      // device: header | images | tile table
    void *hbuf[2] = {nullptr, nullptr};  // pinned host staging (ping-pong)
    cudaEvent_t uploaded[2] = {nullptr, nullptr};
    int flip = 0;
    int sms = 0;                 // SMs of the plan's device
    int grid[kSides] = {};       // resident grid of each side's kernel (0: one CTA per tile)
    size_t smem[kSides] = {};    // its dynamic shared memory
    int nt[kSides] = {};         // its threads per CTA
    BatchKernel fn[kSides] = {};
    // A captured graph per set of sides present.  The graph is kept beside
    // its executable so that the grid of a one-tile-per-CTA node can be set
    // to the tile count of each run.
    struct Captured {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        cudaGraphNode_t node[kSides] = {};
        unsigned grid[kSides] = {};  // grid each node was captured or last set with
    };
    std::map<unsigned, Captured> exec;
    std::mutex mu;
};

namespace {

size_t head_bytes(int max_images) {
    return align256(sizeof(BatchHeader) * kSides) + align256(sizeof(BatchImage) * (size_t)max_images);
}

size_t table_bytes(int max_images, long long max_tiles) {
    return head_bytes(max_images) + sizeof(int) * (size_t)max_tiles;
}

size_t elem_size(int dtype) { return dtype == PENCIL_F16 ? 2 : 4; }

long long tiles_of(const pencil_image &im, int var) {
    const long long ty = (im.h + var_th(var) - 1) / var_th(var);
    const long long tx = (im.w + kTileW - 1) / kTileW;
    return ty * tx;
}

bool image_ok(const pencil_image &im) {
    return im.in && im.out && im.k && im.h > 0 && im.w > 0 && im.ks >= 1 && im.ks <= 15 &&
           (im.ks & 1) && (long long)im.h * im.w <= (1ll << 40);
}

// Every output range must be disjoint from every other output and every input
// and filter range (the restrict rule, per image and across the batch).
bool batch_disjoint(int n, const pencil_image *imgs, size_t esz) {
    struct R { uintptr_t lo, hi; };
    std::vector<R> outs(n), ins;
    ins.reserve(2 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const size_t nb = esz * (size_t)imgs[i].h * imgs[i].w;
        outs[i] = {(uintptr_t)imgs[i].out, (uintptr_t)imgs[i].out + nb};
        ins.push_back({(uintptr_t)imgs[i].in, (uintptr_t)imgs[i].in + nb});
        ins.push_back({(uintptr_t)imgs[i].k, (uintptr_t)imgs[i].k + sizeof(float) * imgs[i].ks * imgs[i].ks});
    }
    std::sort(outs.begin(), outs.end(), [](const R &a, const R &b) { return a.lo < b.lo; });
    for (size_t i = 1; i < outs.size(); ++i)
        if (outs[i].lo < outs[i - 1].hi) return false;
    for (const R &r : ins) {
        // first output starting at or after r.hi cannot overlap; check the one before it
        auto it = std::lower_bound(outs.begin(), outs.end(), r.hi,
                                   [](const R &a, uintptr_t v) { return a.lo < v; });
        if (it != outs.begin() && std::prev(it)->hi > r.lo) return false;
    }
    return true;
}

// Launch parameters of side i's node; a one-tile-per-CTA kernel gets one CTA
// per tile of the side in this run (`tiles`).
cudaKernelNodeParams side_params(const pencil_batch *b, int i, unsigned tiles, void **args) {
    cudaKernelNodeParams p = {};
    p.func = reinterpret_cast<void *>(b->fn[i]);
    p.gridDim = dim3(b->grid[i] > 0 ? (unsigned)b->grid[i] : tiles);
    p.blockDim = dim3((unsigned)b->nt[i]);
    p.sharedMemBytes = (unsigned)b->smem[i];
    p.kernelParams = args;
    return p;
}

// The graph for a set of sides (bit i = side 2i+1): one kernel node per side,
// with no edges between them, so the sides' kernels may run side by side: a
// side whose queue is short (a small wave of requests) leaves SMs to the
// next side at once instead of holding the others back, and at the end of a
// long side the next one fills the SMs it frees.  A resident grid reads its
// tile count from the device header, so its node serves every batch; the
// grid of a one-tile-per-CTA node is set to this run's tile count of its side
// (tiles[i]) whenever that count changes (the update applies to later launches
// of the graph only, never to one already queued).
cudaError_t graph_for(pencil_batch *b, unsigned mask, const unsigned *tiles, cudaGraphExec_t *out) {
    BatchHeader *hdr = static_cast<BatchHeader *>(b->dbuf);
    BatchImage *imgs = reinterpret_cast<BatchImage *>(static_cast<char *>(b->dbuf) +
                                                      align256(sizeof(BatchHeader) * kSides));
    int *tile_img = reinterpret_cast<int *>(static_cast<char *>(b->dbuf) + head_bytes(b->max_images));
    auto it = b->exec.find(mask);
    if (it != b->exec.end()) {
        pencil_batch::Captured &c = it->second;
        for (int i = 0; i < kSides; ++i)
            if ((mask & (1u << i)) && b->grid[i] == 0 && c.grid[i] != tiles[i]) {
                BatchHeader *h = hdr + i;
                void *args[] = {&h, &imgs, &tile_img};
                const cudaKernelNodeParams p = side_params(b, i, tiles[i], args);
                const cudaError_t e = cudaGraphExecKernelNodeSetParams(c.x, c.node[i], &p);
                if (e != cudaSuccess) return e;
                c.grid[i] = tiles[i];
            }
        *out = c.x;
        return cudaSuccess;
    }
    pencil_batch::Captured c;
    cudaError_t e = cudaGraphCreate(&c.g, 0);
    for (int i = kSides - 1; i >= 0 && e == cudaSuccess; --i)
        if (mask & (1u << i)) {
            BatchHeader *h = hdr + i;
            void *args[] = {&h, &imgs, &tile_img};
            const cudaKernelNodeParams p = side_params(b, i, tiles[i], args);
            e = cudaGraphAddKernelNode(&c.node[i], c.g, nullptr, 0, &p);
            c.grid[i] = p.gridDim.x;
        }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c.x, c.g, 0);
    if (e != cudaSuccess) {
        if (c.g) cudaGraphDestroy(c.g);
        return e;
    }
    b->exec[mask] = c;
    *out = c.x;
    return cudaSuccess;
}

void drop_graphs(pencil_batch *b) {
    for (auto &kv : b->exec) {
        cudaGraphExecDestroy(kv.second.x);
        cudaGraphDestroy(kv.second.g);
    }
    b->exec.clear();
}

// Side i runs tile variant v: its kernel, shared memory, CTA size and a
// resident grid of every CTA the SMs hold at once.
cudaError_t load_side(pencil_batch *b, int i, int v) {
    const SideKernel sk = b->dtype == PENCIL_F32 ? side_kernel<float>(i, v) : side_kernel<__half>(i, v);
    cudaError_t e = cudaFuncSetAttribute(sk.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sk.smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sk.fn, sk.nt, sk.smem);
    if (e != cudaSuccess) return e;
    b->fn[i] = sk.fn;
    b->smem[i] = sk.smem;
    b->nt[i] = sk.nt;
    b->grid[i] = var_onetile(v) ? 0 : std::max(1, per_sm) * b->sms;
    return cudaSuccess;
}

void release(pencil_batch *b) {
    drop_graphs(b);
    for (int i = 0; i < 2; ++i) {
        if (b->uploaded[i]) cudaEventDestroy(b->uploaded[i]);
        if (b->hbuf[i]) cudaFreeHost(b->hbuf[i]);
    }
    if (b->dbuf) cudaFree(b->dbuf);
}

}  // namespace

extern "C" {

int pencil_batch_create(int dtype, int max_images, long long max_tiles, pencil_batch **out) {
    if (!out) return PENCIL_ERR_NULL;
    *out = nullptr;
    if ((dtype != PENCIL_F32 && dtype != PENCIL_F16) || max_images <= 0 || max_tiles <= 0 ||
        max_tiles > (1ll << 31) - 1)
        return PENCIL_ERR_ARG;
    pencil_batch *b = new (std::nothrow) pencil_batch;
    if (!b) return PENCIL_ERR_NOMEM;
    b->dtype = dtype;
    b->max_images = max_images;
    b->max_tiles = max_tiles;
    b->bytes = table_bytes(max_images, max_tiles);
    cudaError_t e = cudaMalloc(&b->dbuf, b->bytes);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMallocHost(&b->hbuf[i], b->bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->uploaded[i], cudaEventDisableTiming);
    }
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < kSides && e == cudaSuccess; ++i) e = load_side(b, i, 0);
    if (e != cudaSuccess) {
        release(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? PENCIL_ERR_NOMEM : cuda_fail(e);
    }
    *out = b;
    return PENCIL_OK;
}

int pencil_batch_set_variant(pencil_batch *b, int ks, int variant) {
    if (!b) return PENCIL_ERR_NULL;
    if (ks < 1 || ks > 15 || !(ks & 1) || variant < 0 || variant >= PENCIL_BATCH_VARIANTS)
        return PENCIL_ERR_ARG;
    std::lock_guard<std::mutex> lk(b->mu);
    if (b->var_of_k[ks] == variant) return PENCIL_OK;
    const cudaError_t e = load_side(b, ks / 2, variant);
    if (e != cudaSuccess) return cuda_fail(e);
    b->var_of_k[ks] = (unsigned char)variant;
    drop_graphs(b);  // the captured graphs launch the side's previous kernel
    return PENCIL_OK;
}

int pencil_batch_tiles(const pencil_batch *b, int n, const pencil_image *imgs, long long *tiles) {
    if (!b || !tiles || (n > 0 && !imgs)) return PENCIL_ERR_NULL;
    if (n < 0) return PENCIL_ERR_ARG;
    long long t = 0;
    for (int i = 0; i < n; ++i) {
        if (!image_ok(imgs[i])) return PENCIL_ERR_ARG;
        t += tiles_of(imgs[i], b->var_of_k[imgs[i].ks]);
    }
    *tiles = t;
    return PENCIL_OK;
}

int pencil_batch_run(pencil_batch *b, int n, const pencil_image *imgs, void *stream) {
    if (!b || (n > 0 && !imgs)) return PENCIL_ERR_NULL;
    if (n < 0) return PENCIL_ERR_ARG;
    if (n == 0) return PENCIL_OK;
    if (n > b->max_images) return PENCIL_ERR_NOMEM;
    const size_t esz = elem_size(b->dtype);
    for (int i = 0; i < n; ++i)
        if (!image_ok(imgs[i])) return PENCIL_ERR_ARG;
    if (!batch_disjoint(n, imgs, esz)) return PENCIL_ERR_ALIAS;
    std::lock_guard<std::mutex> lk(b->mu);
    // grouped by filter side (largest first); within a side, more tiles first
    std::vector<int> order(n);
    std::vector<long long> nt(n);
    for (int i = 0; i < n; ++i) {
        order[i] = i;
        nt[i] = tiles_of(imgs[i], b->var_of_k[imgs[i].ks]);
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        if (imgs[x].ks != imgs[y].ks) return imgs[x].ks > imgs[y].ks;
        return nt[x] > nt[y];
    });
    long long total = 0;
    for (int i = 0; i < n; ++i) total += nt[i];
    if (total > b->max_tiles) return PENCIL_ERR_NOMEM;

    const int slot = b->flip;
    b->flip ^= 1;
    cudaError_t e = cudaEventSynchronize(b->uploaded[slot]);  // the copy that last read this staging buffer
    if (e != cudaSuccess) return cuda_fail(e);
    char *h = static_cast<char *>(b->hbuf[slot]);
    BatchHeader *hh = reinterpret_cast<BatchHeader *>(h);
    BatchImage *hi = reinterpret_cast<BatchImage *>(h + align256(sizeof(BatchHeader) * kSides));
    int *ht = reinterpret_cast<int *>(h + head_bytes(b->max_images));
    const int vec = b->dtype == PENCIL_F16 ? 8 : 4;
    for (int i = 0; i < kSides; ++i) hh[i] = BatchHeader{0, 0, 0, 0};
    unsigned mask = 0;
    long long base = 0;
    for (int j = 0; j < n; ++j) {
        const pencil_image &im = imgs[order[j]];
        BatchImage &d = hi[j];
        d.in = im.in;
        d.out = im.out;
        d.k = im.k;
        d.h = im.h;
        d.w = im.w;
        d.ks = im.ks;
        d.var = b->var_of_k[im.ks];
        d.tiles_x = (im.w + kTileW - 1) / kTileW;
        d.tile_base = (int)base;
        d.vec_ok = (im.w % vec == 0) && ((uintptr_t)im.in % 16 == 0) && ((uintptr_t)im.out % 16 == 0);
        d.pad = 0;
        for (long long t = 0; t < nt[order[j]]; ++t) ht[base + t] = j;
        BatchHeader &sh = hh[im.ks / 2];
        if (!(mask & (1u << (im.ks / 2)))) sh.start = (int)base;  // the side's segment begins here
        mask |= 1u << (im.ks / 2);
        sh.total += (int)nt[order[j]];
        base += nt[order[j]];
    }
    unsigned tiles[kSides];
    for (int i = 0; i < kSides; ++i) tiles[i] = (unsigned)hh[i].total;
    cudaGraphExec_t x = nullptr;
    e = graph_for(b, mask, tiles, &x);
    if (e != cudaSuccess) return cuda_fail(e);
    // copy headers + descriptors + the used part of the tile table
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(b->dbuf, h, head_bytes(b->max_images) + sizeof(int) * (size_t)total,
                        cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->uploaded[slot], s);
    if (e == cudaSuccess) e = cudaGraphLaunch(x, s);
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

int pencil_tune(pencil_batch *b, int n, const pencil_image *imgs, int reps, void *stream, int *chosen) {
    if (!b || (n > 0 && !imgs)) return PENCIL_ERR_NULL;
    if (n < 0 || reps < 1) return PENCIL_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!image_ok(imgs[i])) return PENCIL_ERR_ARG;
    if (chosen)
        for (int i = 0; i < kSides; ++i) chosen[i] = -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    int st = ce == cudaSuccess ? PENCIL_OK : cuda_fail(ce);
    std::vector<pencil_image> sub;
    for (int ks = 1; ks <= 15 && st == PENCIL_OK; ks += 2) {
        sub.clear();
        for (int i = 0; i < n; ++i)
            if (imgs[i].ks == ks) sub.push_back(imgs[i]);
        if (sub.empty()) continue;
        float best = 0.0f;
        int best_v = 0;
        for (int v = 0; v < PENCIL_BATCH_VARIANTS && st == PENCIL_OK; ++v) {
            st = pencil_batch_set_variant(b, ks, v);
            if (st == PENCIL_OK) st = pencil_batch_run(b, (int)sub.size(), sub.data(), stream);  // warm-up
            if (st != PENCIL_OK) break;
            ce = cudaEventRecord(e0, (cudaStream_t)stream);
            for (int r = 0; r < reps && ce == cudaSuccess && st == PENCIL_OK; ++r)
                st = pencil_batch_run(b, (int)sub.size(), sub.data(), stream);
            if (ce == cudaSuccess && st == PENCIL_OK) ce = cudaEventRecord(e1, (cudaStream_t)stream);
            if (ce == cudaSuccess && st == PENCIL_OK) ce = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (ce == cudaSuccess && st == PENCIL_OK) ce = cudaEventElapsedTime(&ms, e0, e1);
            if (ce != cudaSuccess) st = cuda_fail(ce);
            if (st == PENCIL_OK && (v == 0 || ms < best)) {
                best = ms;
                best_v = v;
            }
        }
        if (st == PENCIL_OK) st = pencil_batch_set_variant(b, ks, best_v);
        if (st == PENCIL_OK && chosen) chosen[ks / 2] = best_v;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

int pencil_batch_destroy(pencil_batch *b) {
    if (!b) return PENCIL_OK;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2; ++i)
        if (b->uploaded[i]) {
            cudaError_t ei = cudaEventSynchronize(b->uploaded[i]);
            if (e == cudaSuccess) e = ei;
        }
    release(b);
    delete b;
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

}  // extern "C"
