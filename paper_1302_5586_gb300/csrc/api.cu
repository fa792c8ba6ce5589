// api.cu -- the C ABI of libpencilgpu: argument checks, the restrict rule,
// memory-kind checks, the scratch pool of the plain calls, and dispatch.
#include <algorithm>
#include <mutex>
#include <string.h>

#include "internal.cuh"

namespace pencil {

static thread_local int g_last_cuda = 0;

int cuda_fail(cudaError_t e) {
    g_last_cuda = (int)e;
    return PENCIL_ERR_CUDA;
}

namespace {

// Where a pointer lives.  Unregistered host memory is reported as
// cudaMemoryTypeUnregistered by cudaPointerGetAttributes.
enum class Mem { Device, Host, Invalid };

Mem kind_of(const void *p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return Mem::Invalid;
    }
    switch (a.type) {
        case cudaMemoryTypeDevice:
        case cudaMemoryTypeManaged: return Mem::Device;
        default: return Mem::Host;
    }
}

bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return na && nb && x < y + nb && y < x + na;
}

size_t elem_size(int dtype) { return dtype == PENCIL_F16 ? 2 : 4; }

// Plain calls' scratch: grow-only device buffers, the library's copy
// streams, one mutex (plain calls are serialised).
constexpr int kSlots = 16;
constexpr int kBandStreams = 3;

struct Pool {
    std::mutex mu;
    void *buf[kSlots] = {};
    size_t cap[kSlots] = {};
    cudaStream_t streams[kBandStreams] = {};

    // Returns a device buffer of >= bytes in slot i, or nullptr.
    void *get(int i, size_t bytes) {
        if (cap[i] >= bytes) return buf[i];
        if (buf[i]) cudaFree(buf[i]);
        buf[i] = nullptr;
        cap[i] = 0;
        if (cudaMalloc(&buf[i], bytes) != cudaSuccess) {
            cudaGetLastError();
            buf[i] = nullptr;
            return nullptr;
        }
        cap[i] = bytes;
        return buf[i];
    }
    cudaStream_t stream(int i) {
        if (!streams[i] && cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            streams[i] = nullptr;
        }
        return streams[i];
    }
    // A stream-ordered allocation pool per device for temporaries of
    // stream-ordered calls; it keeps its memory for reuse (release threshold
    // = unlimited) until pencil_shutdown, and leaves the device's default pool
    // alone.  Caller holds mu.
    static constexpr int kMaxDev = 64;
    cudaMemPool_t mpool[kMaxDev] = {};
    cudaMemPool_t stream_pool() {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
            cudaGetLastError();
            return nullptr;
        }
        if (!mpool[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if (cudaMemPoolCreate(&mpool[dev], &props) != cudaSuccess) {
                cudaGetLastError();
                mpool[dev] = nullptr;
                return nullptr;
            }
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(mpool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        return mpool[dev];
    }
    void release() {
        for (int d = 0; d < kMaxDev; ++d) {
            if (mpool[d]) cudaMemPoolDestroy(mpool[d]);  // freed once its last block is
            mpool[d] = nullptr;
        }
        for (int i = 0; i < kSlots; ++i) {
            if (buf[i]) cudaFree(buf[i]);
            buf[i] = nullptr;
            cap[i] = 0;
        }
        for (int i = 0; i < kBandStreams; ++i) {
            if (streams[i]) cudaStreamDestroy(streams[i]);
            streams[i] = nullptr;
        }
    }
};

Pool &pool() {
    static Pool p;
    return p;
}

int check_dims(int h, int w) {
    if (h <= 0 || w <= 0) return PENCIL_ERR_ARG;
    if ((int64_t)h * (int64_t)w > ((int64_t)1 << 40)) return PENCIL_ERR_ARG;
    if (h > PENCIL_MAX_ROWS) return PENCIL_ERR_UNSUPPORTED;
    return PENCIL_OK;
}

// A plain-call convolution whose image is in host memory (or mixed): the
// output rows are processed in bands of `band` rows.  A band's input rows,
// widened by the filter's halo (ht rows above, hb below, cut at the image
// edges), are copied into a staging buffer and convolved as a sub-image; the
// band's own rows are copied back.  Inside the sub-image every window of a
// band row reads the same rows as in the whole image (the halo rows are real
// rows; at the true edges the sub-image edge is the image edge), so the
// result is the same bits as one launch over the whole image.  Bands rotate
// over the library's streams, so one band's copies overlap another's kernel.
// The caller holds the pool mutex.  `launch(in, out, h_sub, stream)`.
template <typename Launch>
int banded(int h, int w, int ht, int hb, const float *in, float *out, Launch launch) {
    // a device-memory argument may still be written by earlier work on any
    // stream: a plain call starts from a finished device
    PENCIL_CUDA_TRY(cudaDeviceSynchronize());
    const size_t row = sizeof(float) * (size_t)w;
    int band = (int)std::max<size_t>(32, ((size_t)16 << 20) / row);
    band = std::min(band, h);
    const size_t stage = row * (size_t)(band + ht + hb);
    cudaStream_t st[kBandStreams];
    float *din[kBandStreams], *dout[kBandStreams];
    for (int i = 0; i < kBandStreams; ++i) {
        st[i] = pool().stream(i);
        din[i] = static_cast<float *>(pool().get(4 + 2 * i, stage));
        dout[i] = static_cast<float *>(pool().get(5 + 2 * i, stage));
        if (!st[i]) return cuda_fail(cudaErrorUnknown);
        if (!din[i] || !dout[i]) return PENCIL_ERR_NOMEM;
    }
    int b = 0;
    for (int r0 = 0; r0 < h; r0 += band, ++b) {
        const int r1 = std::min(h, r0 + band);
        const int i0 = std::max(0, r0 - ht), i1 = std::min(h, r1 + hb);
        const int k = b % kBandStreams;
        PENCIL_CUDA_TRY(cudaMemcpyAsync(din[k], in + (size_t)i0 * w, row * (size_t)(i1 - i0),
                                        cudaMemcpyDefault, st[k]));
        PENCIL_CUDA_TRY(launch(din[k], dout[k], i1 - i0, st[k]));
        PENCIL_CUDA_TRY(cudaMemcpyAsync(out + (size_t)r0 * w, dout[k] + (size_t)(r0 - i0) * w,
                                        row * (size_t)(r1 - r0), cudaMemcpyDefault, st[k]));
    }
    for (int i = 0; i < kBandStreams; ++i) PENCIL_CUDA_TRY(cudaStreamSynchronize(st[i]));
    return PENCIL_OK;
}

}  // namespace
}  // namespace pencil

using namespace pencil;

extern "C" {

const char *pencil_strerror(int status) {
    switch (status) {
        case PENCIL_OK: return "ok";
        case PENCIL_ERR_ARG: return "invalid size or flag";
        case PENCIL_ERR_NULL: return "null pointer";
        case PENCIL_ERR_ALIAS: return "output overlaps an input (restrict rule)";
        case PENCIL_ERR_PTR: return "host memory where device memory is required";
        case PENCIL_ERR_NOMEM: return "workspace too small or device allocation failed";
        case PENCIL_ERR_CUDA: return "CUDA error (see pencil_last_cuda_error)";
        case PENCIL_ERR_TIMEOUT: return "bounded wait expired";
        case PENCIL_ERR_UNSUPPORTED: return "valid request the library does not implement";
        default: return "unknown status";
    }
}

// 0.2.0: interleaved layouts, the conv -> Jacobi chain, four batch tile variants.
int pencil_version(void) { return 200; }

int pencil_device_info(char *name, int len, int *sm_count, int *driver_version) {
    int dev = 0;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (name && len > 0) {
        strncpy(name, prop.name, (size_t)len - 1);
        name[len - 1] = 0;
    }
    if (sm_count) *sm_count = prop.multiProcessorCount;
    if (driver_version) {
        e = cudaDriverGetVersion(driver_version);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return PENCIL_OK;
}

int pencil_last_cuda_error(void) { return g_last_cuda; }

int pencil_device_status(void) {
    unsigned n = 0, m = 0;
    unsigned q = 0, r = 0, t = 0;
    cudaError_t e = wait_timeouts(&n, true);
    if (e == cudaSuccess) e = wait_timeouts_hwc(&m, true);
    if (e == cudaSuccess) e = wait_timeouts_cj(&q, true);
    if (e == cudaSuccess) e = wait_timeouts_chain(&r, true);
    if (e == cudaSuccess) e = wait_timeouts_tc(&t, true);
    if (e != cudaSuccess) return cuda_fail(e);
    return n + m + q + r + t ? PENCIL_ERR_TIMEOUT : PENCIL_OK;
}

int pencil_selftest_wait_timeout(unsigned limit_us, int *completed) {
    if (!completed) return PENCIL_ERR_NULL;
    if (limit_us == 0 || limit_us > 1000000) return PENCIL_ERR_ARG;
    cudaError_t e = wait_selftest((uint64_t)limit_us * 1000ull, completed);
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

void pencil_shutdown(void) {
    std::lock_guard<std::mutex> lk(pool().mu);
    pool().release();
}

// Interleaved images: one row of w pixels is w*c elements, an int in the kernels.
int check_layout(int c, int w, int flags) {
    if ((flags & PENCIL_LAYOUT_HWC) && (int64_t)w * c > INT32_MAX) return PENCIL_ERR_UNSUPPORTED;
    return PENCIL_OK;
}

int pencil_conv2d_ex(int c, int h, int w, const void *in, int kh, int kw, const float *k, void *out,
                     int dtype, int flags, void *stream) {
    const int border = (flags >> 8) & 0xF;
    if (c <= 0 || kh <= 0 || kw <= 0 ||
        (flags & ~(PENCIL_CONV_GENERIC | PENCIL_LAYOUT_HWC | PENCIL_CONV_TENSOR | 0xF00)) != 0 ||
        border > PENCIL_BORDER_WRAP)
        return PENCIL_ERR_ARG;
    if (dtype != PENCIL_F32 && dtype != PENCIL_F16) return PENCIL_ERR_ARG;
    int st = check_dims(h, w);
    if (st) return st;
    if (c > PENCIL_MAX_CHANNELS) return PENCIL_ERR_UNSUPPORTED;
    if ((st = check_layout(c, w, flags))) return st;
    if (!in || !k || !out) return PENCIL_ERR_NULL;
    const size_t nb = (size_t)c * h * w * elem_size(dtype);
    if (overlaps(out, nb, in, nb) || overlaps(out, nb, k, sizeof(float) * (size_t)kh * kw))
        return PENCIL_ERR_ALIAS;
    if (kind_of(in) != Mem::Device || kind_of(out) != Mem::Device || kind_of(k) != Mem::Device)
        return PENCIL_ERR_PTR;
    const cudaStream_t s = (cudaStream_t)stream;
    const bool generic = flags & PENCIL_CONV_GENERIC;
    cudaError_t e;
    const bool hwc = (flags & PENCIL_LAYOUT_HWC) && c > 1;  // one channel interleaved is the planar layout
    if ((flags & PENCIL_CONV_TENSOR) && dtype == PENCIL_F16 && !generic && !hwc && kh == kw) {
        bool done = false;
        e = launch_conv2d_tc(c, h, w, in, kh, k, out, border, s, &done);
        if (e != cudaSuccess) return cuda_fail(e);
        if (done) return PENCIL_OK;
    }
    if (hwc)
        e = generic ? launch_conv2d_hwc_generic(dtype, c, h, w, in, kh, kw, k, out, s, border)
                    : launch_conv2d_hwc(dtype, c, h, w, in, kh, kw, k, out, s, border);
    else
        e = generic ? launch_conv2d_generic(dtype, c, h, w, in, kh, kw, k, out, s, border)
                    : launch_conv2d(dtype, c, h, w, in, kh, kw, k, out, s, border);
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

int pencil_conv2d_sep_ex(int c, int h, int w, const void *in, int kx, const float *gx, int ky,
                         const float *gy, void *out, int dtype, int flags, void *stream) {
    const int border = (flags >> 8) & 0xF;
    if (c <= 0 || kx <= 0 || ky <= 0 || (flags & ~(PENCIL_LAYOUT_HWC | 0xF00)) != 0 || border > PENCIL_BORDER_WRAP)
        return PENCIL_ERR_ARG;
    if (dtype != PENCIL_F32 && dtype != PENCIL_F16) return PENCIL_ERR_ARG;
    int st = check_dims(h, w);
    if (st) return st;
    if (c > PENCIL_MAX_CHANNELS) return PENCIL_ERR_UNSUPPORTED;
    if ((st = check_layout(c, w, flags))) return st;
    if (!in || !gx || !gy || !out) return PENCIL_ERR_NULL;
    if (kx > PENCIL_MAX_SPECIALISED_K || ky > PENCIL_MAX_SPECIALISED_K) return PENCIL_ERR_UNSUPPORTED;
    const size_t nb = (size_t)c * h * w * elem_size(dtype);
    if (overlaps(out, nb, in, nb) || overlaps(out, nb, gx, sizeof(float) * kx) ||
        overlaps(out, nb, gy, sizeof(float) * ky))
        return PENCIL_ERR_ALIAS;
    if (kind_of(in) != Mem::Device || kind_of(out) != Mem::Device || kind_of(gx) != Mem::Device ||
        kind_of(gy) != Mem::Device)
        return PENCIL_ERR_PTR;
    cudaError_t e = (flags & PENCIL_LAYOUT_HWC) && c > 1
                        ? launch_conv2d_sep_hwc(dtype, c, h, w, in, kx, gx, ky, gy, out, (cudaStream_t)stream, border)
                        : launch_conv2d_sep(dtype, c, h, w, in, kx, gx, ky, gy, out, (cudaStream_t)stream, border);
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

int pencil_conv2d_jacobi(int c, int h, int w, const float *in, int kh, int kw, const float *k, int sweeps,
                         float *out, int flags, void *stream) {
    if (c <= 0 || kh <= 0 || kw <= 0 || sweeps < 0 || (flags & ~PENCIL_CHAIN_FUSED) != 0) return PENCIL_ERR_ARG;
    int st = check_dims(h, w);
    if (st) return st;
    if (c > PENCIL_MAX_CHANNELS) return PENCIL_ERR_UNSUPPORTED;
    if (!in || !k || !out) return PENCIL_ERR_NULL;
    const size_t plane = (size_t)h * w, nb = sizeof(float) * (size_t)c * plane;
    if (overlaps(out, nb, in, nb) || overlaps(out, nb, k, sizeof(float) * (size_t)kh * kw)) return PENCIL_ERR_ALIAS;
    if (kind_of(in) != Mem::Device || kind_of(out) != Mem::Device || kind_of(k) != Mem::Device)
        return PENCIL_ERR_PTR;
    const bool fusable = sweeps > 0 && conv_jacobi_fusable(h, w, kh, kw, in, out);
    if ((flags & PENCIL_CHAIN_FUSED) && !fusable) return PENCIL_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    int done = 0;  // sweeps already applied
    if (fusable) {
        done = std::min(sweeps, kConvJacobiMaxSweeps);
        e = launch_conv_jacobi_fused(c, h, w, in, kh, k, done, out, s);
    } else {
        e = launch_conv2d(PENCIL_F32, c, h, w, in, kh, kw, k, out, s);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    if (done == sweeps || h < 3 || w < 3) return PENCIL_OK;
    // the remaining sweeps, per channel, through a stream-ordered workspace
    const size_t wsb = jacobi_workspace_bytes(h, w);
    void *ws = nullptr;
    cudaMemPool_t mp = nullptr;
    {
        std::lock_guard<std::mutex> lk(pool().mu);
        mp = pool().stream_pool();
    }
    if (!mp) return PENCIL_ERR_NOMEM;
    e = cudaMallocFromPoolAsync(&ws, wsb, mp, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return PENCIL_ERR_NOMEM;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    for (int ch = 0; ch < c && e == cudaSuccess; ++ch)
        e = jacobi_run(h, w, out + ch * plane, sweeps - done, 0, nullptr, ws, wsb, 0, s);
    const cudaError_t ef = cudaFreeAsync(ws, s);
    if (e == cudaSuccess) e = ef;
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

int pencil_conv2d_chain(int c, int h, int w, const void *in, int kh1, int kw1, const float *k1, int kh2,
                        int kw2, const float *k2, void *out, int dtype, int flags, void *stream) {
    if (c <= 0 || kh1 <= 0 || kw1 <= 0 || kh2 <= 0 || kw2 <= 0 ||
        (flags & ~(PENCIL_CONV_GENERIC | PENCIL_CHAIN_FUSED | 0xF00)) != 0 ||
        ((flags >> 8) & 0xF) > PENCIL_BORDER_WRAP)
        return PENCIL_ERR_ARG;
    if (dtype != PENCIL_F32 && dtype != PENCIL_F16) return PENCIL_ERR_ARG;
    if ((flags >> 8) & 0xF) return PENCIL_ERR_UNSUPPORTED;  // clamp-to-edge only
    int st = check_dims(h, w);
    if (st) return st;
    if (c > PENCIL_MAX_CHANNELS) return PENCIL_ERR_UNSUPPORTED;
    if (!in || !k1 || !k2 || !out) return PENCIL_ERR_NULL;
    if (chain_generic_smem(kh2, kw2) > 200 * 1024) return PENCIL_ERR_UNSUPPORTED;
    const size_t nb = (size_t)c * h * w * elem_size(dtype);
    if (overlaps(out, nb, in, nb) || overlaps(out, nb, k1, sizeof(float) * (size_t)kh1 * kw1) ||
        overlaps(out, nb, k2, sizeof(float) * (size_t)kh2 * kw2))
        return PENCIL_ERR_ALIAS;
    if (kind_of(in) != Mem::Device || kind_of(out) != Mem::Device || kind_of(k1) != Mem::Device ||
        kind_of(k2) != Mem::Device)
        return PENCIL_ERR_PTR;
    cudaStream_t s = (cudaStream_t)stream;
    // fusion wins only for two 3x3 filters (measured on GB300 at 8192 x 8192 x 3:
    // 0.39 vs 0.46 ms; from 5x5 up two passes are faster)
    const bool fuse = (flags & (PENCIL_CONV_GENERIC | PENCIL_CHAIN_FUSED)) != 0 ||
                      (kh1 == 3 && kw1 == 3 && kh2 == 3 && kw2 == 3);
    if (fuse) {
        cudaError_t e = launch_conv2d_chain(dtype, c, h, w, in, kh1, kw1, k1, kh2, kw2, k2, out,
                                            (flags & PENCIL_CONV_GENERIC) != 0, s);
        return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
    }
    // compute-bound chain: two passes through a stream-ordered temporary
    void *tmp = nullptr;
    cudaMemPool_t mp = nullptr;
    {
        std::lock_guard<std::mutex> lk(pool().mu);
        mp = pool().stream_pool();
    }
    if (!mp) return PENCIL_ERR_NOMEM;
    cudaError_t e = cudaMallocFromPoolAsync(&tmp, nb, mp, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return PENCIL_ERR_NOMEM;
    }
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_conv2d(dtype, c, h, w, in, kh1, kw1, k1, tmp, s);
    if (e == cudaSuccess) e = launch_conv2d(dtype, c, h, w, tmp, kh2, kw2, k2, out, s);
    const cudaError_t ef = cudaFreeAsync(tmp, s);
    if (e == cudaSuccess) e = ef;
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

int pencil_conv2d(int h, int w, const float *in, int kh, int kw, const float *k, float *out) {
    if (kh <= 0 || kw <= 0) return PENCIL_ERR_ARG;
    int st = check_dims(h, w);
    if (st) return st;
    if (!in || !k || !out) return PENCIL_ERR_NULL;
    const size_t nb = sizeof(float) * (size_t)h * w;
    const size_t kb = sizeof(float) * (size_t)kh * kw;
    if (overlaps(out, nb, in, nb) || overlaps(out, nb, k, kb)) return PENCIL_ERR_ALIAS;
    const Mem mi = kind_of(in), mk = kind_of(k), mo = kind_of(out);
    if (mi == Mem::Invalid || mk == Mem::Invalid || mo == Mem::Invalid) return PENCIL_ERR_PTR;
    cudaStream_t s = 0;
    if (mi == Mem::Device && mk == Mem::Device && mo == Mem::Device) {
        cudaError_t e = launch_conv2d(PENCIL_F32, 1, h, w, in, kh, kw, k, out, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
    }
    std::lock_guard<std::mutex> lk(pool().mu);
    const float *dk = k;
    if (mk == Mem::Host) {
        void *b = pool().get(1, kb);
        if (!b) return PENCIL_ERR_NOMEM;
        PENCIL_CUDA_TRY(cudaMemcpy(b, k, kb, cudaMemcpyHostToDevice));
        dk = static_cast<const float *>(b);
    }
    if (mi == Mem::Device && mo == Mem::Device) {
        PENCIL_CUDA_TRY(launch_conv2d(PENCIL_F32, 1, h, w, in, kh, kw, dk, out, s));
        PENCIL_CUDA_TRY(cudaStreamSynchronize(s));
        return PENCIL_OK;
    }
    return banded(h, w, kh / 2, kh - 1 - kh / 2, in, out,
                  [&](const float *bi, float *bo, int hs, cudaStream_t bs) {
                      return launch_conv2d(PENCIL_F32, 1, hs, w, bi, kh, kw, dk, bo, bs);
                  });
}

int pencil_conv2d_sep(int h, int w, const float *in, int kx, const float *gx, int ky,
                      const float *gy, float *out) {
    if (kx <= 0 || ky <= 0) return PENCIL_ERR_ARG;
    int st = check_dims(h, w);
    if (st) return st;
    if (!in || !gx || !gy || !out) return PENCIL_ERR_NULL;
    if (kx > PENCIL_MAX_SPECIALISED_K || ky > PENCIL_MAX_SPECIALISED_K) return PENCIL_ERR_UNSUPPORTED;
    const size_t nb = sizeof(float) * (size_t)h * w;
    if (overlaps(out, nb, in, nb) || overlaps(out, nb, gx, sizeof(float) * kx) ||
        overlaps(out, nb, gy, sizeof(float) * ky))
        return PENCIL_ERR_ALIAS;
    const Mem mi = kind_of(in), mx = kind_of(gx), my = kind_of(gy), mo = kind_of(out);
    if (mi == Mem::Invalid || mx == Mem::Invalid || my == Mem::Invalid || mo == Mem::Invalid)
        return PENCIL_ERR_PTR;
    cudaStream_t s = 0;
    std::lock_guard<std::mutex> lk(pool().mu);
    const float *dgx = gx, *dgy = gy;
    if (mx == Mem::Host || my == Mem::Host) {
        float *b = static_cast<float *>(pool().get(1, sizeof(float) * 2 * PENCIL_MAX_SPECIALISED_K));
        if (!b) return PENCIL_ERR_NOMEM;
        if (mx == Mem::Host) {
            PENCIL_CUDA_TRY(cudaMemcpy(b, gx, sizeof(float) * kx, cudaMemcpyHostToDevice));
            dgx = b;
        }
        if (my == Mem::Host) {
            float *by = b + PENCIL_MAX_SPECIALISED_K;
            PENCIL_CUDA_TRY(cudaMemcpy(by, gy, sizeof(float) * ky, cudaMemcpyHostToDevice));
            dgy = by;
        }
    }
    if (mi == Mem::Device && mo == Mem::Device) {
        PENCIL_CUDA_TRY(launch_conv2d_sep(PENCIL_F32, 1, h, w, in, kx, dgx, ky, dgy, out, s));
        PENCIL_CUDA_TRY(cudaStreamSynchronize(s));
        return PENCIL_OK;
    }
    return banded(h, w, ky / 2, ky - 1 - ky / 2, in, out,
                  [&](const float *bi, float *bo, int hs, cudaStream_t bs) {
                      return launch_conv2d_sep(PENCIL_F32, 1, hs, w, bi, kx, dgx, ky, dgy, bo, bs);
                  });
}

size_t pencil_jacobi2d_workspace_size(int h, int w) {
    if (check_dims(h, w)) return 0;
    return jacobi_workspace_bytes(h, w);
}

int pencil_jacobi2d_ex(int h, int w, float *u, int iters, int check_every, double *res_out,
                       void *workspace, size_t ws_bytes, int temporal_t, void *stream) {
    int st = check_dims(h, w);
    if (st) return st;
    if (iters < 0 || check_every < 0 || temporal_t < 0) return PENCIL_ERR_ARG;
    if (!u || !workspace) return PENCIL_ERR_NULL;
    const int nres = check_every > 0 ? iters / check_every : 0;
    if (nres > 0 && !res_out) return PENCIL_ERR_NULL;
    const size_t need = jacobi_workspace_bytes(h, w);
    if (ws_bytes < need) return PENCIL_ERR_NOMEM;
    if ((uintptr_t)workspace % 256 != 0) return PENCIL_ERR_ARG;
    const size_t ub = sizeof(float) * (size_t)h * w;
    if (overlaps(workspace, ws_bytes, u, ub)) return PENCIL_ERR_ALIAS;
    if (nres > 0 && (overlaps(res_out, sizeof(double) * nres, u, ub) ||
                     overlaps(res_out, sizeof(double) * nres, workspace, ws_bytes)))
        return PENCIL_ERR_ALIAS;
    if (kind_of(u) != Mem::Device || kind_of(workspace) != Mem::Device) return PENCIL_ERR_PTR;
    if (nres > 0 && kind_of(res_out) != Mem::Device) return PENCIL_ERR_PTR;
    cudaError_t e = jacobi_run(h, w, u, iters, check_every, res_out, workspace, ws_bytes, temporal_t,
                               (cudaStream_t)stream);
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

// Shared checks of the iterative entry points; returns PENCIL_OK or an error.
static int check_iterative(int h, int w, float *u, int nres, double *res_out, void *workspace,
                           size_t ws_bytes, size_t need) {
    int st = check_dims(h, w);
    if (st) return st;
    if (!u || !workspace) return PENCIL_ERR_NULL;
    if (nres > 0 && !res_out) return PENCIL_ERR_NULL;
    if (ws_bytes < need) return PENCIL_ERR_NOMEM;
    if ((uintptr_t)workspace % 256 != 0) return PENCIL_ERR_ARG;
    const size_t ub = sizeof(float) * (size_t)h * w;
    if (overlaps(workspace, ws_bytes, u, ub)) return PENCIL_ERR_ALIAS;
    if (nres > 0 && (overlaps(res_out, sizeof(double) * nres, u, ub) ||
                     overlaps(res_out, sizeof(double) * nres, workspace, ws_bytes)))
        return PENCIL_ERR_ALIAS;
    if (kind_of(u) != Mem::Device || kind_of(workspace) != Mem::Device) return PENCIL_ERR_PTR;
    if (nres > 0 && kind_of(res_out) != Mem::Device) return PENCIL_ERR_PTR;
    return PENCIL_OK;
}

int pencil_jacobi2d_until(int h, int w, float *u, int max_iters, int check_every, double tol,
                          double *res_out, int *iters_done, void *workspace, size_t ws_bytes,
                          int temporal_t, void *stream) {
    if (!iters_done) return PENCIL_ERR_NULL;
    *iters_done = 0;
    if (max_iters < 0 || check_every < 1 || max_iters % check_every != 0 || temporal_t < 0 ||
        !(tol >= 0.0))
        return PENCIL_ERR_ARG;
    if (int st0 = check_dims(h, w)) return st0;
    int st = check_iterative(h, w, u, max_iters / check_every, res_out, workspace, ws_bytes,
                             jacobi_workspace_bytes(h, w));
    if (st) return st;
    cudaError_t e = jacobi_until(h, w, u, max_iters, check_every, tol, res_out, iters_done, workspace,
                                 ws_bytes, temporal_t, (cudaStream_t)stream);
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

size_t pencil_rbsor2d_workspace_size(int h, int w) {
    if (check_dims(h, w)) return 0;
    return rbsor_workspace_bytes(h, w);
}

int pencil_rbsor2d_ex(int h, int w, float *u, int iters, float omega, int check_every,
                      double *res_out, void *workspace, size_t ws_bytes, void *stream) {
    if (iters < 0 || check_every < 0 || !(omega > 0.0f && omega < 2.0f)) return PENCIL_ERR_ARG;
    if (int st0 = check_dims(h, w)) return st0;
    const int nres = check_every > 0 ? iters / check_every : 0;
    int st = check_iterative(h, w, u, nres, res_out, workspace, ws_bytes, rbsor_workspace_bytes(h, w));
    if (st) return st;
    cudaError_t e = rbsor_run(h, w, u, iters, omega, check_every, res_out, workspace, (cudaStream_t)stream);
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

int pencil_rbsor2d_until(int h, int w, float *u, int max_iters, float omega, int check_every,
                         double tol, double *res_out, int *iters_done, void *workspace,
                         size_t ws_bytes, void *stream) {
    if (!iters_done) return PENCIL_ERR_NULL;
    *iters_done = 0;
    if (max_iters < 0 || check_every < 1 || max_iters % check_every != 0 ||
        !(omega > 0.0f && omega < 2.0f) || !(tol >= 0.0))
        return PENCIL_ERR_ARG;
    if (int st0 = check_dims(h, w)) return st0;
    int st = check_iterative(h, w, u, max_iters / check_every, res_out, workspace, ws_bytes,
                             rbsor_workspace_bytes(h, w));
    if (st) return st;
    cudaError_t e = rbsor_until(h, w, u, max_iters, omega, check_every, tol, res_out, iters_done,
                                workspace, (cudaStream_t)stream);
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

int pencil_residual2d(int h, int w, const float *u, double *res_out, void *workspace,
                      size_t ws_bytes, void *stream) {
    int st = check_dims(h, w);
    if (st) return st;
    if (!u || !res_out || !workspace) return PENCIL_ERR_NULL;
    if (ws_bytes < jacobi_workspace_bytes(h, w)) return PENCIL_ERR_NOMEM;
    if ((uintptr_t)workspace % 256 != 0) return PENCIL_ERR_ARG;
    const size_t ub = sizeof(float) * (size_t)h * w;
    if (overlaps(workspace, ws_bytes, u, ub) || overlaps(res_out, sizeof(double), u, ub) ||
        overlaps(res_out, sizeof(double), workspace, ws_bytes))
        return PENCIL_ERR_ALIAS;
    if (kind_of(u) != Mem::Device || kind_of(res_out) != Mem::Device ||
        kind_of(workspace) != Mem::Device)
        return PENCIL_ERR_PTR;
    cudaError_t e = residual_run(h, w, u, res_out, workspace, (cudaStream_t)stream);
    return e == cudaSuccess ? PENCIL_OK : cuda_fail(e);
}

int pencil_jacobi2d(int h, int w, float *u, int iters) {
    int st = check_dims(h, w);
    if (st) return st;
    if (iters < 0) return PENCIL_ERR_ARG;
    if (!u) return PENCIL_ERR_NULL;
    const Mem mu = kind_of(u);
    if (mu == Mem::Invalid) return PENCIL_ERR_PTR;
    std::lock_guard<std::mutex> lk(pool().mu);
    const size_t ub = sizeof(float) * (size_t)h * w;
    const size_t wsb = jacobi_workspace_bytes(h, w);
    void *ws = pool().get(3, wsb);
    if (!ws) return PENCIL_ERR_NOMEM;
    cudaStream_t s = 0;
    float *du = u;
    if (mu == Mem::Host) {
        void *b = pool().get(0, ub);
        if (!b) return PENCIL_ERR_NOMEM;
        PENCIL_CUDA_TRY(cudaMemcpyAsync(b, u, ub, cudaMemcpyHostToDevice, s));
        du = static_cast<float *>(b);
    }
    PENCIL_CUDA_TRY(jacobi_run(h, w, du, iters, 0, nullptr, ws, wsb, 0, s));
    if (mu == Mem::Host) PENCIL_CUDA_TRY(cudaMemcpyAsync(u, du, ub, cudaMemcpyDeviceToHost, s));
    PENCIL_CUDA_TRY(cudaStreamSynchronize(s));
    return PENCIL_OK;
}

}  // extern "C"
