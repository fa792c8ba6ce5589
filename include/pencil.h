/*
 * pencil.h -- C ABI of libpencilgpu, the GB300 (sm_103a) implementation of
 * the two loop nests PENCIL-style DSL compilers lower image-processing and CFD
 * code to (PENCIL, arXiv:1302.5586, Sec. 1 and Sec. 2): a 2-D convolution with
 * clamp-to-edge borders and an iterated 5-point Jacobi stencil with an FP64
 * residual norm.
 *
 * Calling conventions (the paper's coding rules, Sec. 2.2.1):
 *   - Array arguments follow the C99 VLA rule: each array is a separate,
 *     non-aliasing region ("restrict"); the library checks the byte ranges of
 *     the arrays it writes against those it reads and returns
 *     PENCIL_ERR_ALIAS on overlap.  Under C99 the prototypes below spell the
 *     VLA form; C++ and CUDA callers see the ABI-identical pointer form.
 *   - Images are dense row-major [h][w] (pitch = w elements); multi-channel
 *     images are planar [c][h][w]; filters are row-major [kh][kw] FP32.
 *     Sizes: h*w up to 2^40 elements, h up to PENCIL_MAX_ROWS rows and c up
 *     to PENCIL_MAX_CHANNELS channels (CUDA grid limits); larger return
 *     PENCIL_ERR_UNSUPPORTED.
 *   - Plain calls (no suffix) are synchronous and keep the sequential meaning
 *     of the loop nest (Sec. 2): they accept host or device memory for every
 *     array and return when the result is in place.
 *   - _ex calls are stream-ordered: every array must be device memory
 *     (PENCIL_ERR_PTR otherwise), the work is queued on `stream` (a
 *     cudaStream_t passed as void*, NULL = the legacy default stream) and the
 *     call returns without waiting.
 *   - Ownership: the caller owns every array; the library never frees them.
 *     Scratch for plain calls comes from a library pool released by
 *     pencil_shutdown(); _ex calls take caller-provided workspace.
 *   - Devices: the library works on the calling thread's current CUDA device.
 *     The plain calls' scratch lives on the device that was current when it
 *     was allocated, so a process that moves plain calls to another device
 *     calls pencil_shutdown() first (one process per GPU needs nothing).
 *   - Errors: every call returns 0 (PENCIL_OK) or a negative pencil_status.
 *     Nothing aborts or traps.  After PENCIL_ERR_CUDA the CUDA error code is
 *     kept per thread and readable with pencil_last_cuda_error().
 */
#ifndef PENCIL_H
#define PENCIL_H

#include <stddef.h>
#include <stdint.h>

/* PENCIL_ARR2(T, name, n, m): a [n][m] array parameter.  C99 sees the
 * PENCIL form `T name[restrict const static n][m]`; C++/CUDA see `T *name`,
 * which has the same ABI.  C before C2X converts no `float[n][m]` to a
 * `const float` parameter of this form: declare the input array const, or
 * cast it. */
#ifdef __cplusplus
extern "C" {
#define PENCIL_ARR2(T, name, n, m) T *name
#else
#define PENCIL_ARR2(T, name, n, m) T name[restrict const static n][m]
#endif

typedef enum pencil_status {
    PENCIL_OK = 0,
    PENCIL_ERR_ARG = -1,         /* a size is <= 0, too large, or a flag is unknown */
    PENCIL_ERR_NULL = -2,        /* a required pointer is NULL */
    PENCIL_ERR_ALIAS = -3,       /* an output overlaps an input (restrict rule, Sec. 2.2.1) */
    PENCIL_ERR_PTR = -4,         /* host memory where device memory is required */
    PENCIL_ERR_NOMEM = -5,       /* workspace too small or device allocation failed */
    PENCIL_ERR_CUDA = -6,        /* a CUDA call failed; see pencil_last_cuda_error() */
    PENCIL_ERR_TIMEOUT = -7,     /* a bounded wait expired */
    PENCIL_ERR_UNSUPPORTED = -8  /* a valid request the library does not implement */
} pencil_status;

/* Storage types of images (filters are always FP32; arithmetic is FP32). */
enum { PENCIL_F32 = 0, PENCIL_F16 = 1 };

/* pencil_conv2d_ex flag: run the generic (any-size) kernel even where a
 * specialised one exists.  The result is the same bits; the flag exists so
 * that the fixed per-pixel order can be checked across kernels. */
#define PENCIL_MAX_ROWS 524280      /* 65535 row blocks of 8 */
#define PENCIL_MAX_CHANNELS 65535
#define PENCIL_CONV_GENERIC 1
/* pencil_conv2d_chain: run the fused kernel even where two passes are faster */
#define PENCIL_CHAIN_FUSED 2
/* pencil_conv2d_ex / pencil_conv2d_sep_ex flag: the c channels are
 * interleaved [h][w][c] (channel ch of pixel (i, j) at element
 * (i*w + j)*c + ch, the layout image DSLs hand over, Sec. 1) instead of
 * planar [c][h][w].  Each channel is filtered on its own exactly as the planar
 * layout filters it (the same bits per channel); the output has the input's
 * layout.  3 and 4 channels run tiled kernels over the rows of w*c elements;
 * other channel counts a generic kernel.  w*c must fit an int
 * (PENCIL_ERR_UNSUPPORTED otherwise). */
#define PENCIL_LAYOUT_HWC 4
/* pencil_conv2d_ex flag: binary16 images on the tensor cores.  For planar
 * binary16 images with odd square filters of side 7..15 (where it measured
 * faster than the CUDA cores), rows 16-byte aligned (w a multiple of 8, in and out 16-byte aligned) and the clamp or
 * zero border, each filter row becomes a banded-matrix product on the
 * 5th-generation tensor cores: the weights, scaled by a power of two, are
 * split into two binary16 terms each (about 22 significant bits), products
 * accumulate in FP32 in tensor memory, and the result is rounded to binary16
 * once (Sec. 3.1: precision traded against speed, here within the binary16
 * tolerance -- |out - exact| <= 2^-10 * sum |k| |in| -- but not the same
 * bits as the CUDA-core kernels, whose summation order differs).  Inputs
 * are expected finite: the zeros of a band multiply neighbouring input
 * values too, so an Inf or NaN input can turn outputs up to 16 columns away
 * (not only those whose window holds it) into NaN.  Ignored for FP32 images,
 * with PENCIL_CONV_GENERIC or PENCIL_LAYOUT_HWC, and where the conditions
 * above do not hold (the CUDA-core kernels run). */
#define PENCIL_CONV_TENSOR 16

/* Border modes for the _ex conv2d calls, passed in flags as PENCIL_BORDER(m);
 * index i of an axis of length n reads (the plain calls always clamp):
 *   CLAMP    clamp(i) to [0, n-1]           a a | a b c d | d d
 *   ZERO     a zero outside [0, n-1]        0 0 | a b c d | 0 0
 *   REFLECT  edge repeated, period 2n       b a | a b c d | d c
 *   MIRROR   edge not repeated, period 2n-2 c b | a b c d | c b
 *   WRAP     periodic, period n             c d | a b c d | a b
 * The modes other than CLAMP are the "other border modes" of image DSLs
 * (Sec. 1); they change only which input values a window reads. */
#define PENCIL_BORDER_CLAMP 0
#define PENCIL_BORDER_ZERO 1
#define PENCIL_BORDER_REFLECT 2
#define PENCIL_BORDER_MIRROR 3
#define PENCIL_BORDER_WRAP 4
#define PENCIL_BORDER(m) ((m) << 8)

/* Largest filter side the specialised kernels handle; larger (or non-square)
 * filters take the generic kernel, which has no size limit. */
#define PENCIL_MAX_SPECIALISED_K 15

/* ------------------------------------------------------------------ conv2d
 * out[i][j] = sum_{a<kh} sum_{b<kw} k[a][b] * in[clamp(i+a-kh/2)][clamp(j+b-kw/2)]
 * with clamp(x) = min(max(x, 0), side-1) applied per axis: a correlation (no
 * filter flip) anchored at (kh/2, kw/2), borders replicated ("clamp to
 * edge").  The pixel loops are independent (Sec. 2.2.3, `independent`); the
 * per-pixel sum is a map over output pixels (Sec. 3.2, vector construction).
 * Each output is accumulated in FP32 in one fixed order -- per filter row a
 * chain of fused multiply-adds over b, then the row sums added in order of a
 * -- that does not depend on tiling, batching or stream, so every kernel of
 * this library returns the same bits for the same pixel (Sec. 3.1 on
 * floating-point order and reproducibility).
 */

/* Synchronous, one FP32 channel.  in: h*w, k: kh*kw, out: h*w; each may be
 * host or device memory.  Errors: ARG (h, w, kh, kw <= 0), NULL, ALIAS (out
 * overlaps in or k), NOMEM, CUDA. */
int pencil_conv2d(int h, int w, PENCIL_ARR2(const float, in, h, w), int kh, int kw,
                  PENCIL_ARR2(const float, k, kh, kw), PENCIL_ARR2(float, out, h, w));

/* Stream-ordered, c planar channels, storage dtype PENCIL_F32 or PENCIL_F16
 * (binary16 images; FP32 accumulation; binary16 results rounded to nearest
 * even).  in, out: c*h*w elements of dtype, device memory; k: kh*kw FP32,
 * device memory.  flags: PENCIL_CONV_GENERIC, PENCIL_LAYOUT_HWC,
 * PENCIL_CONV_TENSOR and/or one PENCIL_BORDER(m).
 * Speed, not results, depends on alignment: images whose rows are 16-byte
 * aligned (w a multiple of 4 for FP32, of 8 for binary16, and in and out
 * 16-byte aligned) with the clamp or zero border load their tiles with the
 * tensor memory accelerator; others use cp.async copies as wide as each row
 * allows (large planar images of odd width at filter sides up to 5: one
 * tensor-memory-accelerator copy per staged row).  The call may be
 * captured in a CUDA graph.  Errors: ARG, NULL, ALIAS, PTR, CUDA. */
int pencil_conv2d_ex(int c, int h, int w, const void *in, int kh, int kw, const float *k,
                     void *out, int dtype, int flags, void *stream);

/* Separable filter: the 2-D weights are gy[a] * gx[b] (kx taps along rows,
 * ky taps along columns).  Computed as a row pass then a column pass fused
 * through shared memory (no intermediate in HBM); per pixel the row pass is a
 * chain over b and the column pass a chain over a.  Sides
 * 1..PENCIL_MAX_SPECIALISED_K (odd or even).
 * Synchronous, one FP32 channel; in, gx, gy, out may be host or device memory.
 * Errors: ARG, NULL, ALIAS, UNSUPPORTED (a side above the maximum), NOMEM, CUDA. */
int pencil_conv2d_sep(int h, int w, PENCIL_ARR2(const float, in, h, w), int kx, const float *gx,
                      int ky, const float *gy, PENCIL_ARR2(float, out, h, w));

/* Stream-ordered separable filter over c planar channels of dtype
 * PENCIL_F32 or PENCIL_F16; every array is device memory.  flags:
 * PENCIL_LAYOUT_HWC and/or one PENCIL_BORDER(m).
 * Errors: ARG, NULL, ALIAS, PTR, UNSUPPORTED, CUDA. */
int pencil_conv2d_sep_ex(int c, int h, int w, const void *in, int kx, const float *gx, int ky,
                         const float *gy, void *out, int dtype, int flags, void *stream);

/* Two filters in a row, out = conv(conv(in, k1), k2), in one kernel: the
 * intermediate stays in on-chip memory instead of making a round trip
 * through HBM (the fusion of dependent stencils, Sec. 2.2.3).  The result is
 * bit-identical to two pencil_conv2d_ex calls through a temporary of the same
 * dtype: the intermediate is rounded to the storage type and the second
 * filter reads it clamped at the image edge.  Clamp-to-edge only.  Fusion
 * pays while the chain is bound by memory traffic: for two 3x3 filters the
 * call runs the fused kernel, otherwise two passes through a temporary from
 * a library-owned stream-ordered pool (kept for reuse until pencil_shutdown)
 * -- the same bits either way.
 * PENCIL_CHAIN_FUSED forces the fused kernel (tiled for square odd sides
 * 3, 5, 7), PENCIL_CONV_GENERIC the generic fused one.  Every array is device memory
 * (in, out: c*h*w elements of dtype; k1: kh1*kw1, k2: kh2*kw2 FP32).
 * Errors: ARG, NULL, ALIAS (out overlaps in, k1 or k2), PTR, UNSUPPORTED (a
 * border mode other than clamp, or a second filter too large for on-chip
 * memory), NOMEM (the temporary), CUDA. */
int pencil_conv2d_chain(int c, int h, int w, const void *in, int kh1, int kw1, const float *k1,
                        int kh2, int kw2, const float *k2, void *out, int dtype, int flags,
                        void *stream);

/* A filter pass followed by Jacobi smoothing, out = J^sweeps(conv(in, k)) on
 * each of c planar FP32 channels: conv the clamp-to-edge correlation above,
 * J the 5-point Jacobi sweep below (the image's outer ring fixed).  Where it
 * can, one kernel computes a 128 x 128 window of the filtered image into
 * registers and runs up to 10 sweeps on it before anything goes to HBM (the
 * fusion of dependent stencils, Sec. 2.2.3); further sweeps run as
 * pencil_jacobi2d_ex does.  Fused: square odd filters up to 7, w a multiple of
 * 4, in and out 16-byte aligned; otherwise a conv2d pass into out and the
 * sweeps in place.  Either way the result is the same bits as
 * pencil_conv2d_ex followed by pencil_jacobi2d_ex on each channel.  Sweeps
 * beyond the fused ones take a workspace from a library-owned stream-ordered
 * pool (kept for reuse until pencil_shutdown).  flags: 0, or
 * PENCIL_CHAIN_FUSED to require the fused kernel (UNSUPPORTED where it does
 * not apply).  in, out: c*h*w floats; k: kh*kw floats; all device memory.
 * Errors: ARG (sizes, sweeps < 0, flags), NULL, ALIAS (out overlaps in or k),
 * PTR, UNSUPPORTED, NOMEM, CUDA. */
int pencil_conv2d_jacobi(int c, int h, int w, const float *in, int kh, int kw, const float *k, int sweeps,
                         float *out, int flags, void *stream);

/* ------------------------------------------------------------------- batch
 * Many images, each with its own size and odd filter side 1..15, convolved by
 * ONE graph launch: the captured graph holds one kernel per filter side
 * present (independent graph nodes that may run side by side), each sized to
 * its side's register and shared-memory needs.  A side's tiles form one work
 * list, larger images first, so uneven images keep every SM busy: either a
 * persistent grid (every CTA the SMs hold at once) takes them from the side's
 * queue, or the kernel has one CTA per tile and the hardware block scheduler
 * hands them out -- which of the two, and the tile shape, is the side's tile
 * variant.  Each batched pixel is the same bits as pencil_conv2d_ex on that
 * image alone (the same fixed per-pixel order).  This is the tuned,
 * launch-once form of the independent loop over images and pixels
 * (Sec. 2.2.3); the variant per filter side is chosen by measurement (the
 * auto-tuning step of Sec. 2).
 */
typedef struct pencil_image {
    const void *in;   /* h*w elements of the batch dtype, device memory */
    void *out;        /* h*w elements of the batch dtype, device memory */
    const float *k;   /* ks*ks FP32 weights, row-major, device memory */
    int h, w;         /* image size, both > 0 */
    int ks;           /* odd filter side, 1..15 */
} pencil_image;

/* A reusable batch plan: device and pinned host tables sized for up to
 * max_images images and max_tiles tiles, and the captured graph. */
typedef struct pencil_batch pencil_batch;

/* Tile variants of the batched kernels, each its own kernel per filter side:
 * 0 = 32 x 128 outputs, 128 threads   2 = 64 x 128 outputs, 256 threads
 * 1 = 16 x 128 outputs, 128 threads   3 = 32 x 128 outputs, 256 threads
 * 4 = as 0, one CTA per tile          5 = as 3, one CTA per tile
 * (so tile height, rows per thread, CTA size and schedule differ between
 * them: 0-3 run a persistent grid fed from the side's work queue). */
#define PENCIL_BATCH_VARIANTS 6

/* Create a plan for dtype PENCIL_F32 or PENCIL_F16 (allocates; captures the
 * graph).  All sides start with variant 0.  Errors: NULL, ARG, NOMEM, CUDA. */
int pencil_batch_create(int dtype, int max_images, long long max_tiles, pencil_batch **out);

/* Tile variant used for images whose filter side is ks (odd 1..15).  It swaps
 * the side's kernel and drops the plan's captured graphs (the next run
 * captures again), so call it while no batch of the plan is in flight.
 * Errors: NULL, ARG, CUDA. */
int pencil_batch_set_variant(pencil_batch *b, int ks, int variant);

/* Number of tiles n images need with the plan's current variants (host only).
 * Errors: NULL, ARG. */
int pencil_batch_tiles(const pencil_batch *b, int n, const pencil_image *imgs, long long *tiles);

/* Stream-ordered: convolve n images (descriptors in host memory, read before
 * the call returns) with one graph launch on `stream`.  Outputs must not
 * overlap each other or any input or filter of the batch (PENCIL_ERR_ALIAS).
 * Image buffers must be device memory (not checked per image).  A plan runs
 * on one stream at a time; use one plan per stream for concurrent batches.
 * Errors: NULL, ARG (bad size or side), ALIAS, NOMEM (more images or tiles
 * than the plan holds), CUDA. */
int pencil_batch_run(pencil_batch *b, int n, const pencil_image *imgs, void *stream);

/* Wait for the plan's last uploads, then free it.  Call after its last batch
 * has finished.  NULL is accepted. */
int pencil_batch_destroy(pencil_batch *b);

/* The auto-tuning step of Sec. 2 for a batch plan: for every filter side
 * present in the n images, run that side's images alone under each tile
 * variant (one warm-up run, then `reps` timed runs between CUDA events on
 * `stream`), keep the fastest on the plan and report it in chosen[ks / 2]
 * (chosen has 8 entries for sides 1, 3, ..., 15; -1 for sides not present;
 * may be NULL).  Every variant gives the same bits, so tuning changes only
 * the time.  Synchronous (it reads the events); the images' outputs are
 * overwritten.  Same requirements on the images as pencil_batch_run.
 * Errors: NULL, ARG (bad size or side, reps < 1), ALIAS, NOMEM, CUDA. */
int pencil_tune(pencil_batch *b, int n, const pencil_image *imgs, int reps, void *stream, int *chosen);

/* ------------------------------------------------------------------- arena
 * Byte-offset bookkeeping for one device memory budget, used by the serving
 * loop to admit requests only while their buffers fit (the paper has no
 * serving layer; this is runtime support for the batched path).  First-fit
 * over free blocks kept in address order; freeing merges neighbours.  Host
 * only: it never calls CUDA.  Thread-safe.
 */
typedef struct pencil_arena pencil_arena;

/* capacity: budget in bytes (rounded down to align); align: a power of two.
 * Errors: NULL, ARG, NOMEM. */
int pencil_arena_create(size_t capacity, size_t align, pencil_arena **out);

/* First block of round_up(bytes, align) bytes; its offset in *offset.
 * Errors: NULL, ARG (bytes == 0), NOMEM (no free block is large enough). */
int pencil_arena_alloc(pencil_arena *a, size_t bytes, size_t *offset);

/* Release the block that starts at offset.  Errors: NULL, ARG (no such block). */
int pencil_arena_free(pencil_arena *a, size_t offset);

/* Free bytes in total, and the largest free block (0 for NULL). */
size_t pencil_arena_free_bytes(pencil_arena *a);
size_t pencil_arena_largest_free(pencil_arena *a);

void pencil_arena_destroy(pencil_arena *a);

/* ------------------------------------------------------------------ jacobi
 * One sweep: v[i][j] = 0.25f * ((u[i-1][j] + u[i+1][j]) + (u[i][j-1] + u[i][j+1]))
 * on the interior 1 <= i <= h-2, 1 <= j <= w-2, in FP32 in exactly that order;
 * the boundary ring never changes; u and v are two buffers (a Jacobi step).
 * The sweeps form the sequential outer loop of `untilconverged` (Sec. 3.2);
 * the points of one sweep are independent (Sec. 2.2.3).
 *
 * Residual of an iterate: sqrt(sum over the interior of r^2),
 * r = 4u[i][j] - ((u[i-1][j] + u[i+1][j]) + (u[i][j-1] + u[i][j+1])), r and
 * r^2 in FP32, summed per thread with compensation, then across threads and
 * blocks in FP64 in a fixed order (the `reduction` directive,
 * Sec. 2.2.3).  Grids with h < 3 or w < 3 have no interior: sweeps change
 * nothing and residuals are 0.
 */

/* Synchronous: iters sweeps of u (h*w FP32, host or device) in place.
 * Errors: ARG (h, w <= 0, iters < 0), NULL, NOMEM, CUDA. */
int pencil_jacobi2d(int h, int w, PENCIL_ARR2(float, u, h, w), int iters);

/* Bytes of workspace pencil_jacobi2d_ex needs for an h x w grid. */
size_t pencil_jacobi2d_workspace_size(int h, int w);

/* Stream-ordered: iters sweeps of u (device memory) in place.  When
 * check_every > 0, the residual of the iterate after sweep m*check_every is
 * written to res_out[m-1] (device memory, iters/check_every doubles).
 * workspace: device memory of at least pencil_jacobi2d_workspace_size(h, w)
 * bytes, 256-byte aligned, not overlapping u or res_out.  temporal_t selects
 * how many sweeps one kernel pass performs per HBM round trip (0 = library
 * choice, 1 = one sweep per pass); the iterate is the same bits for every
 * choice.  Errors: ARG, NULL, ALIAS, PTR, NOMEM (workspace too small), CUDA. */
int pencil_jacobi2d_ex(int h, int w, float *u, int iters, int check_every, double *res_out,
                       void *workspace, size_t ws_bytes, int temporal_t, void *stream);

/* Stream-ordered residual of one grid (device memory) into *res_out (device).
 * workspace as for pencil_jacobi2d_ex (not overlapping u or res_out).
 * Errors: ARG, NULL, ALIAS, PTR, NOMEM, CUDA. */
int pencil_residual2d(int h, int w, const float *u, double *res_out, void *workspace,
                      size_t ws_bytes, void *stream);

/* Size of the static scratch array behind pencil_jacobi2d_noalloc: one
 * 2048 x 2048 FP32 grid (16 MiB) plus 1 MiB for residual partials. */
#define PENCIL_NOALLOC_SCRATCH_BYTES ((size_t)17 << 20)

/* pencil_jacobi2d_ex for callers that cannot allocate device memory.  The
 * paper has no counterpart to this entry point; it exists for callers such as
 * a fixed-latency loop that cannot afford the device-wide synchronisation and
 * milliseconds a cudaMalloc/cudaFree may cost, a process whose framework
 * allocator has already reserved the device's memory (so a fresh cudaMalloc
 * fails or fragments it), or code whose rules forbid dynamic allocation after
 * start-up.  Instead of a workspace argument it uses one static device array
 * of PENCIL_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits; it never calls cudaMalloc or cudaFree.
 * Same sweeps, residuals and results as pencil_jacobi2d_ex.  u and res_out
 * are caller-owned device memory.  The first call on each device looks up
 * the array's device address (with that device current) and caches it, so
 * make that first call before any stream capture; after a device reset the
 * next call finds a new context and looks the address up again, so that
 * call too belongs before any capture.  All calls on a device share
 * the one array, which keeps the previous call's contents (every element a
 * call reads it has first written, so nothing needs clearing): calls whose
 * work overlaps on the GPU -- on different streams or from different host
 * threads without ordering -- race and corrupt each other.
 * Errors: ARG, UNSUPPORTED (h above PENCIL_MAX_ROWS, as for every _ex call),
 * NULL, PTR, ALIAS (res_out overlaps u), NOMEM (the grid needs more scratch
 * than PENCIL_NOALLOC_SCRATCH_BYTES: h*w above about 4.4 million points; every
 * grid up to 2048 x 2048 fits), CUDA. */
int pencil_jacobi2d_noalloc(int h, int w, float *u, int iters, int check_every, double *res_out,
                            int temporal_t, void *stream);

/* untilconverged with its threshold (Sec. 3.2): sweeps in chunks of
 * check_every; after each chunk the residual of the iterate is written to
 * res_out[m-1] (device memory, max_iters/check_every doubles), read back, and
 * the loop stops once it is <= tol or max_iters sweeps are done.  *iters_done
 * (host memory) receives the number of sweeps performed; u holds that iterate
 * (the same bits as pencil_jacobi2d_ex with that many sweeps).  Synchronous on
 * `stream` (each chunk ends with a read of one double).  check_every >= 1 and
 * max_iters a multiple of it.  Other arguments as pencil_jacobi2d_ex.
 * Errors: ARG, NULL, ALIAS, PTR, NOMEM, CUDA. */
int pencil_jacobi2d_until(int h, int w, float *u, int max_iters, int check_every, double tol,
                          double *res_out, int *iters_done, void *workspace, size_t ws_bytes,
                          int temporal_t, void *stream);

/* Red-black successive over-relaxation, in place: a sweep updates the
 * interior points with (i + j) even, then those with (i + j) odd (which see
 * the new even values), each as
 *   u <- fma(omega, 0.25f * ((up + down) + (left + right)) - u, u)
 * in FP32 in exactly that order; omega in (0, 2), 1 = red-black Gauss-Seidel.
 * The over-relaxed variant of the sequential untilconverged loop (Sec. 3.2):
 * it needs O(n) sweeps where the Jacobi sweep needs O(n^2).  Residuals every
 * check_every sweeps as for pencil_jacobi2d_ex.  u, res_out, workspace:
 * device memory; workspace of pencil_rbsor2d_workspace_size(h, w) bytes (a
 * second grid for the tiled passes, which read one grid and write the other,
 * and the residual partials).
 * Errors: ARG, NULL, ALIAS, PTR, NOMEM, CUDA. */
size_t pencil_rbsor2d_workspace_size(int h, int w);
int pencil_rbsor2d_ex(int h, int w, float *u, int iters, float omega, int check_every,
                      double *res_out, void *workspace, size_t ws_bytes, void *stream);

/* The same with the convergence stop of pencil_jacobi2d_until. */
int pencil_rbsor2d_until(int h, int w, float *u, int max_iters, float omega, int check_every,
                         double tol, double *res_out, int *iters_done, void *workspace,
                         size_t ws_bytes, void *stream);

/* --------------------------------------------------------------------- op2
 * The indirect increment of the paper's unstructured-mesh example (Sec. 3.1):
 * for every edge i (in order) the cells e2c[2i+1] and e2c[2i] are each
 * incremented by edge[i] (FP64).  Two ways to run it:
 *   PENCIL_OP2_ORDERED  every cell adds its edges in the sequential order
 *                       (from a plan), so the result is the same bits as the
 *                       sequential loop, run after run;
 *   PENCIL_OP2_ATOMIC   one thread per edge with FP64 atomic adds: no plan use,
 *                       but the rounding depends on the order the hardware
 *                       picks (the precision-for-speed switch of Sec. 3.1).
 */
#define PENCIL_OP2_ORDERED 0
#define PENCIL_OP2_ATOMIC 1
typedef struct pencil_op2_plan pencil_op2_plan;

/* Build the per-cell contribution lists of a mesh: e2c is host memory,
 * 2*nedges cell indices in [0, ncells) (edge i joins e2c[2i] and e2c[2i+1]);
 * the plan keeps device copies (lists of at most 8 per cell as a fixed-width
 * table).  Errors: NULL, ARG (an index out of range, sizes), NOMEM, CUDA. */
int pencil_op2_plan_create(int ncells, int nedges, const int *e2c, pencil_op2_plan **out);

/* Stream-ordered: cell[c] += sum of its edges' values.  edge (nedges doubles)
 * and cell (ncells doubles) are device memory and must not overlap.
 * Errors: NULL, ARG (mode), ALIAS, PTR, CUDA. */
int pencil_op2_inc(const pencil_op2_plan *p, const double *edge, double *cell, int mode, void *stream);

/* Free a plan (after its last use has finished).  NULL is accepted. */
int pencil_op2_plan_destroy(pencil_op2_plan *p);

/* ----------------------------------------------------------------- utility */

/* Human-readable text of a pencil_status (static storage). */
const char *pencil_strerror(int status);

/* The current device's name (NUL-terminated, truncated to len), SM count and
 * CUDA driver version; any output pointer may be NULL.  Errors: CUDA. */
int pencil_device_info(char *name, int len, int *sm_count, int *driver_version);

/* Library version as major*10000 + minor*100 + patch. */
int pencil_version(void);

/* The cudaError_t of the calling thread's most recent PENCIL_ERR_CUDA, or 0. */
int pencil_last_cuda_error(void);

/* Status of the device-side waits since the last call: PENCIL_ERR_TIMEOUT if
 * any kernel gave up a bounded wait (a tile load whose completion did not
 * arrive within its limit of about a second; that tile's outputs were not
 * written), else PENCIL_OK.  Clears the count.  Stream-ordered calls report
 * their waits here, so call it after synchronising the streams that ran
 * them.  The library's kernels never wait without a limit.  A CTA whose
 * load timed out waits once more (same limit) for the copy to land before it
 * exits; if even that runs out it exits all the same, and the late copy may
 * then land in shared memory that a later CTA on that SM is using.  So after
 * PENCIL_ERR_TIMEOUT treat every result computed since the previous check as
 * suspect, not only the skipped tiles.  Errors: CUDA. */
int pencil_device_status(void);

/* Self-test of the bounded wait: one CTA waits up to limit_us microseconds
 * (1 .. 1000000) on an mbarrier that no copy completes.  *completed = 0 when
 * the wait ran out as it must (it is then counted, so pencil_device_status
 * reports PENCIL_ERR_TIMEOUT once), 1 if it completed.  Synchronous.
 * Errors: NULL, ARG, CUDA.  (The paper has no counterpart: this checks the
 * library's own failure path without faulting or hanging the GPU.) */
int pencil_selftest_wait_timeout(unsigned limit_us, int *completed);

/* Release the library's device pools (plain calls' scratch, the temporaries
 * of pencil_conv2d_chain).  Call when no library work is in flight, and
 * before moving plain calls to another device.  Safe to call more than once;
 * later calls allocate again. */
void pencil_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* PENCIL_H */
