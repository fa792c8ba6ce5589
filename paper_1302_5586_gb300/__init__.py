"""GB300-native (sm_103a) clamp-to-edge conv2d and 5-point Jacobi stencil.

The computation is the data-parallel loop nest that PENCIL (arXiv:1302.5586)
lets DSL compilers hand to an optimiser: a 2-D convolution over independent
pixel loops (Sec. 2.2.3) and the sweeps of an `untilconverged` loop with an
FP64 reduction for its residual (Sec. 3.2).  The work runs in hand-written
CUDA kernels behind the C ABI in include/pencil.h; this package is the thin
Python binding of that ABI plus the batching and serving layers built on it.
"""
from ._binding import (  # noqa: F401
    HEADER,
    LIB_PATH,
    BORDER_MODES,
    PENCIL_BATCH_VARIANTS,
    PENCIL_BORDER,
    PENCIL_CONV_GENERIC,
    PENCIL_F16,
    PENCIL_F32,
    PENCIL_MAX_SPECIALISED_K,
    PENCIL_NOALLOC_SCRATCH_BYTES,
    PencilError,
    PencilImage,
    declared_symbols,
    lib,
    make_images,
    pencil_arena_alloc,
    pencil_arena_create,
    pencil_arena_destroy,
    pencil_arena_free,
    pencil_arena_free_bytes,
    pencil_arena_largest_free,
    pencil_batch_create,
    pencil_batch_destroy,
    pencil_batch_run,
    pencil_batch_set_variant,
    pencil_batch_tiles,
    pencil_conv2d,
    pencil_conv2d_ex,
    pencil_conv2d_sep,
    pencil_conv2d_sep_ex,
    pencil_device_info,
    pencil_jacobi2d,
    pencil_jacobi2d_ex,
    pencil_jacobi2d_noalloc,
    pencil_jacobi2d_until,
    pencil_rbsor2d_ex,
    pencil_rbsor2d_until,
    pencil_rbsor2d_workspace_size,
    pencil_jacobi2d_workspace_size,
    pencil_last_cuda_error,
    pencil_residual2d,
    pencil_shutdown,
    pencil_strerror,
    pencil_version,
)
