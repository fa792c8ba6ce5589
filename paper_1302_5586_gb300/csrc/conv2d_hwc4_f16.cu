// conv2d_hwc4_f16.cu -- the tiled interleaved-image kernels for 4 channels of
// binary16 (see conv_hwc.cuh).
#include "conv_hwc.cuh"

PENCIL_HWC_UNIT(__half, 4, hwc4_f16)
