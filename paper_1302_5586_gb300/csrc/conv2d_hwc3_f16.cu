// conv2d_hwc3_f16.cu -- the tiled interleaved-image kernels for 3 channels of
// binary16 (see conv_hwc.cuh).
#include "conv_hwc.cuh"

PENCIL_HWC_UNIT(__half, 3, hwc3_f16)
