// conv2d_hwc4_f32.cu -- the tiled interleaved-image kernels for 4 channels of
// FP32 (see conv_hwc.cuh).
#include "conv_hwc.cuh"

PENCIL_HWC_UNIT(float, 4, hwc4_f32)
