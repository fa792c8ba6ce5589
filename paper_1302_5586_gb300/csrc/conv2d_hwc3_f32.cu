// conv2d_hwc3_f32.cu -- the tiled interleaved-image kernels for 3 channels of
// FP32 (see conv_hwc.cuh).
#include "conv_hwc.cuh"

PENCIL_HWC_UNIT(float, 3, hwc3_f32)
