// float values, 256 threads per block.
#include "mr_kernels.cuh"

MRG_INSTANTIATE(float, 256, 4, 6, 2, 4, f32_256)
