// float values, 128 threads per block.
#include "mr_kernels.cuh"

MRG_INSTANTIATE(float, 128, 8, 12, 4, 8, f32_128)
