// float values, 1024 threads per block.
#include "mr_kernels.cuh"

MRG_INSTANTIATE(float, 1024, 1, 1, 1, 1, f32_1024)
