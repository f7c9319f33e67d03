// float values, 512 threads per block.
#include "mr_kernels.cuh"

MRG_INSTANTIATE(float, 512, 2, 3, 1, 2, f32_512)
