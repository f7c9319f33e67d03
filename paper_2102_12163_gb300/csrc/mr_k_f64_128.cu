// double values, 128 threads per block.
#include "mr_kernels.cuh"

MRG_INSTANTIATE(double, 128, 8, 10, 6, 6, f64_128)
