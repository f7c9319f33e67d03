// double values, 256 threads per block.
#include "mr_kernels.cuh"

MRG_INSTANTIATE(double, 256, 4, 5, 3, 3, f64_256)
