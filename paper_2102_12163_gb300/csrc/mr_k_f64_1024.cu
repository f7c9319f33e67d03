// double values, 1024 threads per block.
#include "mr_kernels.cuh"

MRG_INSTANTIATE(double, 1024, 1, 1, 1, 1, f64_1024)
