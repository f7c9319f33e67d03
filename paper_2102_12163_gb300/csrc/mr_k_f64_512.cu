// double values, 512 threads per block.
#include "mr_kernels.cuh"

MRG_INSTANTIATE(double, 512, 2, 2, 2, 2, f64_512)
