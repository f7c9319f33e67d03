// mr_dispatch.cu -- routes a launch to the (precision, block size) instantiation.
#include <cuda_runtime.h>

#include "mr_common.h"

int mrg_launch_f64_128(int, const mrg::LaunchArgs &, cudaStream_t);
int mrg_occ_f64_128(int, int *);
size_t mrg_smem_f64_128(int);
int mrg_launch_f64_256(int, const mrg::LaunchArgs &, cudaStream_t);
int mrg_occ_f64_256(int, int *);
size_t mrg_smem_f64_256(int);
int mrg_launch_f64_512(int, const mrg::LaunchArgs &, cudaStream_t);
int mrg_occ_f64_512(int, int *);
size_t mrg_smem_f64_512(int);
int mrg_launch_f64_1024(int, const mrg::LaunchArgs &, cudaStream_t);
int mrg_occ_f64_1024(int, int *);
size_t mrg_smem_f64_1024(int);
int mrg_launch_f32_128(int, const mrg::LaunchArgs &, cudaStream_t);
int mrg_occ_f32_128(int, int *);
size_t mrg_smem_f32_128(int);
int mrg_launch_f32_256(int, const mrg::LaunchArgs &, cudaStream_t);
int mrg_occ_f32_256(int, int *);
size_t mrg_smem_f32_256(int);
int mrg_launch_f32_512(int, const mrg::LaunchArgs &, cudaStream_t);
int mrg_occ_f32_512(int, int *);
size_t mrg_smem_f32_512(int);
int mrg_launch_f32_1024(int, const mrg::LaunchArgs &, cudaStream_t);
int mrg_occ_f32_1024(int, int *);
size_t mrg_smem_f32_1024(int);

int mrg_launch(bool fp32, int block, int grid, const mrg::LaunchArgs &a, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (fp32) {
        switch (block) {
        case 128: return mrg_launch_f32_128(grid, a, s);
        case 256: return mrg_launch_f32_256(grid, a, s);
        case 512: return mrg_launch_f32_512(grid, a, s);
        case 1024: return mrg_launch_f32_1024(grid, a, s);
        }
    } else {
        switch (block) {
        case 128: return mrg_launch_f64_128(grid, a, s);
        case 256: return mrg_launch_f64_256(grid, a, s);
        case 512: return mrg_launch_f64_512(grid, a, s);
        case 1024: return mrg_launch_f64_1024(grid, a, s);
        }
    }
    return (int)cudaErrorInvalidValue;
}

int mrg_occupancy(bool fp32, int block, int mask_words, int *nb) {
    if (fp32) {
        switch (block) {
        case 128: return mrg_occ_f32_128(mask_words, nb);
        case 256: return mrg_occ_f32_256(mask_words, nb);
        case 512: return mrg_occ_f32_512(mask_words, nb);
        case 1024: return mrg_occ_f32_1024(mask_words, nb);
        }
    } else {
        switch (block) {
        case 128: return mrg_occ_f64_128(mask_words, nb);
        case 256: return mrg_occ_f64_256(mask_words, nb);
        case 512: return mrg_occ_f64_512(mask_words, nb);
        case 1024: return mrg_occ_f64_1024(mask_words, nb);
        }
    }
    return (int)cudaErrorInvalidValue;
}

size_t mrg_smem_bytes(bool fp32, int block, int mask_words) {
    if (fp32) {
        switch (block) {
        case 128: return mrg_smem_f32_128(mask_words);
        case 256: return mrg_smem_f32_256(mask_words);
        case 512: return mrg_smem_f32_512(mask_words);
        case 1024: return mrg_smem_f32_1024(mask_words);
        }
    } else {
        switch (block) {
        case 128: return mrg_smem_f64_128(mask_words);
        case 256: return mrg_smem_f64_256(mask_words);
        case 512: return mrg_smem_f64_512(mask_words);
        case 1024: return mrg_smem_f64_1024(mask_words);
        }
    }
    return 0;
}
