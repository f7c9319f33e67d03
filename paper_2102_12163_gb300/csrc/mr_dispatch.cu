// mr_dispatch.cu -- routes a launch to the (precision, block size) instantiation.
#include <cuda_runtime.h>

#include "mr_common.h"

#define MRG_DECLARE(TAG)                                        \
    int mrg_launch_##TAG(int, const mrg::LaunchArgs &, cudaStream_t, int); \
    int mrg_occ_##TAG(int, int, int *);                         \
    int mrg_minb_##TAG(int);                                    \
    size_t mrg_smem_##TAG(int);
MRG_DECLARE(f64_128)
MRG_DECLARE(f64_256)
MRG_DECLARE(f64_512)
MRG_DECLARE(f64_1024)
MRG_DECLARE(f32_128)
MRG_DECLARE(f32_256)
MRG_DECLARE(f32_512)
MRG_DECLARE(f32_1024)

// CALL(TAG) is expanded for the instantiation of (fp32, block); FAIL otherwise.
#define MRG_ROUTE(CALL, FAIL)                    \
    if (fp32) {                                  \
        switch (block) {                         \
        case 128: return CALL(f32_128);          \
        case 256: return CALL(f32_256);          \
        case 512: return CALL(f32_512);          \
        case 1024: return CALL(f32_1024);        \
        }                                        \
    } else {                                     \
        switch (block) {                         \
        case 128: return CALL(f64_128);          \
        case 256: return CALL(f64_256);          \
        case 512: return CALL(f64_512);          \
        case 1024: return CALL(f64_1024);        \
        }                                        \
    }                                            \
    return FAIL;

int mrg_launch(bool fp32, int block, int grid, const mrg::LaunchArgs &a, void *stream, int priority) {
    cudaStream_t s = (cudaStream_t)stream;
#define MRG_CALL(TAG) mrg_launch_##TAG(grid, a, s, priority)
    MRG_ROUTE(MRG_CALL, (int)cudaErrorInvalidValue)
#undef MRG_CALL
}

int mrg_occupancy(bool fp32, int block, int kind, int mask_words, int *nb) {
#define MRG_CALL(TAG) mrg_occ_##TAG(kind, mask_words, nb)
    MRG_ROUTE(MRG_CALL, (int)cudaErrorInvalidValue)
#undef MRG_CALL
}

int mrg_min_blocks(bool fp32, int block, int kind) {
#define MRG_CALL(TAG) mrg_minb_##TAG(kind)
    MRG_ROUTE(MRG_CALL, 0)
#undef MRG_CALL
}

size_t mrg_smem_bytes(bool fp32, int block, int mask_words) {
#define MRG_CALL(TAG) mrg_smem_##TAG(mask_words)
    MRG_ROUTE(MRG_CALL, (size_t)0)
#undef MRG_CALL
}
