// autotune.cu -- tile order and schedule selection.
//
// chol_default_nb is a fixed table (a pure function of n and precision), so
// the batched and served paths give a matrix the same nb alone and in a mix.
#include "common.cuh"

extern "C" {

int64_t chol_default_nb(int64_t n, int32_t precision) {
    if (precision == CHOL_FP64) {
        // binary64 runs on the CUDA cores at a low per-SM rate: small tiles
        // shorten the POTRF->TRSM->SYRK critical path, which dominates small n
        if (n <= 1024) return 32;
        if (n <= 4096) return 64;
        if (n <= 16384) return 128;
        return 256;
    }
    // tensor-core precisions: tiles are multiples of the 128-row MMA
    if (n <= 8192) return 128;
    if (n <= 32768) return 256;
    return 512;
}

}  // extern "C"
