// score_fp8_fused_w.cu -- fused scoring + top-kappa kernels of the GLV_FP8_E4M3 reduced-row store with
// wide CTAs (512 threads, register row loads), instantiated for the two smaller lane counts.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_WIDE(GLV_FP8_E4M3)
}  // namespace glv
