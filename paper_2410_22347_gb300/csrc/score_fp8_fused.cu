// score_fp8_fused.cu -- fused scoring + top-kappa kernels instantiated for the GLV_FP8_E4M3 reduced-row store.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_FUSED(GLV_FP8_E4M3)
}  // namespace glv
