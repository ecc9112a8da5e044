// score_f32_fused.cu -- fused scoring + top-kappa kernels instantiated for the GLV_F32 reduced-row store.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_FUSED(GLV_F32)
}  // namespace glv
