// score_f32_fused_m0.cu -- fused scoring + top-kappa kernels of the GLV_F32 reduced-row store, gather mode 0
// (register row loads), instantiated for every lane count and row width.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_FUSED(GLV_F32, 0)
}  // namespace glv
