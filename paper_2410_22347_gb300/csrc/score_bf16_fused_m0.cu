// score_bf16_fused_m0.cu -- fused scoring + top-kappa kernels of the GLV_BF16 reduced-row store, gather mode 0
// (register row loads), instantiated for every lane count and row width.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_FUSED(GLV_BF16, 0)
}  // namespace glv
