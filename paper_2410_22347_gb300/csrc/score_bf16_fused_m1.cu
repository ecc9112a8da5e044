// score_bf16_fused_m1.cu -- fused scoring + top-kappa kernels of the GLV_BF16 reduced-row store, gather mode 1
// (pipelined register row loads), instantiated for every lane count and row width.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_FUSED(GLV_BF16, 1)
}  // namespace glv
