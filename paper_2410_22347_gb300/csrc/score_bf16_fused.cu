// score_bf16_fused.cu -- fused scoring + top-kappa kernels instantiated for the GLV_BF16 reduced-row store.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_FUSED(GLV_BF16)
}  // namespace glv
