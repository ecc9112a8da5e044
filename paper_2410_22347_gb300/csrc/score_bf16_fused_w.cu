// score_bf16_fused_w.cu -- fused scoring + top-kappa kernels of the GLV_BF16 reduced-row store with
// wide CTAs (512 threads, register row loads), instantiated for the two smaller lane counts.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_WIDE(GLV_BF16)
}  // namespace glv
