// score_bf16.cu -- scoring kernels instantiated for the GLV_BF16 reduced-row store.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE(GLV_BF16)
}  // namespace glv
