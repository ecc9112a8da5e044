// score_fp8.cu -- scoring kernels instantiated for the GLV_FP8_E4M3 reduced-row store.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE(GLV_FP8_E4M3)
}  // namespace glv
