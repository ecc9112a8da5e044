// score_fp8_plain.cu -- stand-alone scoring kernels instantiated for the GLV_FP8_E4M3 reduced-row store.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_PLAIN(GLV_FP8_E4M3)
}  // namespace glv
