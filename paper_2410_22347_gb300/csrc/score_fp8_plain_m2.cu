// score_fp8_plain_m2.cu -- stand-alone scoring kernels of the GLV_FP8_E4M3 reduced-row store, gather mode 2
// (bulk row copies into shared memory), instantiated for every lane count and row width.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_PLAIN(GLV_FP8_E4M3, 2)
}  // namespace glv
