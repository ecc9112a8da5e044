// score_bf16_plain_m1.cu -- stand-alone scoring kernels of the GLV_BF16 reduced-row store, gather mode 1
// (pipelined register row loads), instantiated for every lane count and row width.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_PLAIN(GLV_BF16, 1)
}  // namespace glv
