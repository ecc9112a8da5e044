// score_f32_plain_m1.cu -- stand-alone scoring kernels of the GLV_F32 reduced-row store, gather mode 1
// (pipelined register row loads), instantiated for every lane count and row width.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_PLAIN(GLV_F32, 1)
}  // namespace glv
