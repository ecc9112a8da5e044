// score_f32_plain.cu -- stand-alone scoring kernels instantiated for the GLV_F32 reduced-row store.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_PLAIN(GLV_F32)
}  // namespace glv
