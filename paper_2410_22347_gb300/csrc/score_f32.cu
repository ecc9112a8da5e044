// score_f32.cu -- scoring kernels instantiated for the GLV_F32 reduced-row store.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE(GLV_F32)
}  // namespace glv
