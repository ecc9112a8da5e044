// score_bf16_plain.cu -- stand-alone scoring kernels instantiated for the GLV_BF16 reduced-row store.
#include "score_variants.cuh"

namespace glv {
GLV_INSTANTIATE_SCORE_PLAIN(GLV_BF16)
}  // namespace glv
