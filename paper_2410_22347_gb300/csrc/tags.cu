// tags.cu -- cluster tags of Eq. (cluster_tag), Section 4:  c_i = argmax_c <x_i, mu_c>.
//
// The C landmarks are staged once per CTA in shared memory.  One warp per database row:
// lane l holds elements l, l+32, ... of the row in registers (a coalesced read of the
// row), and for each landmark the warp forms the dot with an xor-shuffle reduction, which
// leaves the full sum in every lane.  Ties keep the lowest c (strict comparison).
#include "common.cuh"
#include "kernels.cuh"

namespace glv {

template <int NPL>  // row elements per lane (D <= 32 * NPL)
__global__ void __launch_bounds__(256) tags_kernel(const float* __restrict__ X, int64_t N, int D,
                                                   const float* __restrict__ mu, int C,
                                                   uint16_t* __restrict__ tags) {
  extern __shared__ float ms[];  // C x D
  for (int t = threadIdx.x; t < C * D; t += blockDim.x) ms[t] = mu[t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < N;
       i += warps) {
    float x[NPL];
#pragma unroll
    for (int u = 0; u < NPL; ++u) {
      const int e = lane + 32 * u;
      x[u] = e < D ? ld_stream_f32(X + i * D + e) : 0.f;
    }
    float best = -INFINITY;
    int bc = 0;
    for (int c = 0; c < C; ++c) {
      const float* m = ms + c * D;
      float s = 0.f;
#pragma unroll
      for (int u = 0; u < NPL; ++u) {
        const int e = lane + 32 * u;
        if (e < D) s = fmaf(x[u], m[e], s);
      }
      s = warp_sum(s);
      if (s > best) {
        best = s;
        bc = c;
      }
    }
    if (lane == 0) tags[i] = (uint16_t)bc;
  }
}

cudaError_t launch_tags(const float* X, int64_t N, int D, const float* mu, int C, uint16_t* tags,
                        int num_sms, cudaStream_t st) {
  const size_t smem = (size_t)C * D * sizeof(float);
  int64_t blocks = (N + 7) / 8;
  const int64_t cap = (int64_t)num_sms * 8;
  if (blocks > cap) blocks = cap;
#define GLV_TAGS(NPL)                                                                    \
  {                                                                                      \
    auto k = tags_kernel<NPL>;                                                           \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                     \
    if (e != cudaSuccess) return e;                                                      \
    k<<<(unsigned)blocks, 256, smem, st>>>(X, N, D, mu, C, tags);                        \
    return cudaGetLastError();                                                           \
  }
  const int npl = (D + 31) / 32;
  if (npl <= 8) GLV_TAGS(8)
  if (npl <= 16) GLV_TAGS(16)
  if (npl <= 24) GLV_TAGS(24)
  if (npl <= 32) GLV_TAGS(32)
#undef GLV_TAGS
  return cudaErrorInvalidValue;
}

}  // namespace glv
