// topk.cu -- stand-alone per-query top-kappa of candidate scores (Algorithm 1: the main
// step hands kappa candidates to the exact post-processing).  One CTA per query runs
// select_topk() (topk_dev.cuh).  A list of at most kTopkCache entries has its keys cached in
// shared memory for the selection passes; a longer one re-reads its scores each pass (they
// stay L2-resident while the CTA runs).
#include "kernels.cuh"
#include "topk_dev.cuh"

namespace glv {

__global__ void __launch_bounds__(kTopkThreads) topk_kernel(const float* __restrict__ scores,
                                                           const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ ids,
                                                           int kappa, float* __restrict__ out_s,
                                                           int32_t* __restrict__ out_id) {
  __shared__ TopkSmem S;
  extern __shared__ __align__(16) uint32_t kcache[];  // kTopkCache keys, then kappa selected keys and ids
  if (threadIdx.x == 0) {
    S.sel_key = kcache + kTopkCache;
    S.sel_id = reinterpret_cast<int32_t*>(kcache + kTopkCache + kappa);
    S.region = kcache;
    S.region_words = kTopkCache;
  }
  const int64_t j = blockIdx.x;
  const int64_t p0 = off[j];
  const int64_t L = off[j + 1] - p0;
  const float* sj = scores + p0;
  const int32_t* ij = ids + p0;
  const bool cached = L <= kTopkCache;
  if (cached)
    for (int64_t p = threadIdx.x; p < L; p += blockDim.x) kcache[p] = score_key(sj[p]);
  __syncthreads();
  select_topk(
      S, L, kappa, cached, [&](int64_t p) -> uint32_t { return cached ? kcache[p] : score_key(sj[p]); },
      [&](int64_t p) -> int32_t { return ij[p]; }, out_s + j * kappa, out_id + j * kappa);
}

cudaError_t launch_topk(const float* scores, const int64_t* off, const int32_t* ids, int64_t nq,
                        int kappa, float* out_s, int32_t* out_id, cudaStream_t st) {
  const size_t smem = (size_t)kTopkCache * sizeof(uint32_t) + (size_t)kappa * 8;
  cudaError_t e = cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  topk_kernel<<<(unsigned)nq, kTopkThreads, smem, st>>>(scores, off, ids, kappa, out_s, out_id);
  return cudaGetLastError();
}

}  // namespace glv
