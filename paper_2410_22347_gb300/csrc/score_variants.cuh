// score_variants.cuh -- the stand-alone scoring kernel and the fused scoring + top-kappa
// kernel as templates over (store type, lanes per candidate, loads per lane, pipelining),
// with the launchers that instantiate them for one store type (one translation unit per
// store type: score_f32.cu, score_bf16.cu, score_fp8.cu).
#pragma once

#include "kernels.cuh"
#include "score_dev.cuh"
#include "score_launch.cuh"
#include "topk_dev.cuh"

namespace glv {

constexpr int kFusedCache = 2048;  // list entries kept as keys in shared memory

// One CTA per (query, split of its candidate list): the query's C projected views are staged
// once in shared memory, so every candidate, whatever its cluster, finds its q_c on chip (the
// "eager" inner product of the paper).
template <int DT, int G, int NCH, bool PIPE>
__global__ void __launch_bounds__(256) score_kernel(const ScoreArgs a) {
  extern __shared__ __align__(16) float qs[];
  const int64_t j = blockIdx.x;
  stage_qp<DT>(a, j, qs);
  __syncthreads();
  const int64_t p0 = a.off[j], p1 = a.off[j + 1];
  const int64_t per = (p1 - p0 + a.splits - 1) / a.splits;
  const int64_t b0 = p0 + (int64_t)blockIdx.y * per;
  const int64_t b1 = min(p1, b0 + per);
  float* scores = a.scores;
  score_range<DT, G, NCH, PIPE>(a, qs, b0, b1, [scores](int64_t p, float s) { scores[p] = s; });
}

// Gather-score and top-kappa of one query in one CTA: scores stay on chip as order-preserving
// keys in shared memory and the radix selection runs there; a list longer than kFusedCache
// spills its scores to the caller's scratch (L2-resident during the selection passes).
template <int DT, int G, int NCH, bool PIPE>
__global__ void __launch_bounds__(256, PIPE ? 3 : 5) score_topk_kernel(const ScoreArgs a, int kappa, float* out_s,
                                                            int32_t* out_id) {
  extern __shared__ __align__(16) float smem[];
  __shared__ TopkSmem S;
  float* qs = smem;
  uint32_t* kc = reinterpret_cast<uint32_t*>(smem + (size_t)a.C * a.qstride);
  const int64_t j = blockIdx.x;
  stage_qp<DT>(a, j, qs);
  __syncthreads();
  const int64_t p0 = a.off[j], p1 = a.off[j + 1];
  const int64_t L = p1 - p0;
  const bool cached = L <= kFusedCache;
  float* scores = a.scores;
  if (cached)
    score_range<DT, G, NCH, PIPE>(a, qs, p0, p1, [kc, p0](int64_t p, float s) { kc[p - p0] = score_key(s); });
  else
    score_range<DT, G, NCH, PIPE>(a, qs, p0, p1, [scores](int64_t p, float s) { scores[p] = s; });
  __syncthreads();
  const float* sj = scores + p0;
  const int32_t* ij = a.ids + p0;
  select_topk(
      S, L, kappa, [&](int64_t p) -> uint32_t { return cached ? kc[p] : score_key(sj[p]); },
      [&](int64_t p) -> int32_t { return ij[p]; }, out_s + j * kappa, out_id + j * kappa);
}

struct ScoreLaunch {
  const ScoreArgs& a;
  dim3 grid;
  size_t smem;
  cudaStream_t st;
  template <int DT, int G, int NCH, bool PIPE>
  cudaError_t go() {
    auto k = score_kernel<DT, G, NCH, PIPE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
  }
};

struct FusedLaunch {
  const ScoreArgs& a;
  int64_t nq;
  size_t smem;
  int kappa;
  float* out_s;
  int32_t* out_id;
  cudaStream_t st;
  template <int DT, int G, int NCH, bool PIPE>
  cudaError_t go() {
    auto k = score_topk_kernel<DT, G, NCH, PIPE>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)nq, 256, smem, st>>>(a, kappa, out_s, out_id);
    return cudaGetLastError();
  }
};

template <int DT>
cudaError_t launch_score_dt(const ScoreArgs& a, dim3 grid, size_t smem, ScoreConfig cfg, cudaStream_t st) {
  ScoreLaunch f{a, grid, smem, st};
  return dispatch_score<DT>(cfg.G, a.nch, cfg.pipe, f);
}

template <int DT>
cudaError_t launch_fused_dt(const ScoreArgs& a, int64_t nq, size_t smem, int kappa, float* out_s,
                            int32_t* out_id, ScoreConfig cfg, cudaStream_t st) {
  FusedLaunch f{a, nq, smem, kappa, out_s, out_id, st};
  return dispatch_score<DT>(cfg.G, a.nch, cfg.pipe, f);
}

#define GLV_INSTANTIATE_SCORE(DT)                                                                       \
  template cudaError_t launch_score_dt<DT>(const ScoreArgs&, dim3, size_t, ScoreConfig, cudaStream_t); \
  template cudaError_t launch_fused_dt<DT>(const ScoreArgs&, int64_t, size_t, int, float*, int32_t*,    \
                                           ScoreConfig, cudaStream_t);

}  // namespace glv
