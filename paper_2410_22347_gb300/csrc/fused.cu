// fused.cu -- gather-score and top-kappa of one query in one CTA (Algorithm 4 inner-product
// followed by the kappa-candidate cut of Algorithm 1's main step), so the scores of a list
// never leave the chip: they are kept as order-preserving keys in shared memory and the
// radix selection runs there.  A list longer than kFusedCache (2048) entries spills its scores to
// the caller's scratch array (where they stay L2-resident for the selection passes).
// Scores are produced by the same score_range() body as the stand-alone kernel, so the
// result is bit-identical to glv_score_candidates followed by glv_topk.
#include "kernels.cuh"
#include "score_dev.cuh"
#include "topk_dev.cuh"

namespace glv {

constexpr int kFusedCache = 2048;

template <int DT, int G, int NCH>
__global__ void __launch_bounds__(256, 5) score_topk_kernel(const ScoreArgs a, int kappa, float* out_s,
                                                         int32_t* out_id) {
  extern __shared__ __align__(16) float smem[];
  __shared__ TopkSmem S;
  float* qs = smem;
  uint32_t* kc = reinterpret_cast<uint32_t*>(smem + (size_t)a.C * a.qstride);
  const int64_t j = blockIdx.x;
  stage_qp(a, j, qs);
  __syncthreads();
  const int64_t p0 = a.off[j], p1 = a.off[j + 1];
  const int64_t L = p1 - p0;
  const bool cached = L <= kFusedCache;
  float* scores = a.scores;
  if (cached)
    score_range<DT, G, NCH>(a, qs, p0, p1, [kc, p0](int64_t p, float s) { kc[p - p0] = score_key(s); });
  else
    score_range<DT, G, NCH>(a, qs, p0, p1, [scores](int64_t p, float s) { scores[p] = s; });
  __syncthreads();
  const float* sj = scores + p0;
  const int32_t* ij = a.ids + p0;
  select_topk(
      S, L, kappa, [&](int64_t p) -> uint32_t { return cached ? kc[p] : score_key(sj[p]); },
      [&](int64_t p) -> int32_t { return ij[p]; }, out_s + j * kappa, out_id + j * kappa);
}

template <int DT, int G>
static cudaError_t fused_launch_g(const ScoreArgs& a, int nch_lane, int64_t nq, size_t smem, int kappa,
                                  float* out_s, int32_t* out_id, cudaStream_t st) {
#define GLV_FUSED_CASE(n)                                                                \
  case n: {                                                                              \
    auto k = score_topk_kernel<DT, G, n>;                                                \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                     \
    if (e != cudaSuccess) return e;                                                      \
    k<<<(unsigned)nq, 256, smem, st>>>(a, kappa, out_s, out_id);                         \
    return cudaGetLastError();                                                           \
  }
  switch (nch_lane) {
    GLV_FUSED_CASE(1)
    GLV_FUSED_CASE(2)
    GLV_FUSED_CASE(3)
    GLV_FUSED_CASE(4)
    GLV_FUSED_CASE(5)
    GLV_FUSED_CASE(6)
    GLV_FUSED_CASE(7)
    GLV_FUSED_CASE(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef GLV_FUSED_CASE
}

template <int DT>
static cudaError_t fused_launch_dt(const ScoreArgs& a, int64_t nq, size_t smem, int kappa, float* out_s,
                                   int32_t* out_id, cudaStream_t st) {
  constexpr int G0 = default_group<DT>();
  if ((a.nch + G0 - 1) / G0 <= 8)
    return fused_launch_g<DT, G0>(a, (a.nch + G0 - 1) / G0, nq, smem, kappa, out_s, out_id, st);
  return fused_launch_g<DT, 32>(a, (a.nch + 31) / 32, nq, smem, kappa, out_s, out_id, st);
}

size_t fused_smem_bytes(int C, int d, int dt) {
  const int epc = 16 / (dt == GLV_F32 ? 4 : (dt == GLV_BF16 ? 2 : 1));
  const int dpad = (d + epc - 1) / epc * epc;
  return (size_t)C * (dpad + 4) * sizeof(float) + (size_t)kFusedCache * sizeof(uint32_t);
}

cudaError_t launch_score_topk(const ScoreArgs& a0, int dt, int64_t nq, int kappa, float* out_s,
                              int32_t* out_id, int num_sms, cudaStream_t st) {
  // Few queries: one CTA per query would leave the GPU idle, so split the lists over CTAs
  // (stand-alone scoring) and select afterwards.
  if (nq < (int64_t)num_sms * 4) {
    cudaError_t e = launch_score(a0, dt, nq, num_sms, st);
    if (e != cudaSuccess) return e;
    return launch_topk(a0.scores, a0.off, a0.ids, nq, kappa, out_s, out_id, st);
  }
  ScoreArgs a = a0;
  const int epc = 16 / (dt == GLV_F32 ? 4 : (dt == GLV_BF16 ? 2 : 1));
  a.qstride = (a.d + epc - 1) / epc * epc + 4;
  a.splits = 1;
  const size_t smem = fused_smem_bytes(a.C, a.d, dt);
  switch (dt) {
    case GLV_F32: return fused_launch_dt<GLV_F32>(a, nq, smem, kappa, out_s, out_id, st);
    case GLV_BF16: return fused_launch_dt<GLV_BF16>(a, nq, smem, kappa, out_s, out_id, st);
    default: return fused_launch_dt<GLV_FP8_E4M3>(a, nq, smem, kappa, out_s, out_id, st);
  }
}

}  // namespace glv
