// score.cu -- stand-alone gather-score kernel of the eager GleanVec inner product
// (Algorithm 4, procedure inner-product; Eq. GleanVec approximation, Section 4):
//
//     s(j, i) = < q_{j, c_i} , x_i^low >            (times s_i for FP8 rows)
//
// One CTA per (query, split of its candidate list); the query's C projected views (C x d
// floats, <= 192 KB) are staged once in shared memory, so every candidate, whatever its
// cluster, finds its q_c on chip (the "eager" choice of the paper).  The per-candidate body
// is score_range() in score_dev.cuh.
#include "score_dev.cuh"

namespace glv {

template <int DT, int G, int NCH>
__global__ void __launch_bounds__(256) score_kernel(const ScoreArgs a) {
  extern __shared__ __align__(16) float qs[];
  const int64_t j = blockIdx.x;
  stage_qp(a, j, qs);
  __syncthreads();
  const int64_t p0 = a.off[j], p1 = a.off[j + 1];
  const int64_t per = (p1 - p0 + a.splits - 1) / a.splits;
  const int64_t b0 = p0 + (int64_t)blockIdx.y * per;
  const int64_t b1 = min(p1, b0 + per);
  float* scores = a.scores;
  score_range<DT, G, NCH>(a, qs, b0, b1, [scores](int64_t p, float s) { scores[p] = s; });
}

template <int DT, int G>
static cudaError_t launch_g(const ScoreArgs& a, int nch_lane, dim3 grid, size_t smem,
                            cudaStream_t st) {
#define GLV_SCORE_CASE(n)                                                                 \
  case n: {                                                                               \
    auto k = score_kernel<DT, G, n>;                                                      \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                         (int)smem);                                      \
    if (e != cudaSuccess) return e;                                                       \
    k<<<grid, 256, smem, st>>>(a);                                                        \
    return cudaGetLastError();                                                            \
  }
  switch (nch_lane) {
    GLV_SCORE_CASE(1)
    GLV_SCORE_CASE(2)
    GLV_SCORE_CASE(3)
    GLV_SCORE_CASE(4)
    GLV_SCORE_CASE(5)
    GLV_SCORE_CASE(6)
    GLV_SCORE_CASE(7)
    GLV_SCORE_CASE(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef GLV_SCORE_CASE
}

// Lanes per candidate: the fewest (from the dtype's default upward, then 32) that need at
// most 8 chunk loads each.
template <int DT>
static cudaError_t launch_dt(const ScoreArgs& a, dim3 grid, size_t smem, cudaStream_t st) {
  constexpr int G0 = default_group<DT>();
  if ((a.nch + G0 - 1) / G0 <= 8) return launch_g<DT, G0>(a, (a.nch + G0 - 1) / G0, grid, smem, st);
  return launch_g<DT, 32>(a, (a.nch + 31) / 32, grid, smem, st);
}

cudaError_t launch_score(const ScoreArgs& a0, int dt, int64_t nq, int num_sms,
                         cudaStream_t st) {
  ScoreArgs a = a0;
  const int epc = 16 / (dt == GLV_F32 ? 4 : (dt == GLV_BF16 ? 2 : 1));
  const int dpad = (a.d + epc - 1) / epc * epc;
  a.qstride = dpad + 4;  // +16 bytes: consecutive cluster rows start in different banks
  const size_t smem = (size_t)a.C * a.qstride * sizeof(float);
  // enough CTAs to fill the machine a few times over even for few queries
  const int64_t want = (int64_t)num_sms * 8;
  int splits = (int)((want + nq - 1) / nq);
  if (splits < 1) splits = 1;
  if (splits > 64) splits = 64;
  a.splits = splits;
  dim3 grid((unsigned)nq, (unsigned)splits);
  switch (dt) {
    case GLV_F32: return launch_dt<GLV_F32>(a, grid, smem, st);
    case GLV_BF16: return launch_dt<GLV_BF16>(a, grid, smem, st);
    default: return launch_dt<GLV_FP8_E4M3>(a, grid, smem, st);
  }
}

}  // namespace glv
