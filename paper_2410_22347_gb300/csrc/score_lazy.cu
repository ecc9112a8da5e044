// score_lazy.cu -- the lazy GleanVec inner product (Algorithm 3): the projected query of a
// cluster, A_c q, is formed inside the scoring kernel instead of by a preceding batched
// projection (Algorithm 4, eager).  Recomputing A_c q for every candidate would repeat the
// same product for every candidate of a cluster, so each CTA (one query) computes it once per
// cluster its candidate list actually visits: it marks the visited tags, forms A_c q for those
// clusters only (one warp per output element group, A_c streamed from L2), and then scores the
// list exactly like the eager kernel (same layout, same chunk order).  It also reports how
// many distinct clusters each query visited -- the quantity the paper tracks when comparing
// the lazy and eager variants (Section 5.2).
#include "score_dev.cuh"
#include "score_launch.cuh"

namespace glv {

template <int DT, int G, int NCH>
__global__ void __launch_bounds__(256) score_lazy_kernel(const ScoreArgs a, const float* __restrict__ Q, int D,
                                                         const float* __restrict__ A, int32_t* __restrict__ visited) {
  extern __shared__ __align__(16) float smem[];
  float* qs = smem;                                          // C x qstride projected views
  float* qv = qs + (size_t)a.C * a.qstride;                  // the query
  uint8_t* seen = reinterpret_cast<uint8_t*>(qv + D);        // C flags
  constexpr int EPC = Elem<DT>::kPerChunk;
  const int64_t j = blockIdx.x;
  const int64_t p0 = a.off[j], p1 = a.off[j + 1];
  for (int t = threadIdx.x; t < a.C; t += blockDim.x) seen[t] = 0;
  for (int t = threadIdx.x; t < D; t += blockDim.x) qv[t] = Q[j * (int64_t)D + t];
  __syncthreads();
  for (int64_t p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const int64_t id = a.ids[p];
    if (id >= 0 && id < a.N) {
      const int c = a.tags[id];
      if (c < a.C) seen[c] = 1;
    }
  }
  __syncthreads();
  // q_c = A_c q for the visited clusters: warp w computes rows r = w, w + 8, ... of each,
  // lanes split the D-long dot product
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int dpad = a.nch * EPC;
  int nvis = 0;
  for (int c = 0; c < a.C; ++c) {
    if (!seen[c]) continue;
    ++nvis;
    const float* Ac = A + (int64_t)c * a.d * D;
    for (int r = warp; r < dpad; r += nwarps) {
      float v = 0.f;
      if (r < a.d)
        for (int k = lane; k < D; k += 32) v = fmaf(Ac[(int64_t)r * D + k], qv[k], v);
      v = warp_sum(v);
      if (lane == 0) {
        const int ch = r / EPC, e = r - ch * EPC;
        qs[c * a.qstride + ((e >> 2) * a.sbs + ch) * 4 + (e & 3)] = r < a.d ? v : 0.f;
      }
    }
  }
  if (threadIdx.x == 0 && visited) visited[j] = nvis;
  __syncthreads();
  float* scores = a.scores;
  score_range<DT, G, NCH, false>(a, qs, p0, p1, [scores](int64_t p, float s) { scores[p] = s; });
}

struct LazyLaunch {
  const ScoreArgs& a;
  int64_t nq;
  const float* Q;
  int D;
  const float* A;
  int32_t* visited;
  size_t smem;
  cudaStream_t st;
  template <int DT, int G, int NCH, int MODE>
  cudaError_t go() {
    if constexpr (MODE != 0) {
      return cudaErrorInvalidValue;
    } else {
      auto k = score_lazy_kernel<DT, G, NCH>;
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k<<<(unsigned)nq, 256, smem, st>>>(a, Q, D, A, visited);
      return cudaGetLastError();
    }
  }
};

size_t lazy_smem_bytes(int C, int d, int D, int dt) {
  const int eb = dt == GLV_F32 ? 4 : (dt == GLV_BF16 ? 2 : 1);
  const int qstride = qp_qstride((d * eb + 15) / 16, dt);
  return (size_t)C * qstride * 4 + (size_t)D * 4 + (size_t)C + 16;
}

cudaError_t launch_score_lazy(const ScoreArgs& a0, int dt, int64_t nq, const float* Q, int D, const float* A,
                              int32_t* visited, cudaStream_t st) {
  ScoreArgs a = a0;
  a.sbs = qp_sbs(a.nch, dt);
  a.qstride = qp_qstride(a.nch, dt);
  a.splits = 1;
  const size_t smem = lazy_smem_bytes(a.C, a.d, D, dt);
  switch (dt) {
    case GLV_F32: {
      LazyLaunch f{a, nq, Q, D, A, visited, smem, st};
      return dispatch_score_default<GLV_F32>(a.nch, f);
    }
    case GLV_BF16: {
      LazyLaunch f{a, nq, Q, D, A, visited, smem, st};
      return dispatch_score_default<GLV_BF16>(a.nch, f);
    }
    default: {
      LazyLaunch f{a, nq, Q, D, A, visited, smem, st};
      return dispatch_score_default<GLV_FP8_E4M3>(a.nch, f);
    }
  }
}

}  // namespace glv
