// rerank.cu -- post-processing of Algorithm 1: exact inner products <q_j, x_i> in full
// dimension D for each query's kappa survivors, then the top k of them.
//
// One CTA per query; q_j is staged in shared memory.  Each warp scores R survivors at a
// time: every lane issues its 16-byte loads of all R rows (a D-float row is D/128 loads per
// lane) before the FMAs, so a warp has R * D * 4 bytes in flight; shuffles finish the dots.
// The k best (score desc, id asc) come from a bitonic sort of the packed values
// key << 32 | id_rank(id) in one warp (kappa <= 256), else each survivor's rank is counted.
#include "common.cuh"
#include "kernels.cuh"
#include "topk_dev.cuh"

namespace glv {

constexpr int kRerankThreads = 256;

// Warp 0: sort the kappa (<= 32 E) scored survivors, invalid ones packed as 0 (last), and
// write the first min(n_valid, k).
template <int E>
GLV_DEV void rerank_warp_topk(const RerankArgs& a, const uint32_t* skey, const int32_t* sid, const uint8_t* sval,
                              int n, int64_t j) {
  const int lane = threadIdx.x & 31;
  uint64_t v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int t = lane * E + e;
    v[e] = (t < a.kappa && sval[t]) ? ((uint64_t)skey[t] << 32) | id_rank(sid[t]) : 0ull;
  }
  warp_bitonic_sort<E>(v, lane);
  const int m = n < a.k ? n : a.k;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int t = lane * E + e;
    if (t < m) {
      a.out_s[j * a.k + t] = key_score((uint32_t)(v[e] >> 32));
      a.out_id[j * a.k + t] = id_from_rank((uint32_t)v[e]);
    }
  }
}

// VEC: D % 4 == 0 and X, Q 16-byte aligned -> float4 loads; NL = max float4 loads per lane
// per row (D <= 128 * NL), R = rows per warp iteration.
template <bool VEC, int NL, int R>
__global__ void __launch_bounds__(kRerankThreads) rerank_kernel(const RerankArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Dp = (a.D + 3) & ~3;
  float* qs = reinterpret_cast<float*>(smem_raw);
  uint32_t* skey = reinterpret_cast<uint32_t*>(qs + Dp);
  int32_t* sid = reinterpret_cast<int32_t*>(skey + a.kappa);
  uint8_t* sval = reinterpret_cast<uint8_t*>(sid + a.kappa);
  __shared__ int n_valid;

  const int64_t j = blockIdx.x;
  const float* qj = a.Q + j * (int64_t)a.D;
  for (int t = threadIdx.x; t < Dp; t += blockDim.x) qs[t] = t < a.D ? qj[t] : 0.f;
  if (threadIdx.x == 0) n_valid = 0;
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int32_t* sj = a.surv + j * (int64_t)a.kappa;
  for (int t0 = warp * R; t0 < a.kappa; t0 += nwarps * R) {
    int64_t id[R];
    bool ok[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int t = t0 + r;
      id[r] = t < a.kappa ? (int64_t)sj[t] : -1;
      ok[r] = id[r] >= 0 && id[r] < a.N;
    }
    float acc[R];
    if constexpr (VEC) {
      float4 v[R][NL];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float* row = a.X + id[r] * a.D;
#pragma unroll
        for (int u = 0; u < NL; ++u) {
          const int c4 = lane + 32 * u;
          if (ok[r] && 4 * c4 < a.D) {
            uint4 w = ld_stream_v4(row + 4 * c4);
            v[r][u] = make_float4(__uint_as_float(w.x), __uint_as_float(w.y),
                                  __uint_as_float(w.z), __uint_as_float(w.w));
          } else {
            v[r][u] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float s = 0.f;
#pragma unroll
        for (int u = 0; u < NL; ++u) {
          const int c4 = lane + 32 * u;
          if (4 * c4 < a.D) {
            const float4 q = reinterpret_cast<const float4*>(qs)[c4];
            s = fmaf(q.x, v[r][u].x, s);
            s = fmaf(q.y, v[r][u].y, s);
            s = fmaf(q.z, v[r][u].z, s);
            s = fmaf(q.w, v[r][u].w, s);
          }
        }
        acc[r] = s;
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float s = 0.f;
        if (ok[r]) {
          const float* row = a.X + id[r] * a.D;
          for (int e = lane; e < a.D; e += 32) s = fmaf(qs[e], ld_stream_f32(row + e), s);
        }
        acc[r] = s;
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float s = warp_sum(acc[r]);
      const int t = t0 + r;
      if (lane == 0 && t < a.kappa) {
        skey[t] = score_key(s);
        sid[t] = (int32_t)id[r];
        sval[t] = ok[r] ? 1 : 0;
        if (ok[r]) atomicAdd(&n_valid, 1);
        else if (id[r] != -1) report(a.d_status, GLV_ERR_BAD_ID);
      }
    }
  }
  __syncthreads();
  const int n = n_valid;
  if (a.kappa <= 256) {
    if (warp == 0) {
      if (a.kappa <= 64) rerank_warp_topk<2>(a, skey, sid, sval, n, j);
      else if (a.kappa <= 128) rerank_warp_topk<4>(a, skey, sid, sval, n, j);
      else rerank_warp_topk<8>(a, skey, sid, sval, n, j);
    }
  } else {
  for (int e = threadIdx.x; e < a.kappa; e += blockDim.x) {
    if (!sval[e]) continue;
    const uint32_t ke = skey[e];
    const int32_t ie = sid[e];
    int rank = 0;
    for (int f = 0; f < a.kappa; ++f) {
      if (!sval[f]) continue;
      const uint32_t kf = skey[f];
      const int32_t idf = sid[f];
      rank += (ranks_before(kf, idf, ke, ie) || (kf == ke && idf == ie && f < e)) ? 1 : 0;
    }
    if (rank < a.k) {
      a.out_s[j * a.k + rank] = key_score(ke);
      a.out_id[j * a.k + rank] = ie;
    }
  }
  }
  for (int e = n + threadIdx.x; e < a.k; e += blockDim.x) {
    a.out_s[j * a.k + e] = -INFINITY;
    a.out_id[j * a.k + e] = -1;
  }
}

size_t rerank_smem_bytes(int D, int kappa) {
  const int Dp = (D + 3) & ~3;
  return (size_t)Dp * 4 + (size_t)kappa * 9 + 16;
}

cudaError_t launch_rerank(const RerankArgs& a, int64_t nq, bool vec, cudaStream_t st) {
  const size_t smem = rerank_smem_bytes(a.D, a.kappa);
  constexpr int R = 2;
#define GLV_RR(NL)                                                                            \
  {                                                                                           \
    auto kf = rerank_kernel<true, NL, R>;                                                     \
    cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                         (int)smem);                                          \
    if (e != cudaSuccess) return e;                                                           \
    kf<<<(unsigned)nq, kRerankThreads, smem, st>>>(a);                                        \
    return cudaGetLastError();                                                                \
  }
  if (vec) {
    const int nl = (a.D + 127) / 128;
    if (nl <= 2) GLV_RR(2)
    if (nl <= 4) GLV_RR(4)
    if (nl <= 6) GLV_RR(6)
    if (nl <= 8) GLV_RR(8)
  }
#undef GLV_RR
  auto kf = rerank_kernel<false, 1, R>;
  cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kf<<<(unsigned)nq, kRerankThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace glv
