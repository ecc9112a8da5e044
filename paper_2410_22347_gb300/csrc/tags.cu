// tags.cu -- cluster tags of Eq. (cluster_tag), Section 4:  c_i = argmax_c <x_i, mu_c>.
//
// The C landmarks are staged in shared memory (once per CTA when they fit in 96 KB, else in
// tiles of whole landmarks, re-read from L2 for every group of rows).  One warp per database row:
// lane l holds elements l, l+32, ... of the row in registers (a coalesced read of the
// row), and for each landmark the warp forms the dot with an xor-shuffle reduction, which
// leaves the full sum in every lane.  Ties keep the lowest c (strict comparison).
#include "common.cuh"
#include "kernels.cuh"

namespace glv {

template <int NPL>  // row elements per lane (D <= 32 * NPL)
__global__ void __launch_bounds__(256) tags_kernel(const float* __restrict__ X, int64_t N, int D,
                                                   const float* __restrict__ mu, int C, int tile_c,
                                                   uint16_t* __restrict__ tags, float* __restrict__ best_ip) {
  // landmarks are staged tile_c at a time (all of them at once when they fit); a warp keeps its
  // row in registers across the tiles, and the tiles are visited in cluster order so the
  // running argmax keeps the first maximum
  extern __shared__ float ms[];  // tile_c x D
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const bool single = tile_c >= C;
  if (single) {
    for (int t = threadIdx.x; t < C * D; t += blockDim.x) ms[t] = mu[t];
    __syncthreads();
  }
  // block-uniform loop over groups of wpb rows (the tile loop below synchronises the block)
  for (int64_t i0 = (int64_t)blockIdx.x * wpb; i0 < N; i0 += (int64_t)gridDim.x * wpb) {
    const int64_t i = i0 + warp;
    const bool row = i < N;
    float x[NPL];
#pragma unroll
    for (int u = 0; u < NPL; ++u) {
      const int e = lane + 32 * u;
      x[u] = (row && e < D) ? ld_stream_f32(X + i * D + e) : 0.f;
    }
    float best = -INFINITY;
    int bc = 0;
    for (int c0 = 0; c0 < C; c0 += tile_c) {
      const int nc = min(tile_c, C - c0);
      if (!single) {
        __syncthreads();
        for (int t = threadIdx.x; t < nc * D; t += blockDim.x) ms[t] = mu[(int64_t)c0 * D + t];
        __syncthreads();
      }
      for (int c = 0; c < nc; ++c) {
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
          bc = c0 + c;
        }
      }
    }
    if (row && lane == 0) {
      tags[i] = (uint16_t)bc;
      if (best_ip) best_ip[i] = best;
    }
  }
}

// Landmark tile: as many whole landmarks as fit in 96 KB of shared memory (two CTAs per SM).
inline int tags_tile(int C, int D) {
  const int fit = (96 * 1024) / (D * 4);
  return fit < 1 ? 1 : (fit < C ? fit : C);
}

cudaError_t launch_tags(const float* X, int64_t N, int D, const float* mu, int C, uint16_t* tags,
                        float* best_ip, int num_sms, cudaStream_t st) {
  const int tile_c = tags_tile(C, D);
  const size_t smem = (size_t)tile_c * D * sizeof(float);
  int64_t blocks = (N + 7) / 8;
  const int64_t cap = (int64_t)num_sms * 8;
  if (blocks > cap) blocks = cap;
#define GLV_TAGS(NPL)                                                                    \
  {                                                                                      \
    auto k = tags_kernel<NPL>;                                                           \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                                     \
    if (e != cudaSuccess) return e;                                                      \
    k<<<(unsigned)blocks, 256, smem, st>>>(X, N, D, mu, C, tile_c, tags, best_ip);       \
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

// ---- spherical k-means M-step (Appendix A) -------------------------------------------------
//   mu_c = sum_{i: c_i = c} x_i / || . ||_2, rows grouped by cluster (launch_grouping); FP64
//   sums, one CTA per (cluster, 128-column block); a cluster without members (or with a zero
//   sum) keeps its landmark.

namespace glv {

__global__ void __launch_bounds__(128) kmeans_sum_kernel(const float* __restrict__ X, int D, BuildWs g,
                                                         double* __restrict__ sums) {
  const int c = blockIdx.x;
  const int k = blockIdx.y * 128 + threadIdx.x;
  if (k >= D) return;
  const int64_t start = g.seg_start[c], cnt = g.counts[c];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int64_t r = 0;
  for (; r + 4 <= cnt; r += 4) {
    s0 += (double)X[(int64_t)g.perm[start + r] * D + k];
    s1 += (double)X[(int64_t)g.perm[start + r + 1] * D + k];
    s2 += (double)X[(int64_t)g.perm[start + r + 2] * D + k];
    s3 += (double)X[(int64_t)g.perm[start + r + 3] * D + k];
  }
  for (; r < cnt; ++r) s0 += (double)X[(int64_t)g.perm[start + r] * D + k];
  sums[(int64_t)c * D + k] = (s0 + s1) + (s2 + s3);
}

__global__ void __launch_bounds__(256) kmeans_normalize_kernel(const double* __restrict__ sums, int D,
                                                               const int32_t* __restrict__ counts,
                                                               float* __restrict__ mu) {
  __shared__ double part[256];
  const int c = blockIdx.x;
  double q = 0.0;
  for (int k = threadIdx.x; k < D; k += blockDim.x) {
    const double v = sums[(int64_t)c * D + k];
    q += v * v;
  }
  part[threadIdx.x] = q;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  const double nrm = sqrt(part[0]);
  if (counts[c] == 0 || !(nrm > 0.0)) return;  // keep the previous landmark
  for (int k = threadIdx.x; k < D; k += blockDim.x) mu[(int64_t)c * D + k] = (float)(sums[(int64_t)c * D + k] / nrm);
}

size_t kmeans_ws_bytes(int64_t N, int C, int D) {
  return ((size_t)C * D * sizeof(double) + 255) / 256 * 256 + build_ws_bytes(N, C);
}

cudaError_t launch_kmeans_update(const float* X, int64_t N, int D, const uint16_t* tags, int C, float* mu,
                                 int32_t* counts_out, void* ws, int32_t* d_status, cudaStream_t st) {
  double* sums = static_cast<double*>(ws);
  BuildWs g = build_ws_carve(static_cast<char*>(ws) + ((size_t)C * D * sizeof(double) + 255) / 256 * 256, N, C);
  cudaError_t e = launch_grouping(tags, N, C, g, d_status, st);
  if (e != cudaSuccess) return e;
  kmeans_sum_kernel<<<dim3(C, (D + 127) / 128), 128, 0, st>>>(X, D, g, sums);
  kmeans_normalize_kernel<<<C, 256, 0, st>>>(sums, D, g.counts, mu);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (counts_out) e = cudaMemcpyAsync(counts_out, g.counts, sizeof(int32_t) * C, cudaMemcpyDeviceToDevice, st);
  return e;
}

}  // namespace glv
