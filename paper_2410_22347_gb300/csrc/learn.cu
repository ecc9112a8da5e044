// learn.cu -- learning-side kernels: the statistics LeanVec-Sphering is built from and the
// gradient of the inner-product approximation loss used to refine it.
//
// * Second moments (Section 3.2 summary statistics, Algorithm 2 in eigendecomposition form):
//   K = sum_v v v^T over a set of D-vectors, per cluster when tags are given.  FP32 inputs,
//   FP64 products and sums (a product of two FP32 numbers is exact in FP64).  Symmetric: only
//   tiles on or above the diagonal are computed and mirrored.
// * Pair forward: for index pairs (q_p, x_p) with cluster c_p = tag(x_p),
//   u_p = B_c x_p, v_p = A_c q_p (grouped GEMMs over the pairs of each cluster),
//   s_p = <u_p, v_p> (the GleanVec inner product), t_p = <q_p, x_p> (the exact one).
// * Pair backward: given g_p = dL/ds_p,
//   dL/dA_c = sum_{p in c} g_p u_p q_p^T,   dL/dB_c = sum_{p in c} g_p v_p x_p^T,
//   a segmented sum of rank-1 terms = one GEMM over the pairs of each cluster.
// The pairs (or vectors) are grouped by cluster on the device (launch_grouping).
#include "common.cuh"
#include "kernels.cuh"

namespace glv {

// ---- second moments (FP64) -------------------------------------------------------------------

constexpr int kMomT = 64;   // output tile
constexpr int kMomK = 32;   // vectors per chunk

// grid.x: upper-triangle tile index, grid.y: cluster.  perm == nullptr: all n vectors.
__global__ void __launch_bounds__(256) moments_kernel(const float* __restrict__ V, int64_t n, int D,
                                                     const int32_t* __restrict__ perm,
                                                     const int32_t* __restrict__ seg_start,
                                                     const int32_t* __restrict__ counts, double* __restrict__ K) {
  __shared__ double Va[kMomK][kMomT];
  __shared__ double Vb[kMomK][kMomT];
  const int nt = (D + kMomT - 1) / kMomT;
  // decode the upper-triangle tile (ta <= tb)
  int t = blockIdx.x, ta = 0;
  while (t >= nt - ta) {
    t -= nt - ta;
    ++ta;
  }
  const int tb = ta + t;
  const int c = blockIdx.y;
  const int64_t start = perm ? seg_start[c] : 0;
  const int64_t cnt = perm ? counts[c] : n;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  const int a0 = ta * kMomT, b0 = tb * kMomT;
  for (int64_t v0 = 0; v0 < cnt; v0 += kMomK) {
    // 32 vectors x 64 dims for each side: 2048 values, 8 per thread per side
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int r = e >> 6, col = e & 63;
      double xa = 0.0, xb = 0.0;
      if (v0 + r < cnt) {
        const int64_t row = perm ? perm[start + v0 + r] : v0 + r;
        const float* src = V + row * D;
        if (a0 + col < D) xa = (double)src[a0 + col];
        if (b0 + col < D) xb = (double)src[b0 + col];
      }
      Va[r][col] = xa;
      Vb[r][col] = xb;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kMomK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = Va[kk][ty * 4 + i];
        b[i] = Vb[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* Kc = K + (int64_t)c * D * D;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = a0 + ty * 4 + i, q = b0 + tx * 4 + j;
      if (r < D && q < D) {
        Kc[(int64_t)r * D + q] = acc[i][j];
        if (ta != tb) Kc[(int64_t)q * D + r] = acc[i][j];
      }
    }
}

size_t moments_ws_bytes(int64_t n, int C) { return build_ws_bytes(n, C); }

cudaError_t launch_moments(const float* V, int64_t n, int D, const uint16_t* tags, int C, double* K, void* ws,
                           int32_t* d_status, cudaStream_t st) {
  const int nt = (D + kMomT - 1) / kMomT;
  const int ntri = nt * (nt + 1) / 2;
  if (tags == nullptr) {
    moments_kernel<<<dim3(ntri, 1), 256, 0, st>>>(V, n, D, nullptr, nullptr, nullptr, K);
    return cudaGetLastError();
  }
  BuildWs w = build_ws_carve(ws, n, C);
  cudaError_t e = launch_grouping(tags, n, C, w, d_status, st);
  if (e != cudaSuccess) return e;
  moments_kernel<<<dim3(ntri, C), 256, 0, st>>>(V, n, D, w.perm, w.seg_start, w.counts, K);
  return cudaGetLastError();
}

// ---- pairs: grouping ---------------------------------------------------------------------------

struct PairWs {
  uint16_t* ptag;  // P cluster of each pair
  BuildWs g;       // pairs grouped by cluster
};

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

size_t pair_ws_bytes(int64_t P, int C) { return al256(2 * (size_t)P) + build_ws_bytes(P, C); }

static PairWs pair_ws_carve(void* ws, int64_t P, int C) {
  PairWs w;
  w.ptag = static_cast<uint16_t*>(ws);
  w.g = build_ws_carve(static_cast<char*>(ws) + al256(2 * (size_t)P), P, C);
  return w;
}

// Pair p's cluster is the tag of its database vector; a pair with an index out of range gets
// the out-of-range tag C (so the grouping skips it) and is reported.
__global__ void pair_tags_kernel(const int32_t* __restrict__ qi, int64_t nQ, const int32_t* __restrict__ xi,
                                 int64_t nX, const uint16_t* __restrict__ tags, int C, int64_t P,
                                 uint16_t* __restrict__ ptag, int32_t* d_status) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = qi[p], x = xi[p];
    uint16_t t = (uint16_t)C;
    if (q >= 0 && q < nQ && x >= 0 && x < nX) {
      t = tags[x];
      if (t >= C) report(d_status, GLV_ERR_BAD_ID);
    } else {
      report(d_status, GLV_ERR_BAD_ID);
    }
    ptag[p] = t >= C ? (uint16_t)C : t;
  }
}

static cudaError_t group_pairs(const PairWs& w, const int32_t* qi, int64_t nQ, const int32_t* xi, int64_t nX,
                               const uint16_t* tags, int C, int64_t P, int32_t* d_status, cudaStream_t st) {
  const int b = (int)((P + 255) / 256 < 4096 ? (P + 255) / 256 : 4096);
  pair_tags_kernel<<<b, 256, 0, st>>>(qi, nQ, xi, nX, tags, C, P, w.ptag, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  (void)d_status;  // bad pairs are reported by the forward/backward kernels themselves
  return launch_grouping(w.ptag, P, C, w.g, nullptr, st);
}

// ---- pairs: grouped projection  out[p, :] = W_{c_p} . src[idx[p], :] ---------------------------

constexpr int kPM = 32;  // pairs per tile
constexpr int kPN = 64;  // output columns per tile
constexpr int kPK = 32;  // K slice

// grid.x: 32-pair tile (over the grouped order), grid.y: column tile.
__global__ void __launch_bounds__(256) pair_project_kernel(const float* __restrict__ src, int64_t nsrc, int D,
                                                           const int32_t* __restrict__ idx,
                                                           const float* __restrict__ W, int C, int d,
                                                           BuildWs g, float* __restrict__ out) {
  __shared__ float Xs[kPK][kPM];
  __shared__ float Ws[kPK][kPN + 4];
  __shared__ int32_t rows[kPM], pairs[kPM];
  __shared__ int s_c, s_n;
  const int b = blockIdx.x, tid = threadIdx.x;
  if (tid == 0) {
    const int ntiles = g.tile_start[C];
    int c = -1;
    if (b < ntiles) {
      int lo = 0, hi = C - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (g.tile_start[mid] <= b) lo = mid;
        else hi = mid - 1;
      }
      c = lo;
    }
    s_c = c;
    s_n = c >= 0 ? min(kPM, g.counts[c] - (b - g.tile_start[c]) * kPM) : 0;
  }
  __syncthreads();
  const int c = s_c, n = s_n;
  if (c < 0 || n <= 0) return;
  if (tid < kPM) {
    const int t = b - g.tile_start[c];
    const int p = tid < n ? g.perm[g.seg_start[c] + t * kPM + tid] : -1;
    pairs[tid] = p;
    int64_t r = p >= 0 ? (int64_t)idx[p] : -1;
    rows[tid] = (r >= 0 && r < nsrc) ? (int32_t)r : -1;
  }
  __syncthreads();
  const float* Wc = W + (int64_t)c * d * D;
  const int n0 = blockIdx.y * kPN;
  const int ry = tid >> 4, cx = tid & 15;  // rows ry*2..+1, cols cx*4..+3
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  for (int k0 = 0; k0 < D; k0 += kPK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {  // 32 x 32 source values
      const int e = tid + 256 * u;
      const int r = e >> 5, kk = e & 31;
      const int row = rows[r];
      Xs[kk][r] = (row >= 0 && k0 + kk < D) ? src[(int64_t)row * D + k0 + kk] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {  // 64 x 32 weights
      const int e = tid + 256 * u;
      const int col = e >> 5, kk = e & 31;
      Ws[kk][col] = (n0 + col < d && k0 + kk < D) ? Wc[(int64_t)(n0 + col) * D + k0 + kk] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kPK; ++kk) {
      const float x0 = Xs[kk][ry * 2], x1 = Xs[kk][ry * 2 + 1];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float w = Ws[kk][cx * 4 + j];
        acc[0][j] = fmaf(x0, w, acc[0][j]);
        acc[1][j] = fmaf(x1, w, acc[1][j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int r = ry * 2 + i;
    const int p = pairs[r];
    if (r >= n || p < 0) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = n0 + cx * 4 + j;
      if (col < d) out[(int64_t)p * d + col] = rows[r] >= 0 ? acc[i][j] : 0.f;
    }
  }
}

// s_p = <u_p, v_p>,  t_p = <q_p, x_p>  (warp per pair).  A pair with an index out of range or
// a tag out of range gets s = t = 0 and is reported.
__global__ void pair_scores_kernel(const float* __restrict__ Q, int64_t nQ, const float* __restrict__ X,
                                   int64_t nX, int D, const uint16_t* __restrict__ ptag, int C,
                                   const int32_t* __restrict__ qi, const int32_t* __restrict__ xi, int64_t P,
                                   const float* __restrict__ u, const float* __restrict__ v, int d,
                                   float* __restrict__ s, float* __restrict__ t, int32_t* d_status) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); p < P; p += warps) {
    const bool ok = ptag[p] < C;
    float ss = 0.f, tt = 0.f;
    if (ok) {
      for (int r = lane; r < d; r += 32) ss = fmaf(u[p * d + r], v[p * d + r], ss);
      const float* q = Q + (int64_t)qi[p] * D;
      const float* x = X + (int64_t)xi[p] * D;
      for (int k = lane; k < D; k += 32) tt = fmaf(q[k], x[k], tt);
    }
    ss = warp_sum(ss);
    tt = warp_sum(tt);
    if (lane == 0) {
      s[p] = ss;
      t[p] = tt;
      if (!ok) report(d_status, GLV_ERR_BAD_ID);
    }
  }
}

size_t pair_forward_ws(int64_t P, int C) { return pair_ws_bytes(P, C); }

cudaError_t launch_pair_forward(const float* Q, int64_t nQ, const float* X, int64_t nX, int D, const uint16_t* tags,
                                const float* A, const float* B, int C, int d, const int32_t* qi, const int32_t* xi,
                                int64_t P, float* s, float* t, float* u, float* v, void* ws, int32_t* d_status,
                                cudaStream_t st) {
  PairWs w = pair_ws_carve(ws, P, C);
  cudaError_t e = group_pairs(w, qi, nQ, xi, nX, tags, C, P, d_status, st);
  if (e != cudaSuccess) return e;
  // rows of pairs that the grouping skipped (bad indices) are never written: clear u, v first
  if ((e = cudaMemsetAsync(u, 0, sizeof(float) * (size_t)P * d, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(v, 0, sizeof(float) * (size_t)P * d, st)) != cudaSuccess) return e;
  const unsigned tiles = (unsigned)((P + kPM - 1) / kPM + C);
  dim3 grid(tiles, (unsigned)((d + kPN - 1) / kPN));
  pair_project_kernel<<<grid, 256, 0, st>>>(X, nX, D, xi, B, C, d, w.g, u);
  pair_project_kernel<<<grid, 256, 0, st>>>(Q, nQ, D, qi, A, C, d, w.g, v);
  const int sb = (int)((P + 7) / 8 < 8192 ? (P + 7) / 8 : 8192);
  pair_scores_kernel<<<sb, 256, 0, st>>>(Q, nQ, X, nX, D, w.ptag, C, qi, xi, P, u, v, d, s, t, d_status);
  return cudaGetLastError();
}

// ---- pairs: backward --------------------------------------------------------------------------

constexpr int kGT = 64;  // output tile (rows of dA_c / dB_c and columns along D)
constexpr int kGK = 32;  // pairs per chunk

// grid.x: (row tile, column tile) of the d x D gradient, grid.y: cluster, grid.z: 0 = dA, 1 = dB.
//   dA_c[r, k] = sum_{p in c} g_p u_p[r] q_p[k]      dB_c[r, k] = sum_{p in c} g_p v_p[r] x_p[k]
__global__ void __launch_bounds__(256) pair_backward_kernel(const float* __restrict__ Q, const float* __restrict__ X,
                                                            int D, const int32_t* __restrict__ qi,
                                                            const int32_t* __restrict__ xi,
                                                            const float* __restrict__ u, const float* __restrict__ v,
                                                            const float* __restrict__ g, int d, BuildWs grp,
                                                            float* __restrict__ dA, float* __restrict__ dB) {
  __shared__ float Gs[kGK][kGT];  // g_p * (u or v)_p[r0 .. r0+63]
  __shared__ float Ss[kGK][kGT];  // (q or x)_p[k0 .. k0+63]
  const int ntk = (D + kGT - 1) / kGT;
  const int tr = blockIdx.x / ntk, tk = blockIdx.x - tr * ntk;
  const int c = blockIdx.y;
  const bool isB = blockIdx.z == 1;
  const float* coef = isB ? v : u;
  const float* src = isB ? X : Q;
  const int32_t* idx = isB ? xi : qi;
  const int r0 = tr * kGT, k0 = tk * kGT;
  const int64_t start = grp.seg_start[c], cnt = grp.counts[c];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int64_t p0 = 0; p0 < cnt; p0 += kGK) {
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const int e = threadIdx.x + 256 * w;
      const int pr = e >> 6, col = e & 63;
      float gv = 0.f, sv = 0.f;
      if (p0 + pr < cnt) {
        const int64_t p = grp.perm[start + p0 + pr];
        if (r0 + col < d) gv = g[p] * coef[p * d + r0 + col];
        if (k0 + col < D) sv = src[(int64_t)idx[p] * D + k0 + col];
      }
      Gs[pr][col] = gv;
      Ss[pr][col] = sv;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < kGK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = Gs[kk][ty * 4 + i];
        b[i] = Ss[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* out = (isB ? dB : dA) + (int64_t)c * d * D;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty * 4 + i, k = k0 + tx * 4 + j;
      if (r < d && k < D) out[(int64_t)r * D + k] = acc[i][j];
    }
}

cudaError_t launch_pair_backward(const float* Q, int64_t nQ, const float* X, int64_t nX, int D,
                                 const uint16_t* tags, int C, int d, const int32_t* qi, const int32_t* xi, int64_t P,
                                 const float* u, const float* v, const float* g, float* dA, float* dB, void* ws,
                                 int32_t* d_status, cudaStream_t st) {
  PairWs w = pair_ws_carve(ws, P, C);
  cudaError_t e = group_pairs(w, qi, nQ, xi, nX, tags, C, P, d_status, st);
  if (e != cudaSuccess) return e;
  const int tiles = ((d + kGT - 1) / kGT) * ((D + kGT - 1) / kGT);
  pair_backward_kernel<<<dim3(tiles, C, 2), 256, 0, st>>>(Q, X, D, qi, xi, u, v, g, d, w.g, dA, dB);
  return cudaGetLastError();
}

// ---- pairs: loss and its gradient with respect to s -----------------------------------------
//
// L = sum_p (t_p - s_p)^2, the inner-product approximation loss of Section 2.1 over the pairs,
// and g_p = dL/ds_p = -2 (t_p - s_p), scaled by an upstream weight w (dOut/dL; 1 if absent).
// One CTA, a fixed assignment of pairs to threads and a fixed reduction tree: the FP64 loss is
// the same on every call for the same inputs.

constexpr int kLossThreads = 1024;

__global__ void __launch_bounds__(kLossThreads) pair_loss_kernel(const float* __restrict__ s,
                                                               const float* __restrict__ t, int64_t P,
                                                               const double* __restrict__ weight,
                                                               double* __restrict__ loss, float* __restrict__ g) {
  __shared__ double part[kLossThreads / 32];
  const float w = weight ? (float)*weight : 1.f;
  double acc = 0.0;
  for (int64_t p = threadIdx.x; p < P; p += kLossThreads) {
    const float r = t[p] - s[p];
    if (g) g[p] = -2.f * w * r;
    acc = fma((double)r, (double)r, acc);
  }
  if (!loss) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = part[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *loss = v;
  }
}

cudaError_t launch_pair_loss(const float* s, const float* t, int64_t P, const double* weight, double* loss, float* g,
                             cudaStream_t st) {
  pair_loss_kernel<<<1, kLossThreads, 0, st>>>(s, t, P, weight, loss, g);
  return cudaGetLastError();
}

// ---- Adam (Kingma & Ba, 2015) ------------------------------------------------------------------
//
// m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
// param <- param - lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
// The bias corrections are formed on the host in double and passed in.

__global__ void adam_kernel(float* __restrict__ param, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    param[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

cudaError_t launch_adam(float* param, const float* grad, float* m, float* v, int64_t n, float lr, float b1, float b2,
                        float eps, int step, int num_sms, cudaStream_t st) {
  const double c1 = 1.0 - pow((double)b1, (double)step), c2 = 1.0 - pow((double)b2, (double)step);
  const int64_t want = (n + 255) / 256;
  const int blocks = (int)(want < (int64_t)num_sms * 8 ? (want > 0 ? want : 1) : (int64_t)num_sms * 8);
  adam_kernel<<<blocks, 256, 0, st>>>(param, grad, m, v, n, lr, b1, b2, eps, (float)c1, (float)c2);
  return cudaGetLastError();
}

}  // namespace glv
