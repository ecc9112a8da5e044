// project_simt.cu -- FP32 SIMT GEMM for the eager query preprocessing of Algorithm 4:
//
//     Qp[j, c*d + r] = sum_k A[c, r, k] * Q[j, k]      i.e.  Qp = Q . [A_1; ...; A_C]^T
//
// Both operands are K-contiguous ("TN"); the output is row-major nq x (C*d).  Classic
// register-blocked tiling: a 128 x 128 output tile per 256-thread CTA, 8 x 8 outputs per
// thread (split in two 4-row and two 4-column halves so the shared-memory reads are
// conflict-free broadcasts), K in slices of 8 staged through double-buffered shared
// memory with a register prefetch of the next slice.  Products and sums are plain FP32
// FMAs: this is the exact-FP32 path (GLV_F32) that the FP64 oracle checks to ~1e-6.
#include "common.cuh"
#include "kernels.cuh"

namespace glv {

constexpr int kBM = 128, kBN = 128, kBK = 8;

// VEC: K % 4 == 0 and both operand bases 16-byte aligned -> float4 global loads.
template <bool VEC>
__global__ void __launch_bounds__(256) sgemm_tn_kernel(const float* __restrict__ A, int M,
                                                       const float* __restrict__ B, int Nn,
                                                       int K, float* __restrict__ Cm) {
  __shared__ __align__(16) float As[2][kBK][kBM];
  __shared__ __align__(16) float Bs[2][kBK][kBN];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  // loader mapping: 128 rows x 8 k = 256 threads x 4 values
  const int lr = tid >> 1;          // row within tile
  const int lk = (tid & 1) * 4;     // k offset within slice
  const int tx = tid & 15, ty = tid >> 4;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) acc[i][jj] = 0.f;

  float ra[4], rb[4];
  auto load_slice = [&](int k0) {
    const int gm = m0 + lr, gn = n0 + lr;
    if (VEC) {
      float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
      if (gm < M && k0 + lk < K) va = *reinterpret_cast<const float4*>(A + (int64_t)gm * K + k0 + lk);
      if (gn < Nn && k0 + lk < K) vb = *reinterpret_cast<const float4*>(B + (int64_t)gn * K + k0 + lk);
      ra[0] = va.x; ra[1] = va.y; ra[2] = va.z; ra[3] = va.w;
      rb[0] = vb.x; rb[1] = vb.y; rb[2] = vb.z; rb[3] = vb.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kk = k0 + lk + u;
        ra[u] = (gm < M && kk < K) ? A[(int64_t)gm * K + kk] : 0.f;
        rb[u] = (gn < Nn && kk < K) ? B[(int64_t)gn * K + kk] : 0.f;
      }
    }
  };
  auto store_slice = [&](int buf) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      As[buf][lk + u][lr] = ra[u];
      Bs[buf][lk + u][lr] = rb[u];
    }
  };

  const int nslices = (K + kBK - 1) / kBK;
  load_slice(0);
  store_slice(0);
  __syncthreads();
  for (int s = 0; s < nslices; ++s) {
    const int buf = s & 1;
    if (s + 1 < nslices) load_slice((s + 1) * kBK);
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[i][jj] = fmaf(av[i], bv[jj], acc[i][jj]);
    }
    if (s + 1 < nslices) store_slice(buf ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (gm >= M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gn = n0 + h * 64 + tx * 4;
      float* dst = Cm + (int64_t)gm * Nn + gn;
      if (VEC && gn + 3 < Nn && (Nn % 4) == 0) {
        *reinterpret_cast<float4*>(dst) =
            make_float4(acc[i][h * 4 + 0], acc[i][h * 4 + 1], acc[i][h * 4 + 2], acc[i][h * 4 + 3]);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (gn + u < Nn) dst[u] = acc[i][h * 4 + u];
      }
    }
  }
}

cudaError_t launch_project_simt(const float* Q, int64_t nq, int D, const float* A, int64_t Mcols,
                                float* Qp, cudaStream_t st) {
  dim3 grid((unsigned)((Mcols + kBN - 1) / kBN), (unsigned)((nq + kBM - 1) / kBM));
  const bool vec = (D % 4 == 0) && ((uintptr_t)Q % 16 == 0) && ((uintptr_t)A % 16 == 0) &&
                   ((uintptr_t)Qp % 16 == 0);
  if (vec)
    sgemm_tn_kernel<true><<<grid, 256, 0, st>>>(Q, (int)nq, A, (int)Mcols, D, Qp);
  else
    sgemm_tn_kernel<false><<<grid, 256, 0, st>>>(Q, (int)nq, A, (int)Mcols, D, Qp);
  return cudaGetLastError();
}

}  // namespace glv
