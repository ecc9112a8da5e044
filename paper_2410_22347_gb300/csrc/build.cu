// build.cu -- reduced database of Eq. (X_low), Section 4 (read with g):
//
//     x_i^low = B_{c_i} x_i ,  stored as FP32, BF16 or FP8-e4m3 with a per-row scale.
//
// Rows are grouped by cluster on the device (histogram -> scan -> scatter of row ids into a
// permutation), so that every tile of rows of ONE cluster is multiplied by that cluster's
// B_c: a grouped GEMM instead of N separate matrix-vector products.  The GEMM runs on the
// tensor cores (build_tc.cu, FP32-accurate through a TF32 hi/lo split) when D % 4 == 0 and
// d <= 256; otherwise on the FP32 SIMT kernel below, whose CTA keeps its tile's whole reduced
// rows in shared memory, so the epilogue sees each full row and can compute the FP8 row scale
// s_i = max_r |x_ir| / 448 before quantising.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.cuh"

namespace glv {

constexpr int kBuildTM = 32;   // rows per tile
constexpr int kBuildTN = 64;   // output columns per pass
constexpr int kBuildBK = 32;   // K slice

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

size_t build_ws_bytes(int64_t N, int C) {
  return al256(8 * (size_t)C) + al256(4 * (size_t)C) + al256(4 * ((size_t)C + 1)) +
         al256(4 * (size_t)N);
}

BuildWs build_ws_carve(void* ws, int64_t N, int C) {
  char* p = static_cast<char*>(ws);
  BuildWs w;
  w.counts = reinterpret_cast<int32_t*>(p);
  w.cursor = w.counts + C;
  p += al256(8 * (size_t)C);
  w.seg_start = reinterpret_cast<int32_t*>(p);
  p += al256(4 * (size_t)C);
  w.tile_start = reinterpret_cast<int32_t*>(p);
  p += al256(4 * ((size_t)C + 1));
  w.perm = reinterpret_cast<int32_t*>(p);
  (void)N;
  return w;
}

__global__ void build_hist_kernel(const uint16_t* __restrict__ tags, int64_t N, int C,
                                  int32_t* counts, int32_t* d_status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = tags[i];
    if (c < C) atomicAdd(counts + c, 1);
    else report(d_status, GLV_ERR_BAD_ID);
  }
}

// One CTA: exclusive scans of the cluster sizes and of their tile counts.
__global__ void build_scan_kernel(const int32_t* __restrict__ counts, int C, int32_t* seg_start,
                                  int32_t* tile_start) {
  __shared__ int32_t part_rows[1024], part_tiles[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int per = (C + T - 1) / T;
  const int c0 = min(C, t * per), c1 = min(C, c0 + per);
  int32_t rows = 0, tiles = 0;
  for (int c = c0; c < c1; ++c) {
    rows += counts[c];
    tiles += (counts[c] + kBuildTM - 1) / kBuildTM;
  }
  part_rows[t] = rows;
  part_tiles[t] = tiles;
  __syncthreads();
  if (t == 0) {
    int32_t r = 0, q = 0;
    for (int u = 0; u < T; ++u) {
      const int32_t a = part_rows[u], b = part_tiles[u];
      part_rows[u] = r;
      part_tiles[u] = q;
      r += a;
      q += b;
    }
    tile_start[C] = q;
  }
  __syncthreads();
  rows = part_rows[t];
  tiles = part_tiles[t];
  for (int c = c0; c < c1; ++c) {
    seg_start[c] = rows;
    tile_start[c] = tiles;
    rows += counts[c];
    tiles += (counts[c] + kBuildTM - 1) / kBuildTM;
  }
}

__global__ void build_scatter_kernel(const uint16_t* __restrict__ tags, int64_t N, int C,
                                     const int32_t* __restrict__ seg_start, int32_t* cursor,
                                     int32_t* perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = tags[i];
    if (c >= C) continue;
    const int pos = atomicAdd(cursor + c, 1);
    perm[seg_start[c] + pos] = (int32_t)i;
  }
}

struct BuildArgs {
  const float* X;
  int64_t N;
  int D;
  const float* B;
  int C, d, dpad;
  int dt;
  uint8_t* Xred;
  int64_t row_stride;
  float* scales;
  BuildWs ws;
};

template <bool VEC>
__global__ void __launch_bounds__(256) build_gemm_kernel(const BuildArgs a) {
  extern __shared__ __align__(16) float out[];  // kBuildTM x dpad
  __shared__ __align__(16) float Xs[kBuildBK][kBuildTM];
  __shared__ __align__(16) float Bs[kBuildBK][kBuildTN];
  __shared__ int32_t rows[kBuildTM];
  __shared__ int s_c, s_n;

  const int b = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const int ntiles = a.ws.tile_start[a.C];
    int c = -1;
    if (b < ntiles) {  // largest c with tile_start[c] <= b and a non-empty cluster
      int lo = 0, hi = a.C - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (a.ws.tile_start[mid] <= b) lo = mid;
        else hi = mid - 1;
      }
      c = lo;
    }
    s_c = c;
    if (c >= 0) {
      const int t = b - a.ws.tile_start[c];
      s_n = min(kBuildTM, a.ws.counts[c] - t * kBuildTM);
    } else {
      s_n = 0;
    }
  }
  __syncthreads();
  const int c = s_c, n = s_n;
  if (c < 0 || n <= 0) return;
  if (tid < kBuildTM) {
    const int t = b - a.ws.tile_start[c];
    rows[tid] = tid < n ? a.ws.perm[a.ws.seg_start[c] + t * kBuildTM + tid] : -1;
  }
  __syncthreads();

  const float* Bc = a.B + (int64_t)c * a.d * a.D;
  const int ry = tid >> 4, cx = tid & 15;  // rows ry*2..+1, cols cx*4..+3
  for (int n0 = 0; n0 < a.d; n0 += kBuildTN) {
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    for (int k0 = 0; k0 < a.D; k0 += kBuildBK) {
      {  // X tile: 32 rows x 32 k, 4 values per thread
        const int r = tid >> 3, kq = (tid & 7) * 4;
        const int row = rows[r];
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (row >= 0) {
          const float* src = a.X + (int64_t)row * a.D + k0 + kq;
          if (VEC && k0 + kq < a.D) {
            const float4 w = *reinterpret_cast<const float4*>(src);
            v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
          } else if (!VEC) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (k0 + kq + u < a.D) v[u] = src[u];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) Xs[kq + u][r] = v[u];
      }
      {  // B tile: 64 output columns x 32 k, 8 values per thread
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cr = (tid >> 3) + 32 * h, kq = (tid & 7) * 4;
          const int col = n0 + cr;
          float v[4] = {0.f, 0.f, 0.f, 0.f};
          if (col < a.d) {
            const float* src = Bc + (int64_t)col * a.D + k0 + kq;
            if (VEC && k0 + kq < a.D) {
              const float4 w = *reinterpret_cast<const float4*>(src);
              v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
            } else if (!VEC) {
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (k0 + kq + u < a.D) v[u] = src[u];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) Bs[kq + u][cr] = v[u];
        }
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < kBuildBK; ++kk) {
        const float2 xa = *reinterpret_cast<const float2*>(&Xs[kk][ry * 2]);
        const float4 bb = *reinterpret_cast<const float4*>(&Bs[kk][cx * 4]);
        acc[0][0] = fmaf(xa.x, bb.x, acc[0][0]);
        acc[0][1] = fmaf(xa.x, bb.y, acc[0][1]);
        acc[0][2] = fmaf(xa.x, bb.z, acc[0][2]);
        acc[0][3] = fmaf(xa.x, bb.w, acc[0][3]);
        acc[1][0] = fmaf(xa.y, bb.x, acc[1][0]);
        acc[1][1] = fmaf(xa.y, bb.y, acc[1][1]);
        acc[1][2] = fmaf(xa.y, bb.z, acc[1][2]);
        acc[1][3] = fmaf(xa.y, bb.w, acc[1][3]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int col = n0 + cx * 4 + u;
        if (col < a.d) out[(ry * 2 + i) * a.dpad + col] = acc[i][u];
      }
  }
  __syncthreads();

  // epilogue: one warp per row
  const int lane = tid & 31, warp = tid >> 5;
  for (int r = warp; r < n; r += 8) {
    const int64_t row = rows[r];
    const float* v = out + r * a.dpad;
    uint8_t* dst = a.Xred + row * a.row_stride;
    if (a.dt == GLV_F32) {
      const int nw = ((a.d * 4 + 15) / 16) * 4;  // words up to the 16-byte boundary
      float* o = reinterpret_cast<float*>(dst);
      for (int e = lane; e < nw; e += 32) o[e] = e < a.d ? v[e] : 0.f;
    } else if (a.dt == GLV_BF16) {
      const int nw = ((a.d * 2 + 15) / 16) * 4;  // 32-bit words (2 values each)
      uint32_t* o = reinterpret_cast<uint32_t*>(dst);
      for (int w = lane; w < nw; w += 32) {
        const int e = 2 * w;
        const float x0 = e < a.d ? v[e] : 0.f, x1 = e + 1 < a.d ? v[e + 1] : 0.f;
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);  // .x = x0 (low half)
        o[w] = *reinterpret_cast<const uint32_t*>(&h);
      }
    } else {
      float mx = 0.f;
      for (int e = lane; e < a.d; e += 32) mx = fmaxf(mx, fabsf(v[e]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      const float s = mx / 448.0f;  // IEEE division
      if (lane == 0) a.scales[row] = s;
      const int nw = ((a.d + 15) / 16) * 4;  // 32-bit words (4 codes each)
      uint32_t* o = reinterpret_cast<uint32_t*>(dst);
      for (int w = lane; w < nw; w += 32) {
        uint32_t word = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = 4 * w + u;
          uint32_t code = 0;
          if (e < a.d && s != 0.f) {
            const float y = v[e] / s;  // IEEE division
            code = (uint32_t)__nv_cvt_float_to_fp8(y, __NV_SATFINITE, __NV_E4M3);
          }
          word |= code << (8 * u);
        }
        o[w] = word;
      }
    }
  }
}

cudaError_t launch_grouping(const uint16_t* tags, int64_t N, int C, const BuildWs& ws, int32_t* d_status,
                            cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ws.counts, 0, 8 * (size_t)C, st);  // counts + cursor
  if (e != cudaSuccess) return e;
  const int hb = (int)((N + 255) / 256 < 4096 ? (N + 255) / 256 : 4096);
  build_hist_kernel<<<hb, 256, 0, st>>>(tags, N, C, ws.counts, d_status);
  build_scan_kernel<<<1, 1024, 0, st>>>(ws.counts, C, ws.seg_start, ws.tile_start);
  build_scatter_kernel<<<hb, 256, 0, st>>>(tags, N, C, ws.seg_start, ws.cursor, ws.perm);
  return cudaGetLastError();
}

cudaError_t launch_build(const float* X, int64_t N, int D, const uint16_t* tags, const float* B,
                         int C, int d, int dt, void* Xred, int64_t row_stride, float* scales,
                         void* workspace, int32_t* d_status, cudaStream_t st) {
  BuildWs ws = build_ws_carve(workspace, N, C);
  cudaError_t e = launch_grouping(tags, N, C, ws, d_status, st);
  if (e != cudaSuccess) return e;
  if (build_tc_supported(N, D, C, d, X, B)) {  // the tensor-core grouped GEMM (build_tc.cu)
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    return launch_build_tc(X, N, D, B, C, d, dt, Xred, row_stride, scales, ws, d_status, sms, st);
  }

  BuildArgs a;
  a.X = X; a.N = N; a.D = D; a.B = B; a.C = C; a.d = d;
  a.dpad = (d + 3) & ~3;
  a.dt = dt;
  a.Xred = static_cast<uint8_t*>(Xred);
  a.row_stride = row_stride;
  a.scales = scales;
  a.ws = ws;
  const size_t smem = (size_t)kBuildTM * a.dpad * sizeof(float);
  const int64_t max_tiles = (N + kBuildTM - 1) / kBuildTM + C;
  const bool vec = (D % 4 == 0) && ((uintptr_t)X % 16 == 0) && ((uintptr_t)B % 16 == 0);
  if (vec) {
    e = cudaFuncSetAttribute(build_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    build_gemm_kernel<true><<<(unsigned)max_tiles, 256, smem, st>>>(a);
  } else {
    e = cudaFuncSetAttribute(build_gemm_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    build_gemm_kernel<false><<<(unsigned)max_tiles, 256, smem, st>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace glv

// ---------------------------------------------------------------------------------------
// Allocation-free variant of glv_build_reduced: the grouping scratch (cluster counts,
// cursors, offsets, tile table and the row permutation) lives in a file-scope device array
// instead of a caller-provided workspace.  The array is sized for GLV_NOALLOC_MAX_ROWS rows
// and GLV_NOALLOC_MAX_CLUSTERS clusters and stays resident on every device that loads the
// library until the process exits.
// ---------------------------------------------------------------------------------------
#include <mutex>

namespace glv {

constexpr size_t noalloc_al256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kNoAllocScratchBytes =
    noalloc_al256(8 * (size_t)GLV_NOALLOC_MAX_CLUSTERS) + noalloc_al256(4 * (size_t)GLV_NOALLOC_MAX_CLUSTERS) +
    noalloc_al256(4 * ((size_t)GLV_NOALLOC_MAX_CLUSTERS + 1)) + noalloc_al256(4 * (size_t)GLV_NOALLOC_MAX_ROWS);

static __device__ __align__(256) unsigned char g_build_scratch[kNoAllocScratchBytes];

// Device address of g_build_scratch on the current device.  In host code the symbol name is
// only a host-side handle, so the address is looked up once per device (with that device
// current) and cached.
static cudaError_t build_scratch_address(void** out) {
  static std::mutex mu;
  static void* addr[256] = {};
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_build_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
  }
  *out = addr[dev];
  return cudaSuccess;
}

}  // namespace glv

extern "C" glv_status glv_build_reduced_noalloc(const float* X, int64_t N, int32_t D,
                                                const uint16_t* tags, const float* B, int32_t C,
                                                int32_t d, glv_dtype dt, void* Xred,
                                                int64_t row_stride, float* scales,
                                                int32_t* d_status, void* stream) {
  if (N > GLV_NOALLOC_MAX_ROWS || C > GLV_NOALLOC_MAX_CLUSTERS) return GLV_ERR_UNSUPPORTED;
  if (N < 0 || C < 1) return GLV_ERR_INVALID_ARG;
  if (glv::build_ws_bytes(N, C) > glv::kNoAllocScratchBytes) return GLV_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  if (glv::build_scratch_address(&scratch) != cudaSuccess) return GLV_ERR_CUDA;
  return glv_build_reduced(X, N, D, tags, B, C, d, dt, Xred, row_stride, scales, scratch, d_status,
                           stream);
}
