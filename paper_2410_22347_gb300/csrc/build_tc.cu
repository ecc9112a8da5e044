// build_tc.cu -- the reduced database of Eq. (X_low), Section 4 (read with g), on the tensor
// cores:   x_i^low = B_{c_i} x_i,  FP32-accurate, stored as FP32, BF16 or FP8-e4m3 + row scale.
//
// A persistent grouped GEMM over the cluster-sorted rows (the grouping of build.cu: counts,
// segment starts, row permutation): a tile is 128 rows of ONE cluster c times B_c^T (d columns,
// padded to Npad, a multiple of 16, at most 256), K = D in slices of 32 FP32 values.
//
// Operands are FP32 and the product must be FP32-accurate, so every value v is split exactly
// into a TF32 part hi (v with its low 13 mantissa bits cleared) and lo = v - hi, and three
// kind::tf32 MMAs per K step accumulate hi*hi + hi*lo + lo*hi (the lo*lo term is below the
// FP32 rounding of the result) -- the same split as the projection's FP32 mode.
//
// Warp roles (13 warps, one CTA per SM):
//   warp 0      TMEM owner + MMA issuer (one lane); accumulator 128 lanes x Npad columns,
//               double buffered (2 x 256 columns) so a tile's epilogue overlaps the next MMAs;
//   warps 1..4  epilogue, one per TMEM lane quadrant: thread = row; reads its row's d values
//               from TMEM (twice for FP8: the row maximum first), converts, and writes the row
//               of the store (zero padding up to the 16-byte boundary);
//   warps 5..12 loaders: gather the tile's 128 X rows (through the permutation) and B_c's rows
//               with 16-byte asynchronous copies (cp.async) straight into the 128-byte swizzled
//               K-major layout the MMA descriptors read, then split each landed chunk in place
//               into hi and lo; the copies of the next stages - 1 K slices are in flight while
//               one slice is split (three stages of shared memory where they fit, else two).
// Every mbarrier wait is bounded (tc.cuh): a timeout sets GLV_ERR_TIMEOUT, all roles leave,
// the MMAs are drained and the TMEM is freed before the CTA exits.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace glv {

constexpr int kBtM = 128;          // rows per tile (MMA M)
constexpr int kBtK = 32;           // FP32 values of K per stage (one 128-byte swizzle row)
constexpr int kBtMaxStages = 3;    // 3 where they fit in shared memory, else 2
constexpr int kBtLoadWarps = 8;
constexpr int kBtThreads = 32 * (1 + 4 + kBtLoadWarps);
constexpr int kBtMaxClusters = 4096;  // per-cluster tile counts are scanned into shared memory

struct BuildTcArgs {
  const float* X;
  int64_t N;
  int D;
  const float* B;
  int C, d, Npad;
  int stages;
  int dt;
  uint8_t* Xred;
  int64_t row_stride;
  float* scales;
  const int32_t* counts;
  const int32_t* seg_start;
  const int32_t* perm;
  int32_t* d_status;
};

__host__ __device__ inline size_t bt_stage_bytes(int Npad) { return 2 * (size_t)kBtM * 128 + 2 * (size_t)Npad * 128; }
__host__ __device__ inline size_t bt_smem_bytes(int Npad, int C, int stages) {
  return (size_t)stages * bt_stage_bytes(Npad) + 256 + (size_t)(C + 1) * 4 + 1024;
}

// Byte offset of 16-byte chunk c of row r in a 128-byte swizzled K-major tile (8-row atoms
// of 1024 bytes; chunk positions XOR-ed with the row within the atom), as TMA would write it.
GLV_DEV uint32_t sw128_off(int r, int c) { return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4)); }

// 16-byte asynchronous copy global -> shared (cp.async.cg, L1 bypassed); src_bytes = 0 writes
// zeros.  Copies are grouped per commit; wait_group_p(n) waits until at most n groups of this
// thread are pending.
GLV_DEV void bt_cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}
GLV_DEV void bt_cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
GLV_DEV void bt_cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// n is 0 .. kBtMaxStages - 2 (wait_group takes an immediate)
GLV_DEV void bt_cp_async_wait_group_p(int n) {
  if (n <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
  else asm volatile("cp.async.wait_group 1;" ::: "memory");
}

GLV_DEV void split_tf32(float4 v, float4& h, float4& l) {
  h.x = __uint_as_float(__float_as_uint(v.x) & 0xffffe000u);
  h.y = __uint_as_float(__float_as_uint(v.y) & 0xffffe000u);
  h.z = __uint_as_float(__float_as_uint(v.z) & 0xffffe000u);
  h.w = __uint_as_float(__float_as_uint(v.w) & 0xffffe000u);
  l.x = v.x - h.x;  // exact: same sign and exponent
  l.y = v.y - h.y;
  l.z = v.z - h.z;
  l.w = v.w - h.w;
}

__global__ void __launch_bounds__(kBtThreads, 1) build_tc_kernel(const BuildTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const size_t sb = bt_stage_bytes(a.Npad);
  const int nst = a.stages;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + nst * sb);
  uint64_t* empty = full + kBtMaxStages;
  uint64_t* tfull = empty + kBtMaxStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int32_t* tstart = reinterpret_cast<int32_t*>(smem + nst * sb + 256);  // C + 1 tile offsets
  __shared__ int32_t s_part[kBtThreads / 32];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tiles of 128 rows per cluster, scanned into shared memory (C <= kBtMaxClusters)
  {
    const int per = (a.C + blockDim.x - 1) / blockDim.x;
    const int c0 = min(a.C, (int)threadIdx.x * per), c1 = min(a.C, c0 + per);
    int run = 0;
    for (int c = c0; c < c1; ++c) run += (a.counts[c] + kBtM - 1) / kBtM;
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) s_part[warp] = incl;
    __syncthreads();
    int before = incl - run;
    for (int w = 0; w < warp; ++w) before += s_part[w];
    for (int c = c0; c < c1; ++c) {
      tstart[c] = before;
      before += (a.counts[c] + kBtM - 1) / kBtM;
    }
    if (threadIdx.x == blockDim.x - 1) tstart[a.C] = before;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      tc::mbar_init(&full[s], kBtLoadWarps);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 128);
    }
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int ntiles = tstart[a.C];
  const int nkb = (a.D + kBtK - 1) / kBtK;

  // cluster and first row of tile t
  auto tile_of = [&](int t, int& c, int& row0, int& nrows) {
    int lo = 0, hi = a.C - 1;
    while (lo < hi) {  // largest c with tstart[c] <= t (empty clusters share their start)
      const int mid = (lo + hi + 1) / 2;
      if (tstart[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    c = lo;
    const int j = t - tstart[c];
    row0 = a.seg_start[c] + j * kBtM;
    nrows = min(kBtM, a.counts[c] - j * kBtM);
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t idesc = tc::instr_desc(2u, kBtM, (uint32_t)a.Npad);
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        if (!tc::mbar_wait(&tempty[acc], acc_phase ^ 1, abort_flag)) break;
        tc::tc_fence_after();
        const uint32_t d_tmem = tmem + (uint32_t)(acc * 256);
        for (int kb = 0; kb < nkb; ++kb) {
          if (!tc::mbar_wait(&full[stage], phase, abort_flag)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t base = tc::smem_u32(smem + (size_t)stage * sb);
          const uint32_t ahi = base, alo = base + kBtM * 128;
          const uint32_t bhi = base + 2 * kBtM * 128, blo = bhi + (uint32_t)a.Npad * 128;
#pragma unroll
          for (int k = 0; k < 4; ++k) {  // 8 TF32 values (32 bytes) of K per MMA
            const uint32_t acc_in = (kb > 0 || k > 0) ? 1u : 0u;
            const uint64_t dah = tc::sw128_kmajor_desc(ahi + k * 32), dal = tc::sw128_kmajor_desc(alo + k * 32);
            const uint64_t dbh = tc::sw128_kmajor_desc(bhi + k * 32), dbl = tc::sw128_kmajor_desc(blo + k * 32);
            tc::mma_tf32(d_tmem, dah, dbh, idesc, acc_in);  // hi * hi
            tc::mma_tf32(d_tmem, dah, dbl, idesc, 1u);      // hi * lo
            tc::mma_tf32(d_tmem, dal, dbh, idesc, 1u);      // lo * hi
          }
          tc::mma_commit(&empty[stage]);
          if (++stage == nst) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        tc::mma_commit(&tfull[acc]);
        acc ^= 1;
        if (acc == 0) acc_phase ^= 1;
      }
      tc::mma_commit(drain);
      volatile int no_abort = 0;
      tc::mbar_wait(drain, 0, &no_abort);
    }
  } else if (warp <= 4) {
    // ---------------- epilogue: thread = row of the tile ----------------
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const int r = q * 32 + lane;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      int ok = 0;
      if (lane == 0) ok = tc::mbar_wait(&tfull[acc], acc_phase, abort_flag) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      (void)tc::mbar_try_wait(&tfull[acc], acc_phase);
      tc::tc_fence_after();
      int c, row0, nrows;
      tile_of(t, c, row0, nrows);
      const bool live = r < nrows;
      const int64_t row = live ? (int64_t)a.perm[row0 + r] : 0;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 256);
      const int nchunk = (a.d + 31) / 32;
      uint32_t v[32];
      float scale = 1.f;
      if (a.dt == GLV_FP8_E4M3) {  // pass 1: the row maximum
        float mx = 0.f;
        for (int ch = 0; ch < nchunk; ++ch) {
          tc::tmem_ld_32x32b_x32(tbase + (uint32_t)(ch * 32), v);
          tc::tmem_ld_wait(v);
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (ch * 32 + u < a.d) mx = fmaxf(mx, fabsf(__uint_as_float(v[u])));
        }
        scale = mx / 448.0f;  // IEEE division
        if (live) a.scales[row] = scale;
      }
      uint8_t* dst = a.Xred + row * a.row_stride;
      const int eb = a.dt == GLV_F32 ? 4 : (a.dt == GLV_BF16 ? 2 : 1);
      const int row_bytes = (a.d * eb + 15) / 16 * 16;  // data + zero padding to 16 bytes
      for (int ch = 0; ch < nchunk; ++ch) {
        tc::tmem_ld_32x32b_x32(tbase + (uint32_t)(ch * 32), v);
        tc::tmem_ld_wait(v);
        if (!live) continue;
        const int e0 = ch * 32;
        if (a.dt == GLV_F32) {
#pragma unroll
          for (int u4 = 0; u4 < 8; ++u4) {
            const int b = (e0 + u4 * 4) * 4;
            if (b >= row_bytes) break;
            uint4 w;
            w.x = e0 + u4 * 4 + 0 < a.d ? v[u4 * 4 + 0] : 0u;
            w.y = e0 + u4 * 4 + 1 < a.d ? v[u4 * 4 + 1] : 0u;
            w.z = e0 + u4 * 4 + 2 < a.d ? v[u4 * 4 + 2] : 0u;
            w.w = e0 + u4 * 4 + 3 < a.d ? v[u4 * 4 + 3] : 0u;
            *reinterpret_cast<uint4*>(dst + b) = w;
          }
        } else if (a.dt == GLV_BF16) {
#pragma unroll
          for (int u8 = 0; u8 < 4; ++u8) {
            const int b = (e0 + u8 * 8) * 2;
            if (b >= row_bytes) break;
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              const int e = e0 + u8 * 8 + 2 * h;
              const float x0 = e < a.d ? __uint_as_float(v[u8 * 8 + 2 * h]) : 0.f;
              const float x1 = e + 1 < a.d ? __uint_as_float(v[u8 * 8 + 2 * h + 1]) : 0.f;
              const __nv_bfloat162 p = __floats2bfloat162_rn(x0, x1);  // .x = x0 (low half)
              w[h] = *reinterpret_cast<const uint32_t*>(&p);
            }
            *reinterpret_cast<uint4*>(dst + b) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        } else {
#pragma unroll
          for (int u16 = 0; u16 < 2; ++u16) {
            const int b = e0 + u16 * 16;
            if (b >= row_bytes) break;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const int e = e0 + u16 * 16 + u;
              uint32_t code = 0;
              if (e < a.d && scale != 0.f) {
                const float y = __uint_as_float(v[u16 * 16 + u]) / scale;  // IEEE division
                code = (uint32_t)__nv_cvt_float_to_fp8(y, __NV_SATFINITE, __NV_E4M3);
              }
              w[u >> 2] |= code << (8 * (u & 3));
            }
            *reinterpret_cast<uint4*>(dst + b) = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      }
      tc::tc_fence_before();
      tc::mbar_arrive(&tempty[acc]);
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1;
    }
  } else {
    // ---------------- loaders ----------------
    // The K slices of this CTA's tiles form one sequence.  Each thread copies its 16-byte chunks
    // of slice g + P (asynchronously, cp.async: no registers held) while it splits the chunks
    // of slice g, which landed earlier: P = stages - 1 slices are in flight.  A slice's raw FP32
    // chunks land where their hi parts go; the split rewrites them in place and writes lo.
    const int i = threadIdx.x - 5 * 32;  // 0 .. 255
    const int c16 = i & 7;              // the 16-byte chunk of K this thread handles
    const int nb = (a.Npad * 8 + 255) / 256;  // B chunk jobs per thread (<= 8)
    const int P = nst - 1;
    const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = (int64_t)my_tiles * nkb;
    // issue stream state
    int it = 0, ikb = 0, istage = 0;
    uint32_t iphase = 0;
    const float* xr[4] = {nullptr, nullptr, nullptr, nullptr};
    const float* Bc = a.B;
    auto set_tile = [&](int t) {
      int c, row0, nrows;
      tile_of(t, c, row0, nrows);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = (i >> 3) + 32 * u;
        xr[u] = r < nrows ? a.X + (int64_t)a.perm[row0 + r] * a.D : nullptr;
      }
      Bc = a.B + (int64_t)c * a.d * a.D;
    };
    bool ok = true;
    // copies of the next slice of the issue stream into its stage (once the MMAs have freed it)
    auto issue = [&]() -> bool {
      int w_ok = 1;
      if (lane == 0) w_ok = tc::mbar_wait(&empty[istage], iphase ^ 1, abort_flag) ? 1 : 0;
      w_ok = __shfl_sync(0xffffffffu, w_ok, 0);
      if (!w_ok) return false;
      if (ikb == 0) set_tile(blockIdx.x + it * gridDim.x);
      const int k = ikb * kBtK + c16 * 4;
      const bool kin = k < a.D;  // D % 4 == 0: a chunk is all in or all out
      uint8_t* base = smem + (size_t)istage * sb;
      uint8_t* ahi = base;
      uint8_t* bhi = base + 2 * kBtM * 128;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = (i >> 3) + 32 * u;
        const bool in = xr[u] != nullptr && kin;
        bt_cp_async16(ahi + sw128_off(r, c16), in ? xr[u] + k : a.X, in ? 16 : 0);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int r = (i >> 3) + 32 * j;
        if (j < nb && r < a.Npad) {
          const bool in = r < a.d && kin;
          bt_cp_async16(bhi + sw128_off(r, c16), in ? Bc + (int64_t)r * a.D + k : a.B, in ? 16 : 0);
        }
      }
      if (++ikb == nkb) {
        ikb = 0;
        ++it;
      }
      if (++istage == nst) {
        istage = 0;
        iphase ^= 1;
      }
      return true;
    };
    for (int q = 0; q < P; ++q) {  // P groups (empty ones past the end): P pending below
      if (q < total && ok) ok = issue();
      bt_cp_async_commit();
    }
    int sstage = 0;
    for (int64_t g = 0; ok && g < total; ++g) {
      bt_cp_async_wait_group_p(P - 1);  // this thread's copies of slice g have landed
      uint8_t* base = smem + (size_t)sstage * sb;
      uint8_t* ahi = base;
      uint8_t* alo = base + kBtM * 128;
      uint8_t* bhi = base + 2 * kBtM * 128;
      uint8_t* blo = bhi + (size_t)a.Npad * 128;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = (i >> 3) + 32 * u;
        float4 h, l;
        split_tf32(*reinterpret_cast<const float4*>(ahi + sw128_off(r, c16)), h, l);
        *reinterpret_cast<float4*>(ahi + sw128_off(r, c16)) = h;
        *reinterpret_cast<float4*>(alo + sw128_off(r, c16)) = l;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int r = (i >> 3) + 32 * j;
        if (j < nb && r < a.Npad) {
          float4 h, l;
          split_tf32(*reinterpret_cast<const float4*>(bhi + sw128_off(r, c16)), h, l);
          *reinterpret_cast<float4*>(bhi + sw128_off(r, c16)) = h;
          *reinterpret_cast<float4*>(blo + sw128_off(r, c16)) = l;
        }
      }
      tc::fence_proxy_async_smem();  // the MMA reads these through the async proxy
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&full[sstage]);
      if (++sstage == nst) sstage = 0;
      // then the copies of slice g + P, into the stage slice g - 1 leaves (the MMA has it)
      if (g + P < total) ok = issue();
      bt_cp_async_commit();  // (empty when nothing was issued: one group per slice)
    }
    bt_cp_async_wait_all();  // no copy may land in shared memory after the CTA has left
  }

  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && *abort_flag) report(a.d_status, GLV_ERR_TIMEOUT);
}

constexpr size_t kBtSmemLimit = 227 * 1024;

bool build_tc_supported(int64_t N, int D, int C, int d, const void* X, const void* B) {
  const int Npad = (d + 15) / 16 * 16;
  return N > 0 && D % 4 == 0 && Npad <= 256 && C <= kBtMaxClusters && reinterpret_cast<uintptr_t>(X) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(B) % 16 == 0 && bt_smem_bytes(Npad, C, 2) <= kBtSmemLimit;
}

cudaError_t launch_build_tc(const float* X, int64_t N, int D, const float* B, int C, int d, int dt, void* Xred,
                            int64_t row_stride, float* scales, const BuildWs& ws, int32_t* d_status, int num_sms,
                            cudaStream_t st) {
  BuildTcArgs a;
  a.X = X;
  a.N = N;
  a.D = D;
  a.B = B;
  a.C = C;
  a.d = d;
  a.Npad = (d + 15) / 16 * 16;
  a.dt = dt;
  a.Xred = static_cast<uint8_t*>(Xred);
  a.row_stride = row_stride;
  a.scales = scales;
  a.counts = ws.counts;
  a.seg_start = ws.seg_start;
  a.perm = ws.perm;
  a.d_status = d_status;
  a.stages = bt_smem_bytes(a.Npad, C, kBtMaxStages) <= kBtSmemLimit ? kBtMaxStages : 2;
  const size_t smem = bt_smem_bytes(a.Npad, C, a.stages);
  cudaError_t e = cudaFuncSetAttribute(build_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles_max = (N + kBtM - 1) / kBtM + C;
  const int grid = (int)(tiles_max < num_sms ? tiles_max : num_sms);
  build_tc_kernel<<<grid, kBtThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace glv
