// project_tc.cu -- tensor-core (tcgen05 + TMA) GEMM for the eager query preprocessing of
// Algorithm 4:   Qp = Q . [A_1; ...; A_C]^T   (nq x D times D x C*d, FP32 accumulation).
//
// Two operand modes:
//   BF16  : Q and A rounded to bfloat16, one kind::f16 MMA per K-step;
//   TF32x3: each FP32 operand split exactly into hi + lo, hi = the value with its low 13
//           mantissa bits cleared (exactly representable in TF32), lo = value - hi; three
//           kind::tf32 MMAs per K-step accumulate hi*hi + hi*lo + lo*hi, which reproduces the
//           FP32 product to ~2^-20 relative (lo*lo is below that).  This is the FP32 mode.
// One prep launch writes the converted / split operands of Q and A (rows padded with zeros to
// a multiple of 64 along K) into the caller's workspace; TMA then streams 128-byte-wide K
// slices into shared memory in the 128-byte swizzled layout the MMA descriptors expect.
//
// Kernel structure (one persistent CTA per SM, 10 warps):
//   warp 0      TMA producer (one lane): stage ring of S slots, full/empty mbarriers;
//   warp 1      TMEM owner + MMA issuer (one lane): 128 x 256 FP32 accumulator, double
//               buffered in TMEM (2 x 256 columns) so the epilogue of tile t overlaps the
//               MMAs of tile t+1;
//   warps 2..9  epilogue, two warps per TMEM lane quadrant (each half of the columns):
//               tcgen05.ld 32 lanes x 32 columns at a time (the next chunk's load in flight
//               while this one is stored), written to a 4-KB shared-memory tile in the
//               128-byte swizzled layout and sent to Qp by one TMA tensor store per chunk (or,
//               when Qp's rows are not 16-byte multiples, transposed through a padded tile and
//               written by coalesced store instructions).
// Every mbarrier wait is bounded (see tc.cuh); a timeout sets GLV_ERR_TIMEOUT in d_status,
// all roles leave their loops, outstanding TMA loads and MMAs are drained (bounded), and the
// TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace glv {

constexpr int kTcBM = 128;            // rows of Q per tile (MMA M)
constexpr int kTcBN = 256;            // columns of Qp per tile (MMA N)
constexpr int kTcRowBytes = 128;      // K slice per stage: one 128-byte swizzle row
constexpr int kTcKpad = 64;           // operand rows padded to a multiple of 64 elements
constexpr int kTcEpiWarps = 8;      // two per TMEM lane quadrant, each storing half the columns
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;

template <int MODE>  // 0 = BF16, 1 = TF32x3
struct TcCfg {
  static constexpr int kOps = MODE == 0 ? 1 : 2;          // operand copies per side (hi, lo)
  static constexpr int kStages = MODE == 0 ? 4 : 2;
  static constexpr int kABytes = kTcBM * kTcRowBytes;     // 16 KB
  static constexpr int kBBytes = kTcBN * kTcRowBytes;     // 32 KB
  static constexpr int kStageBytes = kOps * (kABytes + kBBytes);
  static constexpr int kElemBytes = MODE == 0 ? 2 : 4;
  static constexpr int kKPerStage = kTcRowBytes / kElemBytes;
  static constexpr int kKPerMma = MODE == 0 ? 16 : 8;     // 32 bytes of K per MMA
  static constexpr int kMmaPerStage = kKPerStage / kKPerMma;
  // epilogue staging: per epilogue warp a 32 x 32 FP32 tile -- rows padded to 33 words for the
  // store-instruction path, or 4 KB in the 128-byte swizzled layout of a TMA tensor store
  static constexpr size_t kEpiBytes = (size_t)kTcEpiWarps * 32 * 33 * sizeof(float);
  static constexpr size_t kSmem = (size_t)kStages * kStageBytes + kEpiBytes + 256 + 1024;
};

struct TcArgs {
  float* out;
  int64_t M;        // rows (queries)
  int64_t N;        // columns (C * d)
  int nkb;          // K stages
  int tiles_n;
  int64_t num_tiles;
  int32_t* d_status;
  int tma_store;    // 1: the epilogue writes Qp with TMA tensor stores (tmOut)
};

template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 1)
    project_tc_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                      const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
                      const __grid_constant__ CUtensorMap tmOut, const TcArgs args) {
  using Cfg = TcCfg<MODE>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // [stages | epilogue staging (1024-aligned) | barriers]
  float* epi = reinterpret_cast<float*>(smem + (size_t)Cfg::kStages * Cfg::kStageBytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)Cfg::kStages * Cfg::kStageBytes + Cfg::kEpiBytes);
  uint64_t* empty = full + Cfg::kStages;
  uint64_t* tfull = empty + Cfg::kStages;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < Cfg::kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 32 * kTcEpiWarps);
    }
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&tmA0);
    tc::prefetch_tmap(&tmB0);
    if (args.tma_store) tc::prefetch_tmap(&tmOut);
    if (MODE == 1) {
      tc::prefetch_tmap(&tmA1);
      tc::prefetch_tmap(&tmB1);
    }
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int stage = 0;
      uint32_t phase = 0;
      bool pending[Cfg::kStages];
      uint32_t pend_phase[Cfg::kStages];
      for (int s = 0; s < Cfg::kStages; ++s) {
        pending[s] = false;
        pend_phase[s] = 0;
      }
      bool ok = true;
      for (int64_t t = blockIdx.x; ok && t < args.num_tiles; t += gridDim.x) {
        const int tm = (int)(t / args.tiles_n), tn = (int)(t % args.tiles_n);
        for (int kb = 0; kb < args.nkb; ++kb) {
          if (!tc::mbar_wait(&empty[stage], phase ^ 1, abort_flag)) {
            ok = false;
            break;
          }
          pending[stage] = false;
          tc::mbar_arrive_expect_tx(&full[stage], Cfg::kStageBytes);
          uint8_t* base = smem + (size_t)stage * Cfg::kStageBytes;
          const int x = kb * Cfg::kKPerStage;
          tc::tma_load_2d(base, &tmA0, x, tm * kTcBM, &full[stage]);
          if (MODE == 1) tc::tma_load_2d(base + Cfg::kABytes, &tmA1, x, tm * kTcBM, &full[stage]);
          uint8_t* bb = base + Cfg::kOps * Cfg::kABytes;
          tc::tma_load_2d(bb, &tmB0, x, tn * kTcBN, &full[stage]);
          if (MODE == 1) tc::tma_load_2d(bb + Cfg::kBBytes, &tmB1, x, tn * kTcBN, &full[stage]);
          pending[stage] = true;
          pend_phase[stage] = phase;
          if (++stage == Cfg::kStages) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // drain: no TMA write may still be in flight into this CTA's shared memory at exit
      volatile int no_abort = 0;
      for (int s = 0; s < Cfg::kStages; ++s)
        if (pending[s]) tc::mbar_wait(&full[s], pend_phase[s], &no_abort);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      constexpr uint32_t idesc = tc::instr_desc(MODE == 0 ? 1u : 2u, kTcBM, kTcBN);
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; ok && t < args.num_tiles; t += gridDim.x) {
        if (!tc::mbar_wait(&tempty[acc], acc_phase ^ 1, abort_flag)) break;
        tc::tc_fence_after();
        const uint32_t d_tmem = tmem + (uint32_t)(acc * kTcBN);
        for (int kb = 0; kb < args.nkb; ++kb) {
          if (!tc::mbar_wait(&full[stage], phase, abort_flag)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t base = tc::smem_u32(smem + (size_t)stage * Cfg::kStageBytes);
          const uint32_t bbase = base + Cfg::kOps * Cfg::kABytes;
#pragma unroll
          for (int k = 0; k < Cfg::kMmaPerStage; ++k) {
            const uint32_t acc_in = (kb > 0 || k > 0) ? 1u : 0u;
            const uint64_t a0 = tc::sw128_kmajor_desc(base + k * 32);
            const uint64_t b0 = tc::sw128_kmajor_desc(bbase + k * 32);
            if (MODE == 0) {
              tc::mma_bf16(d_tmem, a0, b0, idesc, acc_in);
            } else {
              const uint64_t a1 = tc::sw128_kmajor_desc(base + Cfg::kABytes + k * 32);
              const uint64_t b1 = tc::sw128_kmajor_desc(bbase + Cfg::kBBytes + k * 32);
              tc::mma_tf32(d_tmem, a0, b0, idesc, acc_in);  // hi * hi
              tc::mma_tf32(d_tmem, a0, b1, idesc, 1u);      // hi * lo
              tc::mma_tf32(d_tmem, a1, b0, idesc, 1u);      // lo * hi
            }
          }
          tc::mma_commit(&empty[stage]);  // frees the stage once these MMAs have read it
          if (++stage == Cfg::kStages) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        tc::mma_commit(&tfull[acc]);  // accumulator ready for the epilogue
        acc ^= 1;
        if (acc == 0) acc_phase ^= 1;
      }
      // drain: every MMA issued by this thread has completed before TMEM is released
      tc::mma_commit(drain);
      volatile int no_abort = 0;
      tc::mbar_wait(drain, 0, &no_abort);
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    constexpr int kChunks = kTcBN / 32 / (kTcEpiWarps / 4);  // 32-column chunks per warp
    const int ch0 = ((warp - 2) / 4) * kChunks;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int64_t t = blockIdx.x; t < args.num_tiles; t += gridDim.x) {
      // warp-uniform bounded wait (tcgen05.ld below needs the whole warp)
      int ok = 0;
      if (lane == 0) ok = tc::mbar_wait(&tfull[acc], acc_phase, abort_flag) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      (void)tc::mbar_try_wait(&tfull[acc], acc_phase);
      tc::tc_fence_after();
      const int tm = (int)(t / args.tiles_n), tn = (int)(t % args.tiles_n);
      const int64_t row_base = (int64_t)tm * kTcBM + q * 32;
      // lane = row in TMEM; each 32 x 32 chunk goes through the warp's shared-memory tile
      // (conflict-free: rows padded to 33 words) so the global stores write one row segment
      // of 32 consecutive columns (128 bytes) per instruction
      // The TMEM load of the next chunk is issued once this chunk's values are in shared
      // memory, so it lands while this chunk's global stores go out.
      float* stg = epi + (warp - 2) * (32 * 33);
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kTcBN + ch0 * 32);
      uint32_t r[32];
      tc::tmem_ld_32x32b_x32(tbase, r);
      tc::tmem_ld_wait(r);
      if (args.tma_store) {
        // each 32 x 32 chunk goes to the warp's 4-KB staging tile in the 128-byte swizzled layout
        // (row = lane, 16-byte piece c at position c ^ (row & 7): the eight lanes of a quarter
        // warp hit eight different bank groups) and leaves with one TMA tensor store; rows or
        // columns beyond Qp's bounds are clipped by the TMA unit
        uint8_t* tile = reinterpret_cast<uint8_t*>(epi) + (size_t)(warp - 2) * 4096;
#pragma unroll 1
        for (int ch = 0; ch < kChunks; ++ch) {
          if (lane == 0) tc::tma_store_wait_read();  // the previous chunk's store has read the tile
          __syncwarp();
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint4 v = make_uint4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
            *reinterpret_cast<uint4*>(tile + lane * 128 + ((c ^ (lane & 7)) << 4)) = v;
          }
          tc::fence_proxy_async_smem();
          __syncwarp();
          if (ch + 1 < kChunks) tc::tmem_ld_32x32b_x32(tbase + (uint32_t)((ch + 1) * 32), r);
          if (lane == 0) {
            tc::tma_store_2d(&tmOut, tn * kTcBN + (ch0 + ch) * 32, (int)row_base, tile);
            tc::tma_store_commit();
          }
          tc::tmem_ld_wait(r);
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&tempty[acc]);
        acc ^= 1;
        if (acc == 0) acc_phase ^= 1;
        continue;
      }
#pragma unroll 1
      for (int ch = 0; ch < kChunks; ++ch) {
#pragma unroll
        for (int u = 0; u < 32; ++u) stg[lane * 33 + u] = __uint_as_float(r[u]);
        __syncwarp();
        if (ch + 1 < kChunks) tc::tmem_ld_32x32b_x32(tbase + (uint32_t)((ch + 1) * 32), r);
        const int64_t col = (int64_t)tn * kTcBN + (ch0 + ch) * 32 + lane;
        if (col < args.N) {
#pragma unroll 8
          for (int rr = 0; rr < 32; ++rr) {
            const int64_t row = row_base + rr;
            if (row < args.M) args.out[row * args.N + col] = stg[rr * 33 + lane];
          }
        }
        __syncwarp();
        tc::tmem_ld_wait(r);
      }
      tc::tc_fence_before();
      tc::mbar_arrive(&tempty[acc]);
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1;
    }
  }

  if (warp >= 2 && lane == 0 && args.tma_store) tc::tma_store_wait_all();  // Qp written before exit
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && *abort_flag) report(args.d_status, GLV_ERR_TIMEOUT);
}

// ---- operand preparation -------------------------------------------------------------------

// Both operands in one launch: one thread per 4 consecutive K elements of a row, the rows of
// Q first, then those of A; Kp is a multiple of 64, so a group never straddles rows.  Reads
// are 16-byte vectors when D % 4 == 0.
struct PrepPair {
  const float* src[2];
  int64_t rows[2];
};

__global__ void prep_bf16_kernel(PrepPair pp, int D, int Kp, __nv_bfloat16* __restrict__ dst0,
                                 __nv_bfloat16* __restrict__ dst1) {
  const int gpr = Kp / 4;
  const int64_t first = pp.rows[0] * (int64_t)gpr;
  const int64_t total = first + pp.rows[1] * (int64_t)gpr;
  const bool vec = (D % 4) == 0;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < total;
       i0 += (int64_t)gridDim.x * blockDim.x) {
    const int w = i0 < first ? 0 : 1;
    const int64_t i = w ? i0 - first : i0;
    const float* src = pp.src[w];
    __nv_bfloat16* dst = w ? dst1 : dst0;
    const int64_t r = i / gpr;
    const int k = (int)(i - r * gpr) * 4;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    const float* s = src + r * D + k;
    if (vec && k < D) {
      const float4 w = __ldg(reinterpret_cast<const float4*>(s));
      v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k + u < D) v[u] = __ldg(s + u);
    }
    __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
    uint2 packed;
    packed.x = *reinterpret_cast<uint32_t*>(&lo);
    packed.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(dst + r * Kp + k) = packed;
  }
}

__global__ void prep_tf32x3_kernel(PrepPair pp, int D, int Kp, float* __restrict__ hi0, float* __restrict__ lo0,
                                   float* __restrict__ hi1, float* __restrict__ lo1) {
  const int gpr = Kp / 4;
  const int64_t first = pp.rows[0] * (int64_t)gpr;
  const int64_t total = first + pp.rows[1] * (int64_t)gpr;
  const bool vec = (D % 4) == 0;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < total;
       i0 += (int64_t)gridDim.x * blockDim.x) {
    const int w = i0 < first ? 0 : 1;
    const int64_t i = w ? i0 - first : i0;
    const float* src = pp.src[w];
    float* hi = w ? hi1 : hi0;
    float* lo = w ? lo1 : lo0;
    const int64_t r = i / gpr;
    const int k = (int)(i - r * gpr) * 4;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    const float* s = src + r * D + k;
    if (vec && k < D) {
      const float4 w = __ldg(reinterpret_cast<const float4*>(s));
      v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k + u < D) v[u] = __ldg(s + u);
    }
    float h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      h[u] = __uint_as_float(__float_as_uint(v[u]) & 0xffffe000u);
      l[u] = v[u] - h[u];  // exact: v and h share sign and exponent
    }
    *reinterpret_cast<float4*>(hi + r * Kp + k) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(lo + r * Kp + k) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

// ---- host side -------------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// rows x Kp operand, K-major; box = 128 bytes of K x box_rows rows, 128-byte swizzle.
static bool make_operand_map(CUtensorMap* map, const void* base, bool bf16, int64_t rows, int Kp, int box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const int eb = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * eb};
  cuuint32_t box[2] = {(cuuint32_t)(kTcRowBytes / eb), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

size_t project_tc_ws_bytes(int64_t nq, int D, int64_t Mc, int bf16) {
  const int64_t Kp = round_up(D, kTcKpad);
  const int64_t eb = bf16 ? 2 : 4;
  const int64_t ops = bf16 ? 1 : 2;
  return (size_t)(round_up(nq * Kp * eb, 1024) * ops + round_up(Mc * Kp * eb, 1024) * ops);
}

cudaError_t launch_project_tc(const float* Q, int64_t nq, int D, const float* A, int64_t Mc, float* Qp,
                              int bf16, void* ws, int32_t* d_status, int num_sms, cudaStream_t st) {
  const int Kp = (int)round_up(D, kTcKpad);
  const int eb = bf16 ? 2 : 4;
  char* p = static_cast<char*>(ws);
  const size_t qbytes = (size_t)round_up(nq * Kp * eb, 1024), abytes = (size_t)round_up(Mc * Kp * eb, 1024);
  void *q0, *q1 = nullptr, *a0, *a1 = nullptr;
  q0 = p;
  p += qbytes;
  if (!bf16) {
    q1 = p;
    p += qbytes;
  }
  a0 = p;
  p += abytes;
  if (!bf16) {
    a1 = p;
    p += abytes;
  }
  const int pb = num_sms * 8;
  PrepPair pp;
  pp.src[0] = Q;
  pp.rows[0] = nq;
  pp.src[1] = A;
  pp.rows[1] = Mc;
  if (bf16) {
    prep_bf16_kernel<<<pb, 256, 0, st>>>(pp, D, Kp, static_cast<__nv_bfloat16*>(q0), static_cast<__nv_bfloat16*>(a0));
  } else {
    prep_tf32x3_kernel<<<pb, 256, 0, st>>>(pp, D, Kp, static_cast<float*>(q0), static_cast<float*>(q1),
                                           static_cast<float*>(a0), static_cast<float*>(a1));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  CUtensorMap mA0, mA1, mB0, mB1;
  if (!make_operand_map(&mA0, q0, bf16, nq, Kp, kTcBM) || !make_operand_map(&mB0, a0, bf16, Mc, Kp, kTcBN))
    return cudaErrorInvalidValue;
  if (bf16) {
    mA1 = mA0;
    mB1 = mB0;
  } else if (!make_operand_map(&mA1, q1, false, nq, Kp, kTcBM) ||
             !make_operand_map(&mB1, a1, false, Mc, Kp, kTcBN)) {
    return cudaErrorInvalidValue;
  }

  // Qp written by TMA tensor stores when its rows are 16-byte multiples (32 x 32 FP32 boxes,
  // 128-byte swizzle), else by store instructions
  CUtensorMap mOut;
  bool tma_store = (Mc % 4) == 0 && (reinterpret_cast<uintptr_t>(Qp) % 16) == 0;
  if (tma_store) {
    auto enc = tensor_map_encoder();
    cuuint64_t dims[2] = {(cuuint64_t)Mc, (cuuint64_t)nq};
    cuuint64_t strides[1] = {(cuuint64_t)Mc * 4};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    tma_store = enc && enc(&mOut, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Qp, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  if (!tma_store) mOut = mA0;  // unused

  TcArgs args;
  args.tma_store = tma_store ? 1 : 0;
  args.out = Qp;
  args.M = nq;
  args.N = Mc;
  args.nkb = Kp / (kTcRowBytes / eb);
  args.tiles_n = (int)((Mc + kTcBN - 1) / kTcBN);
  args.num_tiles = ((nq + kTcBM - 1) / kTcBM) * (int64_t)args.tiles_n;
  args.d_status = d_status;
  const int grid = (int)(args.num_tiles < num_sms ? args.num_tiles : num_sms);
  if (bf16) {
    auto k = project_tc_kernel<0>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<0>::kSmem);
    if (e != cudaSuccess) return e;
    k<<<grid, kTcThreads, TcCfg<0>::kSmem, st>>>(mA0, mA1, mB0, mB1, mOut, args);
  } else {
    auto k = project_tc_kernel<1>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<1>::kSmem);
    if (e != cudaSuccess) return e;
    k<<<grid, kTcThreads, TcCfg<1>::kSmem, st>>>(mA0, mA1, mB0, mB1, mOut, args);
  }
  return cudaGetLastError();
}

}  // namespace glv
