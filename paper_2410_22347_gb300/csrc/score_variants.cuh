// score_variants.cuh -- the stand-alone scoring kernel and the fused scoring + top-kappa
// kernel as templates over (store type, lanes per candidate G, loads per lane NCH, gather
// mode), with the launchers that instantiate them for one store type (one translation unit
// per store type: score_f32.cu, score_bf16.cu, score_fp8.cu).
#pragma once

#include "kernels.cuh"
#include "score_bulk.cuh"
#include "score_dev.cuh"
#include "score_launch.cuh"
#include "topk_dev.cuh"

namespace glv {

constexpr int kFusedCache = 2048;  // list entries kept as keys in shared memory
constexpr int kBulkSlots = 2;      // ring slots per warp (bulk gather)
constexpr int kScoreThreads = 256;

// Shared-memory carve-up shared by host and device: [projected query | keys | rings | bars].
struct ScoreSmem {
  size_t qs_bytes, keys_bytes, ring_bytes, bar_bytes;
  __host__ __device__ size_t total() const { return qs_bytes + keys_bytes + ring_bytes + bar_bytes; }
};

// keys_bytes (fused only): kFusedCache cached keys, then the kappa selected keys and ids,
// rounded to 128 bytes so the rings stay aligned.
__host__ __device__ inline ScoreSmem score_smem(int C, int qstride, bool fused, int mode, int RB, int nch,
                                                int kappa = 0) {
  ScoreSmem m;
  m.qs_bytes = (((size_t)C * qstride * sizeof(float)) + 127) & ~size_t(127);
  m.keys_bytes = fused ? (((size_t)kFusedCache * sizeof(uint32_t) + (size_t)kappa * 8) + 127) & ~size_t(127) : 0;
  const int warps = kScoreThreads / 32;
  m.ring_bytes = mode == 2 ? (size_t)warps * kBulkSlots * RB * nch * 16 : 0;
  m.bar_bytes = mode == 2 ? (size_t)warps * kBulkSlots * sizeof(uint64_t) : 0;
  return m;
}

// Rows per bulk batch: the largest of 32, 16, 8 whose rings fit next to the rest.
inline int bulk_rows(int C, int qstride, bool fused, int nch, int kappa, size_t limit) {
  for (int RB = 32; RB >= 8; RB /= 2)
    if (score_smem(C, qstride, fused, 2, RB, nch, kappa).total() <= limit) return RB;
  return 0;
}

#ifndef GLV_FUSED_MINB
#define GLV_FUSED_MINB 6  // CTAs per SM the register-gather fused kernel is compiled for
#endif

constexpr int fused_min_blocks_regs(int n) { return n <= 4 ? GLV_FUSED_MINB : n <= 5 ? 5 : n <= 8 ? 4 : 3; }

// CTAs per SM the fused kernel is compiled for: the register budget must hold NCH row chunks
// per lane (x2 when the next candidate's loads are in flight, mode 1) without spilling; the
// FP8 decode costs about one chunk's worth of registers more.
constexpr int fused_min_blocks(int dt, int mode, int nch) {
  return mode == 2 ? 1 : mode == 1 ? 3 : fused_min_blocks_regs(nch + (dt == GLV_FP8_E4M3 ? 1 : 0));
}

template <int DT, int G, int NCH, int MODE, class Sink>
GLV_DEV void score_span(const ScoreArgs& a, uint8_t* smem, const ScoreSmem& L, int RB, int64_t b0, int64_t b1,
                        Sink& sink, volatile int* abort) {
  const float* qs = reinterpret_cast<const float*>(smem);
  if constexpr (MODE == 2) {
    uint8_t* ring = smem + L.qs_bytes + L.keys_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + L.ring_bytes);
    const int warp = threadIdx.x >> 5;
    const size_t per_warp = (size_t)kBulkSlots * RB * a.nch * 16;
    score_range_bulk<DT, G, NCH, kBulkSlots>(a, qs, ring + warp * per_warp, bars + warp * kBulkSlots, RB, b0, b1,
                                             sink, abort);
  } else {
    score_range<DT, G, NCH, MODE == 1>(a, qs, b0, b1, sink);
  }
}

template <int MODE>
GLV_DEV void init_bulk_bars(uint8_t* smem, const ScoreSmem& L) {
  if constexpr (MODE == 2) {
    if (threadIdx.x == 0) {
      uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.qs_bytes + L.keys_bytes + L.ring_bytes);
      for (int t = 0; t < (kScoreThreads / 32) * kBulkSlots; ++t) tc::mbar_init(&bars[t], 1);
      tc::fence_mbar_init();
    }
  }
}

// One CTA per (query, split of its candidate list): the query's C projected views are staged
// once in shared memory, so every candidate, whatever its cluster, finds its q_c on chip (the
// "eager" inner product of the paper).
template <int DT, int G, int NCH, int MODE>
__global__ void __launch_bounds__(kScoreThreads) score_kernel(const ScoreArgs a, int RB) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ int abort_flag;
  const ScoreSmem L = score_smem(a.C, a.qstride, false, MODE, RB, a.nch);
  if (threadIdx.x == 0) abort_flag = 0;
  init_bulk_bars<MODE>(smem, L);
  const int64_t j = blockIdx.x;
  stage_qp<DT>(a, j, reinterpret_cast<float*>(smem));
  __syncthreads();
  const int64_t p0 = a.off[j], p1 = a.off[j + 1];
  // split boundaries on multiples of 64 candidates: every candidate keeps the position parity
  // (and so the summation order, see dot_chunk) it has in the fused kernel
  const int64_t per = ((p1 - p0 + a.splits - 1) / a.splits + 63) / 64 * 64;
  const int64_t b0 = min(p1, p0 + (int64_t)blockIdx.y * per);
  const int64_t b1 = min(p1, b0 + per);
  float* scores = a.scores;
  auto sink = [scores](int64_t p, float s) { scores[p] = s; };
  score_span<DT, G, NCH, MODE>(a, smem, L, RB, b0, b1, sink, &abort_flag);
  if (MODE == 2) {
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) report(a.d_status, GLV_ERR_TIMEOUT);
  }
}

// Gather-score and top-kappa of one query in one CTA: scores stay on chip as order-preserving
// keys in shared memory and the radix selection runs there; a list longer than the key cache
// spills its scores to the caller's scratch (L2-resident during the selection passes).
template <int DT, int G, int NCH, int MODE>
__global__ void __launch_bounds__(kScoreThreads, fused_min_blocks(DT, MODE, NCH))
    score_topk_kernel(const ScoreArgs a, int RB, int kappa, float* out_s, int32_t* out_id) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ TopkSmem S;
  __shared__ int abort_flag;
  const ScoreSmem L = score_smem(a.C, a.qstride, true, MODE, RB, a.nch, kappa);
  uint32_t* kc = reinterpret_cast<uint32_t*>(smem + L.qs_bytes);
  if (threadIdx.x == 0) {
    abort_flag = 0;
    S.sel_key = kc + kFusedCache;
    S.sel_id = reinterpret_cast<int32_t*>(kc + kFusedCache + kappa);
    S.region = kc;
    S.region_words = kFusedCache;
  }
  init_bulk_bars<MODE>(smem, L);
  const int64_t j = blockIdx.x;
  stage_qp<DT>(a, j, reinterpret_cast<float*>(smem));
  __syncthreads();
  const int64_t p0 = a.off[j], p1 = a.off[j + 1];
  const int64_t L_ = p1 - p0;
  const bool cached = L_ <= kFusedCache;
  float* scores = a.scores;
  if (cached) {
    auto sink = [kc, p0](int64_t p, float s) { kc[p - p0] = score_key(s); };
    score_span<DT, G, NCH, MODE>(a, smem, L, RB, p0, p1, sink, &abort_flag);
  } else {
    auto sink = [scores](int64_t p, float s) { scores[p] = s; };
    score_span<DT, G, NCH, MODE>(a, smem, L, RB, p0, p1, sink, &abort_flag);
  }
  __syncthreads();
  if (MODE == 2 && threadIdx.x == 0 && abort_flag) report(a.d_status, GLV_ERR_TIMEOUT);
  const float* sj = scores + p0;
  const int32_t* ij = a.ids + p0;
  select_topk(
      S, L_, kappa, cached, [&](int64_t p) -> uint32_t { return cached ? kc[p] : score_key(sj[p]); },
      [&](int64_t p) -> int32_t { return ij[p]; }, out_s + j * kappa, out_id + j * kappa);
}

// Set kernel k's preferred shared-memory carveout: carve_kb > 0 caps it (when one CTA of
// smem bytes fits under the cap), 0 restores the driver's choice.  The setting stays on the
// function, so every launch sets it.
inline cudaError_t apply_carveout(const void* k, size_t smem, int carve_kb) {
  static int per_sm[64] = {0};
  int pct = cudaSharedmemCarveoutDefault;
  if (carve_kb > 0) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (per_sm[dev] == 0) {
      e = cudaDeviceGetAttribute(&per_sm[dev], cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
      if (e != cudaSuccess) return e;
    }
    const int64_t cap = (int64_t)carve_kb * 1024;
    if (per_sm[dev] > 0 && cap >= (int64_t)smem + 2048 && cap < per_sm[dev])
      pct = (int)(cap * 100 / per_sm[dev]);
  }
  return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

struct ScoreLaunch {
  const ScoreArgs& a;
  dim3 grid;
  int RB;
  int carve_kb;
  cudaStream_t st;
  template <int DT, int G, int NCH, int MODE>
  cudaError_t go() {
    auto k = score_kernel<DT, G, NCH, MODE>;
    const size_t smem = score_smem(a.C, a.qstride, false, MODE, RB, a.nch).total();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = apply_carveout(reinterpret_cast<const void*>(k), smem, carve_kb);
    if (e != cudaSuccess) return e;
    k<<<grid, kScoreThreads, smem, st>>>(a, RB);
    return cudaGetLastError();
  }
};

struct FusedLaunch {
  const ScoreArgs& a;
  int64_t nq;
  int RB;
  int kappa;
  float* out_s;
  int32_t* out_id;
  int carve_kb;
  cudaStream_t st;
  template <int DT, int G, int NCH, int MODE>
  cudaError_t go() {
    auto k = score_topk_kernel<DT, G, NCH, MODE>;
    const size_t smem = score_smem(a.C, a.qstride, true, MODE, RB, a.nch, kappa).total();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = apply_carveout(reinterpret_cast<const void*>(k), smem, carve_kb);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)nq, kScoreThreads, smem, st>>>(a, RB, kappa, out_s, out_id);
    return cudaGetLastError();
  }};

template <int DT>
cudaError_t launch_score_dt(const ScoreArgs& a, dim3 grid, int RB, ScoreConfig cfg, cudaStream_t st) {
  ScoreLaunch f{a, grid, RB, cfg.carve_kb, st};
  return dispatch_score<DT>(cfg.G, a.nch, cfg.mode, f);
}

template <int DT>
cudaError_t launch_fused_dt(const ScoreArgs& a, int64_t nq, int RB, int kappa, float* out_s, int32_t* out_id,
                            ScoreConfig cfg, cudaStream_t st) {
  FusedLaunch f{a, nq, RB, kappa, out_s, out_id, cfg.carve_kb, st};
  return dispatch_score<DT>(cfg.G, a.nch, cfg.mode, f);
}

#define GLV_INSTANTIATE_SCORE_PLAIN(DT) \
  template cudaError_t launch_score_dt<DT>(const ScoreArgs&, dim3, int, ScoreConfig, cudaStream_t);
#define GLV_INSTANTIATE_SCORE_FUSED(DT)                                                            \
  template cudaError_t launch_fused_dt<DT>(const ScoreArgs&, int64_t, int, int, float*, int32_t*, \
                                           ScoreConfig, cudaStream_t);

}  // namespace glv
