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

constexpr int kBulkSlots = 2;      // ring slots per warp (bulk gather)
constexpr int kScoreThreads = 256;
constexpr int kWideThreads = 512;  // fused kernel, wide schedule: twice the warps per staged query
// List entries the fused kernel keeps as keys in shared memory: kWarpThrKeys per thread, the
// most the per-warp threshold selection takes (2048 for 256 threads, 4096 for 512).
constexpr int fused_cache(int threads) { return kWarpThrKeys * threads; }
constexpr int kFusedCache = fused_cache(kScoreThreads);

// Shared-memory carve-up shared by host and device: [projected query | keys | rings | bars].
struct ScoreSmem {
  size_t qs_bytes, keys_bytes, ring_bytes, bar_bytes;
  __host__ __device__ size_t total() const { return qs_bytes + keys_bytes + ring_bytes + bar_bytes; }
};

// keys_bytes (fused only): `cache` cached keys, then the kappa selected keys and ids,
// rounded to 128 bytes so the rings stay aligned.
__host__ __device__ inline ScoreSmem score_smem(int C, int qstride, bool fused, int mode, int RB, int nch,
                                                int kappa = 0, int cache = kFusedCache) {
  ScoreSmem m;
  // the C rows of projected views
  m.qs_bytes = (((size_t)C * qstride * sizeof(float)) + 127) & ~size_t(127);
  m.keys_bytes = fused ? (((size_t)cache * sizeof(uint32_t) + (size_t)kappa * 8) + 127) & ~size_t(127) : 0;
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

constexpr int fused_min_blocks_regs(int n) { return n <= 3 ? GLV_FUSED_MINB : n <= 5 ? 5 : n <= 8 ? 4 : 3; }

// CTAs per SM the fused kernel is compiled for: the register budget must hold NCH row chunks
// per lane (x2 when the next candidate's loads are in flight, mode 1) without spilling; the
// FP8 decode costs about two chunks' worth of registers more.
constexpr int fused_min_blocks(int dt, int mode, int nch) {
  return mode == 2 ? 1 : mode == 1 ? 3 : fused_min_blocks_regs(nch + (dt == GLV_FP8_E4M3 ? 2 : 0));
}
// The same register budget per thread for CTAs of `threads` threads.
constexpr int fused_min_blocks_t(int dt, int mode, int nch, int threads) {
  return fused_min_blocks(dt, mode, nch) * kScoreThreads / threads > 0
             ? fused_min_blocks(dt, mode, nch) * kScoreThreads / threads
             : 1;
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

// Gather-score and top-kappa, persistent: each CTA claims work items (a whole candidate list,
// or a chunk of at most kChunk candidates of a long one) from the plan until none is left.
// Scores stay on chip as order-preserving keys in shared memory and the selection runs
// there; an item longer than the key cache (fused_cache(TPB) keys) spills its scores to the
// caller's scratch.  TPB = 256 or 512 threads: the wide CTA spreads one staged query over
// twice the warps (more row loads in flight per SM for the same shared memory) and keeps
// twice the keys on chip.  A chunk
// of a long list writes its own top-kappa at the start of its part of the scratch (scores then
// ids); the CTA that finishes a query's last chunk (a fenced per-query counter; nothing waits)
// selects the query's top-kappa from the chunks' lists, which contain it: a candidate outside
// its chunk's top-kappa has kappa candidates of that chunk ranked before it.
template <int DT, int G, int NCH, int MODE, int TPB>
__global__ void __launch_bounds__(TPB, fused_min_blocks_t(DT, MODE, NCH, TPB))
    score_topk_kernel(const ScoreArgs a, int kappa, ChunkPlan plan, int direct, float* out_s, int32_t* out_id) {
  static_assert(MODE != 2, "the fused kernel gathers rows into registers");
  constexpr int kCache = fused_cache(TPB);
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ TopkSmem S;
  // work items, double-buffered: slot cur holds the current item, thread 0 fills the other
  // slot with the next one while the current one is being selected
  __shared__ __align__(16) ItemRec s_rec[2];
  __shared__ int s_valid[2], s_last, s_claimed, s_items;  // s_claimed: next item, claimed ahead
  __shared__ int64_t s_staged;
  const ScoreSmem L = score_smem(a.C, a.qstride, true, MODE, 0, a.nch, kappa, kCache);
  float* qs = reinterpret_cast<float*>(smem);
  uint32_t* kc = reinterpret_cast<uint32_t*>(smem + L.qs_bytes);
  if (threadIdx.x == 0) {
    S.sel_key = kc + kCache;
    S.sel_id = reinterpret_cast<int32_t*>(kc + kCache + kappa);
    S.region = kc;
    S.region_words = kCache;
    s_staged = -1;
    if (direct) {  // one CTA per query, no plan: the query's whole list is the only item
      const int64_t q = blockIdx.x, p0 = a.off[q];
      s_rec[0].b0 = p0;
      s_rec[0].len = (int32_t)(a.off[q + 1] - p0);
      s_rec[0].q = (int32_t)q;
      s_rec[0].c = 0;
      s_rec[0].nchunks = 1;
      s_valid[0] = 1;
      s_items = 0;
      s_claimed = 0;
    } else {
      s_items = *plan.n_items;
      const int first = atomicAdd(plan.next, 1);
      s_valid[0] = first < s_items;
      if (s_valid[0]) s_rec[0] = plan.items[first];
      s_claimed = atomicAdd(plan.next, 1);
    }
  }
  __syncthreads();
  float* scores = a.scores;
  for (int cur = 0;; cur ^= 1) {
    if (!s_valid[cur]) break;
    // thread 0: copy the next item's record into the other slot (it lands during this item's
    // gather) and claim the item after it
    if (threadIdx.x == 0) {
      const int claimed = s_claimed;
      const bool has_nxt = claimed < s_items;
      s_valid[cur ^ 1] = has_nxt;
      if (has_nxt) {
        const uint64_t* src = reinterpret_cast<const uint64_t*>(plan.items + claimed);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&s_rec[cur ^ 1]);
#pragma unroll
        for (int w = 0; w < (int)(sizeof(ItemRec) / 8); ++w) cp_async8(dst + w, src + w);
        s_claimed = atomicAdd(plan.next, 1);
      }
    }
    const int64_t j = s_rec[cur].q;
    if (j != s_staged) stage_qp<DT>(a, j, qs);  // else its views were copied during the last selection
    cp_async_wait_all();
    __syncthreads();
    if (threadIdx.x == 0) s_staged = j;
    const int64_t b0 = s_rec[cur].b0, b1 = b0 + s_rec[cur].len;
    if (b1 - b0 <= kCache) {
      auto sink = [kc, b0](int64_t p, float s) { kc[p - b0] = score_key(s); };
      score_range<DT, G, NCH, MODE == 1, TPB == kScoreThreads>(a, qs, b0, b1, sink);
    } else {
      auto sink = [scores](int64_t p, float s) { scores[p] = s; };
      score_range<DT, G, NCH, MODE == 1, TPB == kScoreThreads>(a, qs, b0, b1, sink);
    }
    if (threadIdx.x == 0) cp_async_wait_all();
    __syncthreads();
    // while this item is being selected (the selection does not read qs), the next item's
    // query views are copied into qs asynchronously, and DRAM fetches the next item's first
    // rows (one per thread) into L2
    if (s_valid[cur ^ 1]) {
      const int64_t nb0 = s_rec[cur ^ 1].b0, nq = s_rec[cur ^ 1].q;
      const int nlen = s_rec[cur ^ 1].len;
      if (threadIdx.x < nlen) {
        const int64_t id = a.ids[nb0 + threadIdx.x];
        if (id >= 0 && id < a.N) prefetch_l2_bulk(a.Xred + id * a.row_stride, (uint32_t)a.row_stride);
      }
      const int64_t qbytes = (int64_t)a.C * a.d * 4;
      if (nq != j && qp_async_ok<DT>(a)) {
        stage_qp_async<DT>(a, nq, qs);
        if (threadIdx.x == 0) s_staged = nq;  // read again only after the selection's barriers
      } else if (nq != j && (qbytes & 15) == 0) {
        const int pieces = (int)((qbytes + 4095) / 4096);
        const int t = (int)blockDim.x - 1 - (int)threadIdx.x;
        if (t < pieces) {
          const int64_t o = (int64_t)t * 4096;
          prefetch_l2_bulk(reinterpret_cast<const uint8_t*>(a.Qp) + nq * qbytes + o,
                           (uint32_t)(qbytes - o < 4096 ? qbytes - o : 4096));
        }
      }
    }
    // re-read the item after the barrier (nothing of it stays live across the gather)
    const int nchunks = s_rec[cur].nchunks;
    const int64_t jj = s_rec[cur].q, c0 = s_rec[cur].b0, lc = s_rec[cur].len;
    const bool in_kc = lc <= kCache;
    const float* sj = scores + c0;
    const int32_t* ij = a.ids + c0;
    // FP8 rows leave the kernel issue-bound: the survivors of long on-chip lists are ordered by
    // the bitonic network there (fewer instructions); the other stores keep rank counting
    constexpr bool kNetworkSort = DT == GLV_FP8_E4M3;
    if (nchunks == 1) {
      select_topk(
          S, lc, kappa, in_kc, [&](int64_t p) -> uint32_t { return in_kc ? kc[p] : score_key(sj[p]); },
          [&](int64_t p) -> int32_t { return ij[p]; }, out_s + jj * kappa, out_id + jj * kappa, true,
          kNetworkSort);
    } else {
      // the chunk's unordered top-kappa goes to the start of its own part of the scratch
      // (scores, then ids): every chunk has at least kChunk >= 2 kappa candidates, and its
      // spilled scores have all been read when the list is written
      float* ps = scores + c0;
      select_topk(
          S, lc, kappa, in_kc, [&](int64_t p) -> uint32_t { return in_kc ? kc[p] : score_key(sj[p]); },
          [&](int64_t p) -> int32_t { return ij[p]; }, ps, reinterpret_cast<int32_t*>(ps + kappa), false);
      __threadfence();  // this chunk's list is visible before the count says so
      __syncthreads();
      if (threadIdx.x == 0) s_last = atomicAdd(plan.done + jj, 1) == nchunks - 1;
      __syncthreads();
      if (s_last) {
        __threadfence();
        const int64_t M = (int64_t)nchunks * kappa;
        const float* base = scores + a.off[jj];
        const int64_t kap = kappa;
        auto ent = [base, kap](int64_t e) { return base + (e / kap) * kChunk + (e % kap); };
        const bool mc = M <= kCache;
        if (mc)
          for (int64_t e = threadIdx.x; e < M; e += blockDim.x) kc[e] = score_key(__ldcg(ent(e)));
        __syncthreads();
        select_topk(
            S, M, kappa, mc, [&](int64_t e) -> uint32_t { return mc ? kc[e] : score_key(__ldcg(ent(e))); },
            [&](int64_t e) -> int32_t { return __ldcg(reinterpret_cast<const int32_t*>(ent(e) + kap)); },
            out_s + jj * kappa, out_id + jj * kappa, true, kNetworkSort);
      }
    }
    __syncthreads();
  }
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

template <int TPB>
struct FusedLaunch {
  const ScoreArgs& a;
  unsigned grid;
  int kappa;
  ChunkPlan plan;
  int direct;
  float* out_s;
  int32_t* out_id;
  int carve_kb;
  cudaStream_t st;
  template <int DT, int G, int NCH, int MODE>
  cudaError_t go() {
    if constexpr (MODE == 2) {
      return cudaErrorInvalidValue;  // the launcher maps the bulk gather to register loads
    } else {
      auto k = score_topk_kernel<DT, G, NCH, MODE, TPB>;
      const size_t smem = score_smem(a.C, a.qstride, true, MODE, 0, a.nch, kappa, fused_cache(TPB)).total();
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      e = apply_carveout(reinterpret_cast<const void*>(k), smem, carve_kb);
      if (e != cudaSuccess) return e;
      k<<<grid, TPB, smem, st>>>(a, kappa, plan, direct, out_s, out_id);
      return cudaGetLastError();
    }
  }
};

// One gather mode's launchers; each (store type, mode) is instantiated in a translation unit
// of its own (score_<type>_<kernel>_m<mode>.cu), the host code picks the mode at run time.
template <int DT, int MODE>
cudaError_t launch_score_mode(const ScoreArgs& a, dim3 grid, int RB, ScoreConfig cfg, cudaStream_t st) {
  ScoreLaunch f{a, grid, RB, cfg.carve_kb, st};
  return dispatch_score_mode<DT, MODE>(cfg.G, a.nch, f);
}

template <int DT, int MODE>
cudaError_t launch_fused_mode(const ScoreArgs& a, unsigned grid, int kappa, const ChunkPlan& plan, float* out_s,
                              int32_t* out_id, ScoreConfig cfg, cudaStream_t st) {
  FusedLaunch<kScoreThreads> f{a, grid, kappa, plan, (cfg.sched & 1) ? 0 : 1, out_s, out_id, cfg.carve_kb, st};
  return dispatch_score_mode<DT, MODE>(cfg.G, a.nch, f);
}

// The wide schedule (kWideThreads threads, register gather, the two smaller group sizes).
template <int DT>
cudaError_t launch_fused_wide(const ScoreArgs& a, unsigned grid, int kappa, const ChunkPlan& plan, float* out_s,
                              int32_t* out_id, ScoreConfig cfg, cudaStream_t st) {
  FusedLaunch<kWideThreads> f{a, grid, kappa, plan, (cfg.sched & 1) ? 0 : 1, out_s, out_id, cfg.carve_kb, st};
  return dispatch_score_wide<DT>(cfg.G, a.nch, f);
}

#define GLV_INSTANTIATE_SCORE_PLAIN(DT, MODE) \
  template cudaError_t launch_score_mode<DT, MODE>(const ScoreArgs&, dim3, int, ScoreConfig, cudaStream_t);
#define GLV_INSTANTIATE_SCORE_FUSED(DT, MODE)                                                              \
  template cudaError_t launch_fused_mode<DT, MODE>(const ScoreArgs&, unsigned, int, const ChunkPlan&, float*, \
                                                   int32_t*, ScoreConfig, cudaStream_t);
#define GLV_INSTANTIATE_SCORE_WIDE(DT)                                                                  \
  template cudaError_t launch_fused_wide<DT>(const ScoreArgs&, unsigned, int, const ChunkPlan&, float*, \
                                             int32_t*, ScoreConfig, cudaStream_t);

}  // namespace glv
