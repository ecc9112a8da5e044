// score.cu -- host-side launchers of the gather-score of the eager GleanVec inner product
// (Algorithm 4, procedure inner-product; Eq. GleanVec approximation, Section 4):
//
//     s(j, i) = < q_{j, c_i} , x_i^low >            (times s_i for FP8 rows)
//
// and of the fused scoring + top-kappa, plus the scoring configuration table that the
// autotuner fills (lanes per candidate and row pipelining, per store type).
#include <mutex>

#include "kernels.cuh"
#include "score_launch.cuh"
#include "score_variants.cuh"

namespace glv {

// each (store type, gather mode) pair is instantiated in its own translation unit
#define GLV_EXTERN_MODES(DT)                                                                                     \
  extern template cudaError_t launch_score_mode<DT, 0>(const ScoreArgs&, dim3, int, ScoreConfig, cudaStream_t); \
  extern template cudaError_t launch_score_mode<DT, 1>(const ScoreArgs&, dim3, int, ScoreConfig, cudaStream_t); \
  extern template cudaError_t launch_score_mode<DT, 2>(const ScoreArgs&, dim3, int, ScoreConfig, cudaStream_t); \
  extern template cudaError_t launch_fused_mode<DT, 0>(const ScoreArgs&, unsigned, int, const ChunkPlan&,       \
                                                       float*, int32_t*, ScoreConfig, cudaStream_t);            \
  extern template cudaError_t launch_fused_mode<DT, 1>(const ScoreArgs&, unsigned, int, const ChunkPlan&,       \
                                                       float*, int32_t*, ScoreConfig, cudaStream_t);        \
  extern template cudaError_t launch_fused_wide<DT>(const ScoreArgs&, unsigned, int, const ChunkPlan&, float*,  \
                                                    int32_t*, ScoreConfig, cudaStream_t);
GLV_EXTERN_MODES(GLV_F32)
GLV_EXTERN_MODES(GLV_BF16)
GLV_EXTERN_MODES(GLV_FP8_E4M3)

template <int DT>
static cudaError_t launch_score_dt(const ScoreArgs& a, dim3 grid, int RB, ScoreConfig cfg, cudaStream_t st) {
  switch (cfg.mode) {
    case 1: return launch_score_mode<DT, 1>(a, grid, RB, cfg, st);
    case 2: return launch_score_mode<DT, 2>(a, grid, RB, cfg, st);
    default: return launch_score_mode<DT, 0>(a, grid, RB, cfg, st);
  }
}

template <int DT>
static cudaError_t launch_fused_dt(const ScoreArgs& a, unsigned grid, int kappa, const ChunkPlan& plan, float* out_s,
                                   int32_t* out_id, ScoreConfig cfg, cudaStream_t st) {
  if (cfg.sched & 2) return launch_fused_wide<DT>(a, grid, kappa, plan, out_s, out_id, cfg, st);
  switch (cfg.mode) {
    case 1: return launch_fused_mode<DT, 1>(a, grid, kappa, plan, out_s, out_id, cfg, st);
    default: return launch_fused_mode<DT, 0>(a, grid, kappa, plan, out_s, out_id, cfg, st);  // bulk (2) -> 0
  }
}

constexpr size_t kScoreSmemLimit = 227 * 1024 - 12 * 1024;  // leaves room for static shared memory

static std::mutex g_cfg_mu;
static ScoreConfig g_cfg[3] = {{0, 0, 0, 1}, {0, 0, 0, 1}, {0, 0, 0, 1}};  // G = 0: library default

bool set_score_config(int dt, int G, int mode, int carve_kb, int sched) {
  if (dt < 0 || dt > 2 || mode < 0 || mode > 2 || sched < 0 || sched > 7) return false;
  const bool ok = (G == 0) || G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32;
  if (!ok) return false;
  if (carve_kb != 0 && (carve_kb < 16 || carve_kb > 256)) return false;
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  g_cfg[dt] = {G, mode, carve_kb, sched};
  return true;
}

ScoreConfig get_score_config(int dt) {
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  return g_cfg[dt];
}

static int nch_of(int d, int dt) {
  const int eb = dt == GLV_F32 ? 4 : (dt == GLV_BF16 ? 2 : 1);
  return (d * eb + 15) / 16;
}

// qstride: floats per cluster row of the projected query in shared memory (qp_qstride).
static int qstride_of(int d, int dt) { return qp_qstride(nch_of(d, dt), dt); }

ScoreConfig resolve_config(int dt, int nch) {
  const ScoreConfig t = get_score_config(dt);
  ScoreConfig c;
  switch (dt) {
    case GLV_F32: c = effective_config<GLV_F32>(nch, t.G, t.mode); break;
    case GLV_BF16: c = effective_config<GLV_BF16>(nch, t.G, t.mode); break;
    default: c = effective_config<GLV_FP8_E4M3>(nch, t.G, t.mode); break;
  }
  c.carve_kb = t.carve_kb;
  c.sched = t.sched;
  // the wide fused kernel: register loads with one of the two smaller group sizes
  bool wide_ok = false;
  switch (dt) {
    case GLV_F32: wide_ok = wide_group_supported<GLV_F32>(c.G); break;
    case GLV_BF16: wide_ok = wide_group_supported<GLV_BF16>(c.G); break;
    default: wide_ok = wide_group_supported<GLV_FP8_E4M3>(c.G); break;
  }
  if ((c.sched & 2) && (!wide_ok || c.mode != 0)) c.sched &= ~2;
  return c;
}

void effective_score_config(int dt, int nch, int* G, int* mode, int* carve_kb, int* sched) {
  const ScoreConfig c = resolve_config(dt, nch);
  *G = c.G;
  *mode = c.mode;
  *carve_kb = c.carve_kb;
  *sched = c.sched;
}

// Bulk gather needs its rings in shared memory; if they do not fit, use register loads.
static ScoreConfig with_rings(ScoreConfig cfg, int C, int qstride, bool fused, int nch, int kappa, int* RB) {
  *RB = 0;
  if (cfg.mode == 2) {
    *RB = bulk_rows(C, qstride, fused, nch, kappa, kScoreSmemLimit);
    if (*RB == 0) cfg.mode = 0;
  }
  return cfg;
}

cudaError_t launch_score(const ScoreArgs& a0, int dt, int64_t nq, int num_sms, cudaStream_t st) {
  ScoreArgs a = a0;
  a.qstride = qstride_of(a.d, dt);
  a.sbs = qp_sbs(a.nch, dt);
  // enough CTAs to fill the machine a few times over even for few queries
  const int64_t want = (int64_t)num_sms * 8;
  int splits = (int)((want + nq - 1) / nq);
  if (splits < 1) splits = 1;
  if (splits > 64) splits = 64;
  a.splits = splits;
  dim3 grid((unsigned)nq, (unsigned)splits);
  int RB = 0;
  const ScoreConfig cfg = with_rings(resolve_config(dt, a.nch), a.C, a.qstride, false, a.nch, 0, &RB);
  a.prefetch = (cfg.sched & 4) ? 1 : 0;
  switch (dt) {
    case GLV_F32: return launch_score_dt<GLV_F32>(a, grid, RB, cfg, st);
    case GLV_BF16: return launch_score_dt<GLV_BF16>(a, grid, RB, cfg, st);
    default: return launch_score_dt<GLV_FP8_E4M3>(a, grid, RB, cfg, st);
  }
}

size_t fused_smem_bytes(int C, int d, int dt, int kappa) {
  const int eb = dt == GLV_F32 ? 4 : (dt == GLV_BF16 ? 2 : 1);
  return score_smem(C, qstride_of(d, dt), true, 0, 0, (d * eb + 15) / 16, kappa).total();
}


// ---- work plan of the fused kernel --------------------------------------------------------
// Workspace: [header: next item, item count | chunk_start (nq + 1) | done (nq) | items] with
// at most nq + n_cand / kChunk + 1 items.

static size_t round256(size_t b) { return (b + 255) & ~size_t(255); }
static int64_t max_items(int64_t nq, int64_t n_cand) { return nq + n_cand / kChunk + 1; }

size_t topk_plan_bytes(int64_t nq, int64_t n_cand) {
  return 256 + round256((size_t)(nq + 1) * 4) + round256((size_t)nq * 4) +
         round256((size_t)max_items(nq, n_cand) * sizeof(ItemRec));
}

ChunkPlan topk_plan_layout(void* ws, int64_t nq) {
  uint8_t* b = static_cast<uint8_t*>(ws);
  int32_t* hdr = reinterpret_cast<int32_t*>(b);
  const size_t o_cs = 256, o_done = o_cs + round256((size_t)(nq + 1) * 4), o_items = o_done + round256((size_t)nq * 4);
  return ChunkPlan{hdr, hdr + 1, reinterpret_cast<int32_t*>(b + o_cs), reinterpret_cast<int32_t*>(b + o_done),
                   reinterpret_cast<ItemRec*>(b + o_items)};
}

__host__ __device__ inline int64_t items_of_list(int64_t L) { return L >= 2 * (int64_t)kChunk ? L / kChunk : 1; }

constexpr int kPlanThreads = 1024;
constexpr int kPlanTile = 8192;  // queries per pass (their item counts sit in shared memory)

// One CTA, tiles of kPlanTile queries: the item counts of a tile are read with coalesced,
// independent loads into shared memory, scanned there (each thread a contiguous run of 8
// queries, then a scan of the per-thread sums), and turned into chunk_start, the item records
// and zeroed counters.  Records beyond the workspace's capacity are not written; if the lists
// hold more candidates than n_cand allows for, no item runs and GLV_ERR_INVALID_ARG is
// reported.
__global__ void __launch_bounds__(kPlanThreads) plan_chunks_kernel(const int64_t* __restrict__ off, int64_t nq,
                                                                   int64_t item_cap, ChunkPlan plan,
                                                                   int32_t* d_status) {
  __shared__ int32_t cnt_s[kPlanTile];
  __shared__ int64_t warp_sum_s[kPlanThreads / 32];
  __shared__ int64_t carry_s;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int per = kPlanTile / kPlanThreads;
  if (t == 0) carry_s = 0;
  __syncthreads();
  for (int64_t base = 0; base < nq; base += kPlanTile) {
    const int64_t tile = min((int64_t)kPlanTile, nq - base);
#pragma unroll 4
    for (int i = t; i < kPlanTile; i += kPlanThreads)
      cnt_s[i] = i < tile ? (int32_t)items_of_list(max((int64_t)0, off[base + i + 1] - off[base + i])) : 0;
    __syncthreads();
    int64_t run_sum = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) run_sum += cnt_s[t * per + k];
    int64_t incl = run_sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum_s[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int64_t w = warp_sum_s[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t v = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += v;
      }
      warp_sum_s[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    int64_t run = carry_s + incl - run_sum + (warp > 0 ? warp_sum_s[warp - 1] : 0);
    int64_t o[per + 1];  // this thread's offsets, loaded together
#pragma unroll
    for (int k = 0; k <= per; ++k) o[k] = t * per + k <= tile ? off[base + t * per + k] : 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
      const int i = t * per + k;
      if (i >= tile) continue;
      const int64_t q = base + i, p0 = o[k];
      const int64_t L = max((int64_t)0, o[k + 1] - p0);
      const int64_t n = cnt_s[i];
      plan.done[q] = 0;
      plan.chunk_start[q] = (int32_t)run;
      for (int64_t c = 0; c < n && run + c < item_cap; ++c) {
        ItemRec r;
        r.b0 = p0 + c * kChunk;
        r.len = (int32_t)(c + 1 < n ? (int64_t)kChunk : L - c * kChunk);
        r.q = (int32_t)q;
        r.c = (int32_t)c;
        r.nchunks = (int32_t)n;
        plan.items[run + c] = r;
      }
      run += n;
    }
    __syncthreads();
    if (t == 0) carry_s += warp_sum_s[kPlanThreads / 32 - 1];
    __syncthreads();
  }
  if (t == 0) {
    const int64_t total = carry_s;
    const bool fits = total <= item_cap;
    plan.chunk_start[nq] = (int32_t)(fits ? total : 0);
    *plan.next = 0;
    *plan.n_items = fits ? (int32_t)total : 0;
    if (!fits) report(d_status, GLV_ERR_INVALID_ARG);
  }
}

cudaError_t launch_plan_chunks(const int64_t* off, int64_t nq, int64_t n_cand, void* ws, int32_t* d_status,
                               cudaStream_t st) {
  plan_chunks_kernel<<<1, kPlanThreads, 0, st>>>(off, nq, max_items(nq, n_cand), topk_plan_layout(ws, nq), d_status);
  return cudaGetLastError();
}

cudaError_t launch_score_topk(const ScoreArgs& a0, int dt, int64_t nq, int64_t n_cand, int kappa, void* plan_ws,
                              float* out_s, int32_t* out_id, int num_sms, cudaStream_t st) {
  // Few queries: one CTA per query would leave the GPU idle, so split the lists over CTAs
  // (stand-alone scoring) and select afterwards.
  if (nq < (int64_t)num_sms * 4) {
    cudaError_t e = launch_score(a0, dt, nq, num_sms, st);
    if (e != cudaSuccess) return e;
    return launch_topk(a0.scores, a0.off, a0.ids, nq, kappa, out_s, out_id, st);
  }
  ScoreArgs a = a0;
  a.qstride = qstride_of(a.d, dt);
  a.sbs = qp_sbs(a.nch, dt);
  a.splits = 1;
  ScoreConfig cfg = resolve_config(dt, a.nch);
  // wide CTAs keep twice the keys on chip; where that does not fit, the 256-thread kernel runs
  if ((cfg.sched & 2) &&
      score_smem(a.C, a.qstride, true, 0, 0, a.nch, kappa, fused_cache(kWideThreads)).total() > kScoreSmemLimit)
    cfg.sched &= ~2;
  a.prefetch = (cfg.sched & 4) ? 1 : 0;
  const ChunkPlan plan = topk_plan_layout(plan_ws, nq);
  unsigned grid = (unsigned)nq;  // one CTA per query
  if (cfg.sched & 1) {
    cudaError_t e = launch_plan_chunks(a.off, nq, n_cand, plan_ws, a.d_status, st);
    if (e != cudaSuccess) return e;
    // persistent CTAs claim items dynamically: as many as the SM's thread slots allow (2048
    // threads) covers any occupancy, the extra ones find no item left and exit
    const int64_t items = max_items(nq, n_cand);
    const int64_t per_sm = (cfg.sched & 2) ? 2048 / kWideThreads : 2048 / kScoreThreads;
    grid = (unsigned)(items < (int64_t)num_sms * per_sm ? items : (int64_t)num_sms * per_sm);
  }
  switch (dt) {
    case GLV_F32: return launch_fused_dt<GLV_F32>(a, grid, kappa, plan, out_s, out_id, cfg, st);
    case GLV_BF16: return launch_fused_dt<GLV_BF16>(a, grid, kappa, plan, out_s, out_id, cfg, st);
    default: return launch_fused_dt<GLV_FP8_E4M3>(a, grid, kappa, plan, out_s, out_id, cfg, st);
  }
}

}  // namespace glv
