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

extern template cudaError_t launch_score_dt<GLV_F32>(const ScoreArgs&, dim3, int, ScoreConfig, cudaStream_t);
extern template cudaError_t launch_score_dt<GLV_BF16>(const ScoreArgs&, dim3, int, ScoreConfig, cudaStream_t);
extern template cudaError_t launch_score_dt<GLV_FP8_E4M3>(const ScoreArgs&, dim3, int, ScoreConfig, cudaStream_t);
extern template cudaError_t launch_fused_dt<GLV_F32>(const ScoreArgs&, int64_t, int, int, float*, int32_t*,
                                                     ScoreConfig, cudaStream_t);
extern template cudaError_t launch_fused_dt<GLV_BF16>(const ScoreArgs&, int64_t, int, int, float*, int32_t*,
                                                      ScoreConfig, cudaStream_t);
extern template cudaError_t launch_fused_dt<GLV_FP8_E4M3>(const ScoreArgs&, int64_t, int, int, float*, int32_t*,
                                                          ScoreConfig, cudaStream_t);

constexpr size_t kScoreSmemLimit = 227 * 1024 - 12 * 1024;  // leaves room for static shared memory

static std::mutex g_cfg_mu;
static ScoreConfig g_cfg[3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // G = 0: library default

bool set_score_config(int dt, int G, int mode, int carve_kb) {
  if (dt < 0 || dt > 2 || mode < 0 || mode > 2) return false;
  const bool ok = (G == 0) || G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32;
  if (!ok) return false;
  if (carve_kb != 0 && (carve_kb < 16 || carve_kb > 256)) return false;
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  g_cfg[dt] = {G, mode, carve_kb};
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
  return c;
}

void effective_score_config(int dt, int nch, int* G, int* mode, int* carve_kb) {
  const ScoreConfig c = resolve_config(dt, nch);
  *G = c.G;
  *mode = c.mode;
  *carve_kb = c.carve_kb;
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

cudaError_t launch_score_topk(const ScoreArgs& a0, int dt, int64_t nq, int kappa, float* out_s,
                              int32_t* out_id, int num_sms, cudaStream_t st) {
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
  int RB = 0;
  const ScoreConfig cfg = with_rings(resolve_config(dt, a.nch), a.C, a.qstride, true, a.nch, kappa, &RB);
  switch (dt) {
    case GLV_F32: return launch_fused_dt<GLV_F32>(a, nq, RB, kappa, out_s, out_id, cfg, st);
    case GLV_BF16: return launch_fused_dt<GLV_BF16>(a, nq, RB, kappa, out_s, out_id, cfg, st);
    default: return launch_fused_dt<GLV_FP8_E4M3>(a, nq, RB, kappa, out_s, out_id, cfg, st);
  }
}

}  // namespace glv
