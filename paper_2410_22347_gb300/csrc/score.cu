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

namespace glv {

template <int DT>
cudaError_t launch_score_dt(const ScoreArgs& a, dim3 grid, size_t smem, ScoreConfig cfg, cudaStream_t st);
template <int DT>
cudaError_t launch_fused_dt(const ScoreArgs& a, int64_t nq, size_t smem, int kappa, float* out_s,
                            int32_t* out_id, ScoreConfig cfg, cudaStream_t st);

static std::mutex g_cfg_mu;
static ScoreConfig g_cfg[3] = {{0, false}, {0, false}, {0, false}};  // 0 = library default

bool set_score_config(int dt, int G, bool pipe) {
  if (dt < 0 || dt > 2) return false;
  const bool ok = (G == 0) || G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32;
  if (!ok) return false;
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  g_cfg[dt] = {G, pipe};
  return true;
}

ScoreConfig get_score_config(int dt) {
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  return g_cfg[dt];
}

static int epc_of(int dt) { return 16 / (dt == GLV_F32 ? 4 : (dt == GLV_BF16 ? 2 : 1)); }

// qstride: floats per cluster row in shared memory; +4 (16 bytes) so consecutive cluster
// rows start in different banks.
static int qstride_of(int d, int dt) {
  const int epc = epc_of(dt);
  return (d + epc - 1) / epc * epc + 4;
}

ScoreConfig resolve_config(int dt, int nch) {
  const ScoreConfig t = get_score_config(dt);
  switch (dt) {
    case GLV_F32: return effective_config<GLV_F32>(nch, t.G, t.pipe);
    case GLV_BF16: return effective_config<GLV_BF16>(nch, t.G, t.pipe);
    default: return effective_config<GLV_FP8_E4M3>(nch, t.G, t.pipe);
  }
}

void effective_score_config(int dt, int nch, int* G, int* pipe) {
  const ScoreConfig c = resolve_config(dt, nch);
  *G = c.G;
  *pipe = c.pipe ? 1 : 0;
}

cudaError_t launch_score(const ScoreArgs& a0, int dt, int64_t nq, int num_sms, cudaStream_t st) {
  ScoreArgs a = a0;
  a.qstride = qstride_of(a.d, dt);
  const size_t smem = (size_t)a.C * a.qstride * sizeof(float);
  // enough CTAs to fill the machine a few times over even for few queries
  const int64_t want = (int64_t)num_sms * 8;
  int splits = (int)((want + nq - 1) / nq);
  if (splits < 1) splits = 1;
  if (splits > 64) splits = 64;
  a.splits = splits;
  dim3 grid((unsigned)nq, (unsigned)splits);
  const ScoreConfig cfg = resolve_config(dt, a.nch);
  switch (dt) {
    case GLV_F32: return launch_score_dt<GLV_F32>(a, grid, smem, cfg, st);
    case GLV_BF16: return launch_score_dt<GLV_BF16>(a, grid, smem, cfg, st);
    default: return launch_score_dt<GLV_FP8_E4M3>(a, grid, smem, cfg, st);
  }
}

size_t fused_smem_bytes(int C, int d, int dt) {
  return (size_t)C * qstride_of(d, dt) * sizeof(float) + (size_t)2048 * sizeof(uint32_t);
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
  a.splits = 1;
  const size_t smem = fused_smem_bytes(a.C, a.d, dt);
  const ScoreConfig cfg = resolve_config(dt, a.nch);
  switch (dt) {
    case GLV_F32: return launch_fused_dt<GLV_F32>(a, nq, smem, kappa, out_s, out_id, cfg, st);
    case GLV_BF16: return launch_fused_dt<GLV_BF16>(a, nq, smem, kappa, out_s, out_id, cfg, st);
    default: return launch_fused_dt<GLV_FP8_E4M3>(a, nq, smem, kappa, out_s, out_id, cfg, st);
  }
}

}  // namespace glv
