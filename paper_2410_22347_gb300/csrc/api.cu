// api.cu -- the extern "C" entry points declared in include/glv.h: host-side validation
// (before anything is enqueued) and dispatch to the kernels.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.cuh"

namespace glv {

constexpr size_t kSmemLimit = 227 * 1024;  // opt-in dynamic shared memory per CTA (sm_100+)
constexpr int64_t kMaxGridX = 2147483647;

static int num_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  return n;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }
static int elem_bytes(int dt) { return dt == GLV_F32 ? 4 : (dt == GLV_BF16 ? 2 : 1); }
static bool valid_dt(int dt) { return dt == GLV_F32 || dt == GLV_BF16 || dt == GLV_FP8_E4M3; }

}  // namespace glv

using namespace glv;

namespace {
#define GLV_CHECK(cond, code) \
  do {                        \
    if (!(cond)) return code; \
  } while (0)
static glv_status fill_score_args(ScoreArgs& a, const float* Qp, int64_t nq, int32_t C, int32_t d,
                                  const void* Xred, int64_t row_stride, const float* scales, glv_dtype dt,
                                  const uint16_t* tags, int64_t N, const int64_t* cand_off,
                                  const int32_t* cand_ids, float* scores, int32_t* d_status) {
  GLV_CHECK(nq >= 0 && C >= 1 && C <= 65536 && d >= 1 && N >= 0 && valid_dt(dt), GLV_ERR_INVALID_ARG);
  GLV_CHECK(row_stride >= glv_min_row_stride(d, dt) && row_stride % 16 == 0, GLV_ERR_INVALID_ARG);
  GLV_CHECK((dt == GLV_FP8_E4M3) == (scales != nullptr), GLV_ERR_INVALID_ARG);
  if (nq == 0) return GLV_OK;
  GLV_CHECK(Qp && cand_off && tags && Xred && cand_ids && scores, GLV_ERR_INVALID_ARG);
  GLV_CHECK(aligned(Xred, 16), GLV_ERR_INVALID_ARG);
  GLV_CHECK(nq <= kMaxGridX, GLV_ERR_UNSUPPORTED);
  const int eb = elem_bytes(dt);
  const int64_t bytes = (int64_t)d * eb;
  const int nch = (int)((bytes + 15) / 16);
  GLV_CHECK(nch <= 32 * 10, GLV_ERR_UNSUPPORTED);
  GLV_CHECK((size_t)C * qp_qstride(nch, dt) * 4 <= kSmemLimit, GLV_ERR_UNSUPPORTED);
  a.Qp = Qp;
  a.C = C;
  a.d = d;
  a.qstride = 0;
  a.Xred = static_cast<const uint8_t*>(Xred);
  a.row_stride = row_stride;
  a.scales = scales;
  a.tags = tags;
  a.N = N;
  a.off = cand_off;
  a.ids = cand_ids;
  a.scores = scores;
  a.d_status = d_status;
  a.nch = nch;
  a.tail = (int)(bytes - (int64_t)(nch - 1) * 16);
  a.splits = 1;
  a.sbs = nch;
  a.prefetch = 0;
  return GLV_OK;
}

}  // namespace

// While a composite call (glv_search, glv_search_host) validates the calls it is made of, the
// entry points run their argument checks and return before their first launch: every check
// of every step passes before anything is enqueued.
static thread_local bool g_checks_only = false;

struct ChecksOnly {
  ChecksOnly() { g_checks_only = true; }
  ~ChecksOnly() { g_checks_only = false; }
};

#define GLV_LAUNCH(expr)                            \
  do {                                              \
    if (g_checks_only) return GLV_OK;               \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return GLV_ERR_CUDA;     \
  } while (0)

extern "C" {

int32_t glv_abi_version(void) { return GLV_ABI_VERSION; }

const char* glv_status_string(glv_status s) {
  switch (s) {
    case GLV_OK: return "ok";
    case GLV_ERR_INVALID_ARG: return "invalid argument";
    case GLV_ERR_BAD_ID: return "id or tag out of range";
    case GLV_ERR_UNSUPPORTED: return "unsupported shape";
    case GLV_ERR_CUDA: return "CUDA error";
    case GLV_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

glv_status glv_last_device_status(const int32_t* d_status, void* stream) {
  GLV_CHECK(d_status != nullptr, GLV_ERR_INVALID_ARG);
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GLV_ERR_CUDA;
  int32_t v = 0;
  if (cudaMemcpy(&v, d_status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return GLV_ERR_CUDA;
  return (glv_status)v;
}

int64_t glv_min_row_stride(int32_t d, glv_dtype dt) {
  if (d <= 0 || !valid_dt(dt)) return -1;
  return ((int64_t)d * elem_bytes(dt) + 15) / 16 * 16;
}

glv_status glv_assign_tags(const float* X, int64_t N, int32_t D, const float* mu, int32_t C,
                           uint16_t* tags, float* best_ip, void* stream) {
  GLV_CHECK(N >= 0 && D >= 1 && C >= 1 && C <= 65536, GLV_ERR_INVALID_ARG);
  if (N == 0) return GLV_OK;
  GLV_CHECK(X && mu && tags, GLV_ERR_INVALID_ARG);
  GLV_CHECK(D <= 1024, GLV_ERR_UNSUPPORTED);
  GLV_LAUNCH(launch_tags(X, N, D, mu, C, tags, best_ip, num_sms(), (cudaStream_t)stream));
  return GLV_OK;
}

size_t glv_build_reduced_workspace_size(int64_t N, int32_t C) {
  if (N < 0 || C < 1) return 0;
  return build_ws_bytes(N, C);
}

glv_status glv_build_reduced(const float* X, int64_t N, int32_t D, const uint16_t* tags,
                             const float* B, int32_t C, int32_t d, glv_dtype dt, void* Xred,
                             int64_t row_stride, float* scales, void* workspace,
                             int32_t* d_status, void* stream) {
  GLV_CHECK(N >= 0 && N <= 2147483647LL, GLV_ERR_INVALID_ARG);
  GLV_CHECK(D >= 1 && C >= 1 && C <= 65536 && d >= 1 && d <= D && valid_dt(dt),
            GLV_ERR_INVALID_ARG);
  GLV_CHECK(row_stride >= glv_min_row_stride(d, dt) && row_stride % 16 == 0, GLV_ERR_INVALID_ARG);
  GLV_CHECK((dt == GLV_FP8_E4M3) == (scales != nullptr), GLV_ERR_INVALID_ARG);
  if (N == 0) return GLV_OK;
  GLV_CHECK(X && tags && B && Xred && workspace, GLV_ERR_INVALID_ARG);
  GLV_CHECK(aligned(Xred, 16) && aligned(workspace, 256), GLV_ERR_INVALID_ARG);
  GLV_CHECK((size_t)32 * ((d + 3) & ~3) * 4 <= kSmemLimit - 16 * 1024, GLV_ERR_UNSUPPORTED);
  GLV_CHECK((N + 31) / 32 + C <= kMaxGridX, GLV_ERR_UNSUPPORTED);
  GLV_LAUNCH(launch_build(X, N, D, tags, B, C, d, dt, Xred, row_stride, scales, workspace,
                          d_status, (cudaStream_t)stream));
  return GLV_OK;
}

size_t glv_project_queries_workspace_size(int64_t nq, int32_t D, int32_t C, int32_t d,
                                          glv_dtype compute) {
  if (nq < 0 || D < 1 || C < 1 || d < 1 || (compute != GLV_F32 && compute != GLV_BF16)) return 0;
  return project_tc_ws_bytes(nq, D, (int64_t)C * d, compute == GLV_BF16);
}

glv_status glv_project_queries(const float* Q, int64_t nq, int32_t D, const float* A,
                               int32_t C, int32_t d, glv_dtype compute, float* Qp,
                               void* workspace, int32_t* d_status, void* stream) {
  GLV_CHECK(nq >= 0 && D >= 1 && C >= 1 && C <= 65536 && d >= 1 && d <= D, GLV_ERR_INVALID_ARG);
  GLV_CHECK(compute == GLV_F32 || compute == GLV_BF16, GLV_ERR_INVALID_ARG);
  GLV_CHECK(compute == GLV_F32 || workspace != nullptr, GLV_ERR_INVALID_ARG);
  GLV_CHECK(workspace == nullptr || aligned(workspace, 256), GLV_ERR_INVALID_ARG);
  if (nq == 0) return GLV_OK;
  GLV_CHECK(Q && A && Qp, GLV_ERR_INVALID_ARG);
  const int64_t M = (int64_t)C * d;
  GLV_CHECK(M <= 2147483647LL && nq <= 2147483647LL, GLV_ERR_UNSUPPORTED);
  if (workspace == nullptr) {  // exact FP32 FMA path (no workspace needed)
    GLV_CHECK(nq <= 65535LL * 128, GLV_ERR_UNSUPPORTED);
    GLV_LAUNCH(launch_project_simt(Q, nq, D, A, M, Qp, (cudaStream_t)stream));
    return GLV_OK;
  }
  GLV_LAUNCH(launch_project_tc(Q, nq, D, A, M, Qp, compute == GLV_BF16, workspace, d_status, num_sms(),
                               (cudaStream_t)stream));
  return GLV_OK;
}

glv_status glv_score_candidates(const float* Qp, int64_t nq, int32_t C, int32_t d,
                                const void* Xred, int64_t row_stride, const float* scales,
                                glv_dtype dt, const uint16_t* tags, int64_t N,
                                const int64_t* cand_off, const int32_t* cand_ids,
                                float* scores, int32_t* d_status, void* stream) {
  ScoreArgs a;
  const glv_status st = fill_score_args(a, Qp, nq, C, d, Xred, row_stride, scales, dt, tags, N, cand_off,
                                        cand_ids, scores, d_status);
  if (st != GLV_OK || nq == 0) return st;
  GLV_LAUNCH(launch_score(a, dt, nq, num_sms(), (cudaStream_t)stream));
  return GLV_OK;
}

size_t glv_score_topk_workspace_size(int64_t nq, int64_t n_candidates) {
  if (nq < 0 || n_candidates < 0) return 0;
  return topk_plan_bytes(nq, n_candidates);
}

glv_status glv_score_topk(const float* Qp, int64_t nq, int32_t C, int32_t d, const void* Xred,
                          int64_t row_stride, const float* scales, glv_dtype dt,
                          const uint16_t* tags, int64_t N, const int64_t* cand_off,
                          const int32_t* cand_ids, int64_t n_candidates, int32_t kappa, float* scores_scratch,
                          void* workspace, float* out_s, int32_t* out_id, int32_t* d_status, void* stream) {
  GLV_CHECK(kappa >= 1 && kappa <= GLV_MAX_KAPPA && n_candidates >= 0, GLV_ERR_INVALID_ARG);
  GLV_CHECK(nq + n_candidates / kChunk + 1 <= 2147483647LL, GLV_ERR_UNSUPPORTED);
  ScoreArgs a;
  const glv_status st = fill_score_args(a, Qp, nq, C, d, Xred, row_stride, scales, dt, tags, N, cand_off,
                                        cand_ids, scores_scratch, d_status);
  if (st != GLV_OK || nq == 0) return st;
  GLV_CHECK(out_s && out_id && workspace && aligned(workspace, 256), GLV_ERR_INVALID_ARG);
  GLV_CHECK(fused_smem_bytes(C, d, dt, kappa) <= kSmemLimit - 12 * 1024, GLV_ERR_UNSUPPORTED);  // + static TopkSmem
  GLV_LAUNCH(launch_score_topk(a, dt, nq, n_candidates, kappa, workspace, out_s, out_id, num_sms(),
                               (cudaStream_t)stream));
  return GLV_OK;
}

glv_status glv_score_lazy(const float* Q, int64_t nq, int32_t D, const float* A, int32_t C, int32_t d,
                          const void* Xred, int64_t row_stride, const float* scales, glv_dtype dt,
                          const uint16_t* tags, int64_t N, const int64_t* cand_off, const int32_t* cand_ids,
                          float* scores, int32_t* visited, int32_t* d_status, void* stream) {
  GLV_CHECK(D >= 1 && d <= D, GLV_ERR_INVALID_ARG);
  ScoreArgs a;
  const glv_status st = fill_score_args(a, Q /* placeholder, Qp unused */, nq, C, d, Xred, row_stride, scales, dt,
                                        tags, N, cand_off, cand_ids, scores, d_status);
  if (st != GLV_OK || nq == 0) return st;
  GLV_CHECK(Q && A, GLV_ERR_INVALID_ARG);
  GLV_CHECK(lazy_smem_bytes(C, d, D, dt) <= kSmemLimit, GLV_ERR_UNSUPPORTED);
  a.Qp = nullptr;
  GLV_LAUNCH(launch_score_lazy(a, dt, nq, Q, D, A, visited, (cudaStream_t)stream));
  return GLV_OK;
}

glv_status glv_set_score_config(glv_dtype dt, int32_t lanes_per_candidate, int32_t gather_mode,
                                int32_t smem_carveout_kb, int32_t schedule) {
  GLV_CHECK(valid_dt(dt), GLV_ERR_INVALID_ARG);
  GLV_CHECK(set_score_config(dt, lanes_per_candidate, gather_mode, smem_carveout_kb, schedule), GLV_ERR_INVALID_ARG);
  return GLV_OK;
}

glv_status glv_get_score_config(glv_dtype dt, int32_t d, int32_t* lanes_per_candidate, int32_t* gather_mode,
                                int32_t* smem_carveout_kb, int32_t* schedule) {
  GLV_CHECK(valid_dt(dt) && d >= 1 && lanes_per_candidate && gather_mode && smem_carveout_kb && schedule,
            GLV_ERR_INVALID_ARG);
  const int nch = (int)(((int64_t)d * elem_bytes(dt) + 15) / 16);
  int G = 0, mode = 0, carve = 0, sched = 1;
  effective_score_config(dt, nch, &G, &mode, &carve, &sched);
  *lanes_per_candidate = G;
  *gather_mode = mode;
  *smem_carveout_kb = carve;
  *schedule = sched;
  return GLV_OK;
}

glv_status glv_topk(const float* scores, const int64_t* cand_off, const int32_t* cand_ids,
                    int64_t nq, int32_t kappa, float* out_s, int32_t* out_id, void* stream) {
  GLV_CHECK(nq >= 0 && kappa >= 1 && kappa <= GLV_MAX_KAPPA, GLV_ERR_INVALID_ARG);
  if (nq == 0) return GLV_OK;
  GLV_CHECK(scores && cand_off && cand_ids && out_s && out_id, GLV_ERR_INVALID_ARG);
  GLV_CHECK(nq <= kMaxGridX, GLV_ERR_UNSUPPORTED);
  GLV_LAUNCH(launch_topk(scores, cand_off, cand_ids, nq, kappa, out_s, out_id,
                         (cudaStream_t)stream));
  return GLV_OK;
}

glv_status glv_rerank(const float* X, int64_t N, int32_t D, const float* Q, int64_t nq,
                      const int32_t* surv_id, int32_t kappa, int32_t k, float* out_s,
                      int32_t* out_id, int32_t* d_status, void* stream) {
  GLV_CHECK(N >= 0 && D >= 1 && nq >= 0, GLV_ERR_INVALID_ARG);
  GLV_CHECK(kappa >= 1 && kappa <= GLV_MAX_KAPPA && k >= 1 && k <= kappa, GLV_ERR_INVALID_ARG);
  if (nq == 0) return GLV_OK;
  GLV_CHECK(Q && surv_id && out_s && out_id && (X || N == 0), GLV_ERR_INVALID_ARG);
  GLV_CHECK(nq <= kMaxGridX, GLV_ERR_UNSUPPORTED);
  GLV_CHECK(rerank_smem_bytes(D, kappa) <= kSmemLimit, GLV_ERR_UNSUPPORTED);
  RerankArgs a;
  a.X = X;
  a.N = N;
  a.D = D;
  a.Q = Q;
  a.surv = surv_id;
  a.kappa = kappa;
  a.k = k;
  a.out_s = out_s;
  a.out_id = out_id;
  a.d_status = d_status;
  const bool vec = (D % 4 == 0) && aligned(X, 16) && aligned(Q, 16);
  GLV_LAUNCH(launch_rerank(a, nq, vec, (cudaStream_t)stream));
  return GLV_OK;
}

size_t glv_second_moments_workspace_size(int64_t n, int32_t C) {
  if (n < 0 || C < 1) return 0;
  return moments_ws_bytes(n, C);
}

glv_status glv_second_moments(const float* V, int64_t n, int32_t D, const uint16_t* tags, int32_t C, double* K,
                              void* workspace, int32_t* d_status, void* stream) {
  GLV_CHECK(n >= 0 && n <= 2147483647LL && D >= 1 && C >= 1 && C <= 65535, GLV_ERR_INVALID_ARG);
  GLV_CHECK(tags != nullptr || C == 1, GLV_ERR_INVALID_ARG);
  GLV_CHECK(V || n == 0, GLV_ERR_INVALID_ARG);
  GLV_CHECK(K != nullptr, GLV_ERR_INVALID_ARG);
  GLV_CHECK(tags == nullptr || (workspace && aligned(workspace, 256)), GLV_ERR_INVALID_ARG);
  const int nt = (D + 63) / 64;
  GLV_CHECK((int64_t)nt * (nt + 1) / 2 <= kMaxGridX, GLV_ERR_UNSUPPORTED);
  GLV_LAUNCH(launch_moments(V, n, D, tags, C, K, workspace, d_status, (cudaStream_t)stream));
  return GLV_OK;
}

size_t glv_pair_workspace_size(int64_t P, int32_t C) {
  if (P < 0 || C < 1) return 0;
  return pair_ws_bytes(P, C);
}

glv_status glv_pair_forward(const float* Q, int64_t nQ, const float* X, int64_t nX, int32_t D,
                            const uint16_t* tags, const float* A, const float* B, int32_t C, int32_t d,
                            const int32_t* qi, const int32_t* xi, int64_t P, float* s, float* t, float* u,
                            float* v, void* workspace, int32_t* d_status, void* stream) {
  GLV_CHECK(nQ >= 0 && nX >= 0 && D >= 1 && C >= 1 && C <= 65535 && d >= 1 && d <= D && P >= 0,
            GLV_ERR_INVALID_ARG);
  GLV_CHECK(P <= 2147483647LL, GLV_ERR_UNSUPPORTED);
  if (P == 0) return GLV_OK;
  GLV_CHECK(Q && X && tags && A && B && qi && xi && s && t && u && v && workspace, GLV_ERR_INVALID_ARG);
  GLV_CHECK(aligned(workspace, 256), GLV_ERR_INVALID_ARG);
  GLV_LAUNCH(launch_pair_forward(Q, nQ, X, nX, D, tags, A, B, C, d, qi, xi, P, s, t, u, v, workspace, d_status,
                                 (cudaStream_t)stream));
  return GLV_OK;
}

glv_status glv_pair_backward(const float* Q, int64_t nQ, const float* X, int64_t nX, int32_t D,
                             const uint16_t* tags, int32_t C, int32_t d, const int32_t* qi, const int32_t* xi,
                             int64_t P, const float* u, const float* v, const float* g, float* dA, float* dB,
                             void* workspace, int32_t* d_status, void* stream) {
  GLV_CHECK(nQ >= 0 && nX >= 0 && D >= 1 && C >= 1 && C <= 65535 && d >= 1 && d <= D && P >= 0,
            GLV_ERR_INVALID_ARG);
  GLV_CHECK(P <= 2147483647LL, GLV_ERR_UNSUPPORTED);
  GLV_CHECK(dA && dB, GLV_ERR_INVALID_ARG);
  GLV_CHECK(P == 0 || (Q && X && tags && qi && xi && u && v && g && workspace && aligned(workspace, 256)),
            GLV_ERR_INVALID_ARG);
  if (P == 0) {  // no pairs: zero gradient
    GLV_LAUNCH(cudaMemsetAsync(dA, 0, sizeof(float) * (size_t)C * d * D, (cudaStream_t)stream));
    GLV_LAUNCH(cudaMemsetAsync(dB, 0, sizeof(float) * (size_t)C * d * D, (cudaStream_t)stream));
    return GLV_OK;
  }
  GLV_LAUNCH(launch_pair_backward(Q, nQ, X, nX, D, tags, C, d, qi, xi, P, u, v, g, dA, dB, workspace, d_status,
                                  (cudaStream_t)stream));
  return GLV_OK;
}

glv_status glv_check_bounded_wait(uint32_t limit_us, int32_t* d_status, void* stream) {
  GLV_CHECK(d_status != nullptr && limit_us >= 1 && limit_us <= 1000000, GLV_ERR_INVALID_ARG);
  GLV_LAUNCH(launch_bounded_wait((uint64_t)limit_us * 1000, d_status, (cudaStream_t)stream));
  return GLV_OK;
}

glv_status glv_pair_loss(const float* s, const float* t, int64_t P, const double* weight, double* loss, float* g,
                         void* stream) {
  GLV_CHECK(P >= 0, GLV_ERR_INVALID_ARG);
  GLV_CHECK(loss || g, GLV_ERR_INVALID_ARG);
  GLV_CHECK(P == 0 || (s && t), GLV_ERR_INVALID_ARG);
  GLV_CHECK(aligned(loss, 8), GLV_ERR_INVALID_ARG);
  GLV_LAUNCH(launch_pair_loss(s, t, P, weight, loss, g, (cudaStream_t)stream));
  return GLV_OK;
}

glv_status glv_adam_step(float* param, const float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                         float beta2, float eps, int32_t step, void* stream) {
  GLV_CHECK(n >= 0 && step >= 1, GLV_ERR_INVALID_ARG);
  GLV_CHECK(lr >= 0.f && beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f,
            GLV_ERR_INVALID_ARG);
  if (n == 0) return GLV_OK;
  GLV_CHECK(param && grad && m && v, GLV_ERR_INVALID_ARG);
  GLV_LAUNCH(launch_adam(param, grad, m, v, n, lr, beta1, beta2, eps, step, num_sms(), (cudaStream_t)stream));
  return GLV_OK;
}

size_t glv_kmeans_workspace_size(int64_t N, int32_t D, int32_t C) {
  if (N < 0 || D < 1 || C < 1) return 0;
  return kmeans_ws_bytes(N, C, D);
}

glv_status glv_kmeans_update(const float* X, int64_t N, int32_t D, const uint16_t* tags, int32_t C, float* mu,
                             int32_t* counts, void* workspace, int32_t* d_status, void* stream) {
  GLV_CHECK(N >= 0 && N <= 2147483647LL && D >= 1 && C >= 1 && C <= 65535, GLV_ERR_INVALID_ARG);
  GLV_CHECK(mu && (N == 0 || (X && tags)) && workspace && aligned(workspace, 256), GLV_ERR_INVALID_ARG);
  GLV_LAUNCH(launch_kmeans_update(X, N, D, tags, C, mu, counts, workspace, d_status, (cudaStream_t)stream));
  return GLV_OK;
}

}  // extern "C"

glv_status glv_gather_rows(const void* rows, int64_t row_bytes, int64_t n_rows, const int32_t* ids, int64_t n_ids,
                           float* out, int32_t* d_status, void* stream) {
  GLV_CHECK(row_bytes >= 16 && row_bytes % 16 == 0 && n_rows >= 0 && n_ids >= 0, GLV_ERR_INVALID_ARG);
  GLV_CHECK(row_bytes <= 1024, GLV_ERR_UNSUPPORTED);
  if (n_ids == 0) return GLV_OK;
  GLV_CHECK(rows && ids && out && aligned(rows, 16), GLV_ERR_INVALID_ARG);
  GLV_LAUNCH(launch_gather_rows(rows, row_bytes, n_rows, ids, n_ids, out, d_status, num_sms(),
                                (cudaStream_t)stream));
  return GLV_OK;
}

// ---- one-call search: projection -> fused score + top-kappa -> re-rank ---------------------

static size_t round_up256(size_t b) { return (b + 255) & ~size_t(255); }

size_t glv_search_workspace_size(int64_t nq, int32_t D, int32_t C, int32_t d, glv_dtype compute,
                                 int64_t n_candidates, int32_t kappa) {
  if (nq < 0 || D < 1 || C < 1 || d < 1 || n_candidates < 0 || kappa < 0) return 0;
  size_t b = round_up256((size_t)nq * C * d * sizeof(float));                       // Qp
  b += round_up256(glv_project_queries_workspace_size(nq, D, C, d, compute));        // operands
  b += round_up256((size_t)(n_candidates > 0 ? n_candidates : 1) * sizeof(float));  // scratch
  b += round_up256(glv_score_topk_workspace_size(nq, n_candidates));                 // plan
  if (kappa > 0) b += round_up256((size_t)nq * kappa * 8);                           // survivors
  return b;
}

static glv_status search_steps(const float* X, int64_t N, int32_t D, const float* Q, int64_t nq, const float* A,
                               int32_t C, int32_t d, glv_dtype compute, const void* Xred, int64_t row_stride,
                               const float* scales, glv_dtype dt, const uint16_t* tags, const int64_t* cand_off,
                               const int32_t* cand_ids, int64_t n_candidates, int32_t kappa, int32_t k,
                               void* workspace, float* out_s, int32_t* out_id, int32_t* d_status, void* stream);

glv_status glv_search(const float* X, int64_t N, int32_t D, const float* Q, int64_t nq, const float* A,
                      int32_t C, int32_t d, glv_dtype compute, const void* Xred, int64_t row_stride,
                      const float* scales, glv_dtype dt, const uint16_t* tags, const int64_t* cand_off,
                      const int32_t* cand_ids, int64_t n_candidates, int32_t kappa, int32_t k, void* workspace,
                      float* out_s, int32_t* out_id, int32_t* d_status, void* stream) {
  {
    ChecksOnly guard;
    const glv_status st = search_steps(X, N, D, Q, nq, A, C, d, compute, Xred, row_stride, scales, dt, tags,
                                       cand_off, cand_ids, n_candidates, kappa, k, workspace, out_s, out_id,
                                       d_status, stream);
    if (st != GLV_OK) return st;
  }
  return search_steps(X, N, D, Q, nq, A, C, d, compute, Xred, row_stride, scales, dt, tags, cand_off, cand_ids,
                      n_candidates, kappa, k, workspace, out_s, out_id, d_status, stream);
}

size_t glv_search_host_workspace_size(int64_t nq, int32_t D, int32_t C, int32_t d, glv_dtype compute,
                                      int64_t n_candidates, int32_t kappa, int32_t k) {
  if (nq < 0 || D < 1 || k < 1 || n_candidates < 0) return 0;
  size_t b = round_up256((size_t)nq * D * sizeof(float));                              // queries
  b += round_up256((size_t)(nq + 1) * sizeof(int64_t));                                // list offsets
  b += round_up256((size_t)(n_candidates > 0 ? n_candidates : 1) * sizeof(int32_t));  // candidate ids
  b += round_up256((size_t)nq * k * 8);                                                // top k
  return b + glv_search_workspace_size(nq, D, C, d, compute, n_candidates, kappa);
}

glv_status glv_search_host(const float* X, int64_t N, int32_t D, const float* Q_host, int64_t nq,
                           const float* A, int32_t C, int32_t d, glv_dtype compute, const void* Xred,
                           int64_t row_stride, const float* scales, glv_dtype dt, const uint16_t* tags,
                           const int64_t* cand_off_host, const int32_t* cand_ids_host, int64_t n_candidates,
                           int32_t kappa, int32_t k, void* workspace, float* out_s_host, int32_t* out_id_host,
                           int32_t* d_status, void* stream) {
  GLV_CHECK(nq >= 0 && D >= 1 && k >= 1 && n_candidates >= 0, GLV_ERR_INVALID_ARG);
  if (nq == 0) return GLV_OK;
  GLV_CHECK(Q_host && cand_off_host && out_s_host && out_id_host && (cand_ids_host || n_candidates == 0),
            GLV_ERR_INVALID_ARG);
  GLV_CHECK(workspace && aligned(workspace, 256), GLV_ERR_INVALID_ARG);
  uint8_t* w = static_cast<uint8_t*>(workspace);
  float* Qd = reinterpret_cast<float*>(w);
  w += round_up256((size_t)nq * D * sizeof(float));
  int64_t* offd = reinterpret_cast<int64_t*>(w);
  w += round_up256((size_t)(nq + 1) * sizeof(int64_t));
  int32_t* idsd = reinterpret_cast<int32_t*>(w);
  w += round_up256((size_t)(n_candidates > 0 ? n_candidates : 1) * sizeof(int32_t));
  float* sd = reinterpret_cast<float*>(w);
  int32_t* idd = reinterpret_cast<int32_t*>(w + (size_t)nq * k * sizeof(float));
  w += round_up256((size_t)nq * k * 8);
  {
    ChecksOnly guard;
    const glv_status st = search_steps(X, N, D, Qd, nq, A, C, d, compute, Xred, row_stride, scales, dt, tags, offd,
                                       idsd, n_candidates, kappa, k, w, sd, idd, d_status, stream);
    if (st != GLV_OK) return st;
  }
  const cudaStream_t cs = (cudaStream_t)stream;
  GLV_LAUNCH(cudaMemcpyAsync(Qd, Q_host, (size_t)nq * D * sizeof(float), cudaMemcpyHostToDevice, cs));
  GLV_LAUNCH(cudaMemcpyAsync(offd, cand_off_host, (size_t)(nq + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, cs));
  if (n_candidates > 0)
    GLV_LAUNCH(cudaMemcpyAsync(idsd, cand_ids_host, (size_t)n_candidates * sizeof(int32_t),
                               cudaMemcpyHostToDevice, cs));
  const glv_status st = search_steps(X, N, D, Qd, nq, A, C, d, compute, Xred, row_stride, scales, dt, tags, offd,
                                     idsd, n_candidates, kappa, k, w, sd, idd, d_status, stream);
  if (st != GLV_OK) return st;
  GLV_LAUNCH(cudaMemcpyAsync(out_s_host, sd, (size_t)nq * k * sizeof(float), cudaMemcpyDeviceToHost, cs));
  GLV_LAUNCH(cudaMemcpyAsync(out_id_host, idd, (size_t)nq * k * sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
  return GLV_OK;
}

static glv_status search_steps(const float* X, int64_t N, int32_t D, const float* Q, int64_t nq, const float* A,
                               int32_t C, int32_t d, glv_dtype compute, const void* Xred, int64_t row_stride,
                               const float* scales, glv_dtype dt, const uint16_t* tags, const int64_t* cand_off,
                               const int32_t* cand_ids, int64_t n_candidates, int32_t kappa, int32_t k,
                               void* workspace, float* out_s, int32_t* out_id, int32_t* d_status, void* stream) {
  GLV_CHECK(nq >= 0 && k >= 1 && kappa >= 0 && (kappa == 0 || kappa >= k), GLV_ERR_INVALID_ARG);
  GLV_CHECK(k <= GLV_MAX_KAPPA && kappa <= GLV_MAX_KAPPA && n_candidates >= 0, GLV_ERR_INVALID_ARG);
  GLV_CHECK(compute == GLV_F32 || compute == GLV_BF16, GLV_ERR_INVALID_ARG);
  if (nq == 0) return GLV_OK;
  GLV_CHECK(workspace && aligned(workspace, 256) && out_s && out_id, GLV_ERR_INVALID_ARG);
  uint8_t* w = static_cast<uint8_t*>(workspace);
  float* Qp = reinterpret_cast<float*>(w);
  w += round_up256((size_t)nq * C * d * sizeof(float));
  const size_t pws_bytes = glv_project_queries_workspace_size(nq, D, C, d, compute);
  void* pws = pws_bytes ? static_cast<void*>(w) : nullptr;
  w += round_up256(pws_bytes);
  float* scratch = reinterpret_cast<float*>(w);
  w += round_up256((size_t)(n_candidates > 0 ? n_candidates : 1) * sizeof(float));
  void* tws = w;
  w += round_up256(glv_score_topk_workspace_size(nq, n_candidates));
  glv_status st = glv_project_queries(Q, nq, D, A, C, d, compute, Qp, pws, d_status, stream);
  if (st != GLV_OK) return st;
  if (kappa == 0)  // no re-rank: the top k of the reduced scores
    return glv_score_topk(Qp, nq, C, d, Xred, row_stride, scales, dt, tags, N, cand_off, cand_ids, n_candidates, k,
                          scratch, tws, out_s, out_id, d_status, stream);
  float* surv_s = reinterpret_cast<float*>(w);
  int32_t* surv_id = reinterpret_cast<int32_t*>(w + (size_t)nq * kappa * sizeof(float));
  st = glv_score_topk(Qp, nq, C, d, Xred, row_stride, scales, dt, tags, N, cand_off, cand_ids, n_candidates, kappa,
                      scratch, tws, surv_s, surv_id, d_status, stream);
  if (st != GLV_OK) return st;
  return glv_rerank(X, N, D, Q, nq, surv_id, kappa, k, out_s, out_id, d_status, stream);
}
