// kernels.cuh -- argument blocks and launchers of the libglv kernels (host-side view).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace glv {

struct ScoreArgs {
  const float* Qp;
  int C, d, qstride;  // qstride: floats per cluster row in shared memory (set by the launcher)
  const uint8_t* Xred;
  int64_t row_stride;
  const float* scales;
  const uint16_t* tags;
  int64_t N;
  const int64_t* off;
  const int32_t* ids;
  float* scores;
  int32_t* d_status;
  int nch;     // 16-byte chunks per row that hold data
  int tail;    // bytes of data in the last chunk (16 = full)
  int splits;  // CTAs per query (set by the launcher)
  int sbs;     // float4 stride between the sub-blocks of a projected-query row (set by the launcher)
  int prefetch;  // 1: ask L2 for the next candidate's row one iteration ahead (set by the launcher)
};

// Shared-memory layout of a projected-query row (see dot_chunk in score_dev.cuh): EPC/4
// sub-blocks of sbs float4 each.  BF16 rows: the sub-block stride is padded so that the two
// candidates a quarter-warp serves read opposite halves of the banks (odd candidate groups walk
// the two sub-blocks in swapped order); rows then start on 128-byte boundaries.  FP8 rows:
// sub-blocks are not padded, and the row stride is an odd multiple of 64 bytes, so rows of
// consecutive clusters start in opposite halves of the banks.  FP32 rows: one sub-block, rows
// padded by 16 bytes.
__host__ __device__ inline int qp_sub_blocks(int dt) { return dt == 0 ? 1 : (dt == 1 ? 2 : 4); }
__host__ __device__ inline int qp_sbs(int nch, int dt) {
  if (dt != 1) return nch;
  int s = nch;
  while (s % 8 != 4) ++s;  // 16 * s = 64 (mod 128)
  return s;
}
__host__ __device__ inline int qp_qstride(int nch, int dt) {
  if (dt == 0) return nch * 4 + 4;
  if (dt == 1) return 2 * qp_sbs(nch, dt) * 4;
  return 16 * nch + ((nch & 1) ? 0 : 16);  // 64 * nch bytes, plus 64 when that is a multiple of 128
}

struct RerankArgs {
  const float* X;
  int64_t N;
  int D;
  const float* Q;
  const int32_t* surv;
  int kappa, k;
  float* out_s;
  int32_t* out_id;
  int32_t* d_status;
};

cudaError_t launch_score(const ScoreArgs& a, int dt, int64_t nq, int num_sms, cudaStream_t st);
size_t fused_smem_bytes(int C, int d, int dt, int kappa);

// Work plan of the fused scoring + top-kappa, built on the device (plan_chunks): a query's
// list is one work item, or -- when it holds at least 2 kChunk candidates -- floor(L / kChunk)
// items of kChunk candidates, the last one taking the remainder (so every item has at least
// kChunk >= 2 kappa candidates and can hold its own top-kappa list in its part of the score
// scratch); the item that finishes last merges the items' lists.
constexpr int kChunk = 4096;
struct ItemRec {
  int64_t b0;       // first candidate of the item (a position in cand_ids)
  int32_t len;      // candidates in the item
  int32_t q;        // query
  int32_t c;        // chunk index within the query
  int32_t nchunks;  // items of the query
};
struct ChunkPlan {
  int32_t* next;         // next work item to claim (dynamic scheduling)
  int32_t* n_items;      // number of work items
  int32_t* chunk_start;  // nq + 1: first item of each query
  int32_t* done;         // nq: finished items per query
  ItemRec* items;        // the work items, query-major
};
size_t topk_plan_bytes(int64_t nq, int64_t n_cand);
ChunkPlan topk_plan_layout(void* ws, int64_t nq);
cudaError_t launch_plan_chunks(const int64_t* off, int64_t nq, int64_t n_cand, void* ws, int32_t* d_status,
                               cudaStream_t st);
bool set_score_config(int dt, int G, int mode, int carve_kb, int sched);
void effective_score_config(int dt, int nch, int* G, int* mode, int* carve_kb, int* sched);
cudaError_t launch_score_topk(const ScoreArgs& a, int dt, int64_t nq, int64_t n_cand, int kappa, void* plan_ws,
                              float* out_s, int32_t* out_id, int num_sms, cudaStream_t st);
size_t lazy_smem_bytes(int C, int d, int D, int dt);
cudaError_t launch_score_lazy(const ScoreArgs& a, int dt, int64_t nq, const float* Q, int D, const float* A,
                              int32_t* visited, cudaStream_t st);
cudaError_t launch_topk(const float* scores, const int64_t* off, const int32_t* ids, int64_t nq,
                        int kappa, float* out_s, int32_t* out_id, cudaStream_t st);
cudaError_t launch_rerank(const RerankArgs& a, int64_t nq, bool vec, cudaStream_t st);
cudaError_t launch_bounded_wait(uint64_t limit_ns, int32_t* d_status, cudaStream_t st);
cudaError_t launch_gather_rows(const void* rows, int64_t row_bytes, int64_t n_rows, const int32_t* ids,
                               int64_t n_ids, float* out, int32_t* d_status, int num_sms, cudaStream_t st);
size_t rerank_smem_bytes(int D, int kappa);
cudaError_t launch_project_simt(const float* Q, int64_t nq, int D, const float* A, int64_t Mcols,
                                float* Qp, cudaStream_t st);
size_t project_tc_ws_bytes(int64_t nq, int D, int64_t Mc, int bf16);
cudaError_t launch_project_tc(const float* Q, int64_t nq, int D, const float* A, int64_t Mc, float* Qp,
                              int bf16, void* ws, int32_t* d_status, int num_sms, cudaStream_t st);
// Rows grouped by cluster: counts[c], seg_start[c] (exclusive scan), tile_start[c] (32-row
// tiles), and perm = row ids ordered by cluster (within a cluster in arbitrary order).
struct BuildWs {
  int32_t* counts;      // C
  int32_t* cursor;      // C
  int32_t* seg_start;   // C
  int32_t* tile_start;  // C + 1 (last = number of tiles)
  int32_t* perm;        // N
};
BuildWs build_ws_carve(void* ws, int64_t N, int C);
cudaError_t launch_grouping(const uint16_t* tags, int64_t N, int C, const BuildWs& ws, int32_t* d_status,
                            cudaStream_t st);
size_t build_ws_bytes(int64_t N, int C);
size_t kmeans_ws_bytes(int64_t N, int C, int D);
cudaError_t launch_kmeans_update(const float* X, int64_t N, int D, const uint16_t* tags, int C, float* mu,
                                 int32_t* counts_out, void* ws, int32_t* d_status, cudaStream_t st);
size_t moments_ws_bytes(int64_t n, int C);
cudaError_t launch_moments(const float* V, int64_t n, int D, const uint16_t* tags, int C, double* K, void* ws,
                           int32_t* d_status, cudaStream_t st);
size_t pair_ws_bytes(int64_t P, int C);
cudaError_t launch_pair_forward(const float* Q, int64_t nQ, const float* X, int64_t nX, int D, const uint16_t* tags,
                                const float* A, const float* B, int C, int d, const int32_t* qi, const int32_t* xi,
                                int64_t P, float* s, float* t, float* u, float* v, void* ws, int32_t* d_status,
                                cudaStream_t st);
cudaError_t launch_pair_backward(const float* Q, int64_t nQ, const float* X, int64_t nX, int D,
                                 const uint16_t* tags, int C, int d, const int32_t* qi, const int32_t* xi, int64_t P,
                                 const float* u, const float* v, const float* g, float* dA, float* dB, void* ws,
                                 int32_t* d_status, cudaStream_t st);
cudaError_t launch_pair_loss(const float* s, const float* t, int64_t P, const double* weight, double* loss, float* g,
                             cudaStream_t st);
cudaError_t launch_adam(float* param, const float* grad, float* m, float* v, int64_t n, float lr, float b1, float b2,
                        float eps, int step, int num_sms, cudaStream_t st);
bool build_tc_supported(int64_t N, int D, int C, int d, const void* X, const void* B);
cudaError_t launch_build_tc(const float* X, int64_t N, int D, const float* B, int C, int d, int dt, void* Xred,
                            int64_t row_stride, float* scales, const BuildWs& ws, int32_t* d_status, int num_sms,
                            cudaStream_t st);
cudaError_t launch_build(const float* X, int64_t N, int D, const uint16_t* tags, const float* B,
                         int C, int d, int dt, void* Xred, int64_t row_stride, float* scales,
                         void* workspace, int32_t* d_status, cudaStream_t st);
cudaError_t launch_tags(const float* X, int64_t N, int D, const float* mu, int C, uint16_t* tags,
                        float* best_ip, int num_sms, cudaStream_t st);

}  // namespace glv
