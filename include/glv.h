/*
 * glv.h -- C ABI of the GB300 (sm_103a) GleanVec eager search library (libglv.so).
 *
 * GleanVec (arXiv 2410.22347, Section 4) approximates the inner product of a query q and a
 * database vector x_i by <A_{c_i} q, B_{c_i} x_i>, where c_i is the vector's cluster tag
 * (Eq. cluster_tag) and (A_c, B_c) are per-cluster d x D reduction matrices.  The eager
 * variant (Algorithm 4) projects every query through all C matrices once and then scores
 * each candidate by one d-long dot product against the projected query of its cluster.
 * Search follows the multi-step scheme of Algorithm 1: score the candidates in the
 * reduced space, keep the best kappa, re-rank them exactly in full dimension D, return k.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Every array argument is a DEVICE pointer owned by the caller; the library never
 *    allocates, frees or retains it.  Matrices are row-major.
 *  * `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Every
 *    call enqueues work on that stream and returns without synchronising.
 *  * Arguments are validated on the host before anything is enqueued; an invalid argument
 *    returns GLV_ERR_INVALID_ARG (or GLV_ERR_UNSUPPORTED for a legal shape this build does
 *    not handle) and nothing is enqueued.  A failed launch returns GLV_ERR_CUDA.
 *  * Errors only the device can see (a candidate / survivor id outside [0, N), a tag
 *    outside [0, C)) are written into the caller-provided device word `d_status` (may be
 *    NULL): the first error code wins, later ones are dropped, and the offending item is
 *    skipped (its score is -inf).  Clear the word to GLV_OK before the call and read it
 *    back after synchronising the stream.
 *  * Orderings: results are sorted by score descending, ties broken by the smaller id;
 *    NaN scores rank after every number; a slot with no candidate holds id -1 and score
 *    -inf.
 *  * Sizes: N < 2^31 database rows (ids are int32), 1 <= C <= 65536 clusters (tags are
 *    uint16), 1 <= d <= D.
 */
#ifndef GLV_H_
#define GLV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GLV_OK = 0,
  GLV_ERR_INVALID_ARG = 1, /* bad pointer / size / alignment; nothing enqueued          */
  GLV_ERR_BAD_ID = 2,      /* (device word) an id or tag was out of range; item skipped */
  GLV_ERR_UNSUPPORTED = 3, /* legal shape outside what this build handles               */
  GLV_ERR_CUDA = 4,        /* a CUDA runtime call or a launch failed                    */
  GLV_ERR_TIMEOUT = 5      /* (device word) a bounded device-side wait ran out          */
} glv_status;

/* Storage type of the reduced rows x_i^low (and compute type of the projection).
 * Section 2.1 says the reduced vectors may be scalar-quantised "as in LeanVec" without
 * fixing a scheme; this library offers:
 *   GLV_F32      : FP32 values.
 *   GLV_BF16     : bfloat16, round-to-nearest-even of the FP32 value.
 *   GLV_FP8_E4M3 : OCP FP8 e4m3 codes with one FP32 scale per row,
 *                  s_i = max_j |x_ij| / 448, code_ij = RNE_e4m3(x_ij / s_i) saturating;
 *                  the represented value is s_i * decode(code_ij). */
typedef enum { GLV_F32 = 0, GLV_BF16 = 1, GLV_FP8_E4M3 = 2 } glv_dtype;

#define GLV_ABI_VERSION 4
#define GLV_MAX_KAPPA 1024 /* largest kappa accepted by glv_topk / glv_rerank */

int32_t glv_abi_version(void);
const char* glv_status_string(glv_status s);

/* ---------------------------------------------------------------------------------------
 * Device-detected errors land in a caller-provided int32 status word (d_status arguments):
 * 0 while nothing went wrong, else the first glv_status code recorded.  This helper waits
 * for `stream` (cudaStreamSynchronize), reads the word and returns it (GLV_ERR_CUDA if the
 * wait or the read fails, GLV_ERR_INVALID_ARG for a NULL word).  It does not reset it.
 * ------------------------------------------------------------------------------------- */
glv_status glv_last_device_status(const int32_t* d_status, void* stream);

/* Smallest legal row stride in bytes of a reduced-row store of width d and type dt:
 * d * sizeof(element) rounded up to 16 bytes (rows are read with 16-byte vector loads). */
int64_t glv_min_row_stride(int32_t d, glv_dtype dt);

/* ---------------------------------------------------------------------------------------
 * Cluster tags, Eq. (cluster_tag), Section 4:  c_i = argmax_c <x_i, mu_c>.
 *   X       : N x D float32, rows contiguous.
 *   mu      : C x D float32 landmarks.
 *   tags    : N uint16 output.  Ties go to the lowest c.  FP32 accumulation.
 *   best_ip : N float32 output <x_i, mu_{c_i}> (may be NULL) -- the spherical k-means
 *             objective terms (Appendix A) and the k-means++ seeding weights.
 * Limits: D <= 1024 (else GLV_ERR_UNSUPPORTED); any C <= 65536.
 * ------------------------------------------------------------------------------------- */
glv_status glv_assign_tags(const float* X, int64_t N, int32_t D, const float* mu, int32_t C,
                           uint16_t* tags, float* best_ip, void* stream);

/* ---------------------------------------------------------------------------------------
 * Spherical k-means M-step, Appendix A:  mu_c = sum_{i: tags_i = c} x_i / || . ||_2
 * (FP64 sums; a cluster with no member keeps its landmark).  With glv_assign_tags as the
 * E-step this is the landmark learning of Algorithm 5 (rows are expected L2-normalised).
 *   X : N x D float32;  tags : N uint16;  mu : C x D float32, updated in place.
 *   counts : C int32 output cluster sizes (may be NULL).
 *   workspace : glv_kmeans_workspace_size(N, D, C) bytes, 256-aligned.
 * ------------------------------------------------------------------------------------- */
size_t glv_kmeans_workspace_size(int64_t N, int32_t D, int32_t C);
glv_status glv_kmeans_update(const float* X, int64_t N, int32_t D, const uint16_t* tags,
                             int32_t C, float* mu, int32_t* counts, void* workspace,
                             int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Reduced database, Eq. (X_low), Section 4, read as x_i^low = g_{c_i}(x_i) = B_{c_i} x_i
 * (the equation prints f; the GleanVec approximation that follows it and the definition
 * g_c(x) = B_c x fix g).  Rows are grouped by cluster on the device and each group is
 * multiplied by its B_c (a grouped GEMM, FP32 accumulation); the epilogue stores the
 * row in `dt` (see glv_dtype).
 *   X          : N x D float32.            tags : N uint16, each < C.
 *   B          : C x d x D float32 (B_c row-major, clusters consecutive).
 *   Xred       : N rows of `row_stride` bytes; row i holds d elements of type `dt`,
 *                then zero bytes up to the next 16-byte boundary.  16-byte aligned.
 *   row_stride : multiple of 16, >= glv_min_row_stride(d, dt).
 *   scales     : N float32 per-row scales (FP8 only; must be NULL otherwise).
 *   workspace  : device scratch of glv_build_reduced_workspace_size(N, C) bytes,
 *                256-byte aligned; its contents on entry do not matter.
 *   d_status   : optional device error word (tag >= C -> GLV_ERR_BAD_ID, row skipped).
 * ------------------------------------------------------------------------------------- */
size_t glv_build_reduced_workspace_size(int64_t N, int32_t C);
glv_status glv_build_reduced(const float* X, int64_t N, int32_t D, const uint16_t* tags,
                             const float* B, int32_t C, int32_t d, glv_dtype dt, void* Xred,
                             int64_t row_stride, float* scales, void* workspace,
                             int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * glv_build_reduced_noalloc -- the same build as glv_build_reduced, for callers that cannot
 * allocate device memory.  (This entry point has no counterpart in the paper; it only
 * changes where the build's scratch memory comes from.)
 *
 * Some callers cannot hand the library a workspace: code that runs inside another
 * framework's memory pool or under a fixed device-memory budget it does not control, plugin
 * hosts that only pass through the input and output buffers, and callers on a latency path
 * where cudaMalloc (which may synchronise the device) is not acceptable.  This variant takes
 * the same inputs and outputs as glv_build_reduced but no workspace: its scratch (cluster
 * counts, cursors, offsets, tile table, row permutation) is a fixed array of device memory
 * inside libglv itself, about 4.2 MB, reserved on every GPU that loads the library until the
 * process exits.  It calls no allocator.
 *
 *   Limits: N <= GLV_NOALLOC_MAX_ROWS and C <= GLV_NOALLOC_MAX_CLUSTERS; larger sizes return
 *           GLV_ERR_UNSUPPORTED and enqueue nothing (use glv_build_reduced instead).
 *   Set-up: the first call on each device looks up the array's device address with that
 *           device current (cudaGetSymbolAddress) and caches it; make that first call before
 *           any stream capture on that device.  The cached address belongs to the device's
 *           context of that first call: after cudaDeviceReset() on a device, do not call this
 *           entry point on that device again in the same process.
 *   Sharing: all calls on a device share the one array and it keeps the previous call's
 *           contents (the parts that must start at zero are cleared on the stream by each
 *           call).  Calls whose execution overlaps on the GPU -- on different streams, or
 *           from different host threads -- race on the array: serialise them.
 * All other arguments, results and errors are exactly those of glv_build_reduced.
 * ------------------------------------------------------------------------------------- */
#define GLV_NOALLOC_MAX_ROWS (1LL << 20)
#define GLV_NOALLOC_MAX_CLUSTERS 4096
glv_status glv_build_reduced_noalloc(const float* X, int64_t N, int32_t D, const uint16_t* tags,
                                     const float* B, int32_t C, int32_t d, glv_dtype dt,
                                     void* Xred, int64_t row_stride, float* scales,
                                     int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Query preprocessing of Algorithm 4 (eager):  q_{j,c} = A_c q_j  for every c = 1..C,
 * i.e. one dense GEMM  Qp = Q . [A_1; ...; A_C]^T  of shape nq x (C*d).
 *   Q         : nq x D float32.           A : C x d x D float32.
 *   compute   : GLV_F32  -- FP32-accurate.  With a workspace: tcgen05 tensor cores, each
 *                           operand split exactly into TF32 hi + lo and three MMAs per step
 *                           (hi*hi + hi*lo + lo*hi), ~1e-7 relative; with workspace == NULL:
 *                           a SIMT FP32 FMA kernel (slower, no workspace needed).
 *               GLV_BF16 -- operands rounded to bfloat16, FP32 accumulation on tcgen05
 *                           (workspace required).
 *   Qp        : nq x C x d float32 output (row j holds the C projected views of q_j).
 *   workspace : NULL (GLV_F32 only) or device scratch of
 *               glv_project_queries_workspace_size(nq, D, C, d, compute) bytes, 256-byte
 *               aligned, holding the converted operands; contents on entry do not matter.
 *   d_status  : optional device error word; GLV_ERR_TIMEOUT if a bounded device-side wait
 *               of the tensor-core kernel ran out (the output is then incomplete).
 * ------------------------------------------------------------------------------------- */
size_t glv_project_queries_workspace_size(int64_t nq, int32_t D, int32_t C, int32_t d,
                                          glv_dtype compute);
glv_status glv_project_queries(const float* Q, int64_t nq, int32_t D, const float* A,
                               int32_t C, int32_t d, glv_dtype compute, float* Qp,
                               void* workspace, int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Candidate scoring, Algorithm 4 procedure inner-product and Eq. (GleanVec approximation):
 * for query j and each candidate id i in its list,
 *        s = <q_{j, c_i}, x_i^low>        (times s_i for FP8 rows),
 * FP32 accumulation.  Candidate lists are CSR: list j is
 * cand_ids[cand_off[j] .. cand_off[j+1]); they stand in for the vertices a graph search
 * visits (Algorithm 1, main step).
 *   Qp        : nq x C x d float32 (from glv_project_queries).
 *   Xred, row_stride, scales, dt : the store written by glv_build_reduced.
 *   tags      : N uint16.   cand_off : nq+1 int64, non-decreasing, cand_off[0] = 0.
 *   cand_ids  : int32 ids; an id outside [0, N) scores -inf and sets GLV_ERR_BAD_ID.
 *   scores    : cand_off[nq] float32 output, aligned with cand_ids.
 * Limits: C * d <= 49152 (one query's C projected views are staged in shared memory).
 * ------------------------------------------------------------------------------------- */
glv_status glv_score_candidates(const float* Qp, int64_t nq, int32_t C, int32_t d,
                                const void* Xred, int64_t row_stride, const float* scales,
                                glv_dtype dt, const uint16_t* tags, int64_t N,
                                const int64_t* cand_off, const int32_t* cand_ids,
                                float* scores, int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Lazy candidate scoring, Algorithm 3: the same scores as glv_project_queries followed by
 * glv_score_candidates (up to FP32 rounding of the projection), but the projected views
 * q_c = A_c q are formed inside the scoring kernel, once per cluster that the query's list
 * visits, instead of for all C clusters by a batched projection beforehand.
 *   Q : nq x D float32 queries;  A : C x d x D float32;  other arguments as for
 *   glv_score_candidates.   visited : nq int32 output (may be NULL) -- the number of
 *   distinct clusters among each query's candidates.
 * Limits: C * (d rounded up to 16 bytes + 4) + D floats must fit in shared memory.
 * ------------------------------------------------------------------------------------- */
glv_status glv_score_lazy(const float* Q, int64_t nq, int32_t D, const float* A, int32_t C,
                          int32_t d, const void* Xred, int64_t row_stride, const float* scales,
                          glv_dtype dt, const uint16_t* tags, int64_t N, const int64_t* cand_off,
                          const int32_t* cand_ids, float* scores, int32_t* visited,
                          int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Fused candidate scoring + top-kappa: the same computation and the same results (bit for
 * bit) as glv_score_candidates followed by glv_topk, without writing the scores to memory:
 * they stay on chip and the kappa best are selected there.  Work is planned on the device:
 * a query's list is one work item, or -- when it holds at least 8192 candidates --
 * floor(L / 4096) items (the last one takes the remainder), each selecting its own
 * top-kappa, merged by the item that finishes last (the merged top-kappa is exact);
 * persistent CTAs claim items dynamically, so long lists do not leave a tail of busy CTAs.
 *   Arguments as for glv_score_candidates and glv_topk, and:
 *   n_candidates   : cand_off[nq] - cand_off[0], the number of candidate entries (the
 *                    length of cand_ids).  If the lists hold more, nothing is computed and
 *                    GLV_ERR_INVALID_ARG is reported in d_status.
 *   scores_scratch : n_candidates float32 scratch (per-item top-kappa lists of split
 *                    queries, scores of lists that exceed the on-chip key cache, and the
 *                    scores when nq is small -- the lists are then split over many CTAs and
 *                    the selection runs afterwards); contents on entry do not matter.
 *   workspace      : glv_score_topk_workspace_size(nq, n_candidates) bytes, 256-byte
 *                    aligned (the work plan); contents on entry do not matter.
 *   out_s, out_id  : nq x kappa outputs, as glv_topk.
 * Calls on the same workspace must not overlap in time.
 * ------------------------------------------------------------------------------------- */
size_t glv_score_topk_workspace_size(int64_t nq, int64_t n_candidates);
glv_status glv_score_topk(const float* Qp, int64_t nq, int32_t C, int32_t d, const void* Xred,
                          int64_t row_stride, const float* scales, glv_dtype dt,
                          const uint16_t* tags, int64_t N, const int64_t* cand_off,
                          const int32_t* cand_ids, int64_t n_candidates, int32_t kappa,
                          float* scores_scratch, void* workspace, float* out_s, int32_t* out_id,
                          int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Scoring configuration (the autotuner's hook; no counterpart in the paper).  Per store
 * type: how many lanes of a warp cooperate on one candidate row (1, 2, 4, 8, 16 or 32;
 * 0 = library default) and how rows are gathered (gather_mode): 0 = 16-byte loads into
 * registers; 1 = the same with the next candidate's loads issued before the current dot;
 * 2 = one bulk asynchronous copy per row into a per-warp ring of shared-memory slots (used
 * only where the rings fit in shared memory, else mode 0).  The choice changes only speed
 * and the order in which a row's partial dots are summed (FP32 rounding); the gather mode
 * does not change that order, and glv_score_candidates and glv_score_topk always use the
 * same configuration, so their results stay identical.  smem_carveout_kb caps the shared-
 * memory part of the SM's shared-memory / L1 split for the scoring kernels (0 = the
 * driver's choice, else 16..256 KB; ignored where one CTA would not fit under the cap): the
 * driver sizes that split for the kernel's full occupancy, and the L1 left over stages the
 * gathered rows in flight, so fewer CTAs with more L1 can be faster.  schedule, three bits:
 * bit 0 (fused call) set (1, the default) = the planned work items of glv_score_topk (long
 * lists cut into chunks, persistent CTAs), clear = one CTA per query, no plan (faster when no
 * list is long: no plan launch, no work counter); bit 1 (fused call) set = wide CTAs of 512
 * threads instead of 256 (one query's staged projected views serve twice the warps, and lists
 * of up to 4096 candidates keep their scores on chip), offered with gather mode 0 and the
 * store type's two smaller lane counts (FP32 and BF16: 4, 8; FP8: 2, 4), else ignored; bit 2
 * set = each candidate group asks L2 for the next candidate's row one iteration before loading
 * it (prefetch; stand-alone scoring and 256-thread fused CTAs, ignored by wide ones).  All of these change only speed.  The fused
 * call maps gather mode 2 to mode 0.  A choice that cannot serve a row width falls back to the
 * default for that width; glv_get_score_config reports the configuration used for rows of width d.
 * Process-wide setting.  Errors: GLV_ERR_INVALID_ARG for an unknown dt, lane count, mode,
 * carveout or schedule.
 * ------------------------------------------------------------------------------------- */
glv_status glv_set_score_config(glv_dtype dt, int32_t lanes_per_candidate, int32_t gather_mode,
                                int32_t smem_carveout_kb, int32_t schedule);
glv_status glv_get_score_config(glv_dtype dt, int32_t d, int32_t* lanes_per_candidate,
                                int32_t* gather_mode, int32_t* smem_carveout_kb, int32_t* schedule);

/* ---------------------------------------------------------------------------------------
 * The whole eager multi-step search in one call (Algorithm 1 with Algorithm 4):
 * glv_project_queries -> glv_score_topk (kappa survivors) -> glv_rerank (exact top k), or,
 * with kappa == 0, the top k of the reduced scores without a re-rank.  Same arguments,
 * results and errors as those calls, in that order; the intermediate arrays (projected
 * queries, projection operands, score scratch, work plan, survivors) are carved from one
 * caller-provided workspace of glv_search_workspace_size(nq, D, C, d, compute,
 * n_candidates, kappa) bytes, 256-byte aligned, contents on entry irrelevant.  The arguments
 * of all three steps are checked before the first launch is enqueued.
 *   X : N x D float32 (the re-rank's rows);  Q : nq x D float32;  A : C x d x D float32.
 *   compute : projection operands, GLV_F32 (3xTF32, FP32-accurate) or GLV_BF16.
 *   Xred, row_stride, scales, dt, tags, cand_off, cand_ids, n_candidates : as for
 *   glv_score_topk.   kappa : 0, or k <= kappa <= GLV_MAX_KAPPA.   out_s, out_id : nq x k.
 * ------------------------------------------------------------------------------------- */
size_t glv_search_workspace_size(int64_t nq, int32_t D, int32_t C, int32_t d, glv_dtype compute,
                                 int64_t n_candidates, int32_t kappa);
glv_status glv_search(const float* X, int64_t N, int32_t D, const float* Q, int64_t nq,
                      const float* A, int32_t C, int32_t d, glv_dtype compute, const void* Xred,
                      int64_t row_stride, const float* scales, glv_dtype dt, const uint16_t* tags,
                      const int64_t* cand_off, const int32_t* cand_ids, int64_t n_candidates,
                      int32_t kappa, int32_t k, void* workspace, float* out_s, int32_t* out_id,
                      int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * The same search from HOST buffers (the serving entry point): copies the queries and the
 * candidate lists from host memory into the workspace, runs glv_search on them and copies
 * the top k back to host memory, all enqueued on `stream` in that order (cudaMemcpyAsync;
 * the call returns after enqueueing).  Host buffers should be page-locked (cudaHostAlloc /
 * cudaHostRegister) for the copies to be asynchronous; with pageable memory they still
 * complete correctly but may synchronise the host.  The caller must not touch the host
 * outputs, nor reuse the host inputs or the workspace, until the stream has passed this
 * call.  Two calls on two streams with two workspaces overlap one batch's copies with the
 * other's search.
 *   Q_host : nq x D float32;  cand_off_host : nq + 1 int64;  cand_ids_host : n_candidates
 *   int32 (host);  out_s_host, out_id_host : nq x k (host).   X, A, Xred, scales, tags, as
 *   for glv_search, are device pointers.
 *   workspace : glv_search_host_workspace_size(nq, D, C, d, compute, n_candidates, kappa, k)
 *   bytes of device memory, 256-byte aligned.
 * Every argument of every step is checked before the first copy is enqueued.
 * ------------------------------------------------------------------------------------- */
size_t glv_search_host_workspace_size(int64_t nq, int32_t D, int32_t C, int32_t d, glv_dtype compute,
                                      int64_t n_candidates, int32_t kappa, int32_t k);
glv_status glv_search_host(const float* X, int64_t N, int32_t D, const float* Q_host, int64_t nq,
                           const float* A, int32_t C, int32_t d, glv_dtype compute, const void* Xred,
                           int64_t row_stride, const float* scales, glv_dtype dt, const uint16_t* tags,
                           const int64_t* cand_off_host, const int32_t* cand_ids_host, int64_t n_candidates,
                           int32_t kappa, int32_t k, void* workspace, float* out_s_host, int32_t* out_id_host,
                           int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Gather calibration (no counterpart in the paper; a measuring instrument for the roofline
 * of the gather-score): for every entry p of ids, reads the whole row ids[p] of a row-major
 * store and writes out[p] = the row's 32-bit words summed as floats -- the same bytes in the
 * same random order as the scoring kernels read, without their arithmetic, so its bandwidth
 * is the practical ceiling of random row gathers of that width on this GPU.
 *   rows      : n_rows x row_bytes device bytes, 16-byte aligned; row_bytes a multiple of
 *               16, at most 1024 (else GLV_ERR_UNSUPPORTED).
 *   ids       : n_ids int32 row ids; an id outside [0, n_rows) writes 0 and sets
 *               GLV_ERR_BAD_ID in d_status (optional).   out : n_ids float32.
 * ------------------------------------------------------------------------------------- */
glv_status glv_gather_rows(const void* rows, int64_t row_bytes, int64_t n_rows, const int32_t* ids,
                           int64_t n_ids, float* out, int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Self-check of the bounded device-side waits (no counterpart in the paper).  The tensor-
 * core kernels wait on mbarriers with a time limit (2 s) and report GLV_ERR_TIMEOUT in the
 * status word instead of hanging if a wait never completes; this launches one thread that
 * waits, with a limit of limit_us microseconds (1 .. 10^6), on a barrier nothing completes,
 * so the same timeout path runs and the status word receives GLV_ERR_TIMEOUT (read it with
 * glv_last_device_status).  The GPU is left fully usable.
 * ------------------------------------------------------------------------------------- */
glv_status glv_check_bounded_wait(uint32_t limit_us, int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Per-query top-kappa of the scores (Algorithm 1: the main step hands kappa candidates to
 * the post-processing).  Exact selection (radix select on order-preserving keys), output
 * sorted by score descending, ties to the smaller id, NaN last, padding (-inf, -1) when a
 * list has fewer than kappa entries.
 *   scores, cand_off, cand_ids : as for glv_score_candidates.
 *   out_s, out_id : nq x kappa float32 / int32 outputs.     1 <= kappa <= GLV_MAX_KAPPA.
 * ------------------------------------------------------------------------------------- */
glv_status glv_topk(const float* scores, const int64_t* cand_off, const int32_t* cand_ids,
                    int64_t nq, int32_t kappa, float* out_s, int32_t* out_id, void* stream);

/* ---------------------------------------------------------------------------------------
 * Post-processing of Algorithm 1: exact inner products <q_j, x_i> in full dimension D
 * (FP32 accumulation) for each query's survivors, then the top k of them.
 *   X      : N x D float32.   Q : nq x D float32.
 *   surv_id: nq x kappa int32; -1 marks an empty slot; another id outside [0, N) is
 *            skipped and sets GLV_ERR_BAD_ID.
 *   out_s, out_id : nq x k outputs.   1 <= k <= kappa <= GLV_MAX_KAPPA.
 * ------------------------------------------------------------------------------------- */
glv_status glv_rerank(const float* X, int64_t N, int32_t D, const float* Q, int64_t nq,
                      const int32_t* surv_id, int32_t kappa, int32_t k, float* out_s,
                      int32_t* out_id, int32_t* d_status, void* stream);

/* =======================================================================================
 * Learning side: statistics of LeanVec-Sphering and the gradient used to refine it.
 * ===================================================================================== */

/* ---------------------------------------------------------------------------------------
 * Second moments K = sum_v v v^T (the D x D summary statistics of Section 3.2, from which
 * Algorithm 2 is computed by eigendecompositions: K_Q for the queries, K_{X_c} for the
 * database vectors of each cluster, Algorithm 5).  FP32 inputs, FP64 products and sums.
 *   V    : n x D float32.
 *   tags : n uint16 cluster of each vector, or NULL (then C must be 1: one matrix over all).
 *   K    : C x D x D float64 output (row-major, symmetric; clusters with no vector get 0).
 *   workspace : glv_second_moments_workspace_size(n, C) bytes (256-aligned) when tags are
 *               given, else may be NULL.   d_status : tag >= C -> GLV_ERR_BAD_ID, skipped.
 * ------------------------------------------------------------------------------------- */
size_t glv_second_moments_workspace_size(int64_t n, int32_t C);
glv_status glv_second_moments(const float* V, int64_t n, int32_t D, const uint16_t* tags,
                              int32_t C, double* K, void* workspace, int32_t* d_status,
                              void* stream);

/* ---------------------------------------------------------------------------------------
 * Pair forward of the inner-product approximation loss (the LeanVec problem of Section 2.1
 * restricted to GleanVec pairs, Section 4.1): for P index pairs p = (qi[p], xi[p]) with
 * cluster c = tags[xi[p]],
 *     u_p = B_c x_p,  v_p = A_c q_p  (d each),  s_p = <u_p, v_p>,  t_p = <q_p, x_p>.
 * The loss sum_p (t_p - s_p)^2 and its gradient follow from s, t (see glv_pair_backward).
 *   Q : nQ x D, X : nX x D float32;  A, B : C x d x D float32;  qi, xi : P int32.
 *   s, t : P float32 outputs;  u, v : P x d float32 outputs (kept for the backward).
 *   workspace : glv_pair_workspace_size(P, C) bytes, 256-aligned.
 *   A pair with an index or tag out of range gets s = t = 0, u = v = 0 and GLV_ERR_BAD_ID.
 * ------------------------------------------------------------------------------------- */
size_t glv_pair_workspace_size(int64_t P, int32_t C);
glv_status glv_pair_forward(const float* Q, int64_t nQ, const float* X, int64_t nX, int32_t D,
                            const uint16_t* tags, const float* A, const float* B, int32_t C,
                            int32_t d, const int32_t* qi, const int32_t* xi, int64_t P, float* s,
                            float* t, float* u, float* v, void* workspace, int32_t* d_status,
                            void* stream);

/* ---------------------------------------------------------------------------------------
 * Pair backward (the gather-score backward): given g_p = dL/ds_p,
 *     dA_c = sum_{p: c_p = c} g_p u_p q_p^T,    dB_c = sum_{p: c_p = c} g_p v_p x_p^T,
 * a segmented sum of rank-1 terms per cluster (pairs grouped by cluster on the device, one
 * FP32 GEMM over each cluster's pairs).  For L = sum_p (t_p - s_p)^2, g_p = -2 (t_p - s_p).
 *   u, v : from glv_pair_forward on the same pairs;  g : P float32.
 *   dA, dB : C x d x D float32 outputs (overwritten; clusters without pairs get 0).
 * ------------------------------------------------------------------------------------- */
glv_status glv_pair_backward(const float* Q, int64_t nQ, const float* X, int64_t nX, int32_t D,
                             const uint16_t* tags, int32_t C, int32_t d, const int32_t* qi,
                             const int32_t* xi, int64_t P, const float* u, const float* v,
                             const float* g, float* dA, float* dB, void* workspace,
                             int32_t* d_status, void* stream);

/* ---------------------------------------------------------------------------------------
 * Pair loss, the inner-product approximation loss of Section 2.1 over GleanVec pairs:
 *     loss = sum_p (t_p - s_p)^2       (FP64 accumulation, deterministic order),
 *     g_p  = w * dloss/ds_p = -2 w (t_p - s_p)      (FP32),
 * from the s, t of glv_pair_forward.  weight: device pointer to one double w (the upstream
 * derivative of an outer objective with respect to loss), or NULL for w = 1.  loss: device
 * pointer to one double (8-byte aligned), or NULL;  g: P float32, or NULL (not both NULL).
 * One CTA; meant for minibatches (thousands of pairs).
 * ------------------------------------------------------------------------------------- */
glv_status glv_pair_loss(const float* s, const float* t, int64_t P, const double* weight, double* loss, float* g,
                         void* stream);

/* ---------------------------------------------------------------------------------------
 * One Adam step (Kingma and Ba, 2015) on n FP32 parameters, in place -- the optimiser that
 * refines the Sphering initialisation with the gradients of glv_pair_backward (the paper
 * fixes no optimiser; it has no counterpart there):
 *     m <- beta1 m + (1 - beta1) grad,   v <- beta2 v + (1 - beta2) grad^2,
 *     param <- param - lr * (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps).
 *   param, m, v : n float32, updated (m, v start at zero before step 1).   grad : n float32.
 *   step : 1-based step count.  0 <= beta1, beta2 < 1, eps > 0, lr >= 0.
 * ------------------------------------------------------------------------------------- */
glv_status glv_adam_step(float* param, const float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                         float beta2, float eps, int32_t step, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GLV_H_ */
