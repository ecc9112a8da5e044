/*
 * glv_oracle.c -- plain, slow, FP64 CPU oracle for the GleanVec eager search path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this
 * file: it exists so that tests, the smoke check and the CPU-baseline leg of the
 * benchmark can compare the CUDA library against an implementation that a reader can
 * check against the paper line by line.  It shares no code, header, table or helper
 * with the CUDA library.
 *
 * Every routine reads the FP32 input values exactly as given, widens them to double
 * and does all arithmetic in FP64 with plain loops, in the order the paper states the
 * computation.  No blocking, no BLAS, no fusion.  OpenMP only splits independent queries
 * (or independent database rows) across threads; each output is computed by one thread
 * with the same sequential loop, so results do not depend on the thread count.
 *
 * Paper: "GleanVec: Accelerating vector search with minimalist nonlinear dimensionality
 * reduction" (Tepper, Bhati, Aguerrebere, Willke), arXiv 2410.22347.
 *
 * Readings taken where the paper is silent (kept in one place so a reader can audit them):
 *   R1  Eq. (X_low) writes x_i^low = f_{c_i}(x_i); Eq. (GleanVec approximation) and the
 *       definition g_c(x) = B_c x make it g_{c_i}(x_i) = B_{c_i} x_i.  This file uses g.
 *   R2  argmax ties in Eq. (cluster_tag) go to the lowest cluster index.
 *   R3  top-k orders by score descending, ties by smaller id; NaN scores rank last; a slot
 *       with no candidate gets id -1 and score -inf.
 *   R4  scalar quantisation (Section 2.1 / Section 3 defer it to LeanVec): BF16 is
 *       round-to-nearest-even of the FP32 value; FP8-e4m3 uses one FP32 scale per vector
 *       s_i = fp32(max_j |x_ij| / 448) and code = RNE_e4m3(fp32(x_ij / s_i)), saturating to
 *       +-448.  A vector whose scale is zero is stored as all-zero codes with scale 0.
 *
 * Parity status of each entry point is listed in the comment above it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------ */
/* threads                                                                               */
/* ------------------------------------------------------------------------------------ */

void glvo_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int32_t glvo_get_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* Eq. (cluster_tag), Section 4: c_i = argmax_c <x_i, mu_c>.  Ties: lowest c (R2).         */
/* margin (may be NULL) receives best - second best, so tests can see near-ties.          */
/* Pinned by: brute force against an independent argmax in the tests.                    */
/* ------------------------------------------------------------------------------------ */
void glvo_assign_tags(const float* X, int64_t N, int32_t D, const float* mu, int32_t C,
                      uint16_t* tags, double* margin) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    int32_t best = 0;
    double best_v = -INFINITY, second_v = -INFINITY;
    for (int32_t c = 0; c < C; ++c) {
      double v = 0.0;
      for (int32_t k = 0; k < D; ++k) v += (double)X[i * D + k] * (double)mu[(int64_t)c * D + k];
      if (v > best_v) {
        second_v = best_v;
        best_v = v;
        best = c;
      } else if (v > second_v) {
        second_v = v;
      }
    }
    tags[i] = (uint16_t)best;
    if (margin) margin[i] = best_v - second_v;
  }
}

/* ------------------------------------------------------------------------------------ */
/* Eq. (X_low), Section 4, with reading R1: x_i^low = B_{c_i} x_i.                        */
/* B holds C matrices of shape d x D, row-major, cluster-major: B[(c*d + r)*D + k].       */
/* Pinned by: d = D with B_c = I (identity), and by the M_c = A_c^T B_c route in tests.   */
/* ------------------------------------------------------------------------------------ */
void glvo_build_reduced(const float* X, int64_t N, int32_t D, const uint16_t* tags,
                        const float* B, int32_t C, int32_t d, double* Xr) {
  (void)C;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < N; ++i) {
    const int64_t c = tags[i];
    for (int32_t r = 0; r < d; ++r) {
      double v = 0.0;
      for (int32_t k = 0; k < D; ++k) v += (double)B[(c * d + r) * D + k] * (double)X[i * D + k];
      Xr[i * d + r] = v;
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 4, procedure preprocess(q): q_c = A_c q for every c = 1..C.                  */
/* Qp is nq x C x d: Qp[(j*C + c)*d + r].                                                 */
/* ------------------------------------------------------------------------------------ */
static void project_one(const float* q, int32_t D, const float* A, int32_t C, int32_t d,
                        double* qp) {
  for (int32_t c = 0; c < C; ++c)
    for (int32_t r = 0; r < d; ++r) {
      double v = 0.0;
      for (int32_t k = 0; k < D; ++k)
        v += (double)A[((int64_t)c * d + r) * D + k] * (double)q[k];
      qp[(int64_t)c * d + r] = v;
    }
}

void glvo_project(const float* Q, int64_t nq, int32_t D, const float* A, int32_t C, int32_t d,
                  double* Qp) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < nq; ++j) project_one(Q + j * D, D, A, C, d, Qp + j * (int64_t)C * d);
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 4, procedure inner-product(x_i, q): recover c_i, return <q_{c_i}, x_i^low>.   */
/* Eq. (GleanVec approximation), Section 4.  One score per candidate of query j.          */
/* An id outside [0, N) scores -inf and raises *bad.                                       */
/* ------------------------------------------------------------------------------------ */
static int score_one(const double* qp, int32_t d, const double* Xr, const uint16_t* tags,
                     int64_t N, const int32_t* ids, int64_t L, double* s) {
  int bad = 0;
  for (int64_t p = 0; p < L; ++p) {
    const int64_t i = ids[p];
    if (i < 0 || i >= N) {
      s[p] = -INFINITY;
      bad = 1;
      continue;
    }
    const double* qc = qp + (int64_t)tags[i] * d;
    double v = 0.0;
    for (int32_t r = 0; r < d; ++r) v += qc[r] * Xr[i * d + r];
    s[p] = v;
  }
  return bad;
}

int32_t glvo_score(const double* Qp, int64_t nq, int32_t C, int32_t d, const double* Xr,
                   const uint16_t* tags, int64_t N, const int64_t* off, const int32_t* ids,
                   double* s) {
  int32_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t j = 0; j < nq; ++j)
    bad |= score_one(Qp + j * (int64_t)C * d, d, Xr, tags, N, ids + off[j], off[j + 1] - off[j],
                     s + off[j]);
  return bad;
}

/* ------------------------------------------------------------------------------------ */
/* Top-kappa selection (Algorithm 1, main step returns kappa candidates), ordering R3.    */
/* Plain sort of the whole list, then the first kappa entries.                             */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  double s;
  int32_t id;
} glvo_pair;

/* returns <0 if a ranks before b */
static int pair_cmp(const void* pa, const void* pb) {
  const glvo_pair* a = (const glvo_pair*)pa;
  const glvo_pair* b = (const glvo_pair*)pb;
  const int an = isnan(a->s), bn = isnan(b->s);
  if (an != bn) return an ? 1 : -1; /* NaN last */
  if (!an) {
    if (a->s > b->s) return -1;
    if (a->s < b->s) return 1;
  }
  if (a->id < b->id) return -1;
  if (a->id > b->id) return 1;
  return 0;
}

static void select_sorted(glvo_pair* v, int64_t L, int32_t kappa, double* out_s, int32_t* out_id) {
  qsort(v, (size_t)L, sizeof(glvo_pair), pair_cmp);
  for (int32_t t = 0; t < kappa; ++t) {
    if (t < L) {
      out_s[t] = v[t].s;
      out_id[t] = v[t].id;
    } else {
      out_s[t] = -INFINITY;
      out_id[t] = -1;
    }
  }
}

void glvo_topk(const double* s, const int64_t* off, const int32_t* ids, int64_t nq,
               int32_t kappa, double* out_s, int32_t* out_id) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < nq; ++j) {
    const int64_t L = off[j + 1] - off[j];
    glvo_pair* v = (glvo_pair*)malloc(sizeof(glvo_pair) * (size_t)(L > 0 ? L : 1));
    for (int64_t p = 0; p < L; ++p) {
      v[p].s = s[off[j] + p];
      v[p].id = ids[off[j] + p];
    }
    select_sorted(v, L, kappa, out_s + j * kappa, out_id + j * kappa);
    free(v);
  }
}

/* ------------------------------------------------------------------------------------ */
/* Algorithm 1, post-processing: exact <q, x_i> in full dimension D for the survivors,    */
/* then the top k of them (ordering R3).  Survivor id -1 is an empty slot; an id outside  */
/* [0, N) is skipped and raises the return flag.                                          */
/* ------------------------------------------------------------------------------------ */
static int rerank_one(const float* X, int64_t N, int32_t D, const float* q, const int32_t* surv,
                      int64_t kappa, int32_t k, double* out_s, int32_t* out_id) {
  int bad = 0;
  glvo_pair* v = (glvo_pair*)malloc(sizeof(glvo_pair) * (size_t)(kappa > 0 ? kappa : 1));
  int64_t n = 0;
  for (int64_t t = 0; t < kappa; ++t) {
    const int64_t i = surv[t];
    if (i == -1) continue;
    if (i < 0 || i >= N) {
      bad = 1;
      continue;
    }
    double ip = 0.0;
    for (int32_t e = 0; e < D; ++e) ip += (double)q[e] * (double)X[i * D + e];
    v[n].s = ip;
    v[n].id = (int32_t)i;
    ++n;
  }
  select_sorted(v, n, k, out_s, out_id);
  free(v);
  return bad;
}

int32_t glvo_rerank(const float* X, int64_t N, int32_t D, const float* Q, int64_t nq,
                    const int32_t* surv, int32_t kappa, int32_t k, double* out_s,
                    int32_t* out_id) {
  int32_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t j = 0; j < nq; ++j)
    bad |= rerank_one(X, N, D, Q + j * D, surv + j * (int64_t)kappa, kappa, k, out_s + j * k,
                      out_id + j * k);
  return bad;
}

/* Ground truth of Section 2 (maximum inner product): the exact top k of <q_j, x_i> over  */
/* every candidate of query j.  Same computation as the post-processing step applied to   */
/* the whole candidate list.                                                              */
int32_t glvo_exact_topk(const float* X, int64_t N, int32_t D, const float* Q, int64_t nq,
                        const int64_t* off, const int32_t* ids, int32_t k, double* out_s,
                        int32_t* out_id) {
  int32_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t j = 0; j < nq; ++j)
    bad |= rerank_one(X, N, D, Q + j * D, ids + off[j], off[j + 1] - off[j], k, out_s + j * k,
                      out_id + j * k);
  return bad;
}

/* ------------------------------------------------------------------------------------ */
/* Whole eager multi-step search (Algorithm 1 with Algorithm 4 as the similarity), one    */
/* query at a time: preprocess -> score every candidate -> top kappa -> exact re-rank to  */
/* k.  Xr are the reduced rows as doubles (FP64 oracle rows, or decoded quantised rows).  */
/* kappa == 0 means "no re-rank": the top k of the reduced scores are returned as is.     */
/* This is the routine the CPU baseline times.                                            */
/* ------------------------------------------------------------------------------------ */
int32_t glvo_search(const float* X, int64_t N, int32_t D, const double* Xr,
                    const uint16_t* tags, const float* A, int32_t C, int32_t d, const float* Q,
                    int64_t nq, const int64_t* off, const int32_t* ids, int32_t kappa,
                    int32_t k, double* out_s, int32_t* out_id) {
  int32_t bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t j = 0; j < nq; ++j) {
    const int64_t L = off[j + 1] - off[j];
    double* qp = (double*)malloc(sizeof(double) * (size_t)C * (size_t)d);
    double* s = (double*)malloc(sizeof(double) * (size_t)(L > 0 ? L : 1));
    glvo_pair* v = (glvo_pair*)malloc(sizeof(glvo_pair) * (size_t)(L > 0 ? L : 1));
    project_one(Q + j * D, D, A, C, d, qp);
    bad |= score_one(qp, d, Xr, tags, N, ids + off[j], L, s);
    for (int64_t p = 0; p < L; ++p) {
      v[p].s = s[p];
      v[p].id = ids[off[j] + p];
    }
    if (kappa <= 0) {
      select_sorted(v, L, k, out_s + j * k, out_id + j * k);
    } else {
      double* ss = (double*)malloc(sizeof(double) * (size_t)kappa);
      int32_t* si = (int32_t*)malloc(sizeof(int32_t) * (size_t)kappa);
      select_sorted(v, L, kappa, ss, si);
      bad |= rerank_one(X, N, D, Q + j * D, si, kappa, k, out_s + j * k, out_id + j * k);
      free(ss);
      free(si);
    }
    free(qp);
    free(s);
    free(v);
  }
  return bad;
}

/* ------------------------------------------------------------------------------------ */
/* Scalar quantisation of the reduced rows (reading R4).                                  */
/* ------------------------------------------------------------------------------------ */

static uint32_t f32_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}
static float bits_f32(uint32_t u) {
  float f;
  memcpy(&f, &u, 4);
  return f;
}

/* BF16: sign, 8 exponent bits, 7 stored mantissa bits -- the top half of an FP32 word.  */
/* Round to nearest, ties to even, on the 16 discarded bits.                              */
void glvo_bf16_encode(const float* in, int64_t n, uint16_t* out) {
  for (int64_t t = 0; t < n; ++t) {
    const uint32_t u = f32_bits(in[t]);
    if (isnan(in[t])) {
      out[t] = (uint16_t)((u >> 16) | 0x0040u); /* keep sign, force a quiet NaN */
      continue;
    }
    const uint32_t hi = u >> 16, lo = u & 0xFFFFu;
    uint32_t r = hi;
    if (lo > 0x8000u || (lo == 0x8000u && (hi & 1u))) r = hi + 1u; /* carries into exponent */
    out[t] = (uint16_t)r;
  }
}

void glvo_bf16_decode(const uint16_t* in, int64_t n, double* out) {
  for (int64_t t = 0; t < n; ++t) out[t] = (double)bits_f32((uint32_t)in[t] << 16);
}

/* FP8 E4M3 (OCP 8-bit floating point, "fn" variant): sign bit, 4 exponent bits with      */
/* bias 7, 3 mantissa bits; exponent field 0 is subnormal (m/8 * 2^-6); S.1111.111 is NaN; */
/* no infinities; largest finite magnitude 1.75 * 2^8 = 448.                              */
static double e4m3_value(uint8_t code) {
  const int s = code >> 7, e = (code >> 3) & 0xF, m = code & 7;
  if (e == 15 && m == 7) return NAN;
  double mag = (e == 0) ? ldexp((double)m / 8.0, -6) : ldexp(1.0 + (double)m / 8.0, e - 7);
  return s ? -mag : mag;
}

void glvo_e4m3_decode(const uint8_t* in, int64_t n, double* out) {
  for (int64_t t = 0; t < n; ++t) out[t] = e4m3_value(in[t]);
}

/* Nearest finite E4M3 value, ties to the even code, saturating at +-448; NaN -> 0x7F.    */
/* Magnitude codes 0..126 are strictly increasing in value, so a binary search over them  */
/* finds the two neighbours of |v|.                                                       */
static uint8_t e4m3_encode_one(double v) {
  if (isnan(v)) return 0x7F;
  const uint8_t sign = (v < 0.0 || (v == 0.0 && signbit(v))) ? 0x80 : 0x00;
  const double a = fabs(v);
  if (a >= 448.0) return (uint8_t)(sign | 0x7E);
  int lo = 0, hi = 126; /* invariant: value(lo) <= a < value(hi) */
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (e4m3_value((uint8_t)mid) <= a) lo = mid;
    else hi = mid;
  }
  const double dlo = a - e4m3_value((uint8_t)lo), dhi = e4m3_value((uint8_t)hi) - a;
  int code;
  if (dlo < dhi) code = lo;
  else if (dhi < dlo) code = hi;
  else code = (lo % 2 == 0) ? lo : hi;
  return (uint8_t)(sign | code);
}

void glvo_e4m3_encode(const double* in, int64_t n, uint8_t* out) {
  for (int64_t t = 0; t < n; ++t) out[t] = e4m3_encode_one(in[t]);
}

/* Per-vector FP8 quantisation of FP32 rows (reading R4).  x is rows x d FP32.            */
void glvo_quantize_fp8_rows(const float* x, int64_t rows, int32_t d, uint8_t* codes,
                            float* scales) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < rows; ++i) {
    float mx = 0.0f;
    for (int32_t r = 0; r < d; ++r) {
      const float a = fabsf(x[i * d + r]);
      if (a > mx) mx = a;
    }
    const float s = (float)((double)mx / 448.0); /* = IEEE fp32 division mx / 448 */
    scales[i] = s;
    for (int32_t r = 0; r < d; ++r) {
      if (s == 0.0f) {
        codes[i * d + r] = 0;
        continue;
      }
      const float y = (float)((double)x[i * d + r] / (double)s); /* = fp32 division */
      codes[i * d + r] = e4m3_encode_one((double)y);
    }
  }
}

/* ------------------------------------------------------------------------------------ */
/* Inner-product approximation loss of Section 2.1 (the LeanVec problem) restricted to    */
/* GleanVec pairs (Section 4.1): for pairs p = (q_p, x_p) with x_p in cluster c_p,        */
/*   r_p = <q_p, x_p> - <A_{c_p} q_p, B_{c_p} x_p>,   loss = sum_p r_p^2,                 */
/*   dloss/dA_c = -2 sum_{p: c_p = c} r_p (B_c x_p) q_p^T,                                 */
/*   dloss/dB_c = -2 sum_{p: c_p = c} r_p (A_c q_p) x_p^T.                                 */
/* Pairs are given by index: q = Q[qi[p]], x = X[xi[p]], cluster = tags[xi[p]].            */
/* gA, gB (C x d x D, may be NULL) are overwritten.  Returns the loss.                     */
/* ------------------------------------------------------------------------------------ */
double glvo_pair_loss_grad(const float* Q, const float* X, int32_t D, const uint16_t* tags,
                           const float* A, const float* B, int32_t C, int32_t d,
                           const int32_t* qi, const int32_t* xi, int64_t P, double* gA,
                           double* gB) {
  const int64_t msize = (int64_t)C * d * D;
  if (gA) memset(gA, 0, sizeof(double) * (size_t)msize);
  if (gB) memset(gB, 0, sizeof(double) * (size_t)msize);
  double* aq = (double*)malloc(sizeof(double) * (size_t)d);
  double* bx = (double*)malloc(sizeof(double) * (size_t)d);
  double loss = 0.0;
  for (int64_t p = 0; p < P; ++p) {
    const float* q = Q + (int64_t)qi[p] * D;
    const float* x = X + (int64_t)xi[p] * D;
    const int64_t c = tags[xi[p]];
    double t = 0.0;
    for (int32_t k = 0; k < D; ++k) t += (double)q[k] * (double)x[k];
    double s = 0.0;
    for (int32_t r = 0; r < d; ++r) {
      double va = 0.0, vb = 0.0;
      for (int32_t k = 0; k < D; ++k) {
        va += (double)A[(c * d + r) * D + k] * (double)q[k];
        vb += (double)B[(c * d + r) * D + k] * (double)x[k];
      }
      aq[r] = va;
      bx[r] = vb;
      s += va * vb;
    }
    const double res = t - s;
    loss += res * res;
    for (int32_t r = 0; r < d; ++r)
      for (int32_t k = 0; k < D; ++k) {
        if (gA) gA[(c * d + r) * D + k] += -2.0 * res * bx[r] * (double)q[k];
        if (gB) gB[(c * d + r) * D + k] += -2.0 * res * aq[r] * (double)x[k];
      }
  }
  free(aq);
  free(bx);
  return loss;
}

/* Second moment K = sum_v v v^T of a set of D-vectors (Section 3.2 summary statistics),  */
/* optionally restricted to the rows with tags == cluster (cluster < 0: all rows).        */
void glvo_second_moment(const float* V, int64_t n, int32_t D, const uint16_t* tags,
                        int32_t cluster, double* K) {
#pragma omp parallel for schedule(static)
  for (int32_t a = 0; a < D; ++a)
    for (int32_t b = 0; b < D; ++b) {
      double v = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        if (cluster >= 0 && tags[i] != cluster) continue;
        v += (double)V[i * D + a] * (double)V[i * D + b];
      }
      K[(int64_t)a * D + b] = v;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Spherical k-means, Appendix A: the M-step mu_c = sum_{i: c_i = c} x_i / ||...||_2      */
/* (rows of X are taken as given; the caller normalises them).  A cluster with no member  */
/* (or a zero sum) keeps its previous landmark.  counts (may be NULL) receives |X_c|.     */
/* ------------------------------------------------------------------------------------ */
void glvo_kmeans_update(const float* X, int64_t N, int32_t D, const uint16_t* tags, int32_t C,
                        const float* mu_in, double* mu_out, int64_t* counts) {
  double* sum = (double*)calloc((size_t)C * (size_t)D, sizeof(double));
  int64_t* cnt = (int64_t*)calloc((size_t)C, sizeof(int64_t));
  for (int64_t i = 0; i < N; ++i) {
    const int64_t c = tags[i];
    if (c >= C) continue;
    cnt[c] += 1;
    for (int32_t k = 0; k < D; ++k) sum[c * D + k] += (double)X[i * D + k];
  }
  for (int64_t c = 0; c < C; ++c) {
    double nrm = 0.0;
    for (int32_t k = 0; k < D; ++k) nrm += sum[c * D + k] * sum[c * D + k];
    nrm = sqrt(nrm);
    for (int32_t k = 0; k < D; ++k)
      mu_out[c * D + k] = (cnt[c] > 0 && nrm > 0.0) ? sum[c * D + k] / nrm : (double)mu_in[c * D + k];
    if (counts) counts[c] = cnt[c];
  }
  free(sum);
  free(cnt);
}

/* Spherical k-means objective of Appendix A: sum_i <x_i, mu_{c_i}>. */
double glvo_spherical_objective(const float* X, int64_t N, int32_t D, const float* mu, const uint16_t* tags) {
  double obj = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double v = 0.0;
    for (int32_t k = 0; k < D; ++k) v += (double)X[i * D + k] * (double)mu[(int64_t)tags[i] * D + k];
    obj += v;
  }
  return obj;
}
