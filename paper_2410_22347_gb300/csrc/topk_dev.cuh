// topk_dev.cuh -- exact per-query top-kappa selection in one CTA (Algorithm 1: the main
// step hands kappa candidates to the exact post-processing), shared by the stand-alone
// top-k kernel and the fused score + top-kappa kernel.
//
// Scores are mapped to order-preserving uint32 keys; a 4-pass radix select (8-bit digits,
// most significant first) finds the kappa-th largest key K*.  Every key above K* is taken;
// among keys equal to K* the smallest ids are taken, found by a second radix select on ~id
// only when the tie group is larger than what is left.  The kappa winners are then placed by
// rank ((key desc, id asc) ordering), which needs no sort network and is exact.  Histograms
// use warp-aggregated shared-memory atomics (__match_any_sync), since similar scores pile
// into one bucket.
#pragma once

#include "common.cuh"

namespace glv {

constexpr int kTopkThreads = 256;
constexpr int kTopkCache = 8192;

// Radix histogram and counters; the kappa selected (key, id) pairs live in caller-provided
// shared memory (kappa entries each), so the footprint follows kappa.
struct TopkSmem {
  uint32_t hist[256];
  uint32_t bucket, above, count, n_eq;
  uint32_t* sel_key;
  int32_t* sel_id;
};

// After the histogram is complete: find the digit b whose bucket holds the `want`-th
// largest element (counting from the top), and how many elements lie in buckets above b.
// Executed by warp 0; results land in S.bucket / S.above.
GLV_DEV void find_bucket(TopkSmem& S, uint32_t want) {
  const int lane = threadIdx.x & 31;
  uint32_t c[8];
  uint32_t sum = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    c[t] = S.hist[255 - (lane * 8 + t)];
    sum += c[t];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  const uint32_t excl = incl - sum;
  const unsigned hit = __ballot_sync(0xffffffffu, incl >= want);
  const int first = __ffs(hit) - 1;
  if (lane == first) {
    uint32_t run = excl;
    for (int t = 0; t < 8; ++t) {
      if (run + c[t] >= want) {
        S.bucket = 255 - (lane * 8 + t);
        S.above = run;
        break;
      }
      run += c[t];
    }
  }
}

// Radix select over the keys key_of(p), p in [0, L) with take(p): returns the want-th
// largest key (1-based, want <= number of such p) and sets *rem to how many elements equal
// to it belong to the top `want`.
template <class KeyOf, class Take>
GLV_DEV uint32_t radix_select(TopkSmem& S, int64_t L, uint32_t want, KeyOf key_of, Take take,
                              uint32_t* rem) {
  uint32_t prefix = 0, mask = 0;
  const int lane = threadIdx.x & 31;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int t = threadIdx.x; t < 256; t += blockDim.x) S.hist[t] = 0;
    __syncthreads();
    for (int64_t b = 0; b < L; b += blockDim.x) {
      const int64_t p = b + threadIdx.x;
      uint32_t digit = 0xffffffffu;
      if (p < L && take(p)) {
        const uint32_t k = key_of(p);
        if ((k & mask) == prefix) digit = (k >> shift) & 255u;
      }
      const unsigned peers = __match_any_sync(0xffffffffu, digit);
      if (digit != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&S.hist[digit], __popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < 32) find_bucket(S, want);
    __syncthreads();
    want -= S.above;
    prefix |= S.bucket << shift;
    mask |= 255u << shift;
    __syncthreads();
  }
  *rem = want;
  return prefix;
}

// Select and write the sorted top kappa of L candidates: key_of(p) / id_of(p) give the key
// and id of candidate p in [0, L).  Writes kappa (score, id) pairs to out_s / out_id, padded
// with (-inf, -1).  All threads of the CTA must call it.
template <class KeyOf, class IdOf>
GLV_DEV void select_topk(TopkSmem& S, int64_t L, int kappa, KeyOf key_of, IdOf id_of, float* out_s,
                         int32_t* out_id) {
  if (threadIdx.x == 0) {
    S.count = 0;
    S.n_eq = 0;
  }
  __syncthreads();
  if (L <= kappa) {
    for (int64_t p = threadIdx.x; p < L; p += blockDim.x) {
      S.sel_key[p] = key_of(p);
      S.sel_id[p] = id_of(p);
    }
    if (threadIdx.x == 0) S.count = (uint32_t)L;
  } else {
    uint32_t need_eq = 0;
    const uint32_t kstar =
        radix_select(S, L, (uint32_t)kappa, key_of, [](int64_t) { return true; }, &need_eq);
    // everything strictly above K*: exactly kappa - need_eq entries
    for (int64_t p = threadIdx.x; p < L; p += blockDim.x) {
      const uint32_t k = key_of(p);
      if (k > kstar) {
        const uint32_t slot = atomicAdd(&S.count, 1u);
        if (slot < (uint32_t)kappa) {
          S.sel_key[slot] = k;
          S.sel_id[slot] = id_of(p);
        }
      } else if (k == kstar) {
        atomicAdd(&S.n_eq, 1u);
      }
    }
    __syncthreads();
    // the tie group at K*: all of it, or its need_eq smallest ids
    uint32_t id_cut = 0;
    const bool all_ties = (S.n_eq == need_eq);
    if (!all_ties) {
      uint32_t rem2 = 0;
      id_cut = radix_select(S, L, need_eq, [&](int64_t p) { return ~(uint32_t)id_of(p); },
                            [&](int64_t p) { return key_of(p) == kstar; }, &rem2);
    }
    for (int64_t p = threadIdx.x; p < L; p += blockDim.x) {
      if (key_of(p) != kstar) continue;
      const int32_t id = id_of(p);
      if (all_ties || ~(uint32_t)id >= id_cut) {
        const uint32_t slot = atomicAdd(&S.count, 1u);
        if (slot < (uint32_t)kappa) {  // only repeated (id, score) pairs can overflow
          S.sel_key[slot] = kstar;
          S.sel_id[slot] = id;
        }
      }
    }
  }
  __syncthreads();
  const int n = min((int)S.count, kappa);
  // place by rank; identical entries are ordered by slot so every rank is written once
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const uint32_t ke = S.sel_key[e];
    const int32_t ie = S.sel_id[e];
    int rank = 0;
    for (int f = 0; f < n; ++f) {
      const uint32_t kf = S.sel_key[f];
      const int32_t idf = S.sel_id[f];
      rank += (ranks_before(kf, idf, ke, ie) || (kf == ke && idf == ie && f < e)) ? 1 : 0;
    }
    out_s[rank] = key_score(ke);
    out_id[rank] = ie;
  }
  for (int e = n + threadIdx.x; e < kappa; e += blockDim.x) {
    out_s[e] = -INFINITY;
    out_id[e] = -1;
  }
}

}  // namespace glv
