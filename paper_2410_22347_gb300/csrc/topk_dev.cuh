// topk_dev.cuh -- exact per-query top-kappa selection in one CTA (Algorithm 1: the main
// step hands kappa candidates to the exact post-processing), shared by the stand-alone
// top-k kernel and the fused score + top-kappa kernel.
//
// Scores are mapped to order-preserving uint32 keys; a 4-pass radix select (8-bit digits,
// most significant first) finds the kappa-th largest key K*.  Every key above K* is taken;
// among keys equal to K* the smallest ids are taken, found by a second radix select on id_rank(id)
// only when the tie group is larger than what is left.  Histograms use warp-aggregated
// shared-memory atomics (__match_any_sync), since similar scores pile into one bucket.
//
// Long lists that do not fit the CTA's key cache (kappa <= 256) are filtered first: the radix
// select runs on a 256-key sample of the list to find a threshold T whose expected number of
// list keys >= T is about 2 kappa, one pass copies the keys >= T (with their ids) into the then
// unused key-cache region, and the selection runs there.  If fewer than kappa keys are >= T
// (or the copy overflows), the selection runs on the whole list instead, so the result never
// depends on the sample: when at least kappa keys are >= T, the kappa-th largest key is >= T
// and every key that can be selected (ties included) is in the region.
//
// Lists whose keys are cached in the region with at most 8 per thread skip the block-wide
// radix passes: a per-warp threshold (warp_threshold_filter) that provably leaves at least
// kappa keys, one packing pass, and a rank count over the (typically 1.5 kappa, at most one
// per thread) survivors, which writes the top kappa already sorted.  Wide tie groups take the
// radix path.
//
// The kappa winners are sorted by (key desc, id asc).  After a filtered selection, up to 256
// of them go through a bitonic network across the CTA's threads on the packed 64-bit value
// key << 32 | id_rank(id) (exchanging through the key-cache region, free by then); otherwise each
// entry counts the entries that rank before it.
#pragma once

#include "common.cuh"

namespace glv {

constexpr int kTopkThreads = 256;
constexpr int kTopkCache = 8192;

// Radix histogram and counters.  The kappa selected (key, id) pairs live in caller-provided
// shared memory (kappa entries each), so the footprint follows kappa; `region` (region_words
// 32-bit words, at least 512, 8-byte aligned) is the caller's key cache, reused as scratch.
struct TopkSmem {
  uint32_t hist[256];
  uint32_t bucket, above, count, n_eq, fill, thr;
  uint32_t* sel_key;
  int32_t* sel_id;
  uint32_t* region;
  int region_words;
};

constexpr int kFilterMinList = 1024;  // shorter lists are selected directly
constexpr int kFilterSample = 256;
constexpr int kFilterMaxKappa = 256;

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

// Exact top-kappa of the keys key_of(p), p in [0, L), L > kappa, into S.sel_key / S.sel_id
// (unordered, S.count entries).
template <class KeyOf, class IdOf>
GLV_DEV void select_unordered(TopkSmem& S, int64_t L, int kappa, KeyOf key_of, IdOf id_of) {
  uint32_t need_eq = 0;
  const uint32_t kstar = radix_select(S, L, (uint32_t)kappa, key_of, [](int64_t) { return true; }, &need_eq);
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
    id_cut = radix_select(S, L, need_eq, [&](int64_t p) { return id_rank(id_of(p)); },
                          [&](int64_t p) { return key_of(p) == kstar; }, &rem2);
  }
  for (int64_t p = threadIdx.x; p < L; p += blockDim.x) {
    if (key_of(p) != kstar) continue;
    const int32_t id = id_of(p);
    if (all_ties || id_rank(id) >= id_cut) {
      const uint32_t slot = atomicAdd(&S.count, 1u);
      if (slot < (uint32_t)kappa) {  // only repeated (id, score) pairs can overflow
        S.sel_key[slot] = kstar;
        S.sel_id[slot] = id;
      }
    }
  }
}

// Threshold T from a sample of kFilterSample keys at evenly spread positions: the r-th largest
// sample key, r chosen so that about 2 kappa + 32 list keys are expected to be >= T.  Returns
// 0 (no filtering) when the list is too short for that to pay.
template <class KeyOf>
GLV_DEV uint32_t sample_threshold(TopkSmem& S, int64_t L, int kappa, KeyOf key_of) {
  const int m = kFilterSample;
  const int64_t want_hits = 2 * (int64_t)kappa + 32;
  const int r = (int)((want_hits * m + L - 1) / L);
  if (r < 1 || r > m / 2) return 0u;
  uint32_t rem = 0;
  return radix_select(S, m, (uint32_t)r, [&](int64_t t) { return key_of(t * L / m); },
                      [](int64_t) { return true; }, &rem);
}

// Copy the keys >= T and their ids into the key-cache region (keys in the first half, ids in
// the second); true if it holds between kappa and its capacity (S.fill entries), false if
// the caller must select from the whole list.
template <class KeyOf, class IdOf>
GLV_DEV bool filter_to_region(TopkSmem& S, int64_t L, int kappa, uint32_t T, KeyOf key_of, IdOf id_of) {
  const int cap = S.region_words / 2;
  uint32_t* bk = S.region;
  int32_t* bi = reinterpret_cast<int32_t*>(S.region + cap);
  if (threadIdx.x == 0) S.fill = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // kU keys per thread are loaded before any is used, so their (L2) round trips overlap
  constexpr int kU = 4;
  for (int64_t b = 0; b < L; b += kU * blockDim.x) {
    uint32_t kk[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t p = b + u * blockDim.x + threadIdx.x;
      kk[u] = p < L ? key_of(p) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t p = b + u * blockDim.x + threadIdx.x;
      const bool pass = p < L && kk[u] >= T;
      const unsigned bal = __ballot_sync(0xffffffffu, pass);
      if (bal == 0) continue;
      uint32_t base = 0;
      if (lane == __ffs(bal) - 1) base = atomicAdd(&S.fill, (uint32_t)__popc(bal));
      base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
      if (pass) {
        const uint32_t slot = base + __popc(bal & ((1u << lane) - 1u));
        if (slot < (uint32_t)cap) {
          bk[slot] = kk[u];
          bi[slot] = id_of(p);
        }
      }
    }
  }
  __syncthreads();
  return S.fill >= (uint32_t)kappa && S.fill <= (uint32_t)cap;
}

// Descending sort of 8 keys held in registers (a 19-comparator network).
GLV_DEV void sort8_desc(uint32_t (&v)[8]) {
  constexpr int kNet[19][2] = {{0, 2}, {1, 3}, {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}, {0, 1}, {2, 3},
                               {4, 5}, {6, 7}, {2, 4}, {3, 5}, {1, 4}, {3, 6}, {1, 2}, {3, 4}, {5, 6}};
#pragma unroll
  for (int c = 0; c < 19; ++c) {
    const uint32_t x = v[kNet[c][0]], y = v[kNet[c][1]];
    v[kNet[c][0]] = max(x, y);
    v[kNet[c][1]] = min(x, y);
  }
}

// Keys cached in the region, at most kWarpThrKeys per thread: a threshold T that at least
// kappa of the L keys reach, found with one barrier.  With W warps, each warp pops the
// r = ceil(kappa / W) largest of its own keys (every lane's keys sorted in registers, one
// warp max-reduction per pop), and T is the smallest of the W warps' r-th largest keys, so
// each warp holds r keys >= T and at least W r >= kappa list keys reach T (on random scores
// about 1.5 kappa do).  One pass then packs every key >= T with its id
// (key << 32 | id_rank(id)) into the region as 64-bit values and returns how many there are
// (they hold the top kappa, ties included).  When that is more than one per thread (a wide
// tie group), the keys are put back in the region and -1 is returned, for the radix path.
// The region holds at least 2 blockDim.x words.  S.thr (all ones) and S.fill (0) are set by
// the caller before its barrier.
constexpr int kWarpThrKeys = 8;

template <class KeyOf, class IdOf>
GLV_DEV int warp_threshold_filter(TopkSmem& S, int L, int kappa, KeyOf key_of, IdOf id_of) {
  const int t = threadIdx.x, lane = t & 31, nt = blockDim.x;
  uint32_t v[kWarpThrKeys];
#pragma unroll
  for (int i = 0; i < kWarpThrKeys; ++i) {
    const int p = t + i * nt;
    v[i] = p < L ? key_of(p) : 0u;
  }
  sort8_desc(v);
  const int nw = nt >> 5;
  const int r = (kappa + nw - 1) / nw;
  uint32_t tw = 0;
  for (int s = 0; s < r; ++s) {
    const uint32_t m = __reduce_max_sync(0xffffffffu, v[0]);
    const bool win = lane == __ffs(__ballot_sync(0xffffffffu, v[0] == m)) - 1;
#pragma unroll
    for (int j = 0; j < kWarpThrKeys - 1; ++j) v[j] = win ? v[j + 1] : v[j];
    v[kWarpThrKeys - 1] = win ? 0u : v[kWarpThrKeys - 1];
    tw = m;
  }
  if (lane == 0) atomicMin(&S.thr, tw);
  // the keys again, in list order (the sorted copy is spent), before the region is reused
  uint32_t k[kWarpThrKeys];
#pragma unroll
  for (int i = 0; i < kWarpThrKeys; ++i) {
    const int p = t + i * nt;
    k[i] = p < L ? key_of(p) : 0u;
  }
  __syncthreads();  // T is final, and every key is in registers: the region is free
  const uint32_t T = S.thr;
  uint32_t tot = 0;
#pragma unroll
  for (int i = 0; i < kWarpThrKeys; ++i)
    tot += __popc(__ballot_sync(0xffffffffu, t + i * nt < L && k[i] >= T));
  uint32_t base = 0;
  if (lane == 0 && tot) base = atomicAdd(&S.fill, tot);
  base = __shfl_sync(0xffffffffu, base, 0);
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t cap = (uint32_t)nt;
  uint64_t* xs = reinterpret_cast<uint64_t*>(S.region);
#pragma unroll
  for (int i = 0; i < kWarpThrKeys; ++i) {
    const bool pass = t + i * nt < L && k[i] >= T;
    const unsigned bal = __ballot_sync(0xffffffffu, pass);
    if (pass) {
      const uint32_t slot = base + __popc(bal & lt);
      if (slot < cap) xs[slot] = ((uint64_t)k[i] << 32) | id_rank(id_of(t + i * nt));
    }
    base += __popc(bal);
  }
  __syncthreads();
  const uint32_t n = S.fill;
  if (n <= cap) return (int)n;
#pragma unroll
  for (int i = 0; i < kWarpThrKeys; ++i) {
    const int p = t + i * nt;
    if (p < L) S.region[p] = k[i];
  }
  __syncthreads();
  return -1;
}

// The top kappa of n (kappa <= n <= blockDim.x) packed values xs, written sorted by (key
// desc, id asc): entry t counts the entries that rank before it (identical entries ordered by
// slot, so every rank is written once) and writes itself when its rank is below kappa.
GLV_DEV void rank_place_packed(const uint64_t* xs, int n, int kappa, float* out_s, int32_t* out_id) {
  const int t = threadIdx.x;
  if (t >= n) return;
  const uint64_t ce = xs[t];
  int above = 0, dup = 0;
  const ulonglong2* x2 = reinterpret_cast<const ulonglong2*>(xs);
  const int n2 = n >> 1;
#pragma unroll 4
  for (int f = 0; f < n2; ++f) {
    const ulonglong2 c = x2[f];
    above += (c.x > ce ? 1 : 0) + (c.y > ce ? 1 : 0);
    dup += (c.x == ce && 2 * f < t ? 1 : 0) + (c.y == ce && 2 * f + 1 < t ? 1 : 0);
  }
  if (n & 1) {
    const uint64_t c = xs[n - 1];
    above += c > ce ? 1 : 0;
    dup += (c == ce && n - 1 < t) ? 1 : 0;
  }
  const int rank = above + dup;
  if (rank < kappa) {
    out_s[rank] = key_score((uint32_t)(ce >> 32));
    out_id[rank] = id_from_rank((uint32_t)ce);
  }
}

// The same with a bitonic network (n <= blockDim.x, blockDim.x a power of two): one packed
// value per thread over the first P = 2^ceil(log2 n) threads, partners closer than 32
// exchanged by warp shuffles and farther ones through xs (whose values are all in registers
// before the first exchange); the first kappa of the descending order are written.  Rank
// counting costs about n^2 / 2 compares, the network P log2(P)^2 / 4 but with a barrier pair
// per stage of stride >= 32: fewer instructions, more latency.
// Threads past n hold 0, which sorts last (and equals the packing of a NaN score with id
// INT32_MAX, so either order gives the same output).  All threads of the CTA must call it.
GLV_DEV void bitonic_place_packed(uint64_t* xs, int n, int kappa, float* out_s, int32_t* out_id) {
  const int t = threadIdx.x;
  int P = 2;
  while (P < n) P <<= 1;
  uint64_t v = t < n ? xs[t] : 0ull;
  __syncthreads();
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      uint64_t o = 0;
      if (stride >= 32) {  // block-uniform branch: every thread reaches the barriers
        if (t < P) xs[t] = v;
        __syncthreads();
        if (t < P) o = xs[t ^ stride];
        __syncthreads();
      } else if (t < ((P + 31) & ~31)) {
        o = __shfl_xor_sync(0xffffffffu, v, stride);
      }
      if (t < P) {
        const bool take_max = ((t & stride) == 0) == ((t & size) == 0);
        const uint64_t mx = v > o ? v : o, mn = v > o ? o : v;
        v = take_max ? mx : mn;
      }
    }
  }
  if (t < kappa) {
    out_s[t] = key_score((uint32_t)(v >> 32));
    out_id[t] = id_from_rank((uint32_t)v);
  }
}

// Descending bitonic network over 32 E packed values held E per lane (element i = lane * E +
// j) in one warp; sizes and strides are template parameters, so every register index is a
// compile-time constant.
template <int E, int SIZE, int STRIDE>
GLV_DEV void warp_bitonic_stage(uint64_t (&v)[E], int lane) {
  if constexpr (STRIDE < E) {
#pragma unroll
    for (int j = 0; j < E; ++j) {
      if ((j & STRIDE) == 0) {
        const int jl = j | STRIDE;
        const bool desc = ((lane * E + j) & SIZE) == 0;
        const uint64_t x = v[j], y = v[jl];
        const bool swap = desc ? (x < y) : (x > y);
        v[j] = swap ? y : x;
        v[jl] = swap ? x : y;
      }
    }
  } else {
    constexpr int lx = STRIDE / E;
    const bool lower = (lane & lx) == 0;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, v[j], lx);
      const bool desc = ((lane * E + j) & SIZE) == 0;
      const uint64_t mx = v[j] > o ? v[j] : o, mn = v[j] > o ? o : v[j];
      v[j] = (lower == desc) ? mx : mn;
    }
  }
  if constexpr (STRIDE > 1) warp_bitonic_stage<E, SIZE, STRIDE / 2>(v, lane);
}

template <int E, int SIZE = 2>
GLV_DEV void warp_bitonic_sort(uint64_t (&v)[E], int lane) {
  warp_bitonic_stage<E, SIZE, SIZE / 2>(v, lane);
  if constexpr (SIZE < 32 * E) warp_bitonic_sort<E, SIZE * 2>(v, lane);
}

// Sort the n (<= 256) selected pairs by (key desc, id asc) -- the packed value key << 32 | id_rank(id)
// descending -- with a bitonic network over the first P = 2^ceil(log2 n) threads of the CTA,
// one element per thread: partners closer than 32 are exchanged by warp shuffles, farther ones
// through xs (256 slots of shared memory that are free at this point).  Writes out_s / out_id.
GLV_DEV void block_sort_write(TopkSmem& S, int n, uint64_t* xs, float* out_s, int32_t* out_id) {
  const int t = threadIdx.x;
  int P = 2;
  while (P < n) P <<= 1;
  uint64_t v = t < n ? ((uint64_t)S.sel_key[t] << 32) | id_rank(S.sel_id[t]) : 0ull;
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      uint64_t o = 0;
      if (stride >= 32) {  // block-uniform branch: every thread reaches the barriers
        if (t < P) xs[t] = v;
        __syncthreads();
        if (t < P) o = xs[t ^ stride];
        __syncthreads();
      } else if (t < ((P + 31) & ~31)) {  // whole warps that hold elements
        o = __shfl_xor_sync(0xffffffffu, v, stride);
      }
      if (t < P) {
        const bool take_max = ((t & stride) == 0) == ((t & size) == 0);
        const uint64_t mx = v > o ? v : o, mn = v > o ? o : v;
        v = take_max ? mx : mn;
      }
    }
  }
  if (t < n) {
    out_s[t] = key_score((uint32_t)(v >> 32));
    out_id[t] = id_from_rank((uint32_t)v);
  }
}

// Select and write the top kappa of L candidates: key_of(p) / id_of(p) give the key and id
// of candidate p in [0, L); `in_region` says whether the keys are the ones cached in S.region
// (else S.region is free).  Writes kappa (score, id) pairs to out_s / out_id, sorted and
// padded with (-inf, -1); with sorted == false, writes the min(L, kappa) selected pairs in no
// particular order (a partial list for a later merge).  network_sort: order more than 256
// threshold survivors with the bitonic network instead of rank counting (the choice of
// instruction-bound callers).  All threads of the CTA must call it.
template <class KeyOf, class IdOf>
GLV_DEV void select_topk(TopkSmem& S, int64_t L, int kappa, bool in_region, KeyOf key_of, IdOf id_of,
                         float* out_s, int32_t* out_id, bool sorted = true, bool network_sort = false) {
  if (threadIdx.x == 0) {
    S.count = 0;
    S.n_eq = 0;
    S.fill = 0;
    S.thr = 0xffffffffu;
  }
  __syncthreads();
  if (L <= kappa) {
    for (int64_t p = threadIdx.x; p < L; p += blockDim.x) {
      S.sel_key[p] = key_of(p);
      S.sel_id[p] = id_of(p);
    }
    if (threadIdx.x == 0) S.count = (uint32_t)L;
  } else {
    bool done = false;
    if (in_region && L <= (int64_t)kWarpThrKeys * blockDim.x && kappa <= kFilterMaxKappa &&
        S.region_words >= 2 * (int)blockDim.x) {
      const int n = warp_threshold_filter(S, (int)L, kappa, key_of, id_of);
      uint64_t* xs = reinterpret_cast<uint64_t*>(S.region);
      if (n >= 0) {
        // kappa <= n <= blockDim.x: every rank below kappa is written (n is block-uniform)
        if (network_sort && n > 256) bitonic_place_packed(xs, n, kappa, out_s, out_id);
        else rank_place_packed(xs, n, kappa, out_s, out_id);
        return;
      }
    }
    if (!done && kappa <= kFilterMaxKappa && L >= kFilterMinList) {
      // lists cached on chip: the dense passes over shared memory are short, so they keep the
      // plain path (the threshold's extra barriers cost more latency than they save)
      const uint32_t T = in_region ? 0u : sample_threshold(S, L, kappa, key_of);
      if (T != 0u) {
        if (filter_to_region(S, L, kappa, T, key_of, id_of)) {
          const uint32_t* bk = S.region;
          const int32_t* bi = reinterpret_cast<const int32_t*>(S.region + S.region_words / 2);
          select_unordered(S, (int64_t)S.fill, kappa, [bk](int64_t p) { return bk[p]; },
                           [bi](int64_t p) { return bi[p]; });
          done = true;
        }
      }
    }
    if (!done) select_unordered(S, L, kappa, key_of, id_of);
  }
  __syncthreads();
  const int n = min((int)S.count, kappa);
  if (!sorted) {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      out_s[e] = key_score(S.sel_key[e]);
      out_id[e] = S.sel_id[e];
    }
    return;
  }
  if (!in_region && n <= 256 && S.region_words >= 512 && blockDim.x >= 256) {
    block_sort_write(S, n, reinterpret_cast<uint64_t*>(S.region), out_s, out_id);
  } else if (n <= S.region_words / 2) {
    // place by rank on the packed value key << 32 | id_rank(id) (descending = key desc, id
    // asc),
    // staged in the key-cache region (free now); identical entries are ordered by slot so
    // every rank is written once
    uint64_t* xs = reinterpret_cast<uint64_t*>(S.region);
    for (int e = threadIdx.x; e < n; e += blockDim.x)
      xs[e] = ((uint64_t)S.sel_key[e] << 32) | id_rank(S.sel_id[e]);
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const uint64_t ce = xs[e];
      int above = 0, dup = 0;
#pragma unroll 4
      for (int f = 0; f < n; ++f) {
        const uint64_t cf = xs[f];
        above += cf > ce ? 1 : 0;
        dup += (cf == ce && f < e) ? 1 : 0;
      }
      const int rank = above + dup;
      out_s[rank] = key_score((uint32_t)(ce >> 32));
      out_id[rank] = id_from_rank((uint32_t)ce);
    }
  } else {
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
  }
  for (int e = n + threadIdx.x; e < kappa; e += blockDim.x) {
    out_s[e] = -INFINITY;
    out_id[e] = -1;
  }
}

}  // namespace glv
