// score_bulk.cuh -- gather-score body that moves candidate rows with bulk asynchronous copies
// (cp.async.bulk, the TMA engine's 1-D form) into a per-warp ring of shared-memory slots.
//
// Row bytes in flight no longer occupy registers: each warp keeps NS batches of RB rows in
// flight (lane r of the warp loads candidate r's id and issues the single bulk copy of that
// row; one mbarrier per slot counts the bytes), so an SM can keep far more bytes in flight
// than register-resident loads allow.  The dot products then read the rows from shared
// memory with exactly the chunk order and shuffle tree of score_range(), so the scores are
// bit-identical to the register-gather kernels for the same (G, NCH).
// Every mbarrier wait is bounded (tc.cuh); on a timeout the warp stops issuing, waits
// (bounded) for its copies still in flight, and the CTA reports GLV_ERR_TIMEOUT.
#pragma once

#include "score_dev.cuh"
#include "tc.cuh"

namespace glv {

GLV_DEV void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
      : "memory");
}

GLV_DEV uint4 lds128(const uint8_t* p) { return *reinterpret_cast<const uint4*>(p); }

// Shared-memory bytes of the rings of `warps` warps.
inline size_t bulk_ring_bytes(int warps, int NS, int RB, int row_bytes) {
  return (size_t)warps * NS * RB * row_bytes;
}

// Warp-uniform bounded wait: lane 0 waits, the outcome is broadcast, and every lane then
// observes the completed phase itself (acquire), so all lanes may read the copied bytes.
GLV_DEV bool mbar_wait_warp(uint64_t* bar, uint32_t parity, volatile int* abort) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = tc::mbar_wait(bar, parity, abort) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok) (void)tc::mbar_try_wait(bar, parity);
  return ok != 0;
}

// Score candidates p in [b0, b1) with this warp's ring (NS slots of RB <= 32 rows of
// row_bytes each) and mbarriers bars[0..NS) (initialised with count 1).  Batches are dealt
// round-robin to the CTA's warps.  Returns false if a wait timed out (abort is then set).
template <int DT, int G, int NCH, int NS, class Sink>
GLV_DEV bool score_range_bulk(const ScoreArgs& a, const float* qs, uint8_t* ring, uint64_t* bars, int RB, int64_t b0,
                              int64_t b1, Sink& sink, volatile int* abort) {
  constexpr int GPW = kWarp / G;
  const int PASSES = (RB + GPW - 1) / GPW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int g = lane / G, gl = lane % G;
  const int rb = a.nch * 16;
  const int64_t nb_all = (b1 - b0 + RB - 1) / RB;
  // this warp's batches: warp, warp + nwarps, ...
  const int64_t nb = nb_all > warp ? (nb_all - warp + nwarps - 1) / nwarps : 0;

  int tag_s[NS];
  float sc_s[NS];
  bool ok_s[NS], in_s[NS], pend_s[NS];
  uint32_t par_s[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    tag_s[s] = 0;
    sc_s[s] = 0.f;
    ok_s[s] = in_s[s] = pend_s[s] = false;
    par_s[s] = 0;
  }

  auto issue = [&](int s, int64_t i) {  // batch i of this warp into slot s
    const int64_t p = b0 + (warp + i * nwarps) * RB + lane;
    const bool in = lane < RB && p < b1;
    const int64_t id = in ? (int64_t)__ldg(a.ids + p) : -1;
    const bool okid = in && id >= 0 && id < a.N;
    const unsigned m = __ballot_sync(0xffffffffu, okid);
    if (lane == 0) tc::mbar_arrive_expect_tx(&bars[s], (uint32_t)__popc(m) * (uint32_t)rb);
    __syncwarp();
    if (okid) bulk_g2s(ring + ((size_t)s * RB + lane) * rb, a.Xred + id * a.row_stride, (uint32_t)rb, &bars[s]);
    tag_s[s] = okid ? (int)__ldg(a.tags + id) : 0;
    if constexpr (DT == GLV_FP8_E4M3) sc_s[s] = okid ? __ldg(a.scales + id) : 0.f;
    ok_s[s] = okid;
    in_s[s] = in;
    pend_s[s] = true;
  };

  bool good = true;
#pragma unroll
  for (int s = 0; s < NS; ++s)
    if (s < nb) issue(s, s);

  for (int64_t i0 = 0; good && i0 < nb; i0 += NS) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int64_t i = i0 + s;
      if (i >= nb) break;
      if (!mbar_wait_warp(&bars[s], par_s[s], abort)) {
        good = false;
        break;
      }
      pend_s[s] = false;
      par_s[s] ^= 1u;
      const uint8_t* slot = ring + (size_t)s * RB * rb;
      const int64_t pbase = b0 + (warp + i * nwarps) * RB;
#pragma unroll 1
      for (int pass = 0; pass < PASSES; ++pass) {
        const int r = pass * GPW + g;
        const int rs = r < RB ? r : 0;
        const int tag = __shfl_sync(0xffffffffu, tag_s[s], rs);
        const bool okr = __shfl_sync(0xffffffffu, ok_s[s] ? 1 : 0, rs) != 0;
        const bool inr = (__shfl_sync(0xffffffffu, in_s[s] ? 1 : 0, rs) != 0) && r < RB;
        float sc = 1.f;
        if constexpr (DT == GLV_FP8_E4M3) sc = __shfl_sync(0xffffffffu, sc_s[s], rs);
        const bool ok = okr && inr && tag < a.C;
        const float* qrow = qs + (ok ? tag : 0) * a.qstride;
        const uint8_t* row = slot + (size_t)rs * rb;
        float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < NCH; ++t) {
          const int ch = gl + t * G;
          if (ch < a.nch) {
            uint4 x = ok ? lds128(row + ch * 16) : make_uint4(0, 0, 0, 0);
            if (ch == a.nch - 1 && a.tail < 16) x = keep_bytes(x, a.tail);
            dot_chunk<DT>(acc2, x, qrow, ch, a.sbs, odd_group_swaps<DT>() ? (g & 1) : 0);
          }
        }
        float acc = acc2.x + acc2.y;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (inr && gl == 0) {
          float sv;
          if (!ok) {
            sv = -INFINITY;
            report(a.d_status, GLV_ERR_BAD_ID);
          } else if constexpr (DT == GLV_FP8_E4M3) {
            sv = acc * sc;
          } else {
            sv = acc;
          }
          sink(pbase + r, sv);
        }
      }
      __syncwarp();  // every lane is done with the slot before it is refilled
      if (i + NS < nb) issue(s, i + NS);
    }
  }
  if (!good) {  // no bulk copy may still be writing into this CTA's shared memory at exit
    volatile int no_abort = 0;
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (pend_s[s]) mbar_wait_warp(&bars[s], par_s[s], &no_abort);
  }
  return good;
}

}  // namespace glv
