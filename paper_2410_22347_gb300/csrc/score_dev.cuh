// score_dev.cuh -- device-side body of the gather-score (Algorithm 4, procedure
// inner-product; Eq. GleanVec approximation, Section 4), shared by the stand-alone scoring
// kernel, the fused score + top-kappa kernel and the lazy kernel, so all compute bit-identical
// scores.
//
// A group of G lanes scores one candidate: the lanes issue all of their 16-byte loads of the
// reduced row (NCH each) before any arithmetic, so a warp keeps 32 x NCH x 16 bytes in flight;
// partial dots are combined with xor-shuffles inside the group.  Rows are decoded in
// registers -- FP32 as is, BF16 by shifting into the high half of an FP32 word, FP8-e4m3 two
// codes at a time into f16 (exact: every e4m3 value is an f16 value) and then FP32 -- and
// multiplied with the FP32 projected query by packed two-way FMAs (FP32 accumulation).  The
// row scale of an FP8 row is applied once to the finished dot.
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace glv {

template <int DT>
struct Elem;
template <>
struct Elem<GLV_F32> {
  static constexpr int kPerChunk = 4;
  static constexpr int kBytes = 4;
};
template <>
struct Elem<GLV_BF16> {
  static constexpr int kPerChunk = 8;
  static constexpr int kBytes = 2;
};
template <>
struct Elem<GLV_FP8_E4M3> {
  static constexpr int kPerChunk = 16;
  static constexpr int kBytes = 1;
};

// Four FP8-e4m3 codes (the bytes of x, element 0 in the low byte) against four FP32 query
// elements q: each pair of codes becomes an f16 pair (hardware conversion, exact), each f16 an
// FP32 value (exact), and two packed FMAs accumulate elements 0, 1 into (acc.x, acc.y) and
// then elements 2, 3 into the same pair.
GLV_DEV void fp8_word_dot(uint32_t x, float4 q, float2& acc) {
  float f0, f1, f2, f3;
  asm("{\n\t"
      ".reg .b16 c01, c23, h0, h1, h2, h3;\n\t"
      ".reg .b32 p01, p23;\n\t"
      "mov.b32 {c01, c23}, %4;\n\t"
      "cvt.rn.f16x2.e4m3x2 p01, c01;\n\t"
      "cvt.rn.f16x2.e4m3x2 p23, c23;\n\t"
      "mov.b32 {h0, h1}, p01;\n\t"
      "mov.b32 {h2, h3}, p23;\n\t"
      "cvt.f32.f16 %0, h0;\n\t"
      "cvt.f32.f16 %1, h1;\n\t"
      "cvt.f32.f16 %2, h2;\n\t"
      "cvt.f32.f16 %3, h3;\n\t"
      "}"
      : "=f"(f0), "=f"(f1), "=f"(f2), "=f"(f3)
      : "r"(x));
  acc = __ffma2_rn(make_float2(q.x, q.y), make_float2(f0, f1), acc);
  acc = __ffma2_rn(make_float2(q.z, q.w), make_float2(f2, f3), acc);
}

// Whether the odd lane groups of a quarter-warp walk the sub-blocks of a chunk in swapped
// order (dot_chunk).  BF16 rows do: that keeps the two candidates' shared-memory reads in
// opposite halves of the banks.  For FP8 rows the four selects per chunk cost more than the
// conflicts they avoid (measured), so FP8 rows keep the natural order and their view rows are
// laid out so that rows of consecutive clusters start in opposite bank halves
// (qp_qstride): two candidates then conflict only when their clusters' rows share a half.
template <int DT>
constexpr bool odd_group_swaps() {
  return DT == GLV_BF16;
}

// Dot product of one 16-byte chunk of a reduced row with the matching projected-query
// elements, accumulated into a pair of FP32 partial sums (acc.x + acc.y is the dot once every
// chunk has been added; even elements go to acc.x, odd ones to acc.y).
// The projected query of a cluster is laid out in shared memory as EPC/4
// sub-blocks of float4 (stride sbs), each sub-block holding the same 4-element slice of every
// chunk: element (chunk ch, e) sits at float4 index (e / 4) * sbs + ch.  Lanes that read
// consecutive chunks of one row read consecutive float4 words.  For BF16 rows, when a
// quarter-warp serves two candidates, the odd one (sw = 1) walks the two sub-blocks in
// swapped order, which with the padded sub-block stride puts the two candidates' reads 64
// bytes apart modulo 128 -- in opposite halves of the banks.  The FP32 sums follow the walk
// order, so a BF16 candidate's result depends on the parity of its position in its group,
// which every kernel derives from its offset in the candidate list.  (sw is 0 for the other
// store types: see odd_group_swaps.)
template <int DT>
GLV_DEV void dot_chunk(float2& acc, uint4 v, const float* qrow, int ch, int sbs, int sw) {
  const float4* q4 = reinterpret_cast<const float4*>(qrow);
  if constexpr (DT == GLV_F32) {
    const float4 a = q4[ch];
    acc = __ffma2_rn(make_float2(a.x, a.y), make_float2(__uint_as_float(v.x), __uint_as_float(v.y)), acc);
    acc = __ffma2_rn(make_float2(a.z, a.w), make_float2(__uint_as_float(v.z), __uint_as_float(v.w)), acc);
  } else {
    // odd lane groups walk the two halves of the chunk in swapped order; the words are picked
    // with selects (a runtime index into a register array would put it in local memory)
    const uint32_t x0 = sw ? v.z : v.x, x1 = sw ? v.w : v.y;
    const uint32_t x2 = sw ? v.x : v.z, x3 = sw ? v.y : v.w;
    if constexpr (DT == GLV_BF16) {
      // sub-block 0 holds elements 0..3 (words 0, 1), sub-block 1 elements 4..7 (words 2, 3);
      // the low half of a word is the even element
      const float4 a = q4[sw * sbs + ch], b = q4[(sw ^ 1) * sbs + ch];
      acc = __ffma2_rn(make_float2(a.x, a.y), make_float2(__uint_as_float(x0 << 16), __uint_as_float(x0 & 0xffff0000u)),
                       acc);
      acc = __ffma2_rn(make_float2(a.z, a.w), make_float2(__uint_as_float(x1 << 16), __uint_as_float(x1 & 0xffff0000u)),
                       acc);
      acc = __ffma2_rn(make_float2(b.x, b.y), make_float2(__uint_as_float(x2 << 16), __uint_as_float(x2 & 0xffff0000u)),
                       acc);
      acc = __ffma2_rn(make_float2(b.z, b.w), make_float2(__uint_as_float(x3 << 16), __uint_as_float(x3 & 0xffff0000u)),
                       acc);
    } else {
      // sub-block t holds the four elements of word t (with sw = 1 the words would be taken in
      // the order 2, 3, 0, 1)
      const uint32_t xs[4] = {x0, x1, x2, x3};
#pragma unroll
      for (int t = 0; t < 4; ++t) fp8_word_dot(xs[t], q4[(t ^ (sw << 1)) * sbs + ch], acc);
    }
  }
}

// Zero the bytes at and beyond `nbytes` (0 < nbytes < 16) of a 16-byte chunk.
GLV_DEV uint4 keep_bytes(uint4 v, int nbytes) {
  uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int b = nbytes - 4 * t;
    if (b <= 0) w[t] = 0u;
    else if (b < 4) w[t] &= (1u << (8 * b)) - 1u;
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Stage the C projected views of query j into shared memory in the sub-block layout of
// dot_chunk as FP32 values (rows of a.qstride floats; elements d..dpad-1 are zero).
template <int DT>
GLV_DEV void stage_qp_f32(const ScoreArgs& a, int64_t j, float* qs) {
  constexpr int EPC = Elem<DT>::kPerChunk;
  const float* qj = a.Qp + j * (int64_t)a.C * a.d;
  const int dpad = a.nch * EPC;
  if ((a.d & 3) == 0 && (reinterpret_cast<uintptr_t>(a.Qp) & 15) == 0) {
    // float4 at a time (the four elements of a float4 share a chunk and a sub-block slot),
    // kU loads in flight per thread before their stores
    constexpr int kU = 4;
    const int q4 = dpad >> 2, total4 = a.C * q4;
    for (int t0 = threadIdx.x; t0 < total4; t0 += kU * blockDim.x) {
      float4 v[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int t = t0 + u * blockDim.x;
        const int c = t / q4, r = (t - c * q4) * 4;
        v[u] = (t < total4 && r < a.d) ? *reinterpret_cast<const float4*>(qj + (int64_t)c * a.d + r)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < total4) {
          const int c = t / q4, r = (t - c * q4) * 4;
          const int ch = r / EPC, e = r - ch * EPC;
          *reinterpret_cast<float4*>(qs + c * a.qstride + ((e >> 2) * a.sbs + ch) * 4) = v[u];
        }
      }
    }
    return;
  }
  const int total = a.C * dpad;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int c = t / dpad, r = t - c * dpad;
    const int ch = r / EPC, e = r - ch * EPC;
    qs[c * a.qstride + ((e >> 2) * a.sbs + ch) * 4 + (e & 3)] = (r < a.d) ? qj[(int64_t)c * a.d + r] : 0.f;
  }
}

GLV_DEV float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Stage the C projected views of query j into shared memory in the sub-block layout of
// dot_chunk (rows of a.qstride floats; elements d..dpad-1 are zero).  Called by the whole CTA.
template <int DT>
GLV_DEV void stage_qp(const ScoreArgs& a, int64_t j, float* qs) {
  stage_qp_f32<DT>(a, j, qs);
}

// 16-byte asynchronous copy global -> shared that bypasses L1 (cp.async.cg); src_bytes < 16
// fills the rest of the 16 bytes with zeros.  Completes at cp_async_wait_all.
GLV_DEV void cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}

// Whether stage_qp_async can stage this problem's projected views (the float4 layout).
template <int DT>
GLV_DEV bool qp_async_ok(const ScoreArgs& a) {
  return (a.d & 3) == 0 && (reinterpret_cast<uintptr_t>(a.Qp) & 15) == 0;
}

// stage_qp's float4 path as asynchronous copies: every float4 of the query's C projected views
// (and the zero padding up to dpad) goes straight from global memory to its slot of the
// sub-block layout, without passing through registers; the copies complete at
// cp_async_wait_all.  Needs qp_async_ok(a).
template <int DT>
GLV_DEV void stage_qp_async(const ScoreArgs& a, int64_t j, float* qs) {
  constexpr int EPC = Elem<DT>::kPerChunk;
  const float* qj = a.Qp + j * (int64_t)a.C * a.d;
  const int q4 = (a.nch * EPC) >> 2, total4 = a.C * q4;
  for (int t = threadIdx.x; t < total4; t += blockDim.x) {
    const int c = t / q4, r = (t - c * q4) * 4;
    const int ch = r / EPC, e = r - ch * EPC;
    const bool in = r < a.d;
    cp_async16(qs + c * a.qstride + ((e >> 2) * a.sbs + ch) * 4, in ? qj + (int64_t)c * a.d + r : qj, in ? 16 : 0);
  }
}

// Score candidates p in [b0, b1) with the CTA's warps; sink(p, score) receives each score
// (from lane 0 of the candidate's lane group).  A bad id or tag scores -inf and is reported.
// PIPE: the row loads of the next candidate are issued before the current one is computed
// (twice the registers for row data, a continuous stream of loads per warp).
template <int DT, int G, int NCH, bool PIPE>
struct RowLoad {
  uint4 v[NCH];
  int tag;
  float sc;
  bool ok, in;
  int64_t p;
};

template <int DT, int G, int NCH, bool PIPE>
GLV_DEV void load_row(const ScoreArgs& a, RowLoad<DT, G, NCH, PIPE>& r, int64_t p, int64_t b1, int64_t id,
                      int gl) {
  r.p = p;
  r.in = p < b1;
  r.ok = r.in && id >= 0 && id < a.N;
  r.tag = r.ok ? (int)__ldg(a.tags + id) : 0;
  const uint8_t* row = a.Xred + id * a.row_stride;
#pragma unroll
  for (int t = 0; t < NCH; ++t) {
    const int ch = gl + t * G;
    r.v[t] = (r.ok && ch < a.nch) ? ld_stream_v4(row + (int64_t)ch * 16) : make_uint4(0, 0, 0, 0);
  }
  r.sc = 1.f;
  if constexpr (DT == GLV_FP8_E4M3) r.sc = r.ok ? __ldg(a.scales + id) : 0.f;
}

template <int DT, int G, int NCH, bool PIPE, bool TAIL, class Sink>
GLV_DEV void finish_row(const ScoreArgs& a, const RowLoad<DT, G, NCH, PIPE>& r, const float* qs, int gl, int sw,
                        Sink& sink) {
  const bool ok = r.ok && r.tag < a.C;
  const float* qrow = qs + (ok ? r.tag : 0) * a.qstride;
  float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int t = 0; t < NCH; ++t) {
    const int ch = gl + t * G;
    if (ch < a.nch) {
      uint4 x = r.v[t];
      if constexpr (TAIL) {
        if (ch == a.nch - 1) x = keep_bytes(x, a.tail);
      }
      dot_chunk<DT>(acc2, x, qrow, ch, a.sbs, sw);
    }
  }
  float acc = acc2.x + acc2.y;
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (r.in && gl == 0) {
    float s;
    if (!ok) {
      s = -INFINITY;
      report(a.d_status, GLV_ERR_BAD_ID);
    } else if constexpr (DT == GLV_FP8_E4M3) {
      s = acc * r.sc;
    } else {
      s = acc;
    }
    sink(r.p, s);
  }
}

template <int DT, int G, int NCH, bool PIPE, bool TAIL, bool PF, class Sink>
GLV_DEV void score_range_t(const ScoreArgs& a, const float* qs, int64_t b0, int64_t b1, Sink& sink) {
  constexpr int GPW = kWarp / G;
  const int lane = threadIdx.x & (kWarp - 1);
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int g = lane / G, gl = lane % G;
  const int sw = odd_group_swaps<DT>() ? (g & 1) : 0;
  const int64_t step = (int64_t)nwarps * GPW;
  int64_t base = b0 + (int64_t)warp * GPW;
  // the id of the next candidate is loaded one iteration ahead, so the row loads of an
  // iteration do not wait for an id round trip
  int64_t id_next = (base + g < b1) ? (int64_t)__ldg(a.ids + base + g) : 0;
  if constexpr (!PIPE && PF) {
    // prefetch: ids are loaded two iterations ahead, and each lane of a group asks L2 for one
    // 128-byte line of the next candidate's row one iteration before its loads (a hint: it
    // holds no register and no L1 slot, so the SM keeps twice the row bytes on their way --
    // faster where part of the store sits in L2, slower where every row comes from DRAM; the
    // autotuner chooses)
    int64_t id_next2 = (base + step + g < b1) ? (int64_t)__ldg(a.ids + base + step + g) : 0;
    const int row_bytes = a.nch * 16;
    for (; base < b1; base += step) {
      const int64_t p = base + g;
      const int64_t id = id_next;
      id_next = id_next2;
      id_next2 = (p + 2 * step < b1) ? (int64_t)__ldg(a.ids + p + 2 * step) : 0;
      if (p + step < b1 && id_next >= 0 && id_next < a.N && gl * 128 < row_bytes)
        prefetch_l2_line(a.Xred + id_next * a.row_stride + gl * 128);
      RowLoad<DT, G, NCH, PIPE> r;
      load_row(a, r, p, b1, id, gl);
      finish_row<DT, G, NCH, PIPE, TAIL>(a, r, qs, gl, sw, sink);
    }
  } else if constexpr (!PIPE) {
    for (; base < b1; base += step) {
      const int64_t p = base + g;
      const int64_t id = id_next;
      id_next = (p + step < b1) ? (int64_t)__ldg(a.ids + p + step) : 0;
      RowLoad<DT, G, NCH, PIPE> r;
      load_row(a, r, p, b1, id, gl);
      finish_row<DT, G, NCH, PIPE, TAIL>(a, r, qs, gl, sw, sink);
    }
  } else {
    if (base >= b1) return;
    RowLoad<DT, G, NCH, PIPE> cur, nxt;
    {
      const int64_t p = base + g;
      const int64_t id = id_next;
      id_next = (p + step < b1) ? (int64_t)__ldg(a.ids + p + step) : 0;
      load_row(a, cur, p, b1, id, gl);
    }
    for (; base < b1; base += step) {
      const int64_t pn = base + step + g;
      if (base + step < b1) {
        const int64_t id = id_next;
        id_next = (pn + step < b1) ? (int64_t)__ldg(a.ids + pn + step) : 0;
        load_row(a, nxt, pn, b1, id, gl);
      }
      finish_row<DT, G, NCH, PIPE, TAIL>(a, cur, qs, gl, sw, sink);
      cur = nxt;
    }
  }
}

// Rows whose data end inside a 16-byte chunk (d * element bytes not a multiple of 16) need the
// bytes past the data masked in that chunk, and the L2 prefetch of the next row is an option;
// the loop is compiled in three forms and the kernel-uniform choice is made once, so rows that
// end on a chunk boundary pay nothing for the mask and launches without the prefetch nothing
// for it.  (Rows with a partial last chunk take the form without the prefetch.)
// ALLOW_PF: whether the kernel carries the prefetch form at all (the 512-thread fused kernel
// does not: the third form of the loop cost its other forms 13-18% through code generation).
template <int DT, int G, int NCH, bool PIPE, bool ALLOW_PF = true, class Sink>
GLV_DEV void score_range(const ScoreArgs& a, const float* qs, int64_t b0, int64_t b1, Sink sink) {
  if (a.tail < 16) {
    score_range_t<DT, G, NCH, PIPE, true, false>(a, qs, b0, b1, sink);  // (rare: no prefetch form)
    return;
  }
  if constexpr (ALLOW_PF && !PIPE) {
    if (a.prefetch) {
      score_range_t<DT, G, NCH, PIPE, false, true>(a, qs, b0, b1, sink);
      return;
    }
  }
  score_range_t<DT, G, NCH, PIPE, false, false>(a, qs, b0, b1, sink);
}

// Default lanes per candidate per store type: 8 for FP32 and BF16 rows, 4 for FP8 rows (the
// choices the autotuner made on every measured workload).
template <int DT>
constexpr int default_group() {
  return (DT == GLV_F32) ? 8 : (DT == GLV_BF16 ? 8 : 4);
}

}  // namespace glv
