// score_dev.cuh -- device-side body of the gather-score (Algorithm 4, procedure
// inner-product; Eq. GleanVec approximation, Section 4), shared by the stand-alone scoring
// kernel and the fused score + top-kappa kernel so both compute bit-identical scores.
//
// A group of G lanes scores one candidate: the lanes issue all of their 16-byte loads of
// the reduced row (NCH each) before any arithmetic, so a warp keeps 32 x NCH x 16 bytes in
// flight; partial dots are combined with xor-shuffles inside the group.  Rows are decoded in
// registers: FP32 as is, BF16 by shifting into the high half of an FP32 word.  FP8-e4m3 codes
// are converted two at a time to f16 (exact: every e4m3 value is an f16 value) and multiplied
// with mixed-precision FMAs (f16 x f16 products, FP32 accumulation) against the projected
// query held as two f16 terms per element, q * 2^sigma_c = hi + lo (22 significant bits; the
// power of two 2^sigma_c per cluster keeps both terms in f16's normal range).  The cluster's
// 2^-sigma_c and the row scale are applied once to the finished dot.
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

// Four FP8-e4m3 codes (the bytes of x, element 0 in the low byte) against the projected-query
// terms of the same four elements, q = [hi(0,1), hi(2,3), lo(0,1), lo(2,3)] as f16 pairs:
// sh += sum_e x_e * hi_e, sl += sum_e x_e * lo_e, element by element in order (each product
// exact, each sum rounded to FP32).
GLV_DEV void fp8_word_dot(uint32_t x, float4 q, float& sh, float& sl) {
  asm("{\n\t"
      ".reg .b16 c01, c23, x0, x1, x2, x3, h0, h1, h2, h3, l0, l1, l2, l3;\n\t"
      ".reg .b32 p01, p23;\n\t"
      "mov.b32 {c01, c23}, %2;\n\t"
      "cvt.rn.f16x2.e4m3x2 p01, c01;\n\t"
      "cvt.rn.f16x2.e4m3x2 p23, c23;\n\t"
      "mov.b32 {x0, x1}, p01;\n\t"
      "mov.b32 {x2, x3}, p23;\n\t"
      "mov.b32 {h0, h1}, %3;\n\t"
      "mov.b32 {h2, h3}, %4;\n\t"
      "mov.b32 {l0, l1}, %5;\n\t"
      "mov.b32 {l2, l3}, %6;\n\t"
      "fma.rn.f32.f16 %0, x0, h0, %0;\n\t"
      "fma.rn.f32.f16 %1, x0, l0, %1;\n\t"
      "fma.rn.f32.f16 %0, x1, h1, %0;\n\t"
      "fma.rn.f32.f16 %1, x1, l1, %1;\n\t"
      "fma.rn.f32.f16 %0, x2, h2, %0;\n\t"
      "fma.rn.f32.f16 %1, x2, l2, %1;\n\t"
      "fma.rn.f32.f16 %0, x3, h3, %0;\n\t"
      "fma.rn.f32.f16 %1, x3, l3, %1;\n\t"
      "}"
      : "+f"(sh), "+f"(sl)
      : "r"(x), "r"(__float_as_uint(q.x)), "r"(__float_as_uint(q.y)), "r"(__float_as_uint(q.z)),
        "r"(__float_as_uint(q.w)));
}

// Dot product of one 16-byte chunk of a reduced row with the matching projected-query
// elements.  The projected query of a cluster is laid out in shared memory as EPC/4
// sub-blocks of float4 (stride sbs), each sub-block holding the same 4-element slice of every
// chunk: element (chunk ch, e) sits at float4 index (e / 4) * sbs + ch.  Lanes that read
// consecutive chunks of one row read consecutive float4 words.  When a quarter-warp serves two
// candidates, the odd one (sw = 1) walks the sub-blocks in swapped order (BF16: 1,0; FP8:
// 2,3,0,1), which with the padded sub-block stride puts the two candidates' reads 64 bytes
// apart modulo 128 -- in opposite halves of the banks.  The FP32 sum follows the walk order,
// so a candidate's result depends on the parity of its position in its group, which every
// kernel derives from its offset in the candidate list.
template <int DT>
GLV_DEV float dot_chunk(uint4 v, const float* qrow, int ch, int sbs, int sw) {
  const float4* q4 = reinterpret_cast<const float4*>(qrow);
  if constexpr (DT == GLV_F32) {
    float4 a = q4[ch];
    return a.x * __uint_as_float(v.x) + a.y * __uint_as_float(v.y) + a.z * __uint_as_float(v.z) +
           a.w * __uint_as_float(v.w);
  } else {
    // odd lane groups walk the two halves of the chunk in swapped order; the words are picked
    // with selects (a runtime index into a register array would put it in local memory)
    const uint32_t x0 = sw ? v.z : v.x, x1 = sw ? v.w : v.y;
    const uint32_t x2 = sw ? v.x : v.z, x3 = sw ? v.y : v.w;
    const float4* qa = q4 + sw * sbs + ch;
    const float4* qb = q4 + (sw ^ 1) * sbs + ch;
    float s = 0.f;
    if constexpr (DT == GLV_BF16) {
      // sub-block 0 holds elements 0..3 (words 0, 1), sub-block 1 elements 4..7 (words 2, 3)
      const float4 a = *qa, b = *qb;
      s = fmaf(a.x, __uint_as_float(x0 << 16), s);
      s = fmaf(a.y, __uint_as_float(x0 & 0xffff0000u), s);
      s = fmaf(a.z, __uint_as_float(x1 << 16), s);
      s = fmaf(a.w, __uint_as_float(x1 & 0xffff0000u), s);
      s = fmaf(b.x, __uint_as_float(x2 << 16), s);
      s = fmaf(b.y, __uint_as_float(x2 & 0xffff0000u), s);
      s = fmaf(b.z, __uint_as_float(x3 << 16), s);
      s = fmaf(b.w, __uint_as_float(x3 & 0xffff0000u), s);
    } else {
      // sub-block t holds the terms of the four elements of word t as f16 pairs
      // [hi(0,1), hi(2,3), lo(0,1), lo(2,3)]; odd groups take the words in the order 2, 3, 0, 1.
      // The hi and lo products accumulate in two chains, added at the end.
      const uint32_t xs[4] = {x0, x1, x2, x3};
      float sl = 0.f;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float4 a = q4[(t ^ (sw << 1)) * sbs + ch];
        fp8_word_dot(xs[t], a, s, sl);
      }
      s += sl;
    }
    return s;
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

// FP8 rows: the per-cluster factors 2^-sigma_c follow the C rows of projected views.
GLV_DEV float* qp_scales(const ScoreArgs& a, float* qs) { return qs + (size_t)a.C * a.qstride; }
GLV_DEV const float* qp_scales(const ScoreArgs& a, const float* qs) { return qs + (size_t)a.C * a.qstride; }

// FP8 rows: turn the FP32 projected views staged in the sub-block layout into the f16 term
// pairs dot_chunk reads, in place, one warp per cluster row (rows with seen[c] == 0 skipped
// when seen is given).  sigma_c = 14 - floor(log2 max_e |q_c,e|) (clamped to +-126) puts the
// largest |q| * 2^sigma_c in [2^14, 2^15); hi = f16(q 2^sigma_c), lo = f16(q 2^sigma_c - hi)
// (the difference is exact in FP32), so hi + lo holds q 2^sigma_c to 22 significant bits.
// Each 16-byte slot holding elements 4t..4t+3 of a chunk becomes
// [hi(0,1), hi(2,3), lo(0,1), lo(2,3)], and 2^-sigma_c goes to qp_scales.
GLV_DEV void split_qp_fp8(const ScoreArgs& a, float* qs, const uint8_t* seen) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int slots = a.nch * 4;  // 16-byte slots per row: 4 sub-blocks of nch chunks
  float* qsc = qp_scales(a, qs);
  for (int c = warp; c < a.C; c += nwarps) {
    if (seen && !seen[c]) continue;
    float4* row = reinterpret_cast<float4*>(qs + (size_t)c * a.qstride);
    float m = 0.f;
    for (int t = lane; t < slots; t += 32) {
      const int u = t / a.nch, ch = t - u * a.nch;
      const float4 v = row[u * a.sbs + ch];
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    m = warp_max(m);
    int sigma = 0;
    if (m > 0.f && m <= 3.4e38f) {
      const int e = (int)((__float_as_uint(m) >> 23) & 0xffu) - 127;  // floor(log2 m); -127 if subnormal
      sigma = min(126, max(-126, 14 - e));
    }
    const float up = __uint_as_float((uint32_t)(127 + sigma) << 23);
    const float down = __uint_as_float((uint32_t)(127 - sigma) << 23);
    for (int t = lane; t < slots; t += 32) {
      const int u = t / a.nch, ch = t - u * a.nch;
      const float4 v = row[u * a.sbs + ch];
      const float f[4] = {v.x * up, v.y * up, v.z * up, v.w * up};
      __half h[4], l[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        h[k] = __float2half_rn(f[k]);
        l[k] = __float2half_rn(f[k] - __half2float(h[k]));
      }
      float4 o;
      o.x = __uint_as_float((uint32_t)__half_as_ushort(h[0]) | ((uint32_t)__half_as_ushort(h[1]) << 16));
      o.y = __uint_as_float((uint32_t)__half_as_ushort(h[2]) | ((uint32_t)__half_as_ushort(h[3]) << 16));
      o.z = __uint_as_float((uint32_t)__half_as_ushort(l[0]) | ((uint32_t)__half_as_ushort(l[1]) << 16));
      o.w = __uint_as_float((uint32_t)__half_as_ushort(l[2]) | ((uint32_t)__half_as_ushort(l[3]) << 16));
      row[u * a.sbs + ch] = o;
    }
    if (lane == 0) qsc[c] = down;
  }
}

// Stage the C projected views of query j into shared memory in the sub-block layout of
// dot_chunk (rows of a.qstride floats; elements d..dpad-1 are zero); FP8 rows then get their
// f16 term pairs (split_qp_fp8).  Called by the whole CTA.
template <int DT>
GLV_DEV void stage_qp(const ScoreArgs& a, int64_t j, float* qs) {
  stage_qp_f32<DT>(a, j, qs);
  if constexpr (DT == GLV_FP8_E4M3) {
    __syncthreads();
    split_qp_fp8(a, qs, nullptr);
  }
}

// 16-byte asynchronous copy global -> shared that bypasses L1 (cp.async.cg); src_bytes < 16
// fills the rest of the 16 bytes with zeros.  Completes at cp_async_wait_all.
GLV_DEV void cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}

// Whether stage_qp_async can stage this problem's projected views (the float4 layout; FP8
// rows need the f16 terms computed, so they are staged by stage_qp).
template <int DT>
GLV_DEV bool qp_async_ok(const ScoreArgs& a) {
  return DT != GLV_FP8_E4M3 && (a.d & 3) == 0 && (reinterpret_cast<uintptr_t>(a.Qp) & 15) == 0;
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

template <int DT, int G, int NCH, bool PIPE, class Sink>
GLV_DEV void finish_row(const ScoreArgs& a, const RowLoad<DT, G, NCH, PIPE>& r, const float* qs, int gl, int sw,
                        Sink& sink) {
  const bool ok = r.ok && r.tag < a.C;
  const float* qrow = qs + (ok ? r.tag : 0) * a.qstride;
  float acc = 0.f;
#pragma unroll
  for (int t = 0; t < NCH; ++t) {
    const int ch = gl + t * G;
    if (ch < a.nch) {
      uint4 x = r.v[t];
      if (ch == a.nch - 1 && a.tail < 16) x = keep_bytes(x, a.tail);
      acc += dot_chunk<DT>(x, qrow, ch, a.sbs, sw);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (r.in && gl == 0) {
    float s;
    if (!ok) {
      s = -INFINITY;
      report(a.d_status, GLV_ERR_BAD_ID);
    } else if constexpr (DT == GLV_FP8_E4M3) {
      s = (acc * qp_scales(a, qs)[r.tag]) * r.sc;
    } else {
      s = acc;
    }
    sink(r.p, s);
  }
}

template <int DT, int G, int NCH, bool PIPE, class Sink>
GLV_DEV void score_range(const ScoreArgs& a, const float* qs, int64_t b0, int64_t b1, Sink sink) {
  constexpr int GPW = kWarp / G;
  const int lane = threadIdx.x & (kWarp - 1);
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int g = lane / G, gl = lane % G;
  const int64_t step = (int64_t)nwarps * GPW;
  int64_t base = b0 + (int64_t)warp * GPW;
  // the id of the next candidate is loaded one iteration ahead, so the row loads of an
  // iteration do not wait for an id round trip
  int64_t id_next = (base + g < b1) ? (int64_t)__ldg(a.ids + base + g) : 0;
  if constexpr (!PIPE) {
    for (; base < b1; base += step) {
      const int64_t p = base + g;
      const int64_t id = id_next;
      id_next = (p + step < b1) ? (int64_t)__ldg(a.ids + p + step) : 0;
      RowLoad<DT, G, NCH, PIPE> r;
      load_row(a, r, p, b1, id, gl);
      finish_row(a, r, qs, gl, g & 1, sink);
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
      finish_row(a, cur, qs, gl, g & 1, sink);
      cur = nxt;
    }
  }
}

// Default lanes per candidate per store type: 8 for FP32 and BF16 rows, 4 for FP8 rows (the
// choices the autotuner made on every measured workload).
template <int DT>
constexpr int default_group() {
  return (DT == GLV_F32) ? 8 : (DT == GLV_BF16 ? 8 : 4);
}

}  // namespace glv
