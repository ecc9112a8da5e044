// common.cuh -- small device helpers shared by the libglv kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/glv.h"

#define GLV_DEV __device__ __forceinline__

namespace glv {

constexpr int kWarp = 32;

// Record the first device-side error in the caller's status word (NULL allowed).
GLV_DEV void report(int32_t* d_status, int32_t code) {
  if (d_status) atomicCAS(reinterpret_cast<int*>(d_status), 0, code);
}

// 16-byte streaming load through the non-coherent path without L1 allocation: rows of the
// reduced store and of X are touched once per candidate, so L1 would only be polluted.
// L2 keeps its default policy (rows are re-visited by other queries).
GLV_DEV uint4 ld_stream_v4(const void* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

GLV_DEV float ld_stream_f32(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

GLV_DEV float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Order-preserving map of an FP32 score to uint32 (larger key = better score).  NaN maps
// to 0, below every number including -inf (whose key is 0x007FFFFF); -0.0 maps to the key
// of +0.0 so that the two zeros tie (and are then ordered by id), as they compare equal.
GLV_DEV uint32_t score_key(float s) {
  uint32_t u = __float_as_uint(s);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0u;  // NaN
  if (u == 0x80000000u) u = 0u;                      // -0.0 -> +0.0
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

GLV_DEV float key_score(uint32_t k) {
  if (k == 0u) return __uint_as_float(0x7fc00000u);
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// 8-byte asynchronous copy global -> shared (cp.async; completes at cp_async_wait_all).
GLV_DEV void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
GLV_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Hint: bring `bytes` (a multiple of 16) at the 16-byte aligned global address p into L2.
GLV_DEV void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Hint: bring the 128-byte line holding p into L2 (no register, no completion to wait for).
GLV_DEV void prefetch_l2_line(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Ids as unsigned keys that grow as the (signed) id shrinks: ties between equal scores go to
// the smaller id, negative (invalid) ids included, in every selection path.
GLV_DEV uint32_t id_rank(int32_t id) { return ~((uint32_t)id ^ 0x80000000u); }
GLV_DEV int32_t id_from_rank(uint32_t r) { return (int32_t)(~r ^ 0x80000000u); }

// (score, id) ordering: a ranks before b.
GLV_DEV bool ranks_before(uint32_t ka, int32_t ia, uint32_t kb, int32_t ib) {
  return ka > kb || (ka == kb && ia < ib);
}

}  // namespace glv
