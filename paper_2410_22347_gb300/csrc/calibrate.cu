// calibrate.cu -- gather calibration kernel (no counterpart in the paper): reads, for every
// entry of a candidate-id list, the whole row of a row-major store and writes one float per
// entry (the row's words summed as floats), with no other arithmetic.  It moves the same
// bytes in the same random order as the gather-score, so its bandwidth is the practical
// ceiling of that access pattern on this GPU (random rows cost whole 128-byte lines of
// DRAM access, partial lines included), next to the copy bandwidth of streaming reads.
//
// Layout: G = 8 lanes per row, U = 4 rows in flight per lane group (32 rows per warp), each
// lane loading up to NCH 16-byte chunks per row with streaming (L1 no-allocate) loads; a
// grid-stride loop over the entries with 4 CTAs of 256 threads per SM.
#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace glv {

template <int NCH>
__global__ void __launch_bounds__(256) gather_rows_kernel(const uint8_t* __restrict__ rows, int64_t row_bytes,
                                                          int64_t n_rows, const int32_t* __restrict__ ids,
                                                          int64_t n_ids, float* __restrict__ out,
                                                          int32_t* __restrict__ d_status) {
  constexpr int G = 8, U = 4, GPW = 32 / G;
  const int lane = threadIdx.x & 31, g = lane / G, gl = lane % G;
  const int nch = (int)(row_bytes / 16);
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  for (int64_t base = w * GPW * U; base < n_ids; base += warps * GPW * U) {
    uint4 v[U][NCH];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = base + u * GPW + g;
      const int64_t id = p < n_ids ? (int64_t)__ldg(ids + p) : -1;
      ok[u] = id >= 0 && id < n_rows;
      const uint8_t* row = rows + (ok[u] ? id : 0) * row_bytes;
#pragma unroll
      for (int t = 0; t < NCH; ++t) {
        const int ch = gl + t * G;
        v[u][t] = (ok[u] && ch < nch) ? ld_stream_v4(row + (int64_t)ch * 16) : make_uint4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float s = 0.f;
#pragma unroll
      for (int t = 0; t < NCH; ++t)
        s += (__uint_as_float(v[u][t].x) + __uint_as_float(v[u][t].y)) +
             (__uint_as_float(v[u][t].z) + __uint_as_float(v[u][t].w));
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const int64_t p = base + u * GPW + g;
      if (gl == 0 && p < n_ids) {
        if (!ok[u]) report(d_status, GLV_ERR_BAD_ID);
        out[p] = ok[u] ? s : 0.f;
      }
    }
  }
}

cudaError_t launch_gather_rows(const void* rows, int64_t row_bytes, int64_t n_rows, const int32_t* ids,
                               int64_t n_ids, float* out, int32_t* d_status, int num_sms, cudaStream_t st) {
  const int nch = (int)(row_bytes / 16);
  const unsigned grid = (unsigned)num_sms * 4;
  const uint8_t* r = static_cast<const uint8_t*>(rows);
#define GLV_GATHER(N)                                                                             \
  if (nch <= 8 * (N)) {                                                                           \
    gather_rows_kernel<N><<<grid, 256, 0, st>>>(r, row_bytes, n_rows, ids, n_ids, out, d_status); \
    return cudaGetLastError();                                                                    \
  }
  GLV_GATHER(1)
  GLV_GATHER(2)
  GLV_GATHER(3)
  GLV_GATHER(4)
  GLV_GATHER(6)
  GLV_GATHER(8)
#undef GLV_GATHER
  return cudaErrorInvalidValue;
}

// Self-check of the bounded device-side waits: one thread waits, with the given limit, on an
// mbarrier that nothing will complete (one arrival expected, none made) -- the situation of a
// tensor-core pipeline whose producer has stopped.  The wait gives up after limit_ns, the
// kernel records GLV_ERR_TIMEOUT in the status word and returns normally.
__global__ void bounded_wait_kernel(uint64_t limit_ns, int32_t* d_status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    abort_flag = 0;
    if (!tc::mbar_wait(&bar, 0, &abort_flag, limit_ns)) report(d_status, GLV_ERR_TIMEOUT);
  }
}

cudaError_t launch_bounded_wait(uint64_t limit_ns, int32_t* d_status, cudaStream_t st) {
  bounded_wait_kernel<<<1, 32, 0, st>>>(limit_ns, d_status);
  return cudaGetLastError();
}

}  // namespace glv
