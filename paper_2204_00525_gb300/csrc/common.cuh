// Internal declarations shared by the FiGaRo CUDA translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "figaro.h"

namespace fig {

constexpr int kMaxKeys = 8;
constexpr int kMaxChildren = 8;
constexpr int kWarp = 32;

// ------------------------------------------------------------------ device error word
// Kernels never trap: they record the first failure in a device int and return.
__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ uint64_t shr64(uint64_t x, int s) { return s >= 64 ? 0ull : (x >> s); }
__device__ __forceinline__ uint64_t shl64(uint64_t x, int s) { return s >= 64 ? 0ull : (x << s); }
__device__ __forceinline__ uint64_t mask64(int bits) {
  return bits >= 64 ? ~0ull : ((1ull << bits) - 1ull);
}

// ------------------------------------------------------------------ warp / block reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the whole block; every thread returns the total.  `red` holds >= 33 doubles
// of shared memory.  Contains two __syncthreads().
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    T t = lane < nw ? red[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  T r = red[32];
  return r;
}

// ------------------------------------------------------------------ checked uint64 arithmetic
// Join counts (§5) are exact integers; a product or sum that leaves 64 bits is reported.
__device__ __forceinline__ uint64_t mul_chk(uint64_t a, uint64_t b, int* err) {
  if (__umul64hi(a, b) != 0ull) { set_error(err, FIGARO_ERR_OVERFLOW); return ~0ull; }
  return a * b;
}

// ------------------------------------------------------------------ launch helpers
inline unsigned grid_for(int64_t n, int threads, int64_t cap = 1 << 20) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// ------------------------------------------------------------------ scan primitives (scan.cu)
// Inclusive prefix sum over n_max elements, of which only the first *n_dev (or n_max if
// n_dev is null) are live.  `tmp` must hold scan_tmp_elems(n_max) elements of T.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;
inline int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }
inline int64_t scan_tmp_elems(int64_t n) { return scan_tiles(n) + 1; }

// Flags for the scans that compute group ids.
enum ScanInput : int {
  SCAN_PLAIN_I32 = 0,    // in[i]
  SCAN_KEY_CHANGE = 1,   // 1 if i == 0 or key[i] >> shift != key[i-1] >> shift (uint64 keys)
  SCAN_PLAIN_U64 = 2     // in[i] (uint64)
};

struct ScanSrc {
  int kind;
  const void* in;
  int shift;             // for SCAN_KEY_CHANGE
};

// out[i] = sum_{t <= i} src(t) for i < n; T is int32_t or uint64_t.
template <typename T>
void scan_inclusive(const ScanSrc& src, T* out, int64_t n_max, const int32_t* n_dev, T* tmp,
                    cudaStream_t st, int64_t* launches);
// Exclusive prefix sums of n_max int32 elements (all live).
void scan_exclusive_i32(const ScanSrc& src, int32_t* out, int64_t n_max, int32_t* tmp, cudaStream_t st,
                        int64_t* launches);

}  // namespace fig
