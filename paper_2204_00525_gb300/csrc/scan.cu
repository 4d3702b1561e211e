// Device-wide inclusive prefix sums: reduce tiles, scan the tile sums, scan tiles with
// their offsets.  Sizes may live on the device (groups are counted by earlier kernels),
// so every kernel reads the live length and surplus blocks return at once.
#include "common.cuh"

namespace fig {

template <typename T>
__device__ __forceinline__ T scan_load(const ScanSrc& s, int64_t i) {
  switch (s.kind) {
    case SCAN_KEY_CHANGE: {
      const uint64_t* k = static_cast<const uint64_t*>(s.in);
      if (i == 0) return T(1);
      return shr64(k[i], s.shift) != shr64(k[i - 1], s.shift) ? T(1) : T(0);
    }
    case SCAN_PLAIN_U64: return T(static_cast<const uint64_t*>(s.in)[i]);
    default: return T(static_cast<const int32_t*>(s.in)[i]);
  }
}

__device__ __forceinline__ int64_t live_n(int64_t n_max, const int32_t* n_dev) {
  return n_dev ? (int64_t)(*n_dev) : n_max;
}

// Exclusive scan of one value per thread over the block (blockDim == kScanThreads).
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* warp_tot, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = lane < (kScanThreads / 32) ? warp_tot[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < (kScanThreads / 32)) warp_tot[lane] = wi - w;
    if (lane == (kScanThreads / 32) - 1) *total = wi;
  }
  __syncthreads();
  return warp_tot[warp] + incl - v;
}

template <typename T>
__global__ void k_scan_reduce(ScanSrc src, int64_t n_max, const int32_t* n_dev, T* tile_sum) {
  const int64_t n = live_n(n_max, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  if (base >= n) return;
  __shared__ T red[33];
  T s = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int64_t e = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (e < n) s += scan_load<T>(src, e);
  }
  s = block_sum<T>(s, red);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = s;
}

// One block: exclusive scan of the live tile sums in place.
template <typename T>
__global__ void k_scan_tiles(int64_t n_max, const int32_t* n_dev, T* tile_sum) {
  const int64_t n = live_n(n_max, n_dev);
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  __shared__ T warp_tot[32];
  __shared__ T total;
  T run = 0;
  for (int64_t base = 0; base < nt; base += kScanThreads) {
    int64_t t = base + threadIdx.x;
    T v = t < nt ? tile_sum[t] : T(0);
    T ex = block_excl_scan<T>(v, warp_tot, &total);
    if (t < nt) tile_sum[t] = run + ex;
    run += total;
    __syncthreads();
  }
}

template <typename T>
__global__ void k_scan_apply(ScanSrc src, int64_t n_max, const int32_t* n_dev, const T* tile_off,
                             T* out, int exclusive) {
  const int64_t n = live_n(n_max, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  if (base >= n) return;
  __shared__ T warp_tot[32];
  __shared__ T total;
  T v[kScanItems];
  T s = 0;
  const int64_t first = base + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t e = first + i;
    v[i] = e < n ? scan_load<T>(src, e) : T(0);
    s += v[i];
  }
  T ex = block_excl_scan<T>(s, warp_tot, &total) + tile_off[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t e = first + i;
    const T incl = ex + v[i];
    if (e < n) out[e] = exclusive ? ex : incl;
    ex = incl;
  }
}

template <typename T>
static void scan_any(const ScanSrc& src, T* out, int64_t n_max, const int32_t* n_dev, T* tmp, int exclusive,
                     cudaStream_t st, int64_t* launches) {
  if (n_max <= 0) return;
  const unsigned nt = (unsigned)scan_tiles(n_max);
  k_scan_reduce<T><<<nt, kScanThreads, 0, st>>>(src, n_max, n_dev, tmp);
  k_scan_tiles<T><<<1, kScanThreads, 0, st>>>(n_max, n_dev, tmp);
  k_scan_apply<T><<<nt, kScanThreads, 0, st>>>(src, n_max, n_dev, tmp, out, exclusive);
  if (launches) *launches += 3;
}

template <typename T>
void scan_inclusive(const ScanSrc& src, T* out, int64_t n_max, const int32_t* n_dev, T* tmp,
                    cudaStream_t st, int64_t* launches) {
  scan_any<T>(src, out, n_max, n_dev, tmp, 0, st, launches);
}

void scan_exclusive_i32(const ScanSrc& src, int32_t* out, int64_t n_max, int32_t* tmp, cudaStream_t st,
                        int64_t* launches) {
  scan_any<int32_t>(src, out, n_max, nullptr, tmp, 1, st, launches);
}

template void scan_inclusive<int32_t>(const ScanSrc&, int32_t*, int64_t, const int32_t*, int32_t*,
                                      cudaStream_t, int64_t*);
template void scan_inclusive<uint64_t>(const ScanSrc&, uint64_t*, int64_t, const int32_t*, uint64_t*,
                                       cudaStream_t, int64_t*);

}  // namespace fig
