// Key packing, stable LSD radix sort and segmentation of a relation.
//
// §5 assumes every relation S_i sorted on its join attributes X_i, with a child first
// sorted on the attributes it shares with its parent.  Each relation's key is packed
// into one uint64: the attributes shared with the parent (ascending attribute id) in
// the high bits, then the remaining attributes; each attribute takes the bits needed
// for (value - min) over all relations holding it.  A stable radix sort of the packed
// key gives that order with ties in input order (R does not depend on row order, §1.1
// footnote, so any tie order is valid).  Segment boundaries of X_i (groups) and of
// X_p (parent groups) come from key changes.
#include <climits>

#include "kernels.cuh"

namespace fig {

// ------------------------------------------------------------------ key ranges (plan time)
template <typename K>
__global__ void k_minmax(const K* col, int64_t n, long long* out_min, long long* out_max) {
  long long lo = LLONG_MAX, hi = LLONG_MIN;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    long long v = (long long)col[i];
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    long long a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(out_min, lo);
    atomicMax(out_max, hi);
  }
}

void launch_minmax(const void* col, int key_type, int64_t n, long long* dmin, long long* dmax,
                   cudaStream_t st) {
  unsigned g = grid_for(n, 256, 1024);
  if (key_type == FIGARO_KEY_I32)
    k_minmax<int32_t><<<g, 256, 0, st>>>(static_cast<const int32_t*>(col), n, dmin, dmax);
  else
    k_minmax<long long><<<g, 256, 0, st>>>(static_cast<const long long*>(col), n, dmin, dmax);
}

// ------------------------------------------------------------------ packing
__global__ void k_pack(PackParams p, int64_t n, uint64_t* key, int32_t* perm, int* err) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = 0;
    for (int a = 0; a < p.n_keys; ++a) {
      long long v = p.key_type == FIGARO_KEY_I32 ? (long long)static_cast<const int32_t*>(p.cols[a])[r]
                                                 : static_cast<const long long*>(p.cols[a])[r];
      unsigned long long d = (unsigned long long)(v - p.kmin[a]);
      if (v < p.kmin[a] || shr64(d, p.bits[a]) != 0ull) {
        set_error(err, FIGARO_ERR_KEY_RANGE);
        d = 0;
      }
      k |= shl64(d, p.shift[a]);
    }
    key[r] = k;
    if (perm) perm[r] = (int32_t)r;
  }
}

void launch_pack(const PackParams& p, int64_t n, uint64_t* key, int32_t* perm, int* err,
                 cudaStream_t st, int64_t* launches) {
  k_pack<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(p, n, key, perm, err);
  ++*launches;
}

// Presorted input: keys must be non-decreasing.
__global__ void k_check_sorted(const uint64_t* key, int64_t n, int* err) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x + 1; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    if (key[r] < key[r - 1]) set_error(err, FIGARO_ERR_NOT_SORTED);
}

// ------------------------------------------------------------------ radix sort
// LSD radix sort by digits of up to 11 bits (a relation's packed key of b bits takes
// ceil(b / 11) passes).  One pass: per-tile digit histograms (digit-major, so that one
// exclusive scan yields every tile's output offset per digit), then a stable scatter.
// A tile is 8 warps x 8 rounds x 32 keys; inside a tile keys keep their order (warps,
// rounds and lanes follow key order), so the sort is stable.  Histogram and rank use
// __match_any_sync so that equal digits in a warp (frequent with skewed keys) cost one
// shared-memory update per distinct digit instead of one per key.
constexpr int kRsWarps = 8, kRsRounds = 8;
constexpr int kRsTile = kRsWarps * kRsRounds * 32;   // 2048 keys
constexpr int kRsMaxBits = 11;
constexpr int kRsMaxBins = 1 << kRsMaxBits;

__global__ void __launch_bounds__(256) k_radix_hist(const uint64_t* key, int64_t n, int shift, int bins,
                                                    int32_t* hist, int64_t n_tiles) {
  __shared__ int32_t h[kRsMaxBins];
  for (int d = threadIdx.x; d < bins; d += 256) h[d] = 0;
  __syncthreads();
  const unsigned mask = (unsigned)bins - 1u;
  const int lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * kRsTile;
  for (int i = threadIdx.x; i < kRsTile; i += 256) {
    const int64_t e = base + i;
    const bool ok = e < n;
    const unsigned d = ok ? (unsigned)(key[e] >> shift) & mask : (unsigned)kRsMaxBins + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (ok && lane == __ffs(peers) - 1) atomicAdd(&h[d], __popc(peers));
  }
  __syncthreads();
  for (int d = threadIdx.x; d < bins; d += 256) hist[(int64_t)d * n_tiles + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(256) k_radix_scatter(const uint64_t* key_in, const int32_t* val_in,
                                                       uint64_t* key_out, int32_t* val_out,
                                                       int64_t n, int shift, int bins, const int32_t* off,
                                                       int64_t n_tiles) {
  extern __shared__ int32_t cnt[];                    // [kRsWarps][bins]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned mask = (unsigned)bins - 1u;
  for (int d = lane; d < bins; d += 32) cnt[warp * bins + d] = 0;
  __syncwarp();
  const int64_t base = (int64_t)blockIdx.x * kRsTile + (int64_t)warp * (kRsRounds * 32);
  uint64_t k[kRsRounds];
  int32_t v[kRsRounds];
  int rank[kRsRounds];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kRsRounds; ++j) {
    const int64_t e = base + j * 32 + lane;
    const bool ok = e < n;
    k[j] = ok ? key_in[e] : 0ull;
    v[j] = ok ? val_in[e] : 0;
    const unsigned d = ok ? (unsigned)(k[j] >> shift) & mask : (unsigned)kRsMaxBins + lane;   // unique sentinel
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int before = ok ? cnt[warp * bins + d] : 0;
    __syncwarp();
    if (ok && (peers & lt) == 0) cnt[warp * bins + d] = before + __popc(peers);
    __syncwarp();
    rank[j] = before + __popc(peers & lt);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < bins; d += 256) {      // exclusive scan over warps per digit
    int run = 0;
    for (int w = 0; w < kRsWarps; ++w) {
      const int c = cnt[w * bins + d];
      cnt[w * bins + d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRsRounds; ++j) {
    const int64_t e = base + j * 32 + lane;
    if (e < n) {
      const unsigned d = (unsigned)(k[j] >> shift) & mask;
      const int64_t dst = (int64_t)off[(int64_t)d * n_tiles + blockIdx.x] + cnt[warp * bins + d] + rank[j];
      key_out[dst] = k[j];
      val_out[dst] = v[j];
    }
  }
}

int64_t radix_tiles(int64_t n) { return (n + kRsTile - 1) / kRsTile; }

// The dynamic shared-memory limit is a property of the function, not of a launch: it is
// raised once to the largest size any launch uses (also inside captured graphs).
cudaError_t keys_set_attributes() {
  return cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(kRsWarps * kRsMaxBins * sizeof(int32_t)));
}
int64_t radix_hist_elems(int64_t n) { return (int64_t)kRsMaxBins * radix_tiles(n); }

// Sorts (key, perm) by the low `bits` bits using ping-pong buffers; returns which buffer
// (0 or 1) holds the result.
int radix_sort(uint64_t* key[2], int32_t* perm[2], int64_t n, int bits, int32_t* hist, int32_t* scan_tmp,
               cudaStream_t st, int64_t* launches) {
  int cur = 0;
  const int64_t nt = radix_tiles(n);
  const int passes = (bits + kRsMaxBits - 1) / kRsMaxBits;
  const int width = (bits + passes - 1) / passes;
  const int bins = 1 << width;
  const int64_t hn = (int64_t)bins * nt;
  const size_t smem = (size_t)kRsWarps * bins * sizeof(int32_t);
  for (int shift = 0; shift < bits; shift += width) {
    k_radix_hist<<<(unsigned)nt, 256, 0, st>>>(key[cur], n, shift, bins, hist, nt);
    ScanSrc src{SCAN_PLAIN_I32, hist, 0};
    scan_exclusive_i32(src, hist + hn, hn, scan_tmp, st, launches);
    k_radix_scatter<<<(unsigned)nt, 256, smem, st>>>(key[cur], perm[cur], key[cur ^ 1], perm[cur ^ 1], n, shift,
                                                     bins, hist + hn, nt);
    *launches += 2;
    cur ^= 1;
  }
  return cur;
}

// ------------------------------------------------------------------ segmentation
// row_gid[r] = (inclusive count of key changes up to r) - 1; goff[g] = first sorted row
// of group g, goff[G] = M; gkey[g] = key of group g; sizes[0] = G.
__global__ void k_seg_fill(const uint64_t* skey, const int32_t* incl, int64_t n, int32_t* row_gid,
                           int32_t* goff, uint64_t* gkey, int32_t* sizes) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int32_t g = incl[r] - 1;
    row_gid[r] = g;
    if (r == 0 || skey[r] != skey[r - 1]) {
      goff[g] = (int32_t)r;
      gkey[g] = skey[r];
    }
    if (r == n - 1) {
      goff[g + 1] = (int32_t)n;
      sizes[0] = g + 1;
    }
  }
}

// Parent groups over the groups: g2p[g], pgoff[p] (first group), pgoff[P] = G,
// pkey[p] = gkey >> rest_bits, sizes[1] = P.
__global__ void k_pseg_fill(const uint64_t* gkey, const int32_t* incl, int64_t n_max, int rest_bits,
                            int32_t* g2p, int32_t* pgoff, uint64_t* pkey, int32_t* sizes) {
  const int64_t G = sizes[0];
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
       g += (int64_t)gridDim.x * blockDim.x) {
    int32_t p = incl[g] - 1;
    g2p[g] = p;
    uint64_t pk = shr64(gkey[g], rest_bits);
    if (g == 0 || pk != shr64(gkey[g - 1], rest_bits)) {
      pgoff[p] = (int32_t)g;
      pkey[p] = pk;
    }
    if (g == G - 1) {
      pgoff[p + 1] = (int32_t)G;
      sizes[1] = p + 1;
    }
  }
}

void segment(NodeBuf& b, int64_t n, int rest_bits, cudaStream_t st, int64_t* launches) {
  ScanSrc s1{SCAN_KEY_CHANGE, b.skey, 0};
  scan_inclusive<int32_t>(s1, b.itmp, n, nullptr, b.scan_tmp_i, st, launches);
  k_seg_fill<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(b.skey, b.itmp, n, b.row_gid, b.goff, b.gkey,
                                                         b.sizes);
  ScanSrc s2{SCAN_KEY_CHANGE, b.gkey, rest_bits};
  scan_inclusive<int32_t>(s2, b.itmp, n, b.sizes, b.scan_tmp_i, st, launches);
  k_pseg_fill<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(b.gkey, b.itmp, n, rest_bits, b.g2p, b.pgoff,
                                                          b.pkey, b.sizes);
  *launches += 2;
}

void check_sorted(const uint64_t* key, int64_t n, int* err, cudaStream_t st, int64_t* launches) {
  if (n < 2) return;
  k_check_sorted<<<grid_for(n, 256, 152 * 16), 256, 0, st>>>(key, n, err);
  ++*launches;
}

}  // namespace fig
