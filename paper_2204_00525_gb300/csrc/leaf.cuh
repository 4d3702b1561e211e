// Device helpers of the relation (v = 1) head/tail passes, shared by the scan kernels and
// the fused tails + TSQR leaf: segmented (flag, sum) warp scans in float64 and in
// double-float, and the per-row bookkeeping of a sorted position.
#pragma once

#include "dfloat.cuh"
#include "kernels.cuh"

namespace fig {

// (f, s): f = a segment starts inside the range, s = sum after its last start (or the
// whole range when f == 0).  combine(earlier, later).
__device__ __forceinline__ void pair_scan_incl(int& f, double& s, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int fo = __shfl_up_sync(0xffffffffu, f, o);
    double so = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) {
      s = f ? s : so + s;
      f |= fo;
    }
  }
}

__device__ __forceinline__ void pair_scan_incl_df(int& f, dfl& s, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int fo = __shfl_up_sync(0xffffffffu, f, o);
    const float sh = __shfl_up_sync(0xffffffffu, s.hi, o);
    const float sl = __shfl_up_sync(0xffffffffu, s.lo, o);
    if (lane >= o) {
      if (!f) s = df_add(dfl{sh, sl}, s);
      f |= fo;
    }
  }
}

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  dfl r;
  fast_two(p, e, r.hi, r.lo);
  return r;
}

struct LeafRow {
  int32_t src;   // input row
  int32_t pos;   // position inside the group
  int32_t g;
  bool ok, last;
};

__device__ __forceinline__ LeafRow leaf_row(const LeafParams& p, int64_t e) {
  LeafRow r;
  r.ok = e < p.M;
  if (!r.ok) { r.src = 0; r.pos = 1; r.g = 0; r.last = false; return r; }
  r.src = p.perm ? p.perm[e] : (int32_t)e;
  r.g = p.row_gid[e];
  const int32_t start = p.goff[r.g];
  r.pos = (int32_t)(e - start);
  r.last = (e == (int64_t)p.goff[r.g + 1] - 1);
  return r;
}

// The kHtItems values of column c for one lane's consecutive sorted rows: gathered through
// the permutation (first pass; a copy in sorted order is kept when p.sdata is set), or read
// back from that copy (last pass) with 16-byte loads.
__device__ __forceinline__ void load_leaf_items(const LeafParams& p, const LeafRow (&rw)[kHtItems], int64_t e0,
                                                int c, bool from_copy, double (&xs)[kHtItems]) {
  if (from_copy) {
    const double* col = p.sdata + (int64_t)c * p.lds + e0;
    if (e0 + kHtItems <= p.M) {
#pragma unroll
      for (int i = 0; i < kHtItems; i += 2) {
        const double2 v = *reinterpret_cast<const double2*>(col + i);
        xs[i] = v.x;
        xs[i + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) xs[i] = rw[i].ok ? col[i] : 0.0;
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < kHtItems; ++i) xs[i] = rw[i].ok ? p.data[(int64_t)rw[i].src * p.rs + (int64_t)c * p.cs] : 0.0;
  if (p.sdata) {
    double* col = p.sdata + (int64_t)c * p.lds + e0;
    if (e0 + kHtItems <= p.M) {
#pragma unroll
      for (int i = 0; i < kHtItems; i += 2) *reinterpret_cast<double2*>(col + i) = make_double2(xs[i], xs[i + 1]);
    } else {
#pragma unroll
      for (int i = 0; i < kHtItems; ++i)
        if (rw[i].ok) col[i] = xs[i];
    }
  }
}

}  // namespace fig
