// Tails of a relation formed in registers and triangularised at once: the last head/tail
// pass (Def. "Head and Tail", Alg. 2) fused with the warp Householder QR of the TSQR leaf
// (§7 step 1), for relations of at most 32 data columns, so that the tails block is never
// written to memory.
//
// A warp takes one scan tile (kHtTile sorted rows, whose carry k_tile_carry has computed)
// as S QR tiles of TW rows; in each, lane l holds the RPL consecutive sorted rows starting
// at l * RPL.  Per column, a segmented warp scan of the lanes' (flag, sum) gives every lane
// its exclusive prefix, the running sum then walks the lane's rows, and row p >= 1 of a
// group becomes sqrt(Phi_circ) beta_p (p a_p - S_p) in the QR's registers; the row that
// starts a group (its head, made by the first pass) and rows past the end stay zero, which
// leaves R unchanged.  The QR sees slot (lane, r) as its row lane + 32 r: R does not depend
// on the order of the rows.  One triangle per QR tile; the tree levels follow as for a
// stored block with tiles of TW rows.
#pragma once

#include "leaf.cuh"
#include "tsqr_reg.cuh"

namespace fig {

template <int N>
struct FusedCfg {
  static constexpr int RPL = N <= 8 ? 8 : N <= 16 ? 4 : 2;   // rows per lane, a divisor of kHtItems
  static constexpr int TW = 32 * RPL;                        // rows per QR tile
  static constexpr int S = kHtItems / RPL;                   // QR tiles per scan tile
};

constexpr int kFusedThreads = kRegThreads;
constexpr int kFusedWarps = kFusedThreads / 32;

// RPL consecutive values of column c from sorted position e0 on (zero past the end): from
// the sorted copy when there is one (16-byte loads), else from the input in place.
template <int RPL>
__device__ __forceinline__ void load_fused_items(const LeafParams& p, int64_t e0, int c, double (&xs)[RPL]) {
  if (p.sdata) {
    const double* col = p.sdata + (int64_t)c * p.lds + e0;
    if (e0 + RPL <= p.M) {
#pragma unroll
      for (int r = 0; r < RPL; r += 2) {
        const double2 v = *reinterpret_cast<const double2*>(col + r);
        xs[r] = v.x;
        xs[r + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int r = 0; r < RPL; ++r) xs[r] = e0 + r < p.M ? col[r] : 0.0;
    }
    return;
  }
#pragma unroll
  for (int r = 0; r < RPL; ++r) xs[r] = e0 + r < p.M ? p.data[(e0 + r) * p.rs + (int64_t)c * p.cs] : 0.0;
}

// Triangle of a QR tile (rows 0..n-1 of the register tile), column-major n x n.
template <typename E, int N, int RPL>
__device__ __forceinline__ void store_tri(const E (&a)[RPL][N], int n, int lane, double* tri) {
#pragma unroll
  for (int r = 0; r < RPL; ++r) {
    const int i = lane + 32 * r;
    if (i < n) {
#pragma unroll
      for (int c = 0; c < N; ++c)
        if (c < n) tri[(int64_t)c * n + i] = c >= i ? (double)a[r][c] : 0.0;
    }
  }
}

// Tail rows in float64 on both paths (the mixed path rounds each once to float for its
// float QR, whose arithmetic then runs on the FP32 pipe beside the FP64 tail arithmetic):
// tail = c1 x - c2 S with c1 = sqrt(Phi_circ) p beta_p, c2 = sqrt(Phi_circ) beta_p (both 0
// at p = 0), per cell one add, one FMA and one multiply, as in the stored pass.  With 8 rows
// per lane (S = 1) a lane holds the rows of the first pass's lane, whose exclusive prefix
// that pass stored; otherwise the prefix comes from a warp scan of the lanes' sums.
template <typename E, int N>
__global__ void __launch_bounds__(kFusedThreads) k_tails_qr(LeafParams p, int n, double* tri_out) {
  constexpr int RPL = FusedCfg<N>::RPL, TW = FusedCfg<N>::TW, S = FusedCfg<N>::S;
  __shared__ double2 coef_s[kFusedWarps][TW];
  __shared__ double cin_s[kFusedWarps][N];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n_qr = (p.M + TW - 1) / TW;
  for (int64_t t = gw; t < p.n_tiles; t += nw) {
    if (p.ttail && !p.ttail[t]) {          // single-row groups only: zero triangles
      for (int s = 0; s < S && t * S + s < n_qr; ++s) {
        double* tri = tri_out + (t * S + s) * n * n;
        for (int i = lane; i < n * n; i += 32) tri[i] = 0.0;
      }
      continue;
    }
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
      const int64_t q = t * S + s;
      if (q >= n_qr) break;
      const int64_t e0 = q * TW + (int64_t)lane * RPL;
      uint32_t starts = 0;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int64_t e = e0 + r;
        double2 cf = make_double2(0.0, 0.0);
        if (e < p.M) {
          const int32_t g = p.row_gid[e];
          const int32_t pos = (int32_t)(e - p.goff[g]);
          if (pos == 0) starts |= 1u << r;
          const double2 bt = p.beta[pos];
          const double gs = p.sq_phic[g];
          cf = make_double2(gs * bt.y, gs * bt.x);
        }
        coef_s[w][lane * RPL + r] = cf;
      }
      __syncwarp();
      E a[RPL][N];
#pragma unroll
      for (int c = 0; c < N; ++c) {
        if (c < n) {
          double xs[RPL];
          load_fused_items<RPL>(p, e0, c, xs);
          double run;
          if (S == 1) {
            const int64_t slot = (int64_t)c * p.n_tiles + t;
            const int fe = p.lflag[slot * 32 + lane];
            const double se = p.lsum[slot * 32 + lane];
            run = fe ? se : p.tcarry[slot] + se;
          } else {
            int f = 0;
            double sl = 0.0;
#pragma unroll
            for (int r = 0; r < RPL; ++r) {
              if (starts & (1u << r)) { f = 1; sl = xs[r]; } else { sl += xs[r]; }
            }
            pair_scan_incl(f, sl, lane);
            int fe = __shfl_up_sync(0xffffffffu, f, 1);
            double se = __shfl_up_sync(0xffffffffu, sl, 1);
            if (lane == 0) { fe = 0; se = 0.0; }
            const double cin = s == 0 ? p.tcarry[(int64_t)c * p.n_tiles + t] : cin_s[w][c];
            const int f31 = __shfl_sync(0xffffffffu, f, 31);
            const double s31 = __shfl_sync(0xffffffffu, sl, 31);
            __syncwarp();
            if (lane == 0) cin_s[w][c] = f31 ? s31 : cin + s31;
            run = fe ? se : cin + se;
          }
#pragma unroll
          for (int r = 0; r < RPL; ++r) {
            if (starts & (1u << r)) run = 0.0;
            const double2 cf = coef_s[w][lane * RPL + r];
            a[r][c] = (E)fma(cf.x, xs[r], -(cf.y * run));
            run += xs[r];
          }
        } else {
#pragma unroll
          for (int r = 0; r < RPL; ++r) a[r][c] = E(0);
        }
      }
      RegQR<E, N, RPL, 0>::run(a, TW, lane);
      store_tri<E, N, RPL>(a, n, lane, tri_out + q * n * n);
      __syncwarp();
    }
  }
}

// Persistent grid: at most as many blocks as are resident at once (registers decide).
template <typename K>
static int64_t fused_resident(K kernel) {
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kFusedThreads, 0);
  return (per_sm > 0 && sms > 0) ? (int64_t)per_sm * sms : 152 * 4;
}

inline unsigned fused_blocks(int64_t n_tiles, int64_t resident) {
  int64_t blocks = (n_tiles + kFusedWarps - 1) / kFusedWarps;
  if (blocks > resident) blocks = resident;
  return (unsigned)(blocks < 1 ? 1 : blocks);
}

template <typename E, int N>
void launch_tails_qr(const LeafParams& p, int n, double* tri_out, cudaStream_t st) {
  static const int64_t resident = fused_resident(k_tails_qr<E, N>);
  k_tails_qr<E, N><<<fused_blocks(p.n_tiles, resident), kFusedThreads, 0, st>>>(p, n, tri_out);
}

}  // namespace fig
