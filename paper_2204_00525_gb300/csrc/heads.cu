// Heads and tails (Def. "Head and Tail", Def. "Generalized Head and Tail", Alg. 2) as
// flat segmented scans over key-sorted rows.
//
// The paper loops over join keys in parallel (§6); with Zipf-skewed keys one group can
// hold a sixth of a relation, so here the sorted rows are cut into fixed tiles of
// 256 elements per warp regardless of group boundaries.  Per column, a prefix sum that
// restarts at every group start is computed in three steps: (1) every tile reports
// whether it contains a group start and the sum after its last start, every lane its
// exclusive (flag, sum) inside the tile, and the heads of the groups that begin in the
// tile are written final, (2) one thread block per column scans the tile aggregates into a
// carry per tile, which also completes the one group per tile that began earlier, (3)
// every lane starts its running sum at its carry and writes the tail rows (one add, one FMA
// and one multiply per cell), skipping tiles without a tail row.
//
// Tail of a group with rows a_0..a_{m-1} (0-based position p, exclusive prefix S_p):
//   row p >= 1:  sqrt(Phi_circ) (sqrt(p) a_p - S_p / sqrt(p)) / sqrt(p + 1)
//              = sqrt(Phi_circ) beta_p (p a_p - S_p),   beta_p = 1 / sqrt(p (p + 1)),
//   head:        S_m / sqrt(m).
// Tail row p of group g lands at row (sorted position - g - 1): groups in key order,
// rows in sorted order, m - 1 rows per group.
// Generalized tail of element k of an X_p group with weights v and W_k = sum_{t<k} v_t^2
// (exact integer), P_k = sum_{t<k} v_t D_t:
//   sqrt(Phi_up) (sqrt(W_k) D_k - v_k P_k / sqrt(W_k)) / sqrt(W_k + v_k^2)
//   = gamma_k (W_k D_k - v_k P_k),  gamma_k = sqrt(Phi_up) / sqrt(W_k (W_k + v_k^2)),
//   head: P_n / sqrt(W_n) with W_n = Phi_down(x_p).
#include "dfloat.cuh"
#include "kernels.cuh"
#include "leaf.cuh"

namespace fig {

// Per-position coefficients of the tail formula, {beta_p, p beta_p} with
// beta_p = 1 / sqrt(p (p + 1)), for every position p of every group (the table's length
// is the largest relation's row count + 1).  Read from memory rather than computed, so
// that no FP64 conversion or square root is issued per row; FP64 issues slowly here.
__global__ void k_beta(double2* beta, int64_t len) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < len;
       p += (int64_t)gridDim.x * blockDim.x) {
    const double b = p == 0 ? 0.0 : 1.0 / sqrt((double)p * ((double)p + 1.0));
    beta[p] = make_double2(b, (double)p * b);
  }
}

void beta_table(double2* beta, int64_t len, cudaStream_t st) {
  k_beta<<<grid_for(len, 256, 4096), 256, 0, st>>>(beta, len);
}

// One block of 1024 threads per column: carry[c][t] = sum of the column since the last
// group start before tile t (0 if tile t begins a group).  Each thread reduces a
// contiguous run of tiles, a block-wide scan of (flag, sum) pairs gives every run its
// incoming carry, and the run is then walked again to write the carries.  `live` (if
// set) holds the element count whose tiles are live.
constexpr int kCarryThreads = 1024;

__global__ void __launch_bounds__(kCarryThreads) k_tile_carry(const uint8_t* tflag, const double* tsum,
                                                              double* tcarry, int64_t nt_alloc,
                                                              const int32_t* live) {
  __shared__ int wf[32];
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nt = live ? ((int64_t)live[0] + kHtTile - 1) / kHtTile : nt_alloc;
  const uint8_t* f_in = tflag + (int64_t)blockIdx.x * nt_alloc;
  const double* s_in = tsum + (int64_t)blockIdx.x * nt_alloc;
  double* out = tcarry + (int64_t)blockIdx.x * nt_alloc;
  const int64_t chunk = (nt + kCarryThreads - 1) / kCarryThreads;
  const int64_t t0 = (int64_t)threadIdx.x * chunk;
  const int64_t t1 = t0 + chunk < nt ? t0 + chunk : nt;
  int f = 0;
  double s = 0.0;
  for (int64_t t = t0; t < t1; ++t) {
    if (f_in[t]) { f = 1; s = s_in[t]; } else { s += s_in[t]; }
  }
  int fi = f;
  double si = s;
  pair_scan_incl(fi, si, lane);
  int fe = __shfl_up_sync(0xffffffffu, fi, 1);
  double se = __shfl_up_sync(0xffffffffu, si, 1);
  if (lane == 0) { fe = 0; se = 0.0; }
  if (lane == 31) { wf[warp] = fi; ws[warp] = si; }
  __syncthreads();
  if (warp == 0) {
    int a = wf[lane];
    double b = ws[lane];
    pair_scan_incl(a, b, lane);
    int ae = __shfl_up_sync(0xffffffffu, a, 1);
    double be = __shfl_up_sync(0xffffffffu, b, 1);
    if (lane == 0) { ae = 0; be = 0.0; }
    wf[lane] = ae;
    ws[lane] = be;
  }
  __syncthreads();
  double run = fe ? se : ws[warp] + se;
  for (int64_t t = t0; t < t1; ++t) {
    out[t] = run;
    run = f_in[t] ? s_in[t] : run + s_in[t];
  }
}

// ------------------------------------------------------------------ whole-row gathers
// A row of a column-major table taken at a random position costs one 32-byte sector per
// value, of which 8 bytes are used, and with tables larger than L2 those sectors come from
// HBM.  The gathers below move whole rows instead: a row-major copy of the table (32 x 32
// tiles through shared memory, coalesced on both sides), then every warp reads whole rows
// (contiguous across the lanes) into a shared tile that is written out as column segments
// of 32 consecutive rows.
__global__ void __launch_bounds__(256) k_rows_of(const double* src, int64_t ld, int64_t bound, const int32_t* live,
                                                 int cols, double* dst, int np) {
  __shared__ double tile[32][33];
  const int64_t rows = live ? (int64_t)live[0] : bound;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int ctiles = (cols + 31) >> 5;
  const int64_t tiles = ((rows + 31) >> 5) * ctiles;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t r0 = (t / ctiles) * 32;
    const int c0 = (int)(t % ctiles) * 32;
    for (int k = ty; k < 32; k += 8) {              // tile[column][row]
      const int c = c0 + k;
      const int64_t r = r0 + tx;
      tile[k][tx] = (c < cols && r < rows) ? src[(int64_t)c * ld + r] : 0.0;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
      const int64_t r = r0 + k;
      const int c = c0 + tx;
      if (r < rows && c < cols) dst[r * np + c] = tile[tx][k];
    }
    __syncthreads();
  }
}

// Tables of at most kSlabCols columns: a warp copies a slab of 32 rows and all columns,
// lanes over rows for the loads (one coalesced 256-byte segment per column, all of them in
// flight) and over columns for the stores (whole rows), through its own shared-memory slab.
constexpr int kSlabCols = 64;

__global__ void __launch_bounds__(256) k_rows_of_slab(const double* src, int64_t ld, int64_t bound,
                                                      const int32_t* live, int cols, double* dst, int np) {
  extern __shared__ double slab_all[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ls = cols + 1;                           // odd stride: the row-wise stores hit distinct banks
  double* slab = slab_all + (int64_t)warp * 32 * ls;
  const int64_t rows = live ? (int64_t)live[0] : bound;
  const int64_t slabs = (rows + 31) >> 5;
  for (int64_t q = (int64_t)blockIdx.x * 8 + warp; q < slabs; q += (int64_t)gridDim.x * 8) {
    const int64_t r0 = q * 32, r = r0 + lane;
#pragma unroll 16
    for (int c = 0; c < cols; ++c) slab[lane * ls + c] = r < rows ? src[(int64_t)c * ld + r] : 0.0;
    __syncwarp();
    const int nr = (rows - r0) < 32 ? (int)(rows - r0) : 32;
    for (int i = 0; i < nr; ++i)
      for (int c = lane; c < cols; c += 32) dst[(r0 + i) * np + c] = slab[i * ls + c];
    __syncwarp();
  }
}

size_t rows_of_slab_smem() { return (size_t)8 * 32 * (kSlabCols + 1) * sizeof(double); }

cudaError_t rows_of_set_attributes() {
  return cudaFuncSetAttribute(k_rows_of_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_of_slab_smem());
}

void rows_of(const double* src, int64_t ld, int64_t bound, const int32_t* live, int cols, double* dst, int np,
             cudaStream_t st, int64_t* launches) {
  if (cols <= 0 || bound <= 0) return;
  if (cols <= kSlabCols) {
    const int64_t slabs = (bound + 31) / 32;
    int64_t blocks = (slabs + 7) / 8;
    if (blocks > 152 * 2) blocks = 152 * 2;
    const size_t smem = (size_t)8 * 32 * (cols + 1) * sizeof(double);
    k_rows_of_slab<<<(unsigned)(blocks < 1 ? 1 : blocks), 256, smem, st>>>(src, ld, bound, live, cols, dst, np);
    ++*launches;
    return;
  }
  const int64_t tiles = ((bound + 31) / 32) * ((cols + 31) / 32);
  k_rows_of<<<(unsigned)(tiles < 152 * 8 ? tiles : 152 * 8), 256, 0, st>>>(src, ld, bound, live, cols, dst, np);
  ++*launches;
}

// out[c * ldo + e] = rows[perm[e] * rs + c], 32 sorted positions per tile, 64 columns at a time.
__global__ void __launch_bounds__(256) k_rows_gather(const double* rows, int64_t rs, const int32_t* perm, int64_t M,
                                                     int cols, double* out, int64_t ldo) {
  __shared__ double tile[32][65];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tiles = (M + 31) >> 5;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t e0 = t * 32;
    for (int cc = 0; cc < cols; cc += 64) {
      for (int r = warp; r < 32; r += 8) {
        const int64_t e = e0 + r;
        if (e < M) {
          const double* src = rows + (int64_t)perm[e] * rs + cc;
          tile[r][lane] = cc + lane < cols ? src[lane] : 0.0;
          tile[r][lane + 32] = cc + 32 + lane < cols ? src[lane + 32] : 0.0;
        }
      }
      __syncthreads();
      const int64_t e = e0 + lane;
      for (int c = cc + warp; c < cc + 64 && c < cols; c += 8)
        if (e < M) out[(int64_t)c * ldo + e] = tile[lane][c - cc];
      __syncthreads();
    }
  }
}

void rows_gather(const double* rows, int64_t rs, const int32_t* perm, int64_t M, int cols, double* out,
                 int64_t ldo, cudaStream_t st, int64_t* launches) {
  if (cols <= 0 || M <= 0) return;
  const int64_t tiles = (M + 31) / 32;
  k_rows_gather<<<(unsigned)(tiles < 152 * 8 ? tiles : 152 * 8), 256, 0, st>>>(rows, rs, perm, M, cols, out, ldo);
  ++*launches;
}

// ------------------------------------------------------------------ relations (v = 1)
// Every lane's exclusive (flag, sum) inside the tile and the tile aggregate (lane 31).
__device__ __forceinline__ void store_lane_and_tile(int f, double s, int lane, int64_t slot, int64_t tslot,
                                                    uint8_t* lflag, double* lsum, uint8_t* tflag, double* tsum) {
  pair_scan_incl(f, s, lane);
  int fe = __shfl_up_sync(0xffffffffu, f, 1);
  double se = __shfl_up_sync(0xffffffffu, s, 1);
  if (lane == 0) { fe = 0; se = 0.0; }
  lflag[slot * 32 + lane] = (uint8_t)fe;
  lsum[slot * 32 + lane] = se;
  if (lane == 31) {
    tflag[tslot] = (uint8_t)f;
    tsum[tslot] = s;
  }
}

// Whether the tile holds a tail row (one after its group's first): a tile of single-row
// groups (a key column with distinct values, as the key-fkey joins' dimension and fact
// tables mostly are) has no tails, and the tails pass skips it without reading its data.
__device__ __forceinline__ void mark_tail_tile(const LeafParams& p, const LeafRow (&rw)[kHtItems], int64_t t,
                                               int lane) {
  bool any = false;
#pragma unroll
  for (int i = 0; i < kHtItems; ++i) any = any || (rw[i].ok && rw[i].pos > 0);
  any = __any_sync(0xffffffffu, any);
  if (p.ttail && lane == 0) p.ttail[t] = any ? 1 : 0;
}

// Pass 1: per tile and column, the tile aggregate (for the carry scan), every lane's
// exclusive (flag, sum) inside the tile when a tails pass follows (lflag set), and the head
// of every group that begins in the tile (its sum times 1 / sqrt(rows)), so that the heads
// need no later pass over the data.  The running sum of the lane is the group's sum for
// every group that begins in the lane; only the lane's first group, when it began in an
// earlier lane, waits for the lane's exclusive prefix.  A group that began in an earlier
// tile (at most one ends in each tile) gets its sum from the tile start, and k_heads_fix
// adds the tile's carry and scales it.
__global__ void __launch_bounds__(256, 3) k_leaf_agg(LeafParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = wid; t < p.n_tiles; t += nwarps) {
    const int64_t e0 = t * kHtTile + (int64_t)lane * kHtItems;
    LeafRow rw[kHtItems];
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) rw[i] = leaf_row(p, e0 + i);
    mark_tail_tile(p, rw, t, lane);
    for (int c = 0; c < p.N; ++c) {
      double xs[kHtItems];
      load_leaf_items(p, rw, e0, c, p.sorted_ready != 0, xs);
      int f = 0;
      double s = 0.0;
      int open_g = -1;                     // a group that ends in this lane but began before it
      double open_s = 0.0;
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const double x = xs[i];
        if (rw[i].pos == 0) { f = 1; s = x; } else { s += x; }
        if (rw[i].last) {
          if (f) p.heads[(int64_t)c * p.ldh + rw[i].g] = s * __ldg(p.hrow + rw[i].g);
          else { open_g = rw[i].g; open_s = s; }
        }
      }
      pair_scan_incl(f, s, lane);
      int fe = __shfl_up_sync(0xffffffffu, f, 1);
      double se = __shfl_up_sync(0xffffffffu, s, 1);
      if (lane == 0) { fe = 0; se = 0.0; }
      const int64_t slot = (int64_t)c * p.n_tiles + t;
      if (p.lflag) {
        p.lflag[slot * 32 + lane] = (uint8_t)fe;
        p.lsum[slot * 32 + lane] = se;
      }
      if (lane == 31) {
        p.tflag[slot] = (uint8_t)f;
        p.tsum[slot] = s;
      }
      if (open_g >= 0) {
        const double h = se + open_s;        // began in an earlier tile (fe == 0): k_heads_fix
        p.heads[(int64_t)c * p.ldh + open_g] = fe ? h * __ldg(p.hrow + open_g) : h;
      }
    }
  }
}

// Pass 3 (tails blocks that are materialised): the running sum of every lane starts at its
// carry (tile carry combined with the lane's exclusive partial), so each cell costs one
// add, one FMA and one multiply.
__global__ void __launch_bounds__(256, 2) k_leaf_emit(LeafParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = wid; t < p.n_tiles; t += nwarps) {
    if (p.ttail && !p.ttail[t]) continue;   // single-row groups only: no tail to write
    const int64_t e0 = t * kHtTile + (int64_t)lane * kHtItems;
    LeafRow rw[kHtItems];
    double ca[kHtItems], cb[kHtItems];    // tail = ca x - cb S: ca = g p beta_p, cb = g beta_p
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) {
      rw[i] = leaf_row(p, e0 + i);
      const double2 bt = p.beta[rw[i].ok ? rw[i].pos : 0];
      const double gs = rw[i].ok ? p.sq_phic[rw[i].g] : 0.0;
      ca[i] = gs * bt.y;
      cb[i] = gs * bt.x;
    }
    for (int c = 0; c < p.N; ++c) {
      const int64_t slot = (int64_t)c * p.n_tiles + t;
      const int fe = p.lflag[slot * 32 + lane];
      const double se = p.lsum[slot * 32 + lane];
      double run = fe ? se : p.tcarry[slot] + se;
      double* tcol = p.tails + (int64_t)c * p.ldt;
      double xs[kHtItems];                 // all loads first: the stores below may alias data
      load_leaf_items(p, rw, e0, c, p.sdata != nullptr, xs);
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const double x = xs[i];
        if (rw[i].pos == 0) run = 0.0;
        if (rw[i].pos > 0) tcol[e0 + i - rw[i].g - 1] = fma(ca[i], x, -(cb[i] * run));
        run += x;
      }
    }
  }
}

// ------------------------------------------------------------------ mixed precision (v = 1)
// Same three passes with the prefix sums in double-float arithmetic on the FP32 pipe: the
// FP64 inputs are split exactly enough (2^-47) into float pairs, every running sum and
// p a_p - S_p is formed in double-float, and the tail row is rounded once to float for
// the FP32 TSQR leaf.  Heads stay float64.  Carries between lanes and tiles are kept in
// float64 (one conversion per lane and column).
__global__ void __launch_bounds__(256, 3) k_leaf_agg_mx(LeafParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = wid; t < p.n_tiles; t += nwarps) {
    const int64_t e0 = t * kHtTile + (int64_t)lane * kHtItems;
    LeafRow rw[kHtItems];
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) rw[i] = leaf_row(p, e0 + i);
    mark_tail_tile(p, rw, t, lane);
    for (int c = 0; c < p.N; ++c) {
      double xs[kHtItems];
      load_leaf_items(p, rw, e0, c, p.sorted_ready != 0, xs);
      int f = 0;
      dfl s{0.0f, 0.0f};
      int open_g = -1;                     // as in k_leaf_agg
      dfl open_s{0.0f, 0.0f};
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const dfl x = df_from_double(xs[i]);
        if (rw[i].pos == 0) { f = 1; s = x; } else { s = df_add(s, x); }
        // the pair to float64 by integer instructions (df_to_double_int): a conversion on
        // the FP64 pipe would be if-converted and issued for every element
        if (rw[i].last) {
          if (f) p.heads[(int64_t)c * p.ldh + rw[i].g] = df_to_double_int(s.hi, s.lo) * __ldg(p.hrow + rw[i].g);
          else { open_g = rw[i].g; open_s = s; }
        }
      }
      pair_scan_incl_df(f, s, lane);
      int fe = __shfl_up_sync(0xffffffffu, f, 1);
      float eh = __shfl_up_sync(0xffffffffu, s.hi, 1), el = __shfl_up_sync(0xffffffffu, s.lo, 1);
      if (lane == 0) { fe = 0; eh = 0.0f; el = 0.0f; }
      const int64_t slot = (int64_t)c * p.n_tiles + t;
      if (p.lflag) {
        p.lflag[slot * 32 + lane] = (uint8_t)fe;
        p.lsum[slot * 32 + lane] = df_to_double(dfl{eh, el});
      }
      if (lane == 31) {
        p.tflag[slot] = (uint8_t)f;
        p.tsum[slot] = df_to_double(s);
      }
      if (open_g >= 0) {
        const dfl hs = df_add(dfl{eh, el}, open_s);
        const double h = df_to_double_int(hs.hi, hs.lo);
        p.heads[(int64_t)c * p.ldh + open_g] = fe ? h * __ldg(p.hrow + open_g) : h;
      }
    }
  }
}

// Latency-bound: three blocks per SM on the mixed path (80 registers); the refinement's
// variant (LO, the low floats kept too) holds more state and stays at two.
template <bool LO>
__global__ void __launch_bounds__(256, LO ? 2 : 3) k_leaf_emit_mx(LeafParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = wid; t < p.n_tiles; t += nwarps) {
    if (p.ttail && !p.ttail[t]) continue;   // single-row groups only: no tail to write
    const int64_t e0 = t * kHtTile + (int64_t)lane * kHtItems;
    LeafRow rw[kHtItems];
    dfl gam[kHtItems];                    // sqrt(Phi_circ) beta_p (the low part only when refining)
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) {
      rw[i] = leaf_row(p, e0 + i);
      const bool tail = rw[i].ok && rw[i].pos > 0;
      const double g = tail ? p.sq_phic[rw[i].g] * p.beta[rw[i].pos].x : 0.0;
      gam[i] = LO ? df_from_double(g) : dfl{(float)g, 0.0f};
    }
    for (int c = 0; c < p.N; ++c) {
      const int64_t slot = (int64_t)c * p.n_tiles + t;
      const int fe = p.lflag[slot * 32 + lane];
      const double se = p.lsum[slot * 32 + lane];
      dfl run = df_from_double(fe ? se : p.tcarry[slot] + se);
      float* tcol = p.tails32 + (int64_t)c * p.ldt;
      double xs[kHtItems];
      load_leaf_items(p, rw, e0, c, p.sdata != nullptr, xs);
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const dfl x = df_from_double(xs[i]);
        if (rw[i].pos == 0) run = dfl{0.0f, 0.0f};
        if (rw[i].pos > 0) {
          // p as a float pair, formed again per column (a few FP32 operations) rather than
          // held in registers for the whole tile
          const dfl d = df_add(df_mul(x, df_from_count(rw[i].pos)), df_neg(run));
          const int64_t row = e0 + i - rw[i].g - 1;
          if (LO) {                        // the double-float tail, kept for the refinement's Gram
            const dfl tt = df_mul(d, gam[i]);
            tcol[row] = tt.hi;
            p.tails32lo[(int64_t)c * p.ldt + row] = tt.lo;
          } else {
            tcol[row] = gam[i].hi * (d.hi + d.lo);
          }
        }
        run = df_add(run, x);
      }
    }
  }
}

static unsigned ht_grid(int64_t n_tiles) {
  // 8 warps per block; enough blocks to cover all tiles, capped at 16 blocks per SM
  int64_t blocks = (n_tiles + 7) / 8;
  if (blocks < 1) blocks = 1;
  if (blocks > 152 * 16) blocks = 152 * 16;
  return (unsigned)blocks;
}

// The head of the group that ends in tile t but began in an earlier tile (if any): its sum
// from the tile start, written by the first pass, plus the tile's carry, times
// 1 / sqrt(rows).  One thread per tile and column.
__global__ void k_heads_fix(LeafParams p) {
  const int64_t total = p.n_tiles * (int64_t)p.N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = k / p.n_tiles, t = k - c * p.n_tiles;
    const int64_t e = t * kHtTile;
    const int32_t g = p.row_gid[e];
    if ((int64_t)p.goff[g] >= e || (int64_t)p.goff[g + 1] - 1 >= e + kHtTile) continue;
    double* h = p.heads + c * p.ldh + g;
    *h = (*h + p.tcarry[k]) * p.hrow[g];
  }
}

void leaf_heads(const LeafParams& p, cudaStream_t st, int64_t* launches) {
  if (p.N == 0) return;
  const unsigned g = ht_grid(p.n_tiles);
  if (p.mixed) k_leaf_agg_mx<<<g, 256, 0, st>>>(p);
  else k_leaf_agg<<<g, 256, 0, st>>>(p);
  k_tile_carry<<<p.N, kCarryThreads, 0, st>>>(p.tflag, p.tsum, p.tcarry, p.n_tiles, nullptr);
  k_heads_fix<<<grid_for(p.n_tiles * (int64_t)p.N, 256, 152 * 8), 256, 0, st>>>(p);
  *launches += 3;
}

void leaf_tails(const LeafParams& p, cudaStream_t st, int64_t* launches) {
  if (p.N == 0) return;
  const unsigned g = ht_grid(p.n_tiles);
  if (p.mixed && p.tails32lo) k_leaf_emit_mx<true><<<g, 256, 0, st>>>(p);
  else if (p.mixed) k_leaf_emit_mx<false><<<g, 256, 0, st>>>(p);
  else k_leaf_emit<<<g, 256, 0, st>>>(p);
  ++*launches;
}

// ------------------------------------------------------------------ join + projection
struct GenRow {
  int32_t g, pg, trow, k;   // group, X_p group, output row, position inside the X_p group
  double v;                 // weight sqrt(Theta_down)
  bool ok, last;
};

__device__ __forceinline__ GenRow gen_row(const GenParams& p, int64_t e, int64_t G) {
  GenRow r;
  r.ok = e < G;
  if (!r.ok) { r.g = 0; r.pg = 0; r.trow = 0; r.k = 1; r.v = 0.0; r.last = false; return r; }
  r.g = (int32_t)e;
  r.pg = p.g2p[e];
  const int32_t start = p.pgoff[r.pg];
  r.k = (int32_t)(e - start);
  r.last = (e == (int64_t)p.pgoff[r.pg + 1] - 1);
  r.trow = (int32_t)(e - r.pg - 1);
  r.v = p.vw[e * 3 + 0];
  return r;
}

// Data[x_i : column] of process_and_join_children (Alg. 4) for every group, column-major
// (J[c * ldj + g]): the own heads times prod_j s_j, or the child's passed-up row (looked up
// at x_ij) times sqrt(rows) prod_{j' != j} s_j' (factors in fac; 0 where x_ij is missing).
// The own heads go with lanes over groups (coalesced); the children's rows are read whole
// from their row-major copies (lanes over columns) into a shared tile and written as column
// segments of 32 groups.
constexpr int kGatherMaxCols = 1024;

// x f as a float64, or (PAIRS) as a double-float product stored as the pair's bits
template <bool PAIRS>
__device__ __forceinline__ double scaled(double x, double f) {
  if (!PAIRS) return x * f;
  const dfl r = df_mul(df_from_double(x), df_from_double(f));
  return __hiloint2double(__float_as_int(r.hi), __float_as_int(r.lo));
}

// PAIRS (the mixed path's joined Data): every value and factor is split into a float pair
// (exactly enough, 2^-47, by integer instructions), the product formed in double-float on
// the FP32 pipe and stored as the pair's bits in the float64 slot, so that neither this
// kernel nor the two scans that read it issue FP64 instructions per value.
template <bool PAIRS>
__global__ void __launch_bounds__(256) k_gen_gather(GenParams p, double* J, int64_t ldj) {
  __shared__ double tile[32][33];
  __shared__ int2 cd[kGatherMaxCols];              // column descriptors (N <= 1024)
  __shared__ int32_t qs[kMaxChildren][32];         // the tile's row of every child's table
  __shared__ double fs[kMaxChildren + 1][32];      // the tile's join factors
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nf = 1 + p.n_child;
  const int64_t G = p.sizes[0];
  const int64_t tiles = (G + 31) >> 5;
  for (int c = threadIdx.x; c < p.N; c += blockDim.x) cd[c] = p.coldesc[c];
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t g0 = t * 32;
    __syncthreads();                                 // cd written; the previous tile's reads done
    for (int idx = threadIdx.x; idx < 32 * nf; idx += blockDim.x) {
      const int f = idx >> 5, r = idx & 31;
      const int64_t g = g0 + r;
      fs[f][r] = g < G ? p.fac[g * nf + f] : 0.0;
      if (f > 0) qs[f - 1][r] = g < G ? p.q[(int64_t)(f - 1) * p.M + g] : -1;
    }
    __syncthreads();
    const int64_t g = g0 + lane;
    // own heads: lanes over groups, four columns in flight per warp
    for (int c0 = warp; c0 < p.N; c0 += 32) {
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + 8 * u;
        v[u] = 0.0;
        if (c < p.N && cd[c].x == 0 && g < G) v[u] = p.heads[(int64_t)cd[c].y * p.ldh + g];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + 8 * u;
        if (c < p.N && cd[c].x == 0 && g < G) J[(int64_t)c * ldj + g] = scaled<PAIRS>(v[u], fs[0][lane]);
      }
    }
    // children's rows: lanes over columns, the warp's four rows loaded before they are used
    for (int cc = 0; cc < p.N; cc += 32) {
      const int c = cc + lane;
      const int2 d = c < p.N ? cd[c] : make_int2(0, 0);
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = warp + 8 * u;
        v[u] = 0.0;
        if (d.x > 0) {
          const int32_t q = qs[d.x - 1][r];
          if (q >= 0) v[u] = p.crow[d.x - 1][(int64_t)q * p.cnp[d.x - 1] + d.y];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = warp + 8 * u;
        tile[r][lane] = d.x > 0 ? scaled<PAIRS>(v[u], fs[d.x][r]) : 0.0;
      }
      __syncthreads();
      for (int c2 = cc + warp; c2 < cc + 32 && c2 < p.N; c2 += 8)
        if (cd[c2].x > 0 && g < G) J[(int64_t)c2 * ldj + g] = tile[lane][c2 - cc];
      __syncthreads();
    }
  }
}

// kHtItems joined values of column c for one lane's consecutive groups (16-byte loads)
__device__ __forceinline__ void load_joined(const GenParams& p, const GenRow (&rw)[kHtItems], int64_t e0, int c,
                                            int64_t G, double (&Ds)[kHtItems]) {
  const double* col = p.jdata + (int64_t)c * p.ldj + e0;
  if (e0 + kHtItems <= G) {
#pragma unroll
    for (int i = 0; i < kHtItems; i += 2) {
      const double2 v = *reinterpret_cast<const double2*>(col + i);
      Ds[i] = v.x;
      Ds[i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) Ds[i] = rw[i].ok ? col[i] : 0.0;
  }
}

// The same values of the mixed path's joined Data, stored as float pairs
__device__ __forceinline__ void load_joined_pairs(const GenParams& p, const GenRow (&rw)[kHtItems], int64_t e0,
                                                  int c, int64_t G, dfl (&Ds)[kHtItems]) {
  const float2* col = reinterpret_cast<const float2*>(p.jdata + (int64_t)c * p.ldj + e0);
  if (e0 + kHtItems <= G) {
#pragma unroll
    for (int i = 0; i < kHtItems; i += 2) {
      const float4 v = *reinterpret_cast<const float4*>(col + i);
      Ds[i] = dfl{v.y, v.x};                 // the hi float is the upper half of the slot
      Ds[i + 1] = dfl{v.w, v.z};
    }
  } else {
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) {
      const float2 v = rw[i].ok ? col[i] : make_float2(0.0f, 0.0f);
      Ds[i] = dfl{v.y, v.x};
    }
  }
}

__global__ void __launch_bounds__(256) k_gen_agg(GenParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t G = p.sizes[0];
  const int64_t nt = (G + kHtTile - 1) / kHtTile;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = wid; t < nt; t += nwarps) {
    const int64_t e0 = t * kHtTile + (int64_t)lane * kHtItems;
    GenRow rw[kHtItems];
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) rw[i] = gen_row(p, e0 + i, G);
    for (int c = 0; c < p.N; ++c) {
      double Ds[kHtItems];
      load_joined(p, rw, e0, c, G, Ds);
      int f = 0;
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const double x = rw[i].v * Ds[i];
        if (rw[i].k == 0) { f = 1; s = x; } else { s += x; }
      }
      const int64_t slot = (int64_t)c * p.n_tiles + t;
      store_lane_and_tile(f, s, lane, slot, slot, p.lflag, p.lsum, p.tflag, p.tsum);
    }
  }
}

// Generalized tail gamma (W D - v P) = (gamma W) D - (gamma v) P with P the running sum
// of v D over the earlier groups of the same x_p.
__global__ void __launch_bounds__(256, 2) k_gen_emit(GenParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t G = p.sizes[0];
  const int64_t nt = (G + kHtTile - 1) / kHtTile;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = wid; t < nt; t += nwarps) {
    const int64_t e0 = t * kHtTile + (int64_t)lane * kHtItems;
    GenRow rw[kHtItems];
    double gw[kHtItems], gv[kHtItems];
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) {
      rw[i] = gen_row(p, e0 + i, G);
      const double W = rw[i].ok ? p.vw[(int64_t)rw[i].g * 3 + 1] : 0.0;
      const double gam = rw[i].ok ? p.vw[(int64_t)rw[i].g * 3 + 2] : 0.0;
      gw[i] = gam * W;
      gv[i] = gam * rw[i].v;
    }
    for (int c = 0; c < p.N; ++c) {
      const int64_t slot = (int64_t)c * p.n_tiles + t;
      const int fe = p.lflag[slot * 32 + lane];
      const double se = p.lsum[slot * 32 + lane];
      double run = fe ? se : p.tcarry[slot] + se;
      double Ds[kHtItems];
      load_joined(p, rw, e0, c, G, Ds);
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const double D = Ds[i];
        if (rw[i].k == 0) run = 0.0;
        if (rw[i].k > 0) p.gtails[(int64_t)c * p.M + rw[i].trow] = fma(gw[i], D, -gv[i] * run);
        run = fma(rw[i].v, D, run);
        if (rw[i].last) p.data2[(int64_t)c * p.M + rw[i].pg] = run;   // scaled by gen_heads_finish
      }
    }
  }
}

// ------------------------------------------------------------------ mixed precision (join)
// The generalized head/tail scans of the mixed path on the FP32 pipe: the weights v, W and
// gamma of every group and the joined values are split into float pairs (exactly enough,
// 2^-47), the running sum P of v D and W D - v P are formed in double-float, and each tail
// is rounded once to float for the float TSQR leaf.  Carries between lanes and tiles stay
// float64 (one conversion per lane and column); the X_p group sums are stored as a float
// pair's bits and finished by k_gen_heads_finish.
__global__ void __launch_bounds__(256) k_gen_agg_mx(GenParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t G = p.sizes[0];
  const int64_t nt = (G + kHtTile - 1) / kHtTile;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = wid; t < nt; t += nwarps) {
    const int64_t e0 = t * kHtTile + (int64_t)lane * kHtItems;
    GenRow rw[kHtItems];
    dfl vv[kHtItems];
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) {
      rw[i] = gen_row(p, e0 + i, G);
      vv[i] = df_from_double(rw[i].v);
    }
    for (int c = 0; c < p.N; ++c) {
      dfl Ds[kHtItems];
      load_joined_pairs(p, rw, e0, c, G, Ds);
      int f = 0;
      dfl s{0.0f, 0.0f};
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const dfl x = df_mul(vv[i], Ds[i]);
        if (rw[i].k == 0) { f = 1; s = x; } else { s = df_add(s, x); }
      }
      pair_scan_incl_df(f, s, lane);
      int fe = __shfl_up_sync(0xffffffffu, f, 1);
      float eh = __shfl_up_sync(0xffffffffu, s.hi, 1), el = __shfl_up_sync(0xffffffffu, s.lo, 1);
      if (lane == 0) { fe = 0; eh = 0.0f; el = 0.0f; }
      const int64_t slot = (int64_t)c * p.n_tiles + t;
      p.lflag[slot * 32 + lane] = (uint8_t)fe;
      p.lsum[slot * 32 + lane] = df_to_double(dfl{eh, el});
      if (lane == 31) {
        p.tflag[slot] = (uint8_t)f;
        p.tsum[slot] = df_to_double(s);
      }
    }
  }
}

// gtail = gamma (W D - v P), rounded once to float
__global__ void __launch_bounds__(256, 2) k_gen_emit_mx(GenParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t G = p.sizes[0];
  const int64_t nt = (G + kHtTile - 1) / kHtTile;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = wid; t < nt; t += nwarps) {
    const int64_t e0 = t * kHtTile + (int64_t)lane * kHtItems;
    GenRow rw[kHtItems];
    dfl vv[kHtItems], ww[kHtItems];
    float gam[kHtItems];
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) {
      rw[i] = gen_row(p, e0 + i, G);
      vv[i] = df_from_double(rw[i].v);
      ww[i] = rw[i].ok ? df_from_double(p.vw[(int64_t)rw[i].g * 3 + 1]) : dfl{0.0f, 0.0f};
      gam[i] = rw[i].ok ? df_from_double(p.vw[(int64_t)rw[i].g * 3 + 2]).hi : 0.0f;
    }
    for (int c = 0; c < p.N; ++c) {
      const int64_t slot = (int64_t)c * p.n_tiles + t;
      const int fe = p.lflag[slot * 32 + lane];
      const double se = p.lsum[slot * 32 + lane];
      dfl run = df_from_double(fe ? se : p.tcarry[slot] + se);
      dfl Ds[kHtItems];
      load_joined_pairs(p, rw, e0, c, G, Ds);
      float* tcol = p.gtails32 + (int64_t)c * p.M;
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const dfl D = Ds[i];
        if (rw[i].k == 0) run = dfl{0.0f, 0.0f};
        if (rw[i].k > 0) {
          const dfl d = df_add(df_mul(ww[i], D), df_neg(df_mul(vv[i], run)));
          tcol[rw[i].trow] = gam[i] * (d.hi + d.lo);
        }
        run = df_add(run, df_mul(vv[i], D));
        if (rw[i].last)
          p.data2[(int64_t)c * p.M + rw[i].pg] = __hiloint2double(__float_as_int(run.hi), __float_as_int(run.lo));
      }
    }
  }
}

// Generalized head of every X_p group: the weighted group sum times 1 / sqrt(Phi_down).
__global__ void k_gen_heads_finish(GenParams p) {
  const int64_t P = p.sizes[1];
  const int64_t total = P * p.N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = k / P, q = k - c * P;
    double s = p.data2[c * p.M + q];
    if (p.gtails32) s = df_to_double_int(__int_as_float(__double2hiint(s)), __int_as_float(__double2loint(s)));
    p.data2[c * p.M + q] = s * p.hf[q];
  }
}

static unsigned gather_grid(int64_t rows) {
  const int64_t tiles = (rows + 31) / 32;
  return (unsigned)(tiles < 1 ? 1 : (tiles < 152 * 8 ? tiles : 152 * 8));
}

void gen_heads_tails(const GenParams& p, cudaStream_t st, int64_t* launches) {
  if (p.is_root) {          // Out.append(Data): the joined Data is the root block itself
    k_gen_gather<false><<<gather_grid(p.M), 256, 0, st>>>(p, p.rootrows, p.M);
    ++*launches;
    return;
  }
  if (p.gtails32) k_gen_gather<true><<<gather_grid(p.M), 256, 0, st>>>(p, const_cast<double*>(p.jdata), p.ldj);
  else k_gen_gather<false><<<gather_grid(p.M), 256, 0, st>>>(p, const_cast<double*>(p.jdata), p.ldj);
  const unsigned g = ht_grid(p.n_tiles);
  if (p.gtails32) k_gen_agg_mx<<<g, 256, 0, st>>>(p);
  else k_gen_agg<<<g, 256, 0, st>>>(p);
  k_tile_carry<<<p.N, kCarryThreads, 0, st>>>(p.tflag, p.tsum, p.tcarry, p.n_tiles, p.sizes);
  if (p.gtails32) k_gen_emit_mx<<<g, 256, 0, st>>>(p);
  else k_gen_emit<<<g, 256, 0, st>>>(p);
  k_gen_heads_finish<<<grid_for(p.M * (int64_t)p.N, 256, 152 * 8), 256, 0, st>>>(p);
  *launches += 5;
}

}  // namespace fig
