// Heads and tails (Def. "Head and Tail", Def. "Generalized Head and Tail", Alg. 2) as
// flat segmented scans over key-sorted rows.
//
// The paper loops over join keys in parallel (§6); with Zipf-skewed keys one group can
// hold a sixth of a relation, so here the sorted rows are cut into fixed tiles of
// 256 elements per warp regardless of group boundaries.  Per column, a prefix sum that
// restarts at every group start is computed in three steps: (1) every tile reports
// whether it contains a group start and the sum after its last start, (2) one thread
// block per column scans those tile aggregates into a carry per tile, (3) every tile recomputes its
// prefix sums with the carry and writes tail rows and heads.
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

__device__ __forceinline__ double beta_at(const double* beta, int64_t len, int64_t p) {
  return p < len ? beta[p] : 1.0 / sqrt((double)p * ((double)p + 1.0));
}

__global__ void k_beta(double* beta, int64_t len) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < len;
       p += (int64_t)gridDim.x * blockDim.x)
    beta[p] = p == 0 ? 0.0 : 1.0 / sqrt((double)p * ((double)p + 1.0));
}

void beta_table(double* beta, int64_t len, cudaStream_t st) {
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

// ------------------------------------------------------------------ relations (v = 1)
struct LeafRow {
  int64_t src;   // input row
  int64_t pos;   // position inside the group
  int32_t g;
  bool ok, last;
};

__device__ __forceinline__ LeafRow leaf_row(const LeafParams& p, int64_t e) {
  LeafRow r;
  r.ok = e < p.M;
  if (!r.ok) { r.src = 0; r.pos = 1; r.g = 0; r.last = false; return r; }
  r.src = p.perm ? (int64_t)p.perm[e] : e;
  r.g = p.row_gid[e];
  const int32_t start = p.goff[r.g];
  r.pos = e - start;
  r.last = (e == (int64_t)p.goff[r.g + 1] - 1);
  return r;
}

__global__ void __launch_bounds__(256) k_leaf_agg(LeafParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = wid; t < p.n_tiles; t += nwarps) {
    const int64_t e0 = t * kHtTile + (int64_t)lane * kHtItems;
    LeafRow rw[kHtItems];
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) rw[i] = leaf_row(p, e0 + i);
    for (int c = 0; c < p.N; ++c) {
      int f = 0;
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const double x = p.data[rw[i].src * p.rs + (int64_t)c * p.cs];
        if (rw[i].pos == 0) { f = 1; s = x; } else { s += x; }
      }
      pair_scan_incl(f, s, lane);
      if (lane == 31) {
        p.tflag[(int64_t)c * p.n_tiles + t] = (uint8_t)f;
        p.tsum[(int64_t)c * p.n_tiles + t] = s;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_leaf_emit(LeafParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = wid; t < p.n_tiles; t += nwarps) {
    const int64_t e0 = t * kHtTile + (int64_t)lane * kHtItems;
    LeafRow rw[kHtItems];
    double gam[kHtItems];
#pragma unroll
    for (int i = 0; i < kHtItems; ++i) {
      rw[i] = leaf_row(p, e0 + i);
      gam[i] = (rw[i].ok && rw[i].pos > 0) ? p.sq_phic[rw[i].g] * beta_at(p.beta, p.beta_len, rw[i].pos) : 0.0;
    }
    for (int c = 0; c < p.N; ++c) {
      double x[kHtItems], loc[kHtItems];
      bool use_carry[kHtItems];
      double run = 0.0;
      int seen = 0;
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        x[i] = rw[i].ok ? p.data[rw[i].src * p.rs + (int64_t)c * p.cs] : 0.0;
        if (rw[i].ok && rw[i].pos == 0) { run = 0.0; seen = 1; }
        loc[i] = run;
        use_carry[i] = !seen;
        run += x[i];
      }
      int fi = seen;
      double si = run;
      pair_scan_incl(fi, si, lane);
      int fe = __shfl_up_sync(0xffffffffu, fi, 1);
      double se = __shfl_up_sync(0xffffffffu, si, 1);
      if (lane == 0) { fe = 0; se = 0.0; }
      const double lane_carry = fe ? se : p.tcarry[(int64_t)c * p.n_tiles + t] + se;
      double* tcol = p.tails + (int64_t)c * p.ldt;
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const double S = use_carry[i] ? lane_carry + loc[i] : loc[i];
        if (rw[i].pos > 0)
          tcol[e0 + i - rw[i].g - 1] = gam[i] * fma((double)rw[i].pos, x[i], -S);
        if (rw[i].last)
          p.heads[(int64_t)c * p.ldh + rw[i].g] = (S + x[i]) * p.hrow[rw[i].g];
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

void leaf_heads_tails(const LeafParams& p, cudaStream_t st, int64_t* launches) {
  if (p.N == 0) return;
  const unsigned g = ht_grid(p.n_tiles);
  k_leaf_agg<<<g, 256, 0, st>>>(p);
  k_tile_carry<<<p.N, kCarryThreads, 0, st>>>(p.tflag, p.tsum, p.tcarry, p.n_tiles, nullptr);
  k_leaf_emit<<<g, 256, 0, st>>>(p);
  *launches += 3;
}

// ------------------------------------------------------------------ join + projection
struct GenRow {
  int32_t g, pg, trow;
  int64_t k;       // position inside the X_p group
  double v, W, gam;
  bool ok, last;
};

__device__ __forceinline__ GenRow gen_row(const GenParams& p, int64_t e, int64_t G) {
  GenRow r;
  r.ok = e < G;
  if (!r.ok) { r.g = 0; r.pg = 0; r.trow = 0; r.k = 1; r.v = r.W = r.gam = 0.0; r.last = false; return r; }
  r.g = (int32_t)e;
  r.pg = p.g2p[e];
  const int32_t start = p.pgoff[r.pg];
  r.k = e - start;
  r.last = (e == (int64_t)p.pgoff[r.pg + 1] - 1);
  r.trow = (int32_t)(e - r.pg - 1);
  r.v = p.vw[e * 3 + 0];
  r.W = p.vw[e * 3 + 1];
  r.gam = p.vw[e * 3 + 2];
  return r;
}

// Data[x_i : column] of process_and_join_children (Alg. 4): own heads times prod_j s_j, or
// the child's generalized heads (looked up at x_ij) times sqrt(rows) prod_{j' != j} s_j'.
__device__ __forceinline__ double join_value(const GenParams& p, int32_t g, int2 d) {
  const int nf = 1 + p.n_child;
  double src;
  if (d.x == 0) {
    src = p.heads[(int64_t)d.y * p.ldh + g];
  } else {
    const int32_t q = p.q[(int64_t)(d.x - 1) * p.M + g];
    if (q < 0) return 0.0;
    src = p.cdata[d.x - 1][(int64_t)d.y * p.cld[d.x - 1] + q];
  }
  return src * p.fac[(int64_t)g * nf + d.x];
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
      const int2 d = p.coldesc[c];
      int f = 0;
      double s = 0.0;
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const double x = rw[i].v * join_value(p, rw[i].g, d);
        if (rw[i].k == 0) { f = 1; s = x; } else { s += x; }
      }
      pair_scan_incl(f, s, lane);
      if (lane == 31) {
        p.tflag[(int64_t)c * p.n_tiles + t] = (uint8_t)f;
        p.tsum[(int64_t)c * p.n_tiles + t] = s;
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_gen_emit(GenParams p) {
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
      const int2 d = p.coldesc[c];
      double D[kHtItems], loc[kHtItems];
      bool use_carry[kHtItems];
      double run = 0.0;
      int seen = 0;
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        D[i] = rw[i].ok ? join_value(p, rw[i].g, d) : 0.0;
        if (rw[i].ok && rw[i].k == 0) { run = 0.0; seen = 1; }
        loc[i] = run;
        use_carry[i] = !seen;
        run += rw[i].v * D[i];
      }
      int fi = seen;
      double si = run;
      pair_scan_incl(fi, si, lane);
      int fe = __shfl_up_sync(0xffffffffu, fi, 1);
      double se = __shfl_up_sync(0xffffffffu, si, 1);
      if (lane == 0) { fe = 0; se = 0.0; }
      const double lane_carry = fe ? se : p.tcarry[(int64_t)c * p.n_tiles + t] + se;
#pragma unroll
      for (int i = 0; i < kHtItems; ++i) {
        if (!rw[i].ok) continue;
        const double P = use_carry[i] ? lane_carry + loc[i] : loc[i];
        if (rw[i].k > 0)
          p.gtails[(int64_t)c * p.M + rw[i].trow] = rw[i].gam * fma(rw[i].W, D[i], -rw[i].v * P);
        if (rw[i].last)
          p.data2[(int64_t)c * p.M + rw[i].pg] = fma(rw[i].v, D[i], P) * p.hf[rw[i].pg];
      }
    }
  }
}

// Root: Out.append(Data) -- one row per root group over all N columns.
__global__ void k_root_rows(GenParams p) {
  const int64_t G = p.sizes[0];
  const int64_t total = G * p.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / G, g = i - c * G;
    p.rootrows[c * p.M + g] = join_value(p, (int32_t)g, p.coldesc[c]);
  }
}

void gen_heads_tails(const GenParams& p, cudaStream_t st, int64_t* launches) {
  if (p.is_root) {
    k_root_rows<<<grid_for(p.M * (int64_t)p.N, 256, 152 * 16), 256, 0, st>>>(p);
    ++*launches;
    return;
  }
  const unsigned g = ht_grid(p.n_tiles);
  k_gen_agg<<<g, 256, 0, st>>>(p);
  k_tile_carry<<<p.N, kCarryThreads, 0, st>>>(p.tflag, p.tsum, p.tcarry, p.n_tiles, p.sizes);
  k_gen_emit<<<g, 256, 0, st>>>(p);
  *launches += 3;
}

}  // namespace fig
