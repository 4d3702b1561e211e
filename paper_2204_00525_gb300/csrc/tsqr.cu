// Post-processing of R0 (§7) as a tall-skinny QR.
//
// §7 triangularizes every non-zero block of R0 (tails of a relation, generalized tails
// of a node, the root Data) on its own columns and then the stack of the resulting
// triangles.  Each block is cut into row tiles; every tile is reduced by Householder
// QR to an n x n triangle (leaf), groups of `fan` triangles are stacked and reduced
// again until one triangle per block remains (tree).  The block triangles, placed at
// their global columns, form one more block (the stack) that goes through the same leaf
// and tree kernels; its triangle, sign-normalised, is R.  The paper's own choices were
// Householder (MKL) or per-thread Givens (THIN); the TSQR tree is the GPU form of the
// same block-then-stack scheme.
//
// Two kernels do the QR of a tile:
//   n <= 32: one warp per tile, the tile in registers (k_tsqr_reg), every loop bound a
//            compile-time constant so that no predicated-off FP64 instruction is issued;
//   n >  32: one thread block per tile in shared memory (k_tsqr_cta).
// Both are persistent over the live tiles: the row counts are only known on the device.
//
// Precision: FP64 throughout, or (mixed) FP32 leaf tiles and tree levels with the final QR
// of the stacked block triangles in FP64.
#include "tsqr_reg.cuh"

namespace fig {

constexpr int kQrThreads = 256;   // 8 warps: hh_small's row classes
constexpr int kRedElems = 320;     // reduction scratch ahead of the tile in shared memory
constexpr int kGivensRows = 32;    // rows per thread of the Givens leaf
constexpr size_t kSmemCap = 200 * 1024;

// ------------------------------------------------------------------ block path (n > 32)
// Householder QR of the m x n column-major matrix A (leading dimension lda) by the
// whole thread block.  On return the upper triangle of A[0:min(m,n), :] holds R.
template <typename E>
__device__ void hh_qr(E* A, int lda, int m, int n, E* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int kmax = m < n ? m : n;
  // red[0..32]: block_sum scratch; red[40..42]: the step's scalars (computed by one lane:
  // FP64 square roots and divisions cost some twenty FMA slots each on this part)
  for (int k = 0; k < kmax; ++k) {
    E* ak = A + (int64_t)k * lda;
    E s = 0;
    for (int i = k + 1 + tid; i < m; i += blockDim.x) s = fma(ak[i], ak[i], s);
    s = block_sum<E>(s, red);
    if (s == E(0)) continue;                        // uniform: column already reduced
    if (tid == 0) {
      const E alpha = ak[k];
      const E normx = sqrt(fma(alpha, alpha, s));
      const E beta = alpha >= E(0) ? -normx : normx;
      red[40] = (beta - alpha) / beta;                // tau
      red[41] = E(1) / (alpha - beta);                // scale of v (v_k = 1)
      red[42] = beta;
    }
    __syncthreads();
    const E tau = red[40], scal = red[41];
    for (int i = k + 1 + tid; i < m; i += blockDim.x) ak[i] *= scal;
    __syncthreads();
    if (tid == 0) ak[k] = red[42];
    for (int j = k + 1 + warp; j < n; j += nw) {
      E* aj = A + (int64_t)j * lda;
      const E ajk = aj[k];
      E w = 0;
      for (int i = k + 1 + lane; i < m; i += 32) w = fma(ak[i], aj[i], w);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
      w = (w + ajk) * tau;
      if (lane == 0) aj[k] = ajk - w;
      for (int i = k + 1 + lane; i < m; i += 32) aj[i] = fma(-w, ak[i], aj[i]);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ narrow tiles (n <= 32)
constexpr int kSmallRed = 8 * 32 + 32 + 8;   // per-warp partial dot products, w, scalars

// Householder QR of an m x n tile (n <= 32, column-major in shared memory) by 8 warps,
// shaped for latency: per step one pass of dot products d_j = sum_{i>k} a_ik a_ij
// (j >= k, d_k = sigma) with lane = column and warp = row class, a three-level tree over
// the warps, the scalars in warp 0, and one update pass a_ij -= w_j a_ik with
// w_j = tau (v0 a_kj + d_j); row k becomes a_kj - w_j v0 and a_kk = beta.
template <typename E>
__device__ void hh_small(E* A, int lda, int m, int n, E* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  E* part = red;               // [8][32]
  E* w = red + 256;            // [32]
  E* sc = red + 288;           // v0
  const int kmax = m < n ? m : n;
  for (int k = 0; k < kmax; ++k) {
    const int j = k + lane;
    const E* ak = A + (int64_t)k * lda;
    E d = 0;
    if (j < n) {
      const E* aj = A + (int64_t)j * lda;
      for (int i = k + 1 + warp; i < m; i += 8) d = fma(ak[i], aj[i], d);
    }
    part[warp * 32 + lane] = d;
    __syncthreads();
    if (warp < 4) part[warp * 32 + lane] += part[(warp + 4) * 32 + lane];
    __syncthreads();
    if (warp < 2) part[warp * 32 + lane] += part[(warp + 2) * 32 + lane];
    __syncthreads();
    if (warp == 0) {
      const E dj = part[lane] + part[32 + lane];
      const E sigma = __shfl_sync(0xffffffffu, dj, 0);
      E wj = 0;
      if (!f64_is_zero(sigma)) {                 // warp-uniform
        const E alpha = ak[k];
        const bool mine = j < n && lane > 0;
        E* aj = A + (int64_t)(mine ? j : k) * lda;
        const E akj = mine ? aj[k] : E(0);
        __syncwarp();                            // every read of row k before its writes
        E beta, v0, tau;
        HhScalars<E>::get(alpha, sigma, beta, v0, tau);
        if (mine) {
          wj = tau * fma(v0, akj, dj);
          aj[k] = akj - wj * v0;
        }
        if (lane == 0) A[(int64_t)k * lda + k] = beta;
      }
      w[lane] = wj;
      if (lane == 0) sc[0] = sigma;
    }
    __syncthreads();
    if (sc[0] != E(0) && lane > 0 && j < n) {
      const E wj = w[lane];
      E* aj = A + (int64_t)j * lda;
      for (int i = k + 1 + warp; i < m; i += 8) aj[i] = fma(-wj, ak[i], aj[i]);
    }
    __syncthreads();
  }
}

// Leading dimension of a tile in the block kernel: the tile's row count rounded up to an
// odd number, so that hh_small's lanes (one column each) fall in distinct banks.
__host__ __device__ __forceinline__ int cta_lda(const TsqrBlock& b, bool tree) {
  return (tree ? b.fan * b.n : b.tile) | 1;
}

// One thread block per tile (persistent).  The tile sits in shared memory, or in a
// global scratch slot per block when it does not fit.
// With few_only set (tree levels that the warp-per-tile kernel also serves) it works only
// on levels with fewer than b.warp_min tiles.
template <typename E>
__global__ void __launch_bounds__(kQrThreads) k_tsqr_cta(TsqrBlock b, const double* tri_in, double* tri_out,
                                                         int64_t div_in, E* gscratch, int few_only) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t rows = block_rows(b);
  if (copy_single(b, rows, div_in, tri_in, tri_out)) return;
  if (few_only && level_tiles(b, rows, div_in, tri_in == nullptr) >= b.warp_min) return;
  const int n = b.n;
  const int lda = cta_lda(b, tri_in != nullptr);
  E* red = reinterpret_cast<E*>(smem_raw);
  E* A = gscratch ? gscratch + (int64_t)blockIdx.x * lda * n : red + kRedElems;
  const int64_t nt_in = tri_in ? (rows + div_in - 1) / div_in : 0;
  const int64_t n_tiles = level_tiles(b, rows, div_in, tri_in == nullptr);
  for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    int m;
    if (!tri_in) {
      const int64_t r0 = t * b.tile;
      m = (int)((rows - r0) < b.tile ? (rows - r0) : b.tile);
      if (b.ptr32) {
        for (int c = 0; c < n; ++c)
          for (int i = threadIdx.x; i < m; i += blockDim.x) A[(int64_t)c * lda + i] = (E)b.ptr32[(int64_t)c * b.ld + r0 + i];
      } else {
        for (int c = 0; c < n; ++c)
          for (int i = threadIdx.x; i < m; i += blockDim.x) A[(int64_t)c * lda + i] = (E)b.ptr[(int64_t)c * b.ld + r0 + i];
      }
    } else {
      const int64_t first = t * b.fan;
      const int cnt = (int)((nt_in - first) < b.fan ? (nt_in - first) : b.fan);
      m = cnt * n;
      for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
        const int c = idx / m, rr = idx - c * m;
        const int f = rr / n, r = rr - f * n;
        A[(int64_t)c * lda + rr] = (E)tri_in[(first + f) * n * n + (int64_t)c * n + r];
      }
    }
    __syncthreads();
    if (n <= 32 && m <= 96) hh_small<E>(A, lda, m, n, red);   // short tiles: latency-shaped
    else hh_qr<E>(A, lda, m, n, red);
    double* tri = tri_out + t * n * n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int c = idx / n, r = idx - c * n;
      tri[idx] = (r <= c && r < m) ? (double)A[(int64_t)c * lda + r] : 0.0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ Givens leaf (option)
// The paper's THIN post-processing (§7, after Golub et al.) gives each thread a share of
// a block's rows, which it brings to upper-triangular form by Givens rotations, and then
// combines the threads' triangles.  Here one thread per chunk of kGivensRows rows keeps an
// n x n triangle and rotates every row into it, column by column: rotation (c, s) with
// r = sqrt(T_kk^2 + x_k^2), c = T_kk / r, s = x_k / r turns (T_kj, x_j) into
// (c T_kj + s x_j, -s T_kj + c x_j).  A row entry that is exactly zero needs no rotation
// and is skipped, which is what makes this leaf pay on very sparse blocks (as is an entry
// whose square underflows together with T_kk's, at an error below the format's smallest
// normal); the chunk triangles then go through the same TSQR tree as the Householder
// leaves.
template <typename E, int NMAX>
__global__ void __launch_bounds__(128) k_tsqr_givens(TsqrBlock b, double* tri_out) {
  const int n = b.n;
  const int64_t rows = block_rows(b);
  const int64_t tiles = (rows + kGivensRows - 1) / kGivensRows;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tiles; t += (int64_t)gridDim.x * blockDim.x) {
    E T[NMAX][NMAX];
#pragma unroll
    for (int i = 0; i < NMAX; ++i)
#pragma unroll
      for (int j = 0; j < NMAX; ++j) T[i][j] = E(0);
    const int64_t r0 = t * kGivensRows;
    const int m = (int)(rows - r0 < kGivensRows ? rows - r0 : kGivensRows);
    for (int i = 0; i < m; ++i) {
      E x[NMAX];
#pragma unroll
      for (int c = 0; c < NMAX; ++c)
        x[c] = c < n ? (b.ptr32 ? (E)b.ptr32[(int64_t)c * b.ld + r0 + i] : (E)b.ptr[(int64_t)c * b.ld + r0 + i]) : E(0);
#pragma unroll
      for (int k = 0; k < NMAX; ++k) {
        if (x[k] == E(0)) continue;                   // nothing to rotate away
        const E a = T[k][k];
        const E r = sqrt(fma(a, a, x[k] * x[k]));
        if (r == E(0)) continue;                      // both below the square's underflow
        const E c = a / r, s = x[k] / r;
        T[k][k] = r;
#pragma unroll
        for (int j = k + 1; j < NMAX; ++j) {
          const E tj = T[k][j];
          T[k][j] = fma(c, tj, s * x[j]);
          x[j] = fma(-s, tj, c * x[j]);
        }
      }
    }
    double* tri = tri_out + t * n * n;
#pragma unroll
    for (int c = 0; c < NMAX; ++c)
#pragma unroll
      for (int r = 0; r < NMAX; ++r)
        if (c < n && r < n) tri[(int64_t)c * n + r] = r <= c ? (double)T[r][c] : 0.0;   // T is exact
  }
}

template <typename E>
static void launch_givens(const TsqrBlock& b, cudaStream_t st) {
  const int64_t tiles = (b.bound + kGivensRows - 1) / kGivensRows;
  const unsigned grid = grid_for(tiles, 128, 152 * 16);
  if (b.nreg <= 8) k_tsqr_givens<E, 8><<<grid, 128, 0, st>>>(b, b.tri[0]);
  else k_tsqr_givens<E, 16><<<grid, 128, 0, st>>>(b, b.tri[0]);
}

// ------------------------------------------------------------------ streamed fold (n > 32)
// A wide block is reduced by folding.  A thread block keeps one n x n triangle T, the R of
// the rows it has folded so far, and brings every next chunk X of its rows into it column
// by column: the reflector of column k maps (T_kk, X[:, k]) to (beta, 0) (alpha = T_kk,
// sigma = ||X[:, k]||^2; normalised as in FoldScalars), and for every later column j
// w_j = tau' (T_kj + X[:, k]^T X[:, j] / v0), T_kj -= w_j, X[:, j] -= (w_j / v0) X[:, k].  This is
// Householder QR of the stacked [T; X] with the zeros of T skipped, 2 m n^2 flops per chunk
// of m rows, so a block of M rows costs the 2 M n^2 of one tall QR and no tree work inside a
// thread block.  The leaf gives one triangle per b.seg chunks; tree levels fold b.fan such
// triangles each, several stacked in one chunk when they fit, skipping the rows that are
// zero in the column being reduced (row i of an upper triangle is zero before column i),
// (2/3) n^3 flops per triangle.
//
// Per column k, two passes separated by barriers.  Pass A: warps 0-7 form partial dot
// products of column k with columns k+1.. over row slices (slice s of S takes rows s,
// s + S, ...; thread (column, slice)) while lane 0 of warp 8 forms the scalars from the
// norm and T_kk found in the previous pass.  Pass B: warps 0-7 sum the partials of
// columns k+2.. and update them; warp 8 updates column k+1 and reduces its sum of
// squares over the warp, which the next column's scalars need.
constexpr int kFoldThreads = 288;
constexpr int kFoldWorkers = 256;
constexpr int kFoldPivotWarp = kFoldWorkers / 32;
constexpr int kFoldMaxSlices = 8;
constexpr size_t kFoldSmemF32 = 100 * 1024;   // two float blocks per SM (latency-bound)

__host__ __device__ __forceinline__ int fold_red_elems(int n) {
  const int part = n > kFoldWorkers ? n : kFoldWorkers;
  return ((part + n + 4) + 3) & ~3;
}

// Scalars of the fold's reflector in normalised form: v' = v / v0 = (1, x / v0) and
// tau' = tau v0^2 = |v0| / nu (in [1, 2]), returned with rv = 1 / v0.  Unlike
// tau = 1 / (nu (nu + |alpha|)) this stays finite when sigma is far below the format's
// smallest normal, as the rounding residue of a chunk with fewer rows than columns
// becomes after enough reflections.
template <typename E>
struct FoldScalars {
  __device__ static void get(E alpha, E sigma, E& beta, E& taup, E& rv) {
    const E nu = sqrt(fma(alpha, alpha, sigma));
    beta = alpha >= E(0) ? -nu : nu;
    const E v0 = alpha - beta;
    taup = fabs(v0) / nu;
    rv = E(1) / v0;
  }
};

template <>
struct FoldScalars<double> {
  __device__ static void get(double alpha, double sigma, double& beta, double& taup, double& rv) {
    const double t = fma(alpha, alpha, sigma);
    if (f64_mid_range(t)) {
      // 1/sqrt(t) and 1/v0 by two Newton-Raphson steps each from the float approximations
      // (as in HhScalars<double>); |v0| is in [nu, 2 nu], inside the float range with t
      double y = f64_of_f32_bits(rsqrtf(f32_of_f64_bits(t)));
      const double ht = 0.5 * t;
      y = y * fma(-ht * y, y, 1.5);
      y = y * fma(-ht * y, y, 1.5);
      const double nu = t * y;
      const bool neg = __double_as_longlong(alpha) < 0;
      beta = neg ? nu : -nu;
      const double av0 = fabs(alpha) + nu;           // |v0| = |alpha - beta|
      taup = av0 * y;
      double r = f64_of_f32_bits(__frcp_rn(f32_of_f64_bits(av0)));
      r = r * fma(-av0, r, 2.0);
      r = r * fma(-av0, r, 2.0);
      rv = neg ? -r : r;                             // v0 has the sign of alpha
    } else {
      const double nu = sqrt(t);
      beta = alpha >= 0.0 ? -nu : nu;
      const double v0 = alpha - beta;
      taup = fabs(v0) / nu;
      rv = 1.0 / v0;
    }
  }
};

template <typename E>
__device__ __forceinline__ E fold_warp_sum(E v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// slices for cols columns over the worker threads
__device__ __forceinline__ int fold_slices(int cols) {
  if (cols <= 0) return 0;
  int S = kFoldWorkers / cols;
  if (S > kFoldMaxSlices) S = kFoldMaxSlices;
  return S < 1 ? 1 : S;
}

// Folds X into T.  X holds P row blocks of h rows each (row block p at rows [p h, p h + h),
// leading dimension ldx).  Dense: every row may be non-zero.  tri: every row block holds
// rows [r0, r0 + h) of an upper triangle, so that in column k only its first
// k + 1 - r0 rows can be non-zero.
template <typename E>
__device__ void fold_chunk(E* X, int ldx, int h, int P, int n, int r0, bool tri, E* T, E* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  E* part = red;                                          // [S * cp] partial dots
  E* trow = red + (n > kFoldWorkers ? n : kFoldWorkers);  // T[k][k+1..n-1] of the step
  E* sc = trow + n;                                       // tau', 1/v0, next sigma, next alpha
  auto rows_at = [&](int k) -> int {
    if (!tri) return h;
    const int r = k + 1 - r0;
    return r < 0 ? 0 : (r > h ? h : r);
  };
  // a piece starting at row r0 of a triangle is zero in columns < r0: their reflectors
  // are the identity
  const int kbeg = tri ? (r0 < n ? r0 : n) : 0;
  if (kbeg >= n) return;
  if (warp == kFoldPivotWarp) {
    const int ra = rows_at(kbeg);
    const E* x0 = X + (int64_t)kbeg * ldx;
    E sq = E(0);
    for (int p = 0; p < P; ++p)
      for (int i = lane; i < ra; i += 32) {
        const E v = x0[p * h + i];
        sq = fma(v, v, sq);
      }
    sq = fold_warp_sum(sq);
    if (lane == 0) {
      sc[2] = sq;
      sc[3] = T[(int64_t)kbeg * n + kbeg];
    }
  }
  __syncthreads();
  for (int k = kbeg; k < n; ++k) {
    const int ra = rows_at(k), rb = rows_at(k + 1);   // rows [ra, rb) have X[i][k] = 0
    const int cp = n - 1 - k;                         // columns k+1 .. n-1
    const int S = fold_slices(cp);
    const E* xk = X + (int64_t)k * ldx;
    E* trk = T + (int64_t)k * n;
    if (tid < kFoldWorkers) {
      const int items = S * cp;
      for (int e = tid; e < items; e += kFoldWorkers) {
        const int jc = e % cp, s = e / cp;
        if (s == 0) trow[jc] = trk[k + 1 + jc];
        const E* xj = xk + (int64_t)(jc + 1) * ldx;
        E d0 = E(0), d1 = E(0);
        for (int p = 0; p < P; ++p) {
          const E* a = xk + p * h;
          const E* c = xj + p * h;
          int i = s;
          for (; i + S < ra; i += 2 * S) {
            d0 = fma(a[i], c[i], d0);
            d1 = fma(a[i + S], c[i + S], d1);
          }
          if (i < ra) d0 = fma(a[i], c[i], d0);
        }
        part[e] = d0 + d1;
      }
    } else if (tid == kFoldWorkers) {
      const E sigma = sc[2], alpha = sc[3];
      E beta = alpha, taup = E(0), rv = E(0);           // a zero column: nothing to reflect
      if (!f64_is_zero(sigma)) FoldScalars<E>::get(alpha, sigma, beta, taup, rv);
      trk[k] = beta;
      sc[0] = taup;
      sc[1] = rv;
    }
    __syncthreads();
    const E taup = sc[0], rv = sc[1];
    if (tid < kFoldWorkers) {
      const int cq = cp - 1;                          // columns k+2 .. n-1
      const int S2 = fold_slices(cq);
      const int items = S2 * cq;
      for (int e = tid; e < items; e += kFoldWorkers) {
        const int jc = e % cq + 1, s = e / cq;
        E d = part[jc];
        for (int q = 1; q < S; ++q) d += part[q * cp + jc];
        const E tj = trow[jc];
        const E wt = taup * fma(rv, d, tj);             // w' = tau' (T_kj + d_j / v0)
        if (s == 0) trk[k + 1 + jc] = tj - wt;
        const E w = wt * rv;                              // X[:, j] -= w' (X[:, k] / v0)
        E* xj = X + (int64_t)(k + 1 + jc) * ldx;
        for (int p = 0; p < P; ++p) {
          const E* a = xk + p * h;
          E* c = xj + p * h;
          for (int i = s; i < ra; i += S2) c[i] = fma(-w, a[i], c[i]);
        }
      }
    } else if (cp > 0) {
      // warp 8: column k+1 and the sum of squares of its rows for the next step
      const E alpha_next = lane == 0 ? T[(int64_t)(k + 1) * n + k + 1] : E(0);
      E d = part[0];
      for (int q = 1; q < S; ++q) d += part[q * cp];
      const E tj = trow[0];
      const E wt = taup * fma(rv, d, tj);
      const E w = wt * rv;
      E* xj = X + (int64_t)(k + 1) * ldx;
      E sq = E(0);
      for (int p = 0; p < P; ++p) {
        const E* a = xk + p * h;
        E* c = xj + p * h;
        for (int i = lane; i < rb; i += 32) {
          const E v = fma(-w, a[i], c[i]);
          c[i] = v;
          sq = fma(v, v, sq);
        }
      }
      sq = fold_warp_sum(sq);
      if (lane == 0) {
        trk[k + 1] = tj - wt;
        sc[2] = sq;
        sc[3] = alpha_next;
      }
    }
    __syncthreads();
  }
}

// level 0: the leaf over the block's rows; level l > 0: tree level l over tri_in.
template <typename E>
__global__ void __launch_bounds__(kFoldThreads) k_tsqr_fold(TsqrBlock b, const double* tri_in, double* tri_out,
                                                            int level) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = b.n, mc = b.tile, ldx = mc + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  E* red = reinterpret_cast<E*>(smem_raw);
  E* X = red + fold_red_elems(n);
  E* T = b.fold_tsmem ? X + (int64_t)ldx * n : static_cast<E*>(b.scratch) + (int64_t)blockIdx.x * n * n;
  const int64_t rows = block_rows(b);
  // chunks per leaf triangle from the live rows: the leaf's thread blocks share them evenly
  const int64_t chunks = (rows + mc - 1) / mc;
  int64_t seg = (chunks + b.fold_g0 - 1) / b.fold_g0;
  if (seg > b.seg) seg = b.seg;
  if (seg < 1) seg = 1;
  int64_t live = chunks;                      // leaf: live chunks
  int64_t per = seg;
  if (level > 0) {
    live = (live + seg - 1) / seg;            // live leaf triangles
    for (int l = 1; l < level; ++l) live = (live + b.fan - 1) / b.fan;
    per = b.fan;
    if (live == 1) {                          // one triangle: copied
      if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < n * n; i += blockDim.x) tri_out[i] = tri_in[i];
      return;
    }
  }
  const int stack = mc / n;                   // whole triangles per chunk on tree levels
  int64_t units = (live + per - 1) / per;
  if (units < 1) units = 1;                   // an empty block still leaves a (zero) triangle
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) T[i] = E(0);
    __syncthreads();
    const int64_t q1 = (u + 1) * per < live ? (u + 1) * per : live;
    if (level == 0) {
      for (int64_t q = u * per; q < q1; ++q) {
        const int64_t r0 = q * mc;
        const int m = (int)((rows - r0) < mc ? (rows - r0) : mc);
        for (int c = warp; c < n; c += nwarps) {
          E* dst = X + (int64_t)c * ldx;
          if (b.ptr32) {
            const float* src = b.ptr32 + (int64_t)c * b.ld + r0;
#pragma unroll 4
            for (int i = lane; i < m; i += 32) dst[i] = (E)src[i];
          } else {
            const double* src = b.ptr + (int64_t)c * b.ld + r0;
#pragma unroll 4
            for (int i = lane; i < m; i += 32) dst[i] = (E)src[i];
          }
        }
        __syncthreads();
        fold_chunk<E>(X, ldx, m, 1, n, 0, false, T, red);
      }
    } else if (stack >= 2) {
      for (int64_t q = u * per; q < q1; q += stack) {
        const int cnt = (int)((q1 - q) < stack ? (q1 - q) : stack);
        for (int c = warp; c < n; c += nwarps) {
          E* dst = X + (int64_t)c * ldx;
          for (int idx = lane; idx < cnt * n; idx += 32) {
            const int t = idx / n, r = idx - t * n;
            dst[idx] = (E)tri_in[(q + t) * n * n + (int64_t)c * n + r];
          }
        }
        __syncthreads();
        fold_chunk<E>(X, ldx, n, cnt, n, 0, true, T, red);
      }
    } else {
      for (int64_t q = u * per; q < q1; ++q) {
        const double* src = tri_in + q * n * n;
        for (int r0 = 0; r0 < n; r0 += mc) {
          const int m = (n - r0) < mc ? (n - r0) : mc;
          for (int c = warp; c < n; c += nwarps) {
            E* dst = X + (int64_t)c * ldx;
            for (int i = lane; i < m; i += 32) dst[i] = (E)src[(int64_t)c * n + r0 + i];
          }
          __syncthreads();
          fold_chunk<E>(X, ldx, m, 1, n, r0, true, T, red);
        }
      }
    }
    double* tri = tri_out + u * n * n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int c = idx / n, r = idx - c * n;
      tri[idx] = r <= c ? (double)T[(int64_t)r * n + c] : 0.0;
    }
    __syncthreads();
  }
}

static size_t fold_budget(bool mixed) { return mixed ? kFoldSmemF32 : kSmemCap; }

static size_t fold_smem(const TsqrBlock& b, size_t esz) {
  size_t e = (size_t)fold_red_elems(b.n) + (size_t)(b.tile + 1) * b.n;
  if (b.fold_tsmem) e += (size_t)b.n * b.n;
  return e * esz;
}

static int64_t fold_resident(bool mixed) { return mixed ? 152 * 2 : 152; }

// units (triangles written) at a level, from the allocation bound of the rows
static int64_t fold_units(const TsqrBlock& b, int level) {
  int64_t u = (b.bound + b.tile - 1) / b.tile;
  u = (u + b.seg - 1) / b.seg;                // at most fold_g0 on the device: seg grows with rows
  for (int l = 1; l <= level; ++l) u = (u + b.fan - 1) / b.fan;
  return u < 1 ? 1 : u;
}

template <typename E>
static void launch_fold(const TsqrBlock& b, const double* tri_in, double* tri_out, int level, bool mixed,
                        cudaStream_t st) {
  int64_t grid = fold_units(b, level);
  const int64_t cap = fold_resident(mixed);
  if (grid > cap) grid = cap;
  k_tsqr_fold<E><<<(unsigned)grid, kFoldThreads, fold_smem(b, sizeof(E)), st>>>(b, tri_in, tri_out, level);
}

// ------------------------------------------------------------------ final stack and R
// One thread block places every block's triangle at its global columns: stack rows
// [off_b, off_b + n_b), column-major with leading dimension stack_rows.
__global__ void k_tsqr_stack(const TsqrBlock* blocks, int nb, int stack_rows, int N, double* stack) {
  for (int idx = threadIdx.x; idx < stack_rows * N; idx += blockDim.x) stack[idx] = 0.0;
  __syncthreads();
  int off = 0;
  for (int bi = 0; bi < nb; ++bi) {
    const TsqrBlock& b = blocks[bi];
    const int n = b.n;
    if (block_rows(b) > 0) {
      const double* tri = b.tri[b.top];
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int c = idx / n, r = idx - c * n;
        stack[(int64_t)b.cols[c] * stack_rows + off + r] = tri[idx];
      }
    }
    off += n;
  }
}

// R = the stack's triangle with every row multiplied by the sign of its diagonal entry.
__global__ void k_write_r(const double* tri, int N, double* R, int64_t ldr) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < N * N; idx += gridDim.x * blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    double v = 0.0;
    if (j >= i) {
      const double d = tri[(int64_t)i * N + i];
      v = (d < 0.0 ? -1.0 : 1.0) * tri[(int64_t)j * N + i];
    }
    R[(int64_t)i * ldr + j] = v;
  }
}

// ------------------------------------------------------------------ host planning
static int reg_class(int n) {
  if (n <= 16) return (n + 1) & ~1;          // 2, 4, ..., 16
  if (n <= 32) return (n + 3) & ~3;          // 20, 24, 28, 32
  return 0;
}

static int reg_tile_of(int N) {
  switch (N) {
    case 2: return RegCfg<2>::TW; case 4: return RegCfg<4>::TW; case 6: return RegCfg<6>::TW;
    case 8: return RegCfg<8>::TW; case 10: return RegCfg<10>::TW; case 12: return RegCfg<12>::TW;
    case 14: return RegCfg<14>::TW; case 16: return RegCfg<16>::TW; case 20: return RegCfg<20>::TW;
    case 24: return RegCfg<24>::TW; case 28: return RegCfg<28>::TW; default: return RegCfg<32>::TW;
  }
}

static size_t cta_smem(int lda, int n, size_t esz) { return (kRedElems + (size_t)lda * n) * esz; }

// Fold path for a wide block: the chunk height that fills the shared-memory budget (the
// triangle in shared memory when it takes at most a quarter of it, else in a global slot
// per thread block), one leaf triangle per resident thread block (at most 16 chunks each on
// the float path, whose error grows with the number of folds into one triangle).
static bool fold_plan(TsqrBlock& b, bool mixed, size_t esz) {
  const int n = b.n;
  const size_t budget = fold_budget(mixed);
  const size_t red = (size_t)fold_red_elems(n) * esz;
  if (red >= budget) return false;
  const bool tsm = (size_t)n * n * esz <= budget / 4;
  const size_t rest = budget - red - (tsm ? (size_t)n * n * esz : 0);
  int64_t mc = (int64_t)(rest / (esz * (size_t)n)) - 1;
  mc = (mc / 32) * 32;
  if (mc > 512) mc = 512;
  if (mc < 32) return false;
  b.fold = true;
  b.fold_tsmem = tsm;
  b.warp_min = 0;
  b.tile = (int)mc;
  // tree levels: as many triangles as one chunk stacks (at least 4, at most 16)
  const int64_t stack = mc / n;
  b.fan = (int)(stack < 4 ? 4 : (stack > 16 ? 16 : stack));
  const int64_t chunks = (b.bound + mc - 1) / mc;
  const int64_t res = fold_resident(mixed);
  int64_t seg = (chunks + res - 1) / res;
  if (mixed && seg > 16) seg = 16;
  b.seg = seg < 1 ? 1 : seg;
  int64_t u = (chunks + b.seg - 1) / b.seg;
  b.fold_g0 = u < res ? u : res;
  int levels = 0;
  while (u > 1) {
    u = (u + b.fan - 1) / b.fan;
    ++levels;
  }
  b.levels = levels;
  b.top = levels & 1;
  return true;
}

void tsqr_plan_block(TsqrBlock& b, bool mixed, bool givens) {
  const int n = b.n;
  const size_t esz = mixed ? sizeof(float) : sizeof(double);
  b.nreg = reg_class(n);
  b.givens = givens && b.nreg && b.nreg <= 16;
  if (b.nreg) {
    // one warp's QR of a tile costs about N^2 FP64 instructions at ~70 cycles each: for
    // N <= 16 (tiles of 128-256 rows) it beats a thread block per tile from two tiles
    // on; wider tiles (64 rows) keep the block kernel until the level fills the GPU
    b.warp_min = b.nreg <= 16 ? 2 : 152 * 4;
    b.tile = reg_tile_of(b.nreg);
    // n <= 16: tree tiles fill a register tile (fan = TW / n >= 4); wider blocks reduce
    // their trees with the block-per-tile kernel only, six triangles at a time
    b.fan = b.nreg <= 16 ? b.tile / n : 6;
    if (b.givens) b.tile = kGivensRows;       // leaf chunks of the Givens leaf
  } else if (fold_plan(b, mixed, esz)) {
    return;
  } else {
    b.warp_min = 0;
    int64_t t = (int64_t)(64 * 1024 / (esz * n));
    t = (t / 32) * 32;
    if (t > 2048) t = 2048;
    if (t < n) t = n;
    if (t < 32) t = 32;
    b.tile = (int)t;
    int64_t f = (int64_t)(64 * 1024 / (sizeof(double) * (size_t)n * n));
    if (f < 2) f = 2;
    if (f > 256) f = 256;
    b.fan = (int)f;
  }
  int64_t tiles = (b.bound + b.tile - 1) / b.tile;
  int levels = 0;
  while (tiles > 1) {
    tiles = (tiles + b.fan - 1) / b.fan;
    ++levels;
  }
  b.levels = levels;
  b.top = levels & 1;
}

int64_t tsqr_tri_elems(const TsqrBlock& b) {
  if (b.fold) return fold_units(b, 0) * b.n * b.n;
  int64_t tiles = (b.bound + b.tile - 1) / b.tile;
  if (tiles < 1) tiles = 1;
  return tiles * b.n * b.n;
}

int64_t tsqr_scratch_elems(const TsqrBlock& b, bool mixed) {
  if (b.nreg) return 0;
  if (b.fold) return b.fold_tsmem ? 0 : fold_resident(mixed) * b.n * b.n;   // T slots (as doubles: room for floats)
  const size_t esz = mixed ? sizeof(float) : sizeof(double);
  int64_t need = 0;
  const int64_t grid = 152 * 2;
  if (cta_smem(cta_lda(b, false), b.n, esz) > kSmemCap) need = grid * (int64_t)cta_lda(b, false) * b.n;
  if (cta_smem(cta_lda(b, true), b.n, esz) > kSmemCap) {
    const int64_t r = grid * (int64_t)cta_lda(b, true) * b.n;
    if (r > need) need = r;
  }
  return need;
}

template <typename E>
static void launch_cta(const TsqrBlock& b, const double* tri_in, double* tri_out, int64_t div_in, int64_t tiles,
                       void* scratch, cudaStream_t st, int few_only = 0) {
  const int lda = cta_lda(b, tri_in != nullptr);
  size_t smem = cta_smem(lda, b.n, sizeof(E));
  E* gs = nullptr;
  if (smem > kSmemCap) {
    smem = kRedElems * sizeof(E);
    gs = static_cast<E*>(scratch);
  }
  int64_t blocks = tiles < 1 ? 1 : tiles;
  const int64_t cap = 152 * 2;
  if (blocks > cap) blocks = cap;
  k_tsqr_cta<E><<<(unsigned)blocks, kQrThreads, smem, st>>>(b, tri_in, tri_out, div_in, gs, few_only);
}

cudaError_t tsqr_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_tsqr_cta<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tsqr_cta<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tsqr_fold<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tsqr_fold<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  return e;
}

void tsqr_leaf(const TsqrBlock& b, bool mixed, cudaStream_t st, int64_t* launches) {
  void* scratch = b.scratch;
  const int64_t tiles = (b.bound + b.tile - 1) / b.tile;
  if (tiles < 1) return;
  if (b.givens) {
    // float64 on both paths: rotated in float, the chunk triangles of very sparse
    // blocks lose up to 2e-5 of R^T R (measured), far above the float Householder leaf
    launch_givens<double>(b, st);
    (void)mixed;
    ++*launches;
    return;
  }
  if (b.fold) {
    if (mixed) launch_fold<float>(b, nullptr, b.tri[0], 0, true, st);
    else launch_fold<double>(b, nullptr, b.tri[0], 0, false, st);
  } else if (b.nreg) {
    if (mixed) {
      launch_reg_n<float>(b, nullptr, b.tri[0], 0, tiles, st);
      launch_cta<float>(b, nullptr, b.tri[0], 0, tiles, scratch, st, 1);
    } else {
      launch_reg_n<double>(b, nullptr, b.tri[0], 0, tiles, st);
      launch_cta<double>(b, nullptr, b.tri[0], 0, tiles, scratch, st, 1);
    }
    ++*launches;
  } else if (mixed) {
    launch_cta<float>(b, nullptr, b.tri[0], 0, tiles, scratch, st);
  } else {
    launch_cta<double>(b, nullptr, b.tri[0], 0, tiles, scratch, st);
  }
  ++*launches;
}

// Tree levels in float for the mixed path (the triangles stay stored in float64), in
// float64 otherwise; the final QR of the stacked block triangles is always float64.
void tsqr_reduce(TsqrBlock& b, bool mixed, cudaStream_t st, int64_t* launches) {
  void* scratch = b.scratch;
  int64_t div = b.tile;
  int64_t tiles = (b.bound + b.tile - 1) / b.tile;
  int cur = 0;
  for (int l = 0; l < b.levels; ++l) {
    const int64_t out_tiles = (tiles + b.fan - 1) / b.fan;
    if (b.fold) {
      if (mixed) launch_fold<float>(b, b.tri[cur], b.tri[cur ^ 1], l + 1, true, st);
      else launch_fold<double>(b, b.tri[cur], b.tri[cur ^ 1], l + 1, false, st);
      ++*launches;
    } else if (b.nreg && b.nreg <= 16) {
      if (mixed) {
        launch_reg_n<float>(b, b.tri[cur], b.tri[cur ^ 1], div, out_tiles, st);
        launch_cta<float>(b, b.tri[cur], b.tri[cur ^ 1], div, out_tiles, scratch, st, 1);
      } else {
        launch_reg_n<double>(b, b.tri[cur], b.tri[cur ^ 1], div, out_tiles, st);
        launch_cta<double>(b, b.tri[cur], b.tri[cur ^ 1], div, out_tiles, scratch, st, 1);
      }
      *launches += 2;
    } else {
      if (mixed) launch_cta<float>(b, b.tri[cur], b.tri[cur ^ 1], div, out_tiles, scratch, st);
      else launch_cta<double>(b, b.tri[cur], b.tri[cur ^ 1], div, out_tiles, scratch, st);
      ++*launches;
    }
    cur ^= 1;
    div *= b.fan;
    tiles = out_tiles;
  }
}

void tsqr_final(const TsqrBlock* blocks_dev, int n_blocks, TsqrBlock& stack_blk, double* R, int64_t ldr,
                cudaStream_t st, int64_t* launches) {
  const int N = stack_blk.n;
  k_tsqr_stack<<<1, 256, 0, st>>>(blocks_dev, n_blocks, (int)stack_blk.M, N, const_cast<double*>(stack_blk.ptr));
  ++*launches;
  tsqr_leaf(stack_blk, false, st, launches);
  tsqr_reduce(stack_blk, false, st, launches);
  k_write_r<<<grid_for((int64_t)N * N, 256, 64), 256, 0, st>>>(stack_blk.tri[stack_blk.top], N, R, ldr);
  ++*launches;
}

double tsqr_leaf_flops(int64_t rows, int n) {
  // Householder on the leaf tiles: about 2 m n^2 - 2 n^3 / 3 per tile; summed over
  // the rows of the block this is 2 rows n^2 up to the per-tile correction.
  return 2.0 * (double)rows * n * n;
}

}  // namespace fig
