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
// The kernels:
//   n <= 32:       one warp per tile, the tile in registers (k_tsqr_reg), every loop bound
//                  a compile-time constant so that no predicated-off FP64 instruction is
//                  issued; levels with few tiles take one thread block per tile (k_tsqr_cta);
//   33 <= n <= 1024: the streamed fold (k_tsqr_fold): one resident triangle per thread
//                  block, row chunks folded into it, structured tree levels (above 256
//                  columns the triangle sits in a global slot, its rows staged four
//                  elements per thread, and chunks are 16 to 64 rows high);
//   otherwise:     one thread block per tile in shared memory or a global slot (k_tsqr_cta).
// All are persistent over the live tiles: the row counts are only known on the device.
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
        E beta, v0, tau, tau2;
        HhScalars<E>::get(alpha, sigma, beta, v0, tau, tau2);
        if (mine) {
          wj = tau * fma(v0, akj, dj) * tau2;
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
// thread block.  The leaf gives one triangle per b.seg chunks; a tree level reduces b.fan
// such triangles per unit: T starts as the first and the others are folded in, several
// stacked in one chunk when they fit, skipping the rows that are zero in the column being
// reduced (row i of an upper triangle is zero before column i), (2/3) n^3 flops per
// triangle.
//
// Per column k, two passes separated by barriers.  Pass A: warps 0-7 form partial dot
// products of column k with columns k+1.. over row slices (slice s of S takes rows s,
// s + S, ...; thread (column, slice)) while lane 0 of warp 8 forms the scalars from the
// norm and T_kk found in the previous pass.  Pass B: warps 0-7 sum the partials of
// columns k+2.. and update them; warp 8 updates column k+1 and reduces its sum of
// squares over the warp, which the next column's scalars need.
constexpr int kFoldThreads = 288;
constexpr int kFoldWorkers = 256;
constexpr int kStackStage = 4;                 // the final stack fold: N <= 1024 (staging 4 per thread)
constexpr int kStackFoldMaxN = 1024;
constexpr int kStackMaxBlocks = 256;           // more blocks: none placed, every one folded
constexpr int kFoldPivotWarp = kFoldWorkers / 32;
constexpr int kFoldMaxSlices = 8;
constexpr size_t kFoldSmemF32 = 100 * 1024;   // two float blocks per SM (latency-bound)
constexpr int kTcNb = 16;                      // tensor-core fold: panel width
constexpr int kTcRec = kTcNb;                  // offset of 1/v0 behind tau' in the panel record

// Shared scratch of a fold block, in elements: partial dots [max(256, n)], the step's T row
// [n], scalars [4], and two staging rows [2 n] for T rows read from global memory.
__host__ __device__ __forceinline__ int fold_red_elems(int n) {
  const int part = n > kFoldWorkers ? n : kFoldWorkers;
  return ((part + 3 * n + 4) + 3) & ~3;
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

// One column step of a fold: reflector k, applied to the columns k+1 .. kend-1.  ra rows of
// each of the P row blocks of X can be non-zero in column k, rb in column k+1 (rb >= ra; the
// rows between hold zeros in column k).  T's row k is read from `rowk` (T itself, or the
// staging row that the previous step filled when T is in global memory, tglob); the step
// fills the staging row k+1 the same way, with its loads in flight through both passes.
// rec (may be null) receives tau' and 1/v0 of the reflector.  Both passes end in a barrier.
// ST: elements of a staged T row per thread (n <= ST x kFoldThreads when T is global).
template <typename E, int ST = 1>
__device__ __forceinline__ void fold_step(E* X, int ldx, int h, int P, int n, int k, int kend, int ra, int rb, E* T,
                                          bool tglob, E* red, E* rec) {
  const int tid = threadIdx.x, lane = tid & 31;
  E* part = red;                                          // [S * cp] partial dots
  E* trow = red + (n > kFoldWorkers ? n : kFoldWorkers);  // T[k][k+1..kend-1] of the step
  E* sc = trow + n;                                       // tau', 1/v0, sigma of column k
  E* tbuf = sc + 4;                                       // staging rows, [2][n]
  const int cp = kend - 1 - k;                            // columns k+1 .. kend-1
  const int S = fold_slices(cp);
  const E* xk = X + (int64_t)k * ldx;
  E* trk = T + (int64_t)k * n;
  const E* rowk = tglob ? tbuf + (k & 1) * n : trk;
  E tn[ST];                                               // staging of T[k+1][k+1..n-1]
#pragma unroll
  for (int q = 0; q < ST; ++q) {
    const int idx = tid + q * kFoldThreads;
    tn[q] = (tglob && idx < n - k - 1) ? __ldcg(T + (int64_t)(k + 1) * n + k + 1 + idx) : E(0);
  }
  if (tid < kFoldWorkers) {
    const int items = S * cp;
    for (int e = tid; e < items; e += kFoldWorkers) {
      const int jc = e % cp, s = e / cp;
      const E* xj = xk + (int64_t)(jc + 1) * ldx;
      E d0 = E(0), d1 = E(0), d2 = E(0), d3 = E(0);
      for (int p = 0; p < P; ++p) {
        const E* a = xk + p * h;
        const E* c = xj + p * h;
        int i = s;
        for (; i + 3 * S < ra; i += 4 * S) {   // four rows in flight
          const E a0 = a[i], a1 = a[i + S], a2 = a[i + 2 * S], a3 = a[i + 3 * S];
          const E c0 = c[i], c1 = c[i + S], c2 = c[i + 2 * S], c3 = c[i + 3 * S];
          d0 = fma(a0, c0, d0);
          d1 = fma(a1, c1, d1);
          d2 = fma(a2, c2, d2);
          d3 = fma(a3, c3, d3);
        }
        for (; i < ra; i += S) d0 = fma(a[i], c[i], d0);
      }
      part[e] = (d0 + d1) + (d2 + d3);
      if (s == 0) trow[jc] = rowk[k + 1 + jc];
    }
  } else if (tid == kFoldWorkers) {
    const E sigma = sc[2], alpha = rowk[k];
    E beta = alpha, taup = E(0), rv = E(0);             // a zero column: nothing to reflect
    if (!f64_is_zero(sigma)) FoldScalars<E>::get(alpha, sigma, beta, taup, rv);
    trk[k] = beta;
    sc[0] = taup;
    sc[1] = rv;
    if (rec) {
      rec[0] = taup;
      rec[kTcRec] = rv;
    }
  }
  __syncthreads();
  const E taup = sc[0], rv = sc[1];
  if (tid < kFoldWorkers) {
    const int cq = cp - 1;                                // columns k+2 .. kend-1
    const int S2 = fold_slices(cq);
    const int items = S2 * cq;
    for (int e = tid; e < items; e += kFoldWorkers) {
      const int jc = e % cq + 1, s = e / cq;
      E d = part[jc];
      for (int q = 1; q < S; ++q) d += part[q * cp + jc];
      const E tj = trow[jc];
      const E wt = taup * fma(rv, d, tj);               // w' = tau' (T_kj + d_j / v0)
      if (s == 0) trk[k + 1 + jc] = tj - wt;
      const E w = wt * rv;                                // X[:, j] -= w' (X[:, k] / v0)
      E* xj = X + (int64_t)(k + 1 + jc) * ldx;
      for (int p = 0; p < P; ++p) {
        const E* a = xk + p * h;
        E* c = xj + p * h;
        int i = s;
        for (; i + 3 * S2 < ra; i += 4 * S2) {  // loads of four rows before their stores
          const E a0 = a[i], a1 = a[i + S2], a2 = a[i + 2 * S2], a3 = a[i + 3 * S2];
          const E c0 = c[i], c1 = c[i + S2], c2 = c[i + 2 * S2], c3 = c[i + 3 * S2];
          c[i] = fma(-w, a0, c0);
          c[i + S2] = fma(-w, a1, c1);
          c[i + 2 * S2] = fma(-w, a2, c2);
          c[i + 3 * S2] = fma(-w, a3, c3);
        }
        for (; i < ra; i += S2) c[i] = fma(-w, a[i], c[i]);
      }
    }
  } else if (cp > 0) {
    // warp 8: column k+1 and the sum of squares of its rows for the next step
    E d = part[0];
    for (int q = 1; q < S; ++q) d += part[q * cp];
    const E tj = trow[0];
    const E wt = taup * fma(rv, d, tj);
    const E w = wt * rv;
    E* xj = X + (int64_t)(k + 1) * ldx;
    E sq = E(0), sq2 = E(0);
    for (int p = 0; p < P; ++p) {
      const E* a = xk + p * h;
      E* c = xj + p * h;
      int i = lane;
      for (; i + 96 < rb; i += 128) {
        const E a0 = a[i], a1 = a[i + 32], a2 = a[i + 64], a3 = a[i + 96];
        const E c0 = c[i], c1 = c[i + 32], c2 = c[i + 64], c3 = c[i + 96];
        const E v0 = fma(-w, a0, c0), v1 = fma(-w, a1, c1), v2 = fma(-w, a2, c2), v3 = fma(-w, a3, c3);
        c[i] = v0;
        c[i + 32] = v1;
        c[i + 64] = v2;
        c[i + 96] = v3;
        sq = fma(v0, v0, sq);
        sq2 = fma(v1, v1, sq2);
        sq = fma(v2, v2, sq);
        sq2 = fma(v3, v3, sq2);
      }
      for (; i < rb; i += 32) {
        const E v = fma(-w, a[i], c[i]);
        c[i] = v;
        sq = fma(v, v, sq);
      }
    }
    sq = fold_warp_sum(sq + sq2);
    if (lane == 0) {
      trk[k + 1] = tj - wt;
      sc[2] = sq;
    }
  }
#pragma unroll
  for (int q = 0; q < ST; ++q) {
    const int idx = tid + q * kFoldThreads;
    if (tglob && idx < n - k - 1) tbuf[((k + 1) & 1) * n + k + 1 + idx] = tn[q];
  }
  __syncthreads();
}

// Sum of squares of column k of X over ra rows of its P row blocks into sc[2], and (T in
// global memory) T's row k into its staging row; ends in a barrier.
template <typename E>
__device__ __forceinline__ void fold_column_start(const E* X, int ldx, int h, int P, int n, int k, int ra,
                                                  const E* T, bool tglob, E* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  E* sc = red + (n > kFoldWorkers ? n : kFoldWorkers) + n;
  E* tbuf = sc + 4;
  if (tglob)
    for (int idx = tid; idx < n - k; idx += kFoldThreads) tbuf[(k & 1) * n + k + idx] = __ldcg(T + (int64_t)k * n + k + idx);
  if (warp == kFoldPivotWarp) {
    const E* x0 = X + (int64_t)k * ldx;
    E sq = E(0);
    for (int p = 0; p < P; ++p)
      for (int i = lane; i < ra; i += 32) {
        const E v = x0[p * h + i];
        sq = fma(v, v, sq);
      }
    sq = fold_warp_sum(sq);
    if (lane == 0) sc[2] = sq;
  }
  __syncthreads();
}

// Folds X into T.  X holds P row blocks of h rows each (row block p at rows [p h, p h + h),
// leading dimension ldx).  Dense: every row may be non-zero.  tri: every row block holds
// rows [r0, r0 + h) of an upper triangle, so that in column k only its first
// k + 1 - r0 rows can be non-zero.
template <typename E, int ST = 1>
__device__ void fold_chunk(E* X, int ldx, int h, int P, int n, int r0, bool tri, E* T, bool tglob, E* red) {
  auto rows_at = [&](int k) -> int {
    if (!tri) return h;
    const int r = k + 1 - r0;
    return r < 0 ? 0 : (r > h ? h : r);
  };
  // a piece starting at row r0 of a triangle is zero in columns < r0: their reflectors
  // are the identity
  const int kbeg = tri ? (r0 < n ? r0 : n) : 0;
  if (kbeg >= n) return;
  fold_column_start<E>(X, ldx, h, P, n, kbeg, rows_at(kbeg), T, tglob, red);
  for (int k = kbeg; k < n; ++k)
    fold_step<E, ST>(X, ldx, h, P, n, k, n, rows_at(k), rows_at(k + 1), T, tglob, red, nullptr);
}

// ------------------------------------------------------------------ tensor-core fold (float leaf)
// The float leaf folds a chunk by panels of kTcNb columns.  The panel's reflectors come from
// the column steps above, restricted to the panel; the trailing columns then take all of
// them at once in compact WY form: Q = H_0 ... H_{b-1} = I - Y Tw Y^T with
// y_q = (e_{p0+q} on T's rows, x_q / v0_q on X's rows), Tw upper triangular (Tw_qq = tau'_q,
// Tw[0:q, q] = -tau'_q Tw[0:q, 0:q] z, z_r = y_r^T y_q = (x_r^T x_q) / (v0_r v0_q)), so that
//   P  = X_v^T [X_panel X_trail]                 (tensor cores; its panel part gives x_r^T x_q)
//   W  = T[p0.., trail] + diag(1/v0) P_trail,  W' = Tw^T W,
//   T[p0.., trail] -= W',  X_trail -= X_v diag(1/v0) W'   (tensor cores).
// The tensor-core products are tf32 with every operand split into three tf32 parts
// (a = a0 + a1 + a2 exactly to 2^-33 |a|) and the six products of order <= 2 kept, which is
// better than float; every k-step of 8 starts from a zero accumulator and is added to the
// running sums in float on the CUDA cores, so the accumulation rounds like a float dot.
constexpr int kTcLdw = 20;      // leading dimension of the column-by-panel staging buffer

__host__ __device__ __forceinline__ int fold_tc_extra(int n) {
  return ((n * kTcLdw + kTcNb * kTcNb + 2 * kTcNb) + 3) & ~3;
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = p0 + p1 + p2, all tf32 (each remainder is exact in float)
__device__ __forceinline__ void split3_tf32(float x, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
  p0 = to_tf32(x);
  const float r1 = x - __uint_as_float(p0);
  p1 = to_tf32(r1);
  p2 = to_tf32(r1 - __uint_as_float(p1));
}

// d += a b, one m16n8k8 tf32 product with float accumulation
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// d = a b (16 x 8 x 8) from a zero accumulator: the six split products, smallest first
__device__ __forceinline__ void mma_6xtf32(float (&d)[4], const float (&a)[4], const float (&b)[2]) {
  uint32_t a0[4], a1[4], a2[4], b0[2], b1[2], b2[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) split3_tf32(a[i], a0[i], a1[i], a2[i]);
#pragma unroll
  for (int i = 0; i < 2; ++i) split3_tf32(b[i], b0[i], b1[i], b2[i]);
  d[0] = d[1] = d[2] = d[3] = 0.f;
  mma_tf32(d, a2, b0);
  mma_tf32(d, a1, b1);
  mma_tf32(d, a0, b2);
  mma_tf32(d, a1, b0);
  mma_tf32(d, a0, b1);
  mma_tf32(d, a0, b0);
}

// Folds the dense chunk X (m rows, leading dimension ldx = 4 mod 32, against bank
// conflicts of the fragment loads) into T.  ext: kTcLdw x n staging, Tw, tau', 1/v0.
// Fragment layouts of mma.m16n8k8 (g = lane / 4, t = lane % 4): A (16 x 8) a0 = (g, t),
// a1 = (g + 8, t), a2 = (g, t + 4), a3 = (g + 8, t + 4); B (8 x 8) b0 = (t, g),
// b1 = (t + 4, g); C (16 x 8) c0 = (g, 2t), c1 = (g, 2t + 1), c2 = (g + 8, 2t),
// c3 = (g + 8, 2t + 1).
__device__ void fold_chunk_tc(float* X, int ldx, int m, int n, float* T, bool tglob, float* red, float* ext) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  float* Ps = ext;                         // [n][kTcLdw]: P (column j - p0), then diag(1/v0) W'
  float* Tw = ext + n * kTcLdw;            // Tw[r * kTcNb + q]
  float* tpv = Tw + kTcNb * kTcNb;         // tau' of the panel's reflectors
  float* rvv = tpv + kTcRec;               // 1/v0 of the panel's reflectors
  fold_column_start<float>(X, ldx, m, 1, n, 0, m, T, tglob, red);
  for (int p0 = 0; p0 < n; p0 += kTcNb) {
    const int b = (n - p0) < kTcNb ? (n - p0) : kTcNb;
    const int kend = p0 + b;
    for (int k = p0; k < kend; ++k) fold_step<float>(X, ldx, m, 1, n, k, kend, m, m, T, tglob, red, tpv + (k - p0));
    const int c = n - kend;                  // trailing columns
    if (c <= 0) break;
    const float* Xv = X + (int64_t)p0 * ldx; // x_q = column p0 + q
    // ---- P = X_v^T [X_panel X_trail]: 16 x (n - p0), K = m
    {
      const int ncol = n - p0;
      const int NT = (ncol + 7) >> 3, KT = (m + 7) >> 3;
      if (warp < kFoldPivotWarp) {
        for (int nt = warp; nt < NT; nt += kFoldPivotWarp) {
          float sum[4] = {0.f, 0.f, 0.f, 0.f};
          const int jb = nt * 8 + g;
          const bool jok = jb < ncol;
          const float* xb = Xv + (int64_t)jb * ldx;
          const float* xa0 = Xv + (int64_t)g * ldx;
          const float* xa1 = Xv + (int64_t)(g + 8) * ldx;
          const bool q0ok = g < b, q1ok = g + 8 < b;
          for (int kt = 0; kt < KT; kt += 2) {   // two independent k-steps in flight
            float d[2][4];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
              const int i0 = (kt + h2) * 8 + t4, i1 = i0 + 4;
              const bool r0ok = i0 < m, r1ok = i1 < m;
              const float a[4] = {(q0ok && r0ok) ? xa0[i0] : 0.f, (q1ok && r0ok) ? xa1[i0] : 0.f,
                                  (q0ok && r1ok) ? xa0[i1] : 0.f, (q1ok && r1ok) ? xa1[i1] : 0.f};
              const float bb[2] = {(jok && r0ok) ? xb[i0] : 0.f, (jok && r1ok) ? xb[i1] : 0.f};
              mma_6xtf32(d[h2], a, bb);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) sum[i] += d[0][i] + d[1][i];
          }
          const int j0 = nt * 8 + 2 * t4;
          if (j0 < ncol) {
            Ps[j0 * kTcLdw + g] = sum[0];
            Ps[j0 * kTcLdw + g + 8] = sum[2];
          }
          if (j0 + 1 < ncol) {
            Ps[(j0 + 1) * kTcLdw + g] = sum[1];
            Ps[(j0 + 1) * kTcLdw + g + 8] = sum[3];
          }
        }
      }
    }
    __syncthreads();
    // ---- Tw, column by column (one warp; Ps[q][s] = x_s^T x_q for s < q)
    if (warp == 0) {
      for (int q = 0; q < b; ++q) {
        const float tq = tpv[q], rq = rvv[q];
        float val = 0.f;
        if (lane < q) {
          float acc = 0.f;
          for (int s2 = lane; s2 < q; ++s2) acc = fmaf(Tw[lane * kTcNb + s2], Ps[q * kTcLdw + s2] * rvv[s2] * rq, acc);
          val = -tq * acc;
        } else if (lane == q) {
          val = tq;
        }
        __syncwarp();
        if (lane <= q) Tw[lane * kTcNb + q] = val;
        __syncwarp();
      }
    }
    __syncthreads();
    // ---- W' = Tw^T (T[p0.., j] + diag(1/v0) P[:, j]) per trailing column; T rows updated
    for (int jj = tid; jj < c; jj += blockDim.x) {
      const int j = kend + jj, jr = b + jj;
      float w[kTcNb];
#pragma unroll
      for (int q = 0; q < kTcNb; ++q)
        w[q] = q < b ? fmaf(rvv[q], Ps[jr * kTcLdw + q], T[(int64_t)(p0 + q) * n + j]) : 0.f;
#pragma unroll
      for (int q = kTcNb - 1; q >= 0; --q) {   // in place from the last row: w[r], r <= q, still W
        if (q < b) {
          float acc = 0.f;
#pragma unroll
          for (int r = 0; r <= q; ++r) acc = fmaf(Tw[r * kTcNb + q], w[r], acc);
          w[q] = acc;
        }
      }
#pragma unroll
      for (int q = 0; q < kTcNb; ++q) {
        if (q < b) {
          T[(int64_t)(p0 + q) * n + j] -= w[q];
          Ps[jr * kTcLdw + q] = rvv[q] * w[q];
        } else {
          Ps[jr * kTcLdw + q] = 0.f;
        }
      }
    }
    __syncthreads();
    // ---- X_trail -= X_v B, B = diag(1/v0) W' (K = 16)
    {
      const int MT = (m + 15) >> 4, NT = (c + 7) >> 3;
      if (warp < kFoldPivotWarp) {
        for (int u = warp; u < MT * NT; u += kFoldPivotWarp) {
          const int mt = u % MT, nt = u / MT;
          const int r0 = mt * 16 + g, r1 = r0 + 8;
          const int jc0 = nt * 8 + 2 * t4, jb = nt * 8 + g;
          const bool r0ok = r0 < m, r1ok = r1 < m, c0ok = jc0 < c, c1ok = jc0 + 1 < c, jok = jb < c;
          float* x0 = X + (int64_t)(kend + jc0) * ldx;
          float* x1 = x0 + ldx;
          float prod[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int kt = 0; kt < 2; ++kt) {
            const int q0 = kt * 8 + t4, q1 = q0 + 4;
            const float* v0p = Xv + (int64_t)q0 * ldx;
            const float* v1p = Xv + (int64_t)q1 * ldx;
            const bool q0ok = q0 < b, q1ok = q1 < b;
            const float a[4] = {(r0ok && q0ok) ? v0p[r0] : 0.f, (r1ok && q0ok) ? v0p[r1] : 0.f,
                                (r0ok && q1ok) ? v1p[r0] : 0.f, (r1ok && q1ok) ? v1p[r1] : 0.f};
            const float bb[2] = {jok ? Ps[(b + jb) * kTcLdw + q0] : 0.f, jok ? Ps[(b + jb) * kTcLdw + q1] : 0.f};
            float d[4];
            mma_6xtf32(d, a, bb);
#pragma unroll
            for (int i = 0; i < 4; ++i) prod[i] += d[i];
          }
          if (c0ok && r0ok) x0[r0] -= prod[0];
          if (c1ok && r0ok) x1[r0] -= prod[1];
          if (c0ok && r1ok) x0[r1] -= prod[2];
          if (c1ok && r1ok) x1[r1] -= prod[3];
        }
      }
    }
    __syncthreads();
    // ---- the next panel's first column: its sum of squares (its T row is staged already)
    if (warp == kFoldPivotWarp) {
      const float* xn = X + (int64_t)kend * ldx;
      float sq = 0.f;
      for (int i = lane; i < m; i += 32) sq = fmaf(xn[i], xn[i], sq);
      sq = fold_warp_sum(sq);
      if (lane == 0) red[(n > kFoldWorkers ? n : kFoldWorkers) + n + 2] = sq;
    }
    __syncthreads();
  }
}

template <typename E>
struct FoldLeafTc {
  __device__ static bool run(E*, int, int, int, E*, bool, E*, E*) { return false; }
};
template <>
struct FoldLeafTc<float> {
  __device__ static bool run(float* X, int ldx, int m, int n, float* T, bool tglob, float* red, float* ext) {
    fold_chunk_tc(X, ldx, m, n, T, tglob, red, ext);
    return true;
  }
};

// level 0: the leaf over the block's rows; level l > 0: tree level l over tri_in.  ST: T-row
// staging per thread (4 for blocks wider than the 256 worker threads, up to 1,024 columns).
template <typename E, int ST = 1>
__global__ void __launch_bounds__(kFoldThreads, sizeof(E) == 4 ? 2 : 1)
    k_tsqr_fold(TsqrBlock b, const double* tri_in, double* tri_out, int level) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = b.n, mc = b.tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const bool tc = b.fold_tc && level == 0;    // tensor-core panels (float leaf)
  const int ldx_alloc = mc + (b.fold_tc ? 4 : 1);
  E* red = reinterpret_cast<E*>(smem_raw);
  E* ext = red + fold_red_elems(n);
  E* X = ext + (b.fold_tc ? fold_tc_extra(n) : 0);
  E* T = b.fold_tsmem ? X + (int64_t)ldx_alloc * n : static_cast<E*>(b.scratch) + (int64_t)blockIdx.x * n * n;
  const bool tglob = !b.fold_tsmem;
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
  const int ldx = tc ? mc + 4 : mc + 1;      // odd for the column steps, 4 mod 32 for the fragments
  const int stack = mc / n;                   // whole triangles per chunk on tree levels
  int64_t units = (live + per - 1) / per;
  if (units < 1) units = 1;                   // an empty block still leaves a (zero) triangle
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t q1 = (u + 1) * per < live ? (u + 1) * per : live;
    int64_t qs = u * per;
    if (level > 0) {
      // T starts as the unit's first triangle (folding it into a zero T would only
      // reproduce it), and the others are folded in
      const double* src = tri_in + qs * n * n;
      for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        const int r = i / n, c = i - r * n;
        T[i] = r <= c ? (E)src[(int64_t)c * n + r] : E(0);
      }
      ++qs;
    } else {
      for (int i = threadIdx.x; i < n * n; i += blockDim.x) T[i] = E(0);
    }
    __syncthreads();
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
        if (!(tc && FoldLeafTc<E>::run(X, ldx, m, n, T, tglob, red, ext)))
          fold_chunk<E, ST>(X, ldx, m, 1, n, 0, false, T, tglob, red);
      }
    } else if (stack >= 2) {
      for (int64_t q = qs; q < q1; q += stack) {
        const int cnt = (int)((q1 - q) < stack ? (q1 - q) : stack);
        for (int c = warp; c < n; c += nwarps) {
          E* dst = X + (int64_t)c * ldx;
          for (int idx = lane; idx < cnt * n; idx += 32) {
            const int t = idx / n, r = idx - t * n;
            dst[idx] = (E)tri_in[(q + t) * n * n + (int64_t)c * n + r];
          }
        }
        __syncthreads();
        fold_chunk<E, ST>(X, ldx, n, cnt, n, 0, true, T, tglob, red);
      }
    } else {
      for (int64_t q = qs; q < q1; ++q) {
        const double* src = tri_in + q * n * n;
        for (int r0 = 0; r0 < n; r0 += mc) {
          const int m = (n - r0) < mc ? (n - r0) : mc;
          for (int c = warp; c < n; c += nwarps) {
            E* dst = X + (int64_t)c * ldx;
            for (int i = lane; i < m; i += 32) dst[i] = (E)src[(int64_t)c * n + r0 + i];
          }
          __syncthreads();
          fold_chunk<E, ST>(X, ldx, m, 1, n, r0, true, T, tglob, red);
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
  size_t e = (size_t)fold_red_elems(b.n) + (size_t)(b.tile + (b.fold_tc ? 4 : 1)) * b.n;
  if (b.fold_tc) e += (size_t)fold_tc_extra(b.n);
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
  const int64_t cap = b.fold_res > 0 ? b.fold_res : fold_resident(mixed);
  if (grid > cap) grid = cap;
  if (b.n > kFoldWorkers)
    k_tsqr_fold<E, kStackStage><<<(unsigned)grid, kFoldThreads, fold_smem(b, sizeof(E)), st>>>(b, tri_in, tri_out,
                                                                                               level);
  else
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

// Final QR of the stacked block triangles by folding (N <= 1024, at most kStackMaxBlocks
// blocks): the triangles of blocks with pairwise disjoint column sets are placed in T as
// they are, and every other block triangle, embedded at its global columns, is folded in as
// row pieces of an upper triangle: row r of a block triangle is zero before global column
// cols[r] >= cols[0] + r, so a piece starting at row p is the tri case of fold_chunk with
// r0 = cols[p].  The stack's zeros are skipped, where the dense stack of S rows would cost
// 2 S N^2 flops in a leaf and a tree.
__global__ void __launch_bounds__(kFoldThreads, 1)
    k_tsqr_stack_fold(const TsqrBlock* blocks, int nb, int N, int mc, int tsm, double* Tglob, double* tri_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* red = reinterpret_cast<double*>(smem_raw);
  double* X = red + fold_red_elems(N);
  const int ldx = mc + 1;
  double* T = tsm ? X + (int64_t)ldx * N : Tglob;
  const bool tglob = !tsm;
  // Blocks whose column sets are disjoint need no fold: their triangles are placed in T as
  // they are (row r of a block lands in T's row cols[r], still upper triangular).  One
  // thread picks them greedily by rank (non-zero rows of the triangle, min(n, live rows)),
  // largest first; the others are folded in that order, each only over its non-zero rows.
  __shared__ int order[kStackMaxBlocks];
  __shared__ unsigned char placed[kStackMaxBlocks];
  __shared__ uint32_t used[kStackFoldMaxN / 32];
  __shared__ int n_order;
  if (threadIdx.x == 0) {
    int cnt = 0;
    for (int bi = 0; bi < nb && bi < kStackMaxBlocks; ++bi) {
      placed[bi] = 0;
      if (block_rows(blocks[bi]) > 0) order[cnt++] = bi;
    }
    auto rank = [&](int bi) {
      const int64_t r = block_rows(blocks[bi]);
      return r < blocks[bi].n ? (int)r : blocks[bi].n;
    };
    for (int i = 0; i < cnt; ++i)                    // selection sort, rank descending
      for (int j = i + 1; j < cnt; ++j)
        if (rank(order[j]) > rank(order[i])) { const int t = order[i]; order[i] = order[j]; order[j] = t; }
    for (int w = 0; w < (N + 31) / 32; ++w) used[w] = 0u;
    for (int i = 0; i < cnt; ++i) {
      const TsqrBlock& b = blocks[order[i]];
      bool free_cols = nb <= kStackMaxBlocks;
      for (int c = 0; c < b.n && free_cols; ++c) free_cols = !(used[b.cols[c] >> 5] & (1u << (b.cols[c] & 31)));
      if (!free_cols) continue;
      placed[order[i]] = 1;
      for (int c = 0; c < b.n; ++c) used[b.cols[c] >> 5] |= 1u << (b.cols[c] & 31);
    }
    n_order = cnt;
  }
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) T[idx] = 0.0;
  __syncthreads();
  for (int i = 0; i < n_order; ++i) {
    const TsqrBlock& b = blocks[order[i]];
    if (!placed[order[i]]) continue;
    const int n = b.n;
    const double* tri = b.tri[b.top];               // column-major n x n, upper
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int c = idx / n, r = idx - c * n;
      if (r <= c) T[(int64_t)b.cols[r] * N + b.cols[c]] = tri[idx];
    }
  }
  __syncthreads();
  for (int i = 0; i < n_order; ++i) {
    const int bi = order[i];
    if (placed[bi]) continue;
    const TsqrBlock& b = blocks[bi];
    const int n = b.n;
    const int64_t live = block_rows(b);
    const int nz = live < n ? (int)live : n;        // the triangle's rows below nz are zero
    const double* tri = b.tri[b.top];               // column-major n x n, upper
    for (int p = 0; p < nz; p += mc) {
      const int h = (nz - p) < mc ? (nz - p) : mc;
      for (int idx = threadIdx.x; idx < ldx * N; idx += blockDim.x) X[idx] = 0.0;
      __syncthreads();
      for (int idx = threadIdx.x; idx < h * n; idx += blockDim.x) {
        const int c = idx / h, r = idx - c * h;     // local column c, piece row r (block row p + r)
        if (p + r <= c) X[(int64_t)b.cols[c] * ldx + r] = tri[(int64_t)c * n + p + r];
      }
      __syncthreads();
      fold_chunk<double, kStackStage>(X, ldx, h, 1, N, b.cols[p], true, T, tglob, red);
    }
  }
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int c = idx / N, r = idx - c * N;
    tri_out[idx] = r <= c ? (tglob ? __ldcg(T + (int64_t)r * N + c) : T[(int64_t)r * N + c]) : 0.0;
  }
}

// Shared-memory plan of k_tsqr_stack_fold: rows per piece and whether T fits beside X.
static void stack_fold_plan(int N, int& mc, int& tsm, size_t& smem) {
  const size_t red = (size_t)fold_red_elems(N) * sizeof(double);
  const size_t tbytes = (size_t)N * N * sizeof(double);
  tsm = tbytes <= kSmemCap / 4 ? 1 : 0;
  const size_t rest = kSmemCap - red - (tsm ? tbytes : 0);
  int64_t m = (int64_t)(rest / (sizeof(double) * (size_t)N)) - 1;
  m = m >= 32 ? (m / 32) * 32 : (m / 8) * 8;  // rows per piece: at least 16 up to N = 1024
  if (m > 512) m = 512;
  mc = (int)m;
  smem = red + (size_t)(mc + 1) * N * sizeof(double) + (tsm ? tbytes : 0);
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
static bool fold_plan(TsqrBlock& b, bool mixed, size_t esz, bool tcgen05, const TsqrTune* tn) {
  const int n = b.n;
  if (n > kStackFoldMaxN) return false;        // T rows are staged at most four elements per thread
  const bool wide = n > kFoldWorkers;          // no tensor-core panels (their staging is per worker)
  size_t budget = fold_budget(mixed);
  if (tn && tn->fold_budget_kib > 0 && (size_t)tn->fold_budget_kib * 1024 < budget)
    budget = (size_t)tn->fold_budget_kib * 1024;
  const bool tc = mixed && !wide;             // float leaf: tensor-core panels
  const size_t red = ((size_t)fold_red_elems(n) + (tc ? (size_t)fold_tc_extra(n) : 0)) * esz;
  if (red >= budget) return false;
  const bool tsm = (size_t)n * n * esz <= budget / 4;
  const size_t rest = budget - red - (tsm ? (size_t)n * n * esz : 0);
  int64_t mc = (int64_t)(rest / (esz * (size_t)n)) - (tc ? 4 : 1);
  mc = (wide && mc < 32) ? (mc / 16) * 16 : (mc / 32) * 32;   // wide blocks: 16-row chunks at least
  if (mc > 512) mc = 512;
  if (mc < (wide ? 16 : 32)) return false;
  b.fold = true;
  b.fold_tsmem = tsm;
  b.fold_tc = tc;
  b.warp_min = 0;
  b.tile = (int)mc;
  // the float leaf on tcgen05 where its shared-memory layout fits (unless the mma.sync
  // fold was asked for): 128-row chunks (the tree levels fold with the same chunk height),
  // one thread block per SM
  b.fold_tc5 = tcgen05 && mixed && !wide && fold_tc_fits(n);
  if (b.fold_tc5) {
    b.fold_tc = false;
    b.tile = 128;
    mc = 128;
  }
  // tree levels: a unit copies its first triangle and folds the others in, as many per
  // chunk as one chunk stacks, so one chunk per unit and level: fan = stack + 1 (2..16)
  const int64_t stack = mc / n;
  b.fan = (int)(stack + 1 < 2 ? 2 : (stack + 1 > 16 ? 16 : stack + 1));
  if (tn && tn->fan >= 2) b.fan = tn->fan;
  const int64_t chunks = (b.bound + mc - 1) / mc;
  // thread blocks resident at once: one per SM for the tcgen05 leaf, else as many as the
  // budget leaves room for (its tree levels keep the float fold's two per SM)
  int64_t res = b.fold_tc5 ? 152 : fold_resident(mixed);
  if (!b.fold_tc5 && tn && tn->fold_budget_kib > 0) res = 152 * (int64_t)(kSmemCap / budget);
  b.fold_res = (int)(b.fold_tc5 ? fold_resident(true) : res);
  int64_t seg = (chunks + res - 1) / res;
  if (mixed && seg > 16) seg = 16;             // the float path's error grows with the folds per triangle
  if (tn && tn->seg_cap > 0 && seg > tn->seg_cap) seg = tn->seg_cap;
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

void tsqr_plan_block(TsqrBlock& b, bool mixed, bool givens, bool tcgen05, const TsqrTune* tune) {
  const int n = b.n;
  const size_t esz = mixed ? sizeof(float) : sizeof(double);
  // a block may be planned again (the autotuner's choice after the rule): the fold fields of
  // an earlier plan must not survive into a plan of another path
  b.fold = b.fold_tsmem = b.fold_tc = b.fold_tc5 = false;
  b.seg = b.fold_g0 = 0;
  b.fold_res = 0;
  b.nreg = reg_class(n);
  b.givens = givens && b.nreg && b.nreg <= 16;
  b.fused = b.fused && b.kind == BLK_TAILS && b.nreg && !b.givens;
  if (b.nreg) {
    // one warp's QR of a tile costs about N^2 FP64 instructions at ~70 cycles each: for
    // N <= 16 (tiles of 128-256 rows) it beats a thread block per tile from two tiles
    // on; wider tiles (64 rows) keep the block kernel until the level fills the GPU
    b.warp_min = b.nreg <= 16 ? 2 : 152 * 4;
    b.tile = reg_tile_of(b.nreg);
    // n <= 16: tree tiles fill a register tile (fan = TW / n >= 4); wider blocks reduce
    // their trees with the block-per-tile kernel only, six triangles at a time
    b.fan = b.nreg <= 16 ? b.tile / n : 6;
    if (tune && tune->warp_min > 0) b.warp_min = tune->warp_min;
    if (tune && tune->fan >= 2 && (b.nreg > 16 || tune->fan * n <= b.tile)) b.fan = tune->fan;
    if (b.givens) b.tile = kGivensRows;       // leaf chunks of the Givens leaf
    // tails formed in the leaf (tails_qr): QR tiles of 32 lanes x 8, 4 or 2 sorted rows
    else if (b.fused) b.tile = 32 * (b.nreg <= 8 ? 8 : b.nreg <= 16 ? 4 : 2);
  } else if (fold_plan(b, mixed, esz, tcgen05, tune)) {
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
  if (b.fold)                                  // T slots (as doubles: room for floats)
    return b.fold_tsmem ? 0 : (b.fold_res > 0 ? b.fold_res : fold_resident(mixed)) * (int64_t)b.n * b.n;
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
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tsqr_fold<double, kStackStage>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemCap);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tsqr_fold<float, kStackStage>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemCap);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tsqr_stack_fold, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  if (e == cudaSuccess) e = fold_tc_set_attributes();
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
    if (mixed && b.fold_tc5) launch_fold_tc(b, b.tri[0], b.err, st);
    else if (mixed) launch_fold<float>(b, nullptr, b.tri[0], 0, true, st);
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
  // Up to 32 columns the dense stack goes through the register leaf in a launch or two,
  // which beats the fold's single block walking the pieces one Householder step at a time.
  if (N > 32 && N <= kStackFoldMaxN && n_blocks <= kStackMaxBlocks) {
    int mc = 0, tsm = 0;
    size_t smem = 0;
    stack_fold_plan(N, mc, tsm, smem);
    k_tsqr_stack_fold<<<1, kFoldThreads, smem, st>>>(blocks_dev, n_blocks, N, mc, tsm, stack_blk.tri[1],
                                                     stack_blk.tri[0]);
    k_write_r<<<grid_for((int64_t)N * N, 256, 64), 256, 0, st>>>(stack_blk.tri[0], N, R, ldr);
    *launches += 2;
    return;
  }
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
