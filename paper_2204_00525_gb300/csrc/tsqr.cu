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
  int64_t tiles = (b.bound + b.tile - 1) / b.tile;
  if (tiles < 1) tiles = 1;
  return tiles * b.n * b.n;
}

int64_t tsqr_scratch_elems(const TsqrBlock& b, bool mixed) {
  if (b.nreg) return 0;
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
  if (b.nreg) {
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
    if (b.nreg && b.nreg <= 16) {
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
