// Post-processing of R0 (§7) as a tall-skinny QR.
//
// §7 triangularizes every non-zero block of R0 (tails of a relation, generalized tails
// of a node, the root Data) on its own columns and then the stack of the resulting
// triangles.  Each block is cut into row tiles; every tile is reduced by Householder
// QR to an n x n triangle (leaf), groups of `fan` triangles are stacked and reduced
// again until one triangle per block remains (tree), and the block triangles, placed
// at their global columns, are reduced by a final QR to R.  The paper's own choices
// were Householder (MKL) or per-thread Givens (THIN); the TSQR tree is the GPU form of
// the same block-then-stack scheme.
//
// Precision: FP64 throughout, or (mixed) FP32 leaf tiles with FP64 tree and final QR.
#include "kernels.cuh"

namespace fig {

constexpr int kQrThreads = 256;
constexpr size_t kSmemCap = 200 * 1024;

__device__ __forceinline__ int64_t block_rows(const TsqrBlock& b) {
  const int32_t G = b.sizes[0], P = b.sizes[1];
  switch (b.kind) {
    case BLK_TAILS: return b.M - G;
    case BLK_GEN: return (int64_t)G - P;
    default: return G;
  }
}

// Householder QR of the m x n column-major matrix A (leading dimension lda) by the
// whole block.  On return the upper triangle of A[0:min(m,n), :] holds R (diagonal of
// either sign); the reflector of column k is x -> beta e_1 with beta = -sign(x_0)||x||.
template <typename E>
__device__ void hh_qr(E* A, int lda, int m, int n, E* red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int kmax = m < n ? m : n;
  for (int k = 0; k < kmax; ++k) {
    E* ak = A + (int64_t)k * lda;
    E s = 0;
    for (int i = k + 1 + tid; i < m; i += blockDim.x) s = fma(ak[i], ak[i], s);
    s = block_sum<E>(s, red);
    const E alpha = ak[k];
    if (s == E(0)) continue;                         // column already reduced below k
    const E normx = sqrt(fma(alpha, alpha, s));
    const E beta = alpha >= E(0) ? -normx : normx;
    const E tau = (beta - alpha) / beta;
    const E scal = E(1) / (alpha - beta);
    __syncthreads();                                  // alpha read by everyone
    for (int i = k + 1 + tid; i < m; i += blockDim.x) ak[i] *= scal;   // v, with v_k = 1
    if (tid == 0) ak[k] = beta;
    __syncthreads();
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

// Leaf: tile blockIdx.x of the block's rows -> n x n triangle (zeros below the diagonal).
template <typename E>
__global__ void __launch_bounds__(kQrThreads) k_tsqr_leaf(TsqrBlock b, E* gscratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t rows = block_rows(b);
  const int64_t r0 = (int64_t)blockIdx.x * b.tile;
  if (r0 >= rows) return;
  const int n = b.n, T = b.tile;
  const int m = (int)((rows - r0) < T ? (rows - r0) : T);
  E* red = reinterpret_cast<E*>(smem_raw);
  E* A = gscratch ? gscratch + (int64_t)blockIdx.x * T * n : red + 64;
  for (int c = 0; c < n; ++c)
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      A[(int64_t)c * T + i] = (E)b.ptr[(int64_t)c * b.ld + r0 + i];
  __syncthreads();
  hh_qr<E>(A, T, m, n, red);
  double* tri = b.tri[0] + (int64_t)blockIdx.x * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int c = idx / n, r = idx - c * n;
    tri[idx] = (r <= c && r < m) ? (double)A[(int64_t)c * T + r] : 0.0;
  }
}

// Tree level: stack `fan` triangles of the previous level and reduce them to one.
__global__ void __launch_bounds__(kQrThreads) k_tsqr_reduce(TsqrBlock b, const double* tri_in, double* tri_out,
                                                           int64_t div_in, double* gscratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t rows = block_rows(b);
  const int64_t nt_in = (rows + div_in - 1) / div_in;
  const int64_t first = (int64_t)blockIdx.x * b.fan;
  if (first >= nt_in) return;
  const int n = b.n, F = b.fan;
  const int cnt = (int)((nt_in - first) < F ? (nt_in - first) : F);
  const int lda = F * n, m = cnt * n;
  double* red = reinterpret_cast<double*>(smem_raw);
  double* A = gscratch ? gscratch + (int64_t)blockIdx.x * lda * n : red + 64;
  for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
    const int c = idx / m, rr = idx - c * m;
    const int f = rr / n, r = rr - f * n;
    A[(int64_t)c * lda + rr] = tri_in[(first + f) * n * n + (int64_t)c * n + r];
  }
  __syncthreads();
  hh_qr<double>(A, lda, m, n, red);
  double* tri = tri_out + (int64_t)blockIdx.x * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int c = idx / n, r = idx - c * n;
    tri[idx] = (r <= c && r < m) ? A[(int64_t)c * lda + r] : 0.0;
  }
}

// Final: place every block's triangle at its global columns, QR the stack, write R
// row-major with a non-negative diagonal and zeros below it.
__global__ void __launch_bounds__(kQrThreads) k_tsqr_final(const TsqrBlock* blocks, int nb, int stack_rows,
                                                          int N, double* stack, double* R, int64_t ldr,
                                                          int use_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* red = reinterpret_cast<double*>(smem_raw);
  double* A = use_smem ? red + 64 : stack;
  const int lda = stack_rows;
  for (int idx = threadIdx.x; idx < stack_rows * N; idx += blockDim.x) A[idx] = 0.0;
  __syncthreads();
  int off = 0;
  for (int bi = 0; bi < nb; ++bi) {
    const TsqrBlock& b = blocks[bi];
    const int n = b.n;
    if (block_rows(b) > 0) {
      const double* tri = b.tri[b.top];
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int c = idx / n, r = idx - c * n;
        A[(int64_t)b.cols[c] * lda + off + r] = tri[idx];
      }
    }
    off += n;
  }
  __syncthreads();
  hh_qr<double>(A, lda, stack_rows, N, red);
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    double v = 0.0;
    if (j >= i && i < stack_rows) {
      const double d = A[(int64_t)i * lda + i];
      v = (d < 0.0 ? -1.0 : 1.0) * A[(int64_t)j * lda + i];
    }
    R[(int64_t)i * ldr + j] = v;
  }
}

// ------------------------------------------------------------------ host planning
static size_t leaf_smem(int tile, int n, size_t esz) { return (64 + (size_t)tile * n) * esz; }
static size_t reduce_smem(int fan, int n) { return (64 + (size_t)fan * n * n) * sizeof(double); }

void tsqr_plan_block(TsqrBlock& b, bool mixed) {
  const int n = b.n;
  const size_t esz = mixed ? sizeof(float) : sizeof(double);
  // leaf tile: about 64 KB of shared memory, at least n rows, a multiple of 32
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
  const size_t esz = mixed ? sizeof(float) : sizeof(double);
  int64_t need = 0;
  const int64_t tiles = (b.bound + b.tile - 1) / b.tile;
  if (leaf_smem(b.tile, b.n, esz) > kSmemCap) need = tiles * b.tile * b.n;
  if (reduce_smem(b.fan, b.n) > kSmemCap) {
    const int64_t rt = (tiles + b.fan - 1) / b.fan;
    const int64_t r = rt * b.fan * b.n * b.n;
    if (r > need) need = r;
  }
  return need;
}

template <typename E>
static void launch_leaf(const TsqrBlock& b, E* scratch, cudaStream_t st) {
  const int64_t tiles = (b.bound + b.tile - 1) / b.tile;
  if (tiles < 1) return;
  size_t smem = leaf_smem(b.tile, b.n, sizeof(E));
  if (smem > kSmemCap) smem = 64 * sizeof(E); else scratch = nullptr;
  cudaFuncSetAttribute(k_tsqr_leaf<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_tsqr_leaf<E><<<(unsigned)tiles, kQrThreads, smem, st>>>(b, scratch);
}

void tsqr_leaf(const TsqrBlock& b, bool mixed, void* scratch, cudaStream_t st, int64_t* launches) {
  if (mixed) launch_leaf<float>(b, static_cast<float*>(scratch), st);
  else launch_leaf<double>(b, static_cast<double*>(scratch), st);
  ++*launches;
}

void tsqr_reduce(TsqrBlock& b, void* scratch, cudaStream_t st, int64_t* launches) {
  int64_t div = b.tile;
  int64_t tiles = (b.bound + b.tile - 1) / b.tile;
  size_t smem = reduce_smem(b.fan, b.n);
  double* gs = nullptr;
  if (smem > kSmemCap) { smem = 64 * sizeof(double); gs = static_cast<double*>(scratch); }
  cudaFuncSetAttribute(k_tsqr_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int cur = 0;
  for (int l = 0; l < b.levels; ++l) {
    const int64_t out_tiles = (tiles + b.fan - 1) / b.fan;
    k_tsqr_reduce<<<(unsigned)out_tiles, kQrThreads, smem, st>>>(b, b.tri[cur], b.tri[cur ^ 1], div, gs);
    ++*launches;
    cur ^= 1;
    div *= b.fan;
    tiles = out_tiles;
  }
}

void tsqr_final(const TsqrBlock* blocks_dev, int n_blocks, int stack_rows, int N, double* stack,
                double* R, int64_t ldr, cudaStream_t st, int64_t* launches) {
  size_t smem = (64 + (size_t)stack_rows * N) * sizeof(double);
  int use_smem = smem <= kSmemCap;
  if (!use_smem) smem = 64 * sizeof(double);
  cudaFuncSetAttribute(k_tsqr_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_tsqr_final<<<1, kQrThreads, smem, st>>>(blocks_dev, n_blocks, stack_rows, N, stack, R, ldr, use_smem);
  ++*launches;
}

double tsqr_leaf_flops(int64_t rows, int n) {
  // Householder on the leaf tiles: about 2 m n^2 - 2 n^3 / 3 per tile; summed over
  // the rows of the block this is 2 rows n^2 up to the per-tile correction.
  return 2.0 * (double)rows * n * n;
}

}  // namespace fig
