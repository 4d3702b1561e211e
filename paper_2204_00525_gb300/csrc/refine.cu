// CholeskyQR2-style refinement of the mixed-precision R (FIGARO_PREC_MIXED_REFINED).
// Not a step of the paper: its §7 takes R0 to R by a QR in one precision.  Here R~ comes
// from float32 TSQR; with A^T A = R0^T R0 (the Theorem of §6) accumulated accurately,
//   X = R~^-T (A^T A) R~^-1 = C^T C   (Cholesky, C upper),   R = C R~
// satisfies R^T R = R~^T X R~ = A^T A, and X is close to the identity, so its Cholesky
// factorisation is well conditioned whenever float32 TSQR resolved A.
//
// A^T A is the sum over the R0 blocks of each block's Gram matrix placed at the block's
// columns.  The Gram sums run in double-float arithmetic on the FP32 pipe: the tail rows
// of the mixed path arrive as unevaluated float pairs (hi + lo, the emit's double-float
// value before rounding), the float64 blocks are split into pairs exactly enough
// (2^-47); per-thread double-float partial sums over row slices, then float64 sums of
// the per-block partials in a fixed order (deterministic).
#include "dfloat.cuh"
#include "tsqr_reg.cuh"

namespace fig {

constexpr int kGramThreads = 256;
constexpr int kGramEnt = 4;             // Gram entries per thread when they outnumber threads
constexpr int kGramChunksPerCta = 16;

// Rows staged in shared memory per round: 64, fewer for wide blocks (at most 192 KB).
__host__ __device__ __forceinline__ int gram_chunk(int n) {
  const int c = 24576 / (n > 0 ? n : 1);
  return c < 1 ? 1 : (c > 64 ? 64 : c);
}

__device__ __forceinline__ void df_fma_acc(dfl& acc, dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);                   // exact error of the leading product
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  dfl t;
  fast_two(p, e, t.hi, t.lo);
  acc = df_add(acc, t);
}

// Entry e of the packed upper triangle (row-major over i <= j) -> (i, j).
__device__ __forceinline__ void tri_index(int e, int n, int& i, int& j) {
  i = 0;
  int rem = e;
  while (rem >= n - i) { rem -= n - i; ++i; }
  j = i + rem;
}

// Partial Gram matrices of one R0 block: CTA x writes partial[x][e] for the ne = n(n+1)/2
// entries of blockIdx.y's entry range.  Threads = entries x row slices.
__global__ void __launch_bounds__(kGramThreads) k_gram(TsqrBlock b, const float* lo32, double* partial,
                                                       int ne_cta) {
  extern __shared__ __align__(16) float gsm[];      // [2][chunk][n] hi, lo
  const int n = b.n;
  const int kGramChunk = gram_chunk(n);
  const int64_t rows = block_rows(b);
  const int ne = n * (n + 1) / 2;
  const int e0 = blockIdx.y * ne_cta;
  const int ne_here = ne - e0 < ne_cta ? ne - e0 : ne_cta;
  const int slices = ne_here >= kGramThreads ? 1 : kGramThreads / ne_here;
  const int t = threadIdx.x;
  const int slice = t / (ne_here < kGramThreads ? ne_here : kGramThreads);
  int ei[kGramEnt], ej[kGramEnt];
  bool on[kGramEnt];
  dfl acc[kGramEnt];
#pragma unroll
  for (int q = 0; q < kGramEnt; ++q) {
    const int el = ne_here >= kGramThreads ? t + q * kGramThreads : (q == 0 ? t % ne_here : ne_here);
    on[q] = slice < slices && el < ne_here;
    int i = 0, j = 0;
    if (on[q]) tri_index(e0 + el, n, i, j);
    ei[q] = i;
    ej[q] = j;
    acc[q] = dfl{0.0f, 0.0f};
  }
  float* shi = gsm;
  float* slo = gsm + kGramChunk * n;
  // this CTA's rows: [blockIdx.x * span, (blockIdx.x + 1) * span) in chunks (short-lived
  // CTAs, so that work on higher-priority streams is scheduled in between)
  const int64_t span = (int64_t)kGramChunk * kGramChunksPerCta;
  const int64_t r_end = (blockIdx.x + 1) * span < rows ? (blockIdx.x + 1) * span : rows;
  for (int64_t r0 = (int64_t)blockIdx.x * span; r0 < r_end; r0 += kGramChunk) {
    const int m = (int)(r_end - r0 < kGramChunk ? r_end - r0 : kGramChunk);
    __syncthreads();
    for (int idx = t; idx < m * n; idx += kGramThreads) {
      const int c = idx / m, r = idx - c * m;
      const int64_t g = (int64_t)c * b.ld + r0 + r;
      dfl v;
      if (b.ptr32) v = dfl{b.ptr32[g], lo32 ? lo32[g] : 0.0f};
      else v = df_from_double(b.ptr[g]);
      shi[r * n + c] = v.hi;
      slo[r * n + c] = v.lo;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kGramEnt; ++q) {
      if (!on[q]) continue;
      for (int r = slice; r < m; r += slices)
        df_fma_acc(acc[q], dfl{shi[r * n + ei[q]], slo[r * n + ei[q]]}, dfl{shi[r * n + ej[q]], slo[r * n + ej[q]]});
    }
  }
  // sum the slices of every entry (float64, fixed order) and write the CTA's partial
  __syncthreads();
  double* red = reinterpret_cast<double*>(gsm);     // [kGramThreads * kGramEnt]
#pragma unroll
  for (int q = 0; q < kGramEnt; ++q) red[q * kGramThreads + t] = on[q] ? df_to_double(acc[q]) : 0.0;
  __syncthreads();
  if (slices > 1) {
    if (t < ne_here) {
      double s = 0.0;
      for (int sl = 0; sl < slices; ++sl) s += red[sl * ne_here + t];
      partial[(int64_t)blockIdx.x * ne + e0 + t] = s;
    }
  } else {
#pragma unroll
    for (int q = 0; q < kGramEnt; ++q) {
      const int el = t + q * kGramThreads;
      if (el < ne_here) partial[(int64_t)blockIdx.x * ne + e0 + el] = red[q * kGramThreads + t];
    }
  }
}

// G += the sum over CTAs of a block's partial Gram matrices, at the block's columns
// (both triangles).  One warp per entry: lanes sum strided partials, then a butterfly
// (fixed order, deterministic).  Only the CTAs that held rows are read.
__global__ void k_gram_add(TsqrBlock b, const double* partial, double* G, int N) {
  const int n = b.n;
  const int ne = n * (n + 1) / 2;
  const int64_t rows = block_rows(b);
  const int64_t span = (int64_t)gram_chunk(n) * kGramChunksPerCta;
  const int live = (int)((rows + span - 1) / span);
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < ne; e += warps) {
    double s = 0.0;
    for (int x = lane; x < live; x += 32) s += partial[(int64_t)x * ne + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      int i, j;
      tri_index(e, n, i, j);
      const int gi = b.cols[i], gj = b.cols[j];
      G[(int64_t)gi * N + gj] += s;
      if (gi != gj) G[(int64_t)gj * N + gi] += s;
    }
  }
}

// R (row-major, upper, leading dimension ldr) <- C R with C = chol(R^-T G R^-1), in one
// block of threads.  Every step is right-looking (one row or column finished, then a
// parallel update of the rest), so the sequential depth is O(N), not O(N^2).
// W1, W2: N x N work arrays.  On a zero or non-finite pivot R is left as it is and
// *ok = 0; otherwise *ok = 1.
__global__ void __launch_bounds__(1024) k_refine(double* R, int64_t ldr, const double* G, int N, double* W1,
                                                 double* W2, int* ok) {
  __shared__ int bad;
  extern __shared__ double rinv[];                  // [N]: 1 / R[i][i]
  const int t = threadIdx.x, nt = blockDim.x;
  const int64_t NN = (int64_t)N * N;
  if (t == 0) bad = 0;
  __syncthreads();
  for (int i = t; i < N; i += nt) {
    const double d = R[(int64_t)i * ldr + i];
    if (!(d != 0.0) || !isfinite(d)) bad = 1;
    rinv[i] = 1.0 / d;                               // all divisions at once, in parallel
  }
  for (int64_t idx = t; idx < NN; idx += nt) W1[idx] = G[idx];
  __syncthreads();
  if (!bad) {
    // W1 <- R^-T W1 (forward substitution, all columns at once): row i is final after the
    // division; rows below lose R[i][i'] times it
    for (int i = 0; i < N; ++i) {
      const double ri = rinv[i];
      for (int c = t; c < N; c += nt) W1[(int64_t)i * N + c] *= ri;
      __syncthreads();
      for (int64_t idx = t; idx < (int64_t)(N - i - 1) * N; idx += nt) {
        const int i2 = i + 1 + (int)(idx / N), c = (int)(idx % N);
        W1[(int64_t)i2 * N + c] = fma(-R[(int64_t)i * ldr + i2], W1[(int64_t)i * N + c], W1[(int64_t)i2 * N + c]);
      }
      __syncthreads();
    }
    // W1 <- W1 R^-1 (all rows at once): column j final after the division; columns to the
    // right lose R[j][j'] times it
    for (int j = 0; j < N; ++j) {
      const double rj = rinv[j];
      for (int rr = t; rr < N; rr += nt) W1[(int64_t)rr * N + j] *= rj;
      __syncthreads();
      for (int64_t idx = t; idx < (int64_t)N * (N - j - 1); idx += nt) {
        const int rr = (int)(idx / (N - j - 1)), j2 = j + 1 + (int)(idx % (N - j - 1));
        W1[(int64_t)rr * N + j2] = fma(-W1[(int64_t)rr * N + j], R[(int64_t)j * ldr + j2], W1[(int64_t)rr * N + j2]);
      }
      __syncthreads();
    }
    // Cholesky of the symmetric part, upper factor in W2: X = C^T C
    for (int64_t idx = t; idx < NN; idx += nt) {
      const int i = (int)(idx / N), j = (int)(idx % N);
      W2[idx] = j >= i ? 0.5 * (W1[(int64_t)i * N + j] + W1[(int64_t)j * N + i]) : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < N; ++k) {
      if (t == 0) {
        const double p = W2[(int64_t)k * N + k];
        if (!(p > 0.0) || !isfinite(p)) {
          bad = 1;
        } else {
          double beta, v0, tau, tau2;                 // 1 / sqrt(p) by the Newton steps of
          HhScalars<double>::get(0.0, p, beta, v0, tau, tau2);   // the Householder scalars:
          rinv[0] = -beta;                            // nu = sqrt(p), tau tau2 = 1 / p
          rinv[1] = -beta * tau * tau2;               // 1 / sqrt(p)
        }
      }
      __syncthreads();
      if (bad) break;
      if (t == 0) W2[(int64_t)k * N + k] = rinv[0];
      const double ck_inv = rinv[1];
      for (int j = k + 1 + t; j < N; j += nt) W2[(int64_t)k * N + j] *= ck_inv;
      __syncthreads();
      const int rem = N - k - 1;
      for (int64_t idx = t; idx < (int64_t)rem * rem; idx += nt) {
        const int i = k + 1 + (int)(idx / rem), j = k + 1 + (int)(idx % rem);
        if (j >= i) W2[(int64_t)i * N + j] = fma(-W2[(int64_t)k * N + i], W2[(int64_t)k * N + j], W2[(int64_t)i * N + j]);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (!bad) {
    // W1 = C R (upper times upper), then copy back into R
    for (int64_t idx = t; idx < NN; idx += nt) {
      const int i = (int)(idx / N), j = (int)(idx % N);
      double s = 0.0;
      if (j >= i)
        for (int k = i; k <= j; ++k) s = fma(W2[(int64_t)i * N + k], R[(int64_t)k * ldr + j], s);
      W1[idx] = s;
    }
    __syncthreads();
    for (int64_t idx = t; idx < NN; idx += nt) {
      const int i = (int)(idx / N), j = (int)(idx % N);
      R[(int64_t)i * ldr + j] = W1[idx];
    }
  }
  if (t == 0) *ok = bad ? 0 : 1;
}

int gram_grid(int64_t bound, int n) {
  const int64_t span = (int64_t)gram_chunk(n) * kGramChunksPerCta;
  const int64_t g = (bound + span - 1) / span;
  return (int)(g < 1 ? 1 : g);
}

int gram_entry_groups(int n) {
  const int ne = n * (n + 1) / 2;
  const int per = kGramThreads * kGramEnt;
  return (ne + per - 1) / per;
}

int64_t gram_partial_elems(const TsqrBlock& b) {
  return (int64_t)gram_grid(b.bound, b.n) * b.n * (b.n + 1) / 2;
}

static size_t gram_smem(int n) {
  const size_t stage = (size_t)2 * gram_chunk(n) * n * sizeof(float);
  const size_t red = (size_t)kGramThreads * kGramEnt * sizeof(double);
  return stage > red ? stage : red;
}

cudaError_t refine_set_attributes() {
  return cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void gram_block(const TsqrBlock& b, const float* lo32, double* partial, cudaStream_t st, int64_t* launches) {
  const int grid = gram_grid(b.bound, b.n);
  const int groups = gram_entry_groups(b.n);
  const int ne_cta = kGramThreads * kGramEnt;
  k_gram<<<dim3(grid, groups), kGramThreads, gram_smem(b.n), st>>>(b, lo32, partial, ne_cta);
  ++*launches;
}

void gram_add(const TsqrBlock& b, const double* partial, double* G, int N, cudaStream_t st, int64_t* launches) {
  const int ne = b.n * (b.n + 1) / 2;
  k_gram_add<<<grid_for((int64_t)ne * 32, 256, 152 * 8), 256, 0, st>>>(b, partial, G, N);
  ++*launches;
}

void refine_r(double* R, int64_t ldr, const double* G, int N, double* W1, double* W2, int* ok, cudaStream_t st,
              int64_t* launches) {
  k_refine<<<1, 1024, (size_t)(N > 2 ? N : 2) * sizeof(double), st>>>(R, ldr, G, N, W1, W2, ok);
  ++*launches;
}

}  // namespace fig
