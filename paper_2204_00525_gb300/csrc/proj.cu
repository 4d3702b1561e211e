// Projections of the join matrix, A X for a small X (Q = A R^-1, U = A V Sigma^-1, the
// principal-component scores A V_k): §8.1-8.3 of the paper express Q, U and the scores
// through R and V; their row count is the join size, so they are formed only when the
// caller provides room for every join row.
//
// Row tau of A X is the sum over the relations k of y_{tau_k}^T X[Y_k, :], so every
// relation's rows are first multiplied by their block of X (P_k = Y_k X[Y_k, :]), and
// every output row then decodes which tuple of each relation it combines and adds their
// P_k rows.  The join rows are enumerated in a fixed order: the root's tuples in sorted
// order; below a tuple t of node i, the combinations of its children's subtrees in mixed
// radix (first child most significant, radix Phi_down_c at t's key); inside child c's
// X_p group, its tuples in sorted order, each covering Theta_down(g) / rows(g)
// combinations of its own subtree (Alg. 3's counts, exact in uint64).
#include "kernels.cuh"

namespace fig {

// X <- R^-1 for upper-triangular R (row-major, ld ldr): X starts as the identity.
__global__ void __launch_bounds__(1024) k_tri_inverse(const double* R, int64_t ldr, int N, double* X, int* err) {
  const int t = threadIdx.x, nt = blockDim.x;
  __shared__ int bad;
  if (t == 0) bad = 0;
  __syncthreads();
  for (int i = t; i < N; i += nt) {
    const double d = R[(int64_t)i * ldr + i];
    if (!(d != 0.0) || !isfinite(d)) bad = 1;
  }
  for (int64_t idx = t; idx < (int64_t)N * N; idx += nt) X[idx] = (idx / N == idx % N) ? 1.0 : 0.0;
  __syncthreads();
  if (bad) {
    if (t == 0) set_error(err, FIGARO_ERR_SINGULAR);
    return;
  }
  tri_solve_upper_rows(R, ldr, X, N);
}

// X[i][c] = V[i][c] / sigma[c] (U's columns), or V[i][c] (scores), for c < k.
__global__ void k_scale_v(const double* V, const double* sigma, int N, int k, int divide, double* X, int* err) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)N * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / k), c = (int)(idx % k);
    double v = V[(int64_t)i * N + c];
    if (divide) {
      const double s = sigma[c];
      if (!(s > 0.0)) { set_error(err, FIGARO_ERR_SINGULAR); v = 0.0; }
      else v /= s;
    }
    X[idx] = v;
  }
}

// P[row][c] = sum_b data[row][b] X[col_off + b][c] (row-major P, input row order).
__global__ void k_proj_rows(const double* data, int64_t rs, int64_t cs, int64_t M, int Ni, const double* X,
                            int64_t ldx, int col_off, int k, double* P) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < M * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / k;
    const int c = (int)(idx % k);
    double s = 0.0;
    for (int b = 0; b < Ni; ++b) s = fma(data[row * rs + (int64_t)b * cs], X[(int64_t)(col_off + b) * ldx + c], s);
    P[idx] = s;
  }
}

// First index g in [lo, hi) with incl[g] > v (incl non-decreasing); hi if none.
__device__ __forceinline__ int64_t upper_bound_u64(const uint64_t* incl, int64_t lo, int64_t hi, uint64_t v) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (incl[mid] > v) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// One output row per thread (grid-stride).  nodes[] is in pre-order (nodes[0] = root).
__global__ void k_project(const ProjNode* nodes, int r, int k, uint64_t total, double* out, int64_t ldo) {
  for (uint64_t row = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; row < total;
       row += (uint64_t)gridDim.x * blockDim.x) {
    int64_t e[kMaxRel];              // sorted position of the tuple chosen in each node
    uint64_t j[kMaxRel];             // index among the combinations below that tuple
    uint64_t d[kMaxRel];             // index among the node's combinations at its X_p key
    int32_t x[kMaxRel];              // the node's X_p group (child-side index of the key)
    bool ok = true;
    for (int v = 0; v < r && ok; ++v) {
      const ProjNode& n = nodes[v];
      int64_t lo, hi;
      uint64_t base, want;
      if (v == 0) {
        lo = 0;
        hi = n.sizes[0];
        base = 0;
        want = row;
      } else {
        lo = n.pgoff[x[v]];
        hi = n.pgoff[x[v] + 1];
        base = lo > 0 ? n.theta_incl[lo - 1] : 0;
        want = base + d[v];
      }
      const int64_t g = upper_bound_u64(n.theta_incl, lo, hi, want);
      if (g >= hi) { ok = false; break; }
      const uint64_t before = n.theta_incl[g] - n.theta[g];
      const uint64_t local = want - before;
      const uint64_t rows = (uint64_t)(n.goff[g + 1] - n.goff[g]);
      const uint64_t w = n.theta[g] / rows;          // combinations below each tuple
      e[v] = n.goff[g] + (int64_t)(local / w);
      j[v] = local % w;
      // digits of j[v] for the children (first child most significant)
      uint64_t rem = j[v];
      for (int c = n.n_child - 1; c >= 0; --c) {
        const int cv = n.child[c];
        const int32_t q = n.q[(int64_t)c * n.M + g];
        const uint64_t radix = q < 0 ? 0 : nodes[cv].phid[q];
        if (radix == 0) { ok = false; break; }
        d[cv] = rem % radix;
        rem /= radix;
        x[cv] = q;
      }
    }
    if (!ok) continue;                                // unreachable for consistent counts
    for (int c = 0; c < k; ++c) {
      double s = 0.0;
      for (int v = 0; v < r; ++v) {
        const ProjNode& n = nodes[v];
        if (!n.P) continue;
        const int64_t src = n.perm ? n.perm[e[v]] : e[v];
        s += n.P[src * k + c];
      }
      out[row * ldo + c] = s;
    }
  }
}

void tri_inverse(const double* R, int64_t ldr, int N, double* X, int* err, cudaStream_t st) {
  k_tri_inverse<<<1, 1024, 0, st>>>(R, ldr, N, X, err);
}

void scale_v(const double* V, const double* sigma, int N, int k, bool divide, double* X, int* err, cudaStream_t st) {
  k_scale_v<<<grid_for((int64_t)N * k, 256, 64), 256, 0, st>>>(V, sigma, N, k, divide ? 1 : 0, X, err);
}

void proj_rows(const double* data, int64_t rs, int64_t cs, int64_t M, int Ni, const double* X, int64_t ldx,
               int col_off, int k, double* P, cudaStream_t st) {
  k_proj_rows<<<grid_for(M * k, 256, 152 * 16), 256, 0, st>>>(data, rs, cs, M, Ni, X, ldx, col_off, k, P);
}

void project(const ProjNode* nodes, int r, int k, uint64_t total, double* out, int64_t ldo, cudaStream_t st) {
  const int64_t blocks = (int64_t)((total + 255) / 256);
  k_project<<<(unsigned)(blocks < 152 * 16 ? (blocks < 1 ? 1 : blocks) : 152 * 16), 256, 0, st>>>(nodes, r, k, total,
                                                                                                 out, ldo);
}

}  // namespace fig
