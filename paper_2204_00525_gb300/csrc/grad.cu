// Gradients of a loss on R with respect to every relation's data columns.
//
// The paper computes R (§7) but does not differentiate it.  R depends on the join matrix
// A only through A^T A, and for full column rank the derivative of the QR factor gives
//   dL/dA = A W,  W = R^-1 copyltu(R Rbar^T) R^-T      (Rbar = dL/dR, N x N symmetric W)
// (copyltu mirrors the lower triangle).  The gradient for tuple t of relation S_k is the
// sum of dL/dA over the join rows that contain t:
//   dL/dy_t = m(t)^T W[:, Y_k],   m(t) = sum of the join rows of A that contain t,
// and m(t) = c(t) y_t on Y_k (c(t) = Phi_circ of t's group, Fig. 4) plus, on every other
// relation's columns, sums that come from messages over the join tree keyed by the
// attributes that neighbours share (the counts are Alg. 3's Phi_down / Phi_up):
//   up_i[x]   (post-order) sum over the join of S_i's subtree, restricted to key x of X_p,
//             of the rows' subtree columns;
//   down_j[x] (pre-order)  the same over the rest of the tree for key x of child j's X_p.
// All tuples of a group x_i join alike, so messages are formed from the group sums
// S_i(g) = head(g) sqrt(rows) and the per-tuple work is one small matrix-vector product.
// Message sums use FP64 atomics combined per warp first: the gradient is accurate to
// rounding but not bitwise reproducible from call to call.
#include "kernels.cuh"

namespace fig {

constexpr int kGradChunk = 8;     // gradient columns formed together per pass

// ------------------------------------------------------------------ W
// One block.  M = R Rbar^T, S = copyltu(M), X = R^-1 S, W = (R^-1 X^T)^T, with the
// triangular solves right-looking (row i final, then the rows above updated).  A zero
// diagonal of R sets FIGARO_ERR_SINGULAR.  T1, T2: N x N work arrays.
__global__ void __launch_bounds__(1024) k_grad_w(const double* R, int64_t ldr, const double* Rbar, int64_t ldb,
                                                 int N, double* W, double* T1, double* T2, int* err) {
  __shared__ int bad;
  const int t = threadIdx.x, nt = blockDim.x;
  const int64_t NN = (int64_t)N * N;
  if (t == 0) bad = 0;
  __syncthreads();
  for (int i = t; i < N; i += nt) {
    const double d = R[(int64_t)i * ldr + i];
    if (!(d != 0.0) || !isfinite(d)) bad = 1;
  }
  // T1 = M = R Rbar^T (R upper: M_ij = sum_{k >= i} R_ik Rbar_jk)
  for (int64_t idx = t; idx < NN; idx += nt) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    double s = 0.0;
    for (int k = i; k < N; ++k) s = fma(R[(int64_t)i * ldr + k], Rbar[(int64_t)j * ldb + k], s);
    T1[idx] = s;
  }
  __syncthreads();
  if (bad) {
    if (t == 0) set_error(err, FIGARO_ERR_SINGULAR);
    return;
  }
  // T2 = S = copyltu(M)
  for (int64_t idx = t; idx < NN; idx += nt) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    T2[idx] = i >= j ? T1[idx] : T1[(int64_t)j * N + i];
  }
  __syncthreads();
  tri_solve_upper_rows(R, ldr, T2, N);          // T2 = X = R^-1 S
  for (int64_t idx = t; idx < NN; idx += nt) {  // T1 = X^T
    const int i = (int)(idx / N), j = (int)(idx % N);
    T1[idx] = T2[(int64_t)j * N + i];
  }
  __syncthreads();
  tri_solve_upper_rows(R, ldr, T1, N);          // T1 = R^-1 X^T = W^T
  for (int64_t idx = t; idx < NN; idx += nt) {  // W (symmetric in exact arithmetic)
    const int i = (int)(idx / N), j = (int)(idx % N);
    W[idx] = 0.5 * (T1[idx] + T1[(int64_t)j * N + i]);
  }
}

// ------------------------------------------------------------------ messages
__device__ __forceinline__ double child_count(const GradNode& g, int c, int32_t grp) {
  const int32_t q = g.q[(int64_t)c * g.M + grp];
  return q < 0 ? 0.0 : (double)g.cphid[c][q];
}

// Group sum of column a of S_i: head * sqrt(rows) = head * rows / sqrt(rows).
__device__ __forceinline__ double group_sum(const GradNode& g, int32_t grp, int a) {
  const double rows = (double)(g.goff[grp + 1] - g.goff[grp]);
  return g.heads[(int64_t)a * g.ldh + grp] * rows * g.hrow[grp];
}

// Column col of the join-sum over the combinations of group grp with the rest of the
// tree: S_i's own columns, a child's subtree, or the rest of the tree (the message
// received from the parent).  skip = a child whose subtree is left out (the message sent
// down to it) or -1; cd = Phi_up at the group's X_p key (1 at the root, and for up
// messages, which stop at S_i); cu[c] = Phi_down of child c at the group's key.  With
// per_tuple the sum is for one tuple of the group (m(t)), else for all of them.
__device__ double group_message(const GradNode& g, int32_t grp, int col, int skip, double cd, bool up,
                                const double* cu, bool per_tuple = false) {
  const int kind = g.colkind[col];
  const double rows = per_tuple ? 1.0 : (double)(g.goff[grp + 1] - g.goff[grp]);
  if (kind == 0) {
    double coef = cd;
    for (int c = 0; c < g.n_child; ++c)
      if (c != skip) coef *= cu[c];
    return coef == 0.0 ? 0.0 : coef * group_sum(g, grp, col - g.col_off);
  }
  if (kind <= kMaxChildren) {
    const int c = kind - 1;
    if (c == skip) return 0.0;
    double coef = rows * cd;
    for (int c2 = 0; c2 < g.n_child; ++c2)
      if (c2 != skip && c2 != c) coef *= cu[c2];
    const int32_t q = g.q[(int64_t)c * g.M + grp];
    if (coef == 0.0 || q < 0) return 0.0;
    return coef * g.cup[c][(int64_t)col * g.cld[c] + q];
  }
  if (up || g.is_root) return 0.0;                  // the rest of the tree: not in an up message
  double coef = rows;
  for (int c = 0; c < g.n_child; ++c)
    if (c != skip) coef *= cu[c];
  if (coef == 0.0) return 0.0;
  return coef * g.dn[(int64_t)col * g.ldd + g.g2p[grp]];
}

// base[idx] += v over the lanes with `on`, lanes with equal idx combined first.  All 32
// lanes of the warp must call it.
__device__ __forceinline__ void warp_add_f64(double* base, int32_t idx, double v, bool on) {
  const int lane = threadIdx.x & 31;
  const bool live = on && v != 0.0;
  const unsigned peers = __match_any_sync(0xffffffffu, live ? idx : -1 - lane);
  if (!__any_sync(0xffffffffu, __popc(peers) > 1)) {   // warp-uniform: no lane has a partner
    if (live) atomicAdd(base + idx, v);
    return;
  }
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    const double o = __shfl_sync(0xffffffffu, v, t);
    if ((peers >> t) & 1u) s += o;
  }
  if (live && lane == __ffs(peers) - 1) atomicAdd(base + idx, s);
}

// Same for non-decreasing idx across the lanes (runs of equal idx are contiguous): a
// segmented inclusive scan, and the last lane of every run adds.
__device__ __forceinline__ void warp_add_sorted_f64(double* base, int32_t idx, double v, bool on) {
  const int lane = threadIdx.x & 31;
  const int32_t key = on ? idx : -1 - lane;
  double s = on ? v : 0.0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double so = __shfl_up_sync(0xffffffffu, s, o);
    const int32_t ko = __shfl_up_sync(0xffffffffu, key, o);
    if (lane >= o && ko == key) s += so;
  }
  const int32_t next = __shfl_down_sync(0xffffffffu, key, 1);
  if (on && (lane == 31 || next != key) && s != 0.0) atomicAdd(base + idx, s);
}

__global__ void k_grad_clear(double* a, int64_t ld, const int32_t* sizes, int N) {
  const int64_t P = sizes[1];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P * N; k += (int64_t)gridDim.x * blockDim.x)
    a[(k / P) * ld + k % P] = 0.0;
}

// up_i[x_p][col] += contribution of every group (thread = group, blockIdx.y = column).
// Grid-stride loops keep warps whole for warp_add_f64.
__global__ void k_grad_up(GradNode g) {
  const int col = blockIdx.y;
  if (g.colkind[col] == 255) return;                 // not a column of the subtree
  const int64_t G = g.sizes[0];
  const int lane = threadIdx.x & 31;
  for (int64_t grp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; grp - lane < G;
       grp += (int64_t)gridDim.x * blockDim.x) {
    const bool on = grp < G;
    double v = 0.0;
    int32_t target = 0;
    if (on) {
      double cu[kMaxChildren];
      for (int c = 0; c < g.n_child; ++c) cu[c] = child_count(g, c, (int32_t)grp);
      v = group_message(g, (int32_t)grp, col, -1, 1.0, true, cu);
      target = g.g2p[grp];
    }
    warp_add_sorted_f64(g.up + (int64_t)col * g.ldu, target, v, on);   // groups are sorted by X_p
  }
}

// down_j[x_ij][col] += contribution of every group of S_i to child j (blockIdx.y = column).
__global__ void k_grad_down(GradNode g, int j, double* dn_child, int64_t ld_child) {
  const int col = blockIdx.y;
  const int kind = g.colkind[col];
  if (kind == 1 + j) return;                          // child j's own subtree
  const int64_t G = g.sizes[0];
  const int lane = threadIdx.x & 31;
  for (int64_t grp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; grp - lane < G;
       grp += (int64_t)gridDim.x * blockDim.x) {
    const bool on = grp < G;
    double v = 0.0;
    int32_t target = -1;
    if (on) {
      target = g.q[(int64_t)j * g.M + grp];
      if (target >= 0) {
        double cu[kMaxChildren];
        for (int c = 0; c < g.n_child; ++c) cu[c] = child_count(g, c, (int32_t)grp);
        const double cd = g.is_root ? 1.0 : (double)g.phiu[g.g2p[grp]];
        v = group_message(g, (int32_t)grp, col, j, cd, false, cu);
      }
    }
    warp_add_f64(dn_child + (int64_t)col * ld_child, target < 0 ? 0 : target, v, on && target >= 0);
  }
}

// phi(g)[a] = sum over the columns outside Y_k of m(g)[col] W[col][col_off + a]: the
// part of the gradient shared by all tuples of group g.  Thread per group: m(g) column by
// column, accumulated into kGradChunk outputs at a time (no cross-lane sums: every FP64
// instruction does useful work in every lane).
__global__ void k_grad_group(GradNode g) {
  const int64_t G = g.sizes[0];
  for (int64_t grp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; grp < G;
       grp += (int64_t)gridDim.x * blockDim.x) {
    double cu[kMaxChildren];
    for (int c = 0; c < g.n_child; ++c) cu[c] = child_count(g, c, (int32_t)grp);
    const double cd = g.is_root ? 1.0 : (double)g.phiu[g.g2p[grp]];
    for (int a0 = 0; a0 < g.Ni; a0 += kGradChunk) {
      double acc[kGradChunk];
#pragma unroll
      for (int q = 0; q < kGradChunk; ++q) acc[q] = 0.0;
      for (int col = 0; col < g.N; ++col) {
        if (g.colkind[col] == 0) continue;
        const double m = group_message(g, (int32_t)grp, col, -1, cd, false, cu, true);
        if (m == 0.0) continue;
        const double* wrow = g.W + (int64_t)col * g.N + g.col_off + a0;
#pragma unroll
        for (int q = 0; q < kGradChunk; ++q)
          if (a0 + q < g.Ni) acc[q] = fma(m, wrow[q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < kGradChunk; ++q)
        if (a0 + q < g.Ni) g.phi[(int64_t)(a0 + q) * g.M + grp] = acc[q];
    }
  }
}

// dL/dy_t[a] = Phi_circ(g) sum_b y_t[b] W[col_off + b][col_off + a] + phi(g)[a], written at
// the tuple's input row.  Thread per sorted row: its values come from the sorted copy of
// the data that the forward pass kept (coalesced), all its columns at once.
__global__ void k_grad_rows(GradNode g) {
  const int64_t M = g.M;
  const double* Wk = g.W + (int64_t)g.col_off * g.N + g.col_off;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t grp = g.row_gid[e];
    const int64_t src = g.perm ? g.perm[e] : e;
    const double c = (double)g.phic[grp];
    for (int a0 = 0; a0 < g.Ni; a0 += kGradChunk) {
      double s[kGradChunk];
#pragma unroll
      for (int q = 0; q < kGradChunk; ++q) s[q] = 0.0;
      if (c != 0.0)
        for (int b = 0; b < g.Ni; ++b) {
          const double y = g.sdata ? g.sdata[(int64_t)b * g.lds + e] : g.data[src * g.rs + (int64_t)b * g.cs];
          const double* wrow = Wk + (int64_t)b * g.N + a0;
#pragma unroll
          for (int q = 0; q < kGradChunk; ++q)
            if (a0 + q < g.Ni) s[q] = fma(y, wrow[q], s[q]);
        }
#pragma unroll
      for (int q = 0; q < kGradChunk; ++q)
        if (a0 + q < g.Ni)
          g.grad[(int64_t)(a0 + q) * g.ldg + src] = fma(c, s[q], g.phi[(int64_t)(a0 + q) * g.M + grp]);
    }
  }
}

void grad_w(const double* R, int64_t ldr, const double* Rbar, int64_t ldb, int N, double* W, double* T1, double* T2,
            int* err, cudaStream_t st) {
  k_grad_w<<<1, 1024, 0, st>>>(R, ldr, Rbar, ldb, N, W, T1, T2, err);
}

void grad_clear(double* a, int64_t ld, const int32_t* sizes, int N, int64_t bound, cudaStream_t st) {
  k_grad_clear<<<grid_for(bound * N, 256, 152 * 8), 256, 0, st>>>(a, ld, sizes, N);
}

void grad_up(const GradNode& g, int64_t bound, cudaStream_t st) {
  k_grad_up<<<dim3(grid_for(bound, 256, 152 * 8), g.N), 256, 0, st>>>(g);
}

void grad_down(const GradNode& g, int j, double* dn_child, int64_t ld_child, int64_t bound, cudaStream_t st) {
  k_grad_down<<<dim3(grid_for(bound, 256, 152 * 8), g.N), 256, 0, st>>>(g, j, dn_child, ld_child);
}

void grad_rows(const GradNode& g, int64_t bound, cudaStream_t st) {
  if (g.Ni == 0) return;
  k_grad_group<<<grid_for(bound, 256, 152 * 8), 256, 0, st>>>(g);
  k_grad_rows<<<grid_for(bound, 256, 152 * 8), 256, 0, st>>>(g);
}

}  // namespace fig
