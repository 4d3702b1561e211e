// Count aggregates of §5 (Alg. 3) on the device, exact in uint64.
//
// pass 1 (post-order over the join tree), one thread per group x_i of S_i:
//   rows_per_key(x_i) = group size, Theta_down(x_i) = rows * prod_children Phi_down_j(x_ij),
//   Phi_down_i(x_p) += Theta_down(x_i)   (integer atomics: order-independent, exact).
// The atomics are combined per warp first (one atomic per distinct target and warp): with
// Zipf-skewed keys thousands of groups add into the same few x_p.
// pass 2 (pre-order):
//   full_join_size(x_i) = Theta_down(x_i) * Phi_up_i(x_p)  (1 at the root),
//   Phi_up_j(x_ij) += full_join_size(x_i) for every child j,
//   Phi_circ(x_i) = full_join_size(x_i) / rows_per_key(x_i);
// then, per child, Phi_up_j(x) /= Phi_down_j(x).
// x_ij is located in the child's table of X_p keys (sorted, distinct) by binary search.
// A key with no partner in a child gets Theta_down = 0, hence weight 0 everywhere:
// such tuples are not in the join, so dropping them is exact.
#include "kernels.cuh"

namespace fig {

__device__ __forceinline__ int32_t find_key(const uint64_t* keys, int32_t n, uint64_t x) {
  int32_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    int32_t mid = (lo + hi) >> 1;
    uint64_t v = keys[mid];
    if (v == x) return mid;
    if (v < x) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__device__ __forceinline__ uint64_t project_key(const ChildLink& c, uint64_t key) {
  uint64_t x = 0;
  for (int a = 0; a < c.n_attr; ++a)
    x |= shl64(shr64(key, c.src_shift[a]) & mask64(c.bits[a]), c.dst_shift[a]);
  return x;
}

// arr[idx] += v for every lane with `on`; all 32 lanes of the warp must call it.  Lanes
// with equal idx are summed first (checked for overflow), and their lowest lane adds.
__device__ __forceinline__ void warp_combined_add(uint64_t* arr, int32_t idx, uint64_t v, bool on, int* err) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, on ? idx : -1 - lane);
  uint64_t sum = 0;
  bool wrap = false;
#pragma unroll
  for (int t = 0; t < 32; ++t) {
    const uint64_t o = __shfl_sync(0xffffffffu, v, t);
    if ((peers >> t) & 1u) {
      wrap |= sum + o < sum;
      sum += o;
    }
  }
  if (on && lane == __ffs(peers) - 1 && sum) {
    const unsigned long long old = atomicAdd((unsigned long long*)&arr[idx], (unsigned long long)sum);
    if (wrap || old + sum < old) set_error(err, FIGARO_ERR_OVERFLOW);
  }
}

// Zeroes Phi_down and Phi_up over the P parent groups of a relation.
__global__ void k_counts_clear(uint64_t* phid, uint64_t* phiu, const int32_t* sizes) {
  const int64_t P = sizes[1];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
    phid[q] = 0ull;
    phiu[q] = 0ull;
  }
}

// Grid-stride loops below keep whole warps together (g - lane is warp-uniform) so that
// the warp-combined atomics see all 32 lanes.
__global__ void k_counts_pass1(CountParams p, int* err) {
  const int64_t G = p.sizes[0];
  const int lane = threadIdx.x & 31;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g - lane < G;
       g += (int64_t)gridDim.x * blockDim.x) {
    const bool on = g < G;
    uint64_t theta = 0;
    int32_t pg = 0;
    if (on) {
      theta = (uint64_t)(p.goff[g + 1] - p.goff[g]);
      for (int j = 0; j < p.n_child; ++j) {
        const ChildLink& c = p.ch[j];
        int32_t q = find_key(c.pkey, c.sizes[1], project_key(c, p.gkey[g]));
        c.q[g] = q;
        theta = q < 0 ? 0ull : mul_chk(theta, c.phid[q], err);
      }
      p.theta[g] = theta;
      pg = p.is_root ? 0 : p.g2p[g];
    }
    if (!p.is_root) warp_combined_add(p.phid, pg, theta, on && theta, err);
  }
}

__global__ void k_counts_pass2(CountParams p, int* err) {
  const int64_t G = p.sizes[0];
  const int lane = threadIdx.x & 31;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g - lane < G;
       g += (int64_t)gridDim.x * blockDim.x) {
    const bool on = g < G;
    uint64_t full = 0;
    if (on) {
      const uint64_t rows = (uint64_t)(p.goff[g + 1] - p.goff[g]);
      const uint64_t up = p.is_root ? 1ull : p.phiu[p.g2p[g]];
      full = mul_chk(p.theta[g], up, err);
      p.full[g] = full;
      const uint64_t circ = full / rows;
      p.phic[g] = circ;
      if (p.require_reduced && circ == 0) set_error(err, FIGARO_ERR_NOT_REDUCED);
      p.sq_phic[g] = sqrt((double)circ);
      p.hrow[g] = 1.0 / sqrt((double)rows);
    }
    for (int j = 0; j < p.n_child; ++j) {
      const ChildLink& c = p.ch[j];
      const int32_t q = on ? c.q[g] : -1;
      warp_combined_add(c.phiu, q, full, q >= 0 && full, err);
    }
  }
}

__global__ void k_counts_finalize(ChildLink c) {
  const int64_t P = c.sizes[1];
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P;
       q += (int64_t)gridDim.x * blockDim.x) {
    uint64_t d = c.phid[q];
    c.phiu[q] = d ? c.phiu[q] / d : 0ull;
    c.sq_phid[q] = sqrt((double)d);
  }
}

// Per-group factors of process_and_join_children and the weights of the generalized
// head/tail of project_away_join_attributes (Alg. 4), for an internal node:
//   s_j = scales_j[x_ij] = sqrt(Phi_down_j(x_ij)), sr = sqrt(rows_per_key(x_i))
//   fac[g][0]   = prod_j s_j                 (own columns Y_i: H(S^{x_i}) * prod_j s_j)
//   fac[g][1+j] = sr * prod_{j' != j} s_j'   (columns of the subtree of child j)
//   v = scales[x_i] = sr * prod_j s_j;  W = sum of v^2 = Theta_down over the earlier
//   groups of the same x_p (exact integer prefix); gamma = sqrt(Phi_up_i(x_p)) /
//   sqrt(W (W + v^2)) scales the generalized tail row (0 for the first group of an x_p,
//   for groups of weight 0 and for groups after only weight-0 groups);
//   hf[x_p] = 1 / sqrt(Phi_down_i(x_p)) turns the running sum into the generalized head.
__global__ void k_join_prep(CountParams p) {
  const int64_t G = p.sizes[0];
  const int nf = 1 + p.n_child;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
       g += (int64_t)gridDim.x * blockDim.x) {
    double s[kMaxChildren];
    double all = 1.0;
    for (int j = 0; j < p.n_child; ++j) {
      int32_t q = p.ch[j].q[g];
      s[j] = q >= 0 ? p.ch[j].sq_phid[q] : 0.0;
      all *= s[j];
    }
    const uint64_t rows = (uint64_t)(p.goff[g + 1] - p.goff[g]);
    const double sr = (double)rows * p.hrow[g];        // sqrt(rows) = rows / sqrt(rows)
    p.fac[g * nf] = all;
    for (int j = 0; j < p.n_child; ++j) {
      double o = sr;
      for (int jj = 0; jj < p.n_child; ++jj)
        if (jj != j) o *= s[jj];
      p.fac[g * nf + 1 + j] = o;
    }
    const double v = sr * all;
    double W = 0.0, gam = 0.0;
    if (!p.is_root) {
      const int32_t pg = p.g2p[g];
      const int32_t start = p.pgoff[pg];
      const uint64_t th = p.theta[g];
      const uint64_t before = p.theta_incl[g] - th - (start > 0 ? p.theta_incl[start - 1] : 0ull);
      W = (double)before;
      if (g > start && th && before) {
        const double Wn = (double)(before + th);
        gam = sqrt((double)p.phiu[pg]) / sqrt(W * Wn);
      }
      if (g == start) {
        const uint64_t d = p.phid[pg];
        p.hf[pg] = d ? 1.0 / sqrt((double)d) : 0.0;
      }
    }
    p.vw[g * 3 + 0] = v;    // 0 exactly when Theta_down(x_i) = 0
    p.vw[g * 3 + 1] = W;
    p.vw[g * 3 + 2] = gam;
  }
}

void counts_clear(NodeBuf& b, int64_t bound, cudaStream_t st, int64_t* launches) {
  k_counts_clear<<<grid_for(bound, 256, 152 * 4), 256, 0, st>>>(b.phid, b.phiu, b.sizes);
  ++*launches;
}

void counts_pass1(const CountParams& p, cudaStream_t st, int* err, int64_t* launches) {
  k_counts_pass1<<<grid_for(p.M, 256, 152 * 16), 256, 0, st>>>(p, err);
  ++*launches;
}

void counts_pass2(const CountParams& p, cudaStream_t st, int* err, int64_t* launches) {
  k_counts_pass2<<<grid_for(p.M, 256, 152 * 16), 256, 0, st>>>(p, err);
  ++*launches;
}

void counts_finalize_child(const ChildLink& c, int64_t bound, cudaStream_t st, int64_t* launches) {
  k_counts_finalize<<<grid_for(bound, 256, 152 * 16), 256, 0, st>>>(c);
  ++*launches;
}

void join_prep(const CountParams& p, cudaStream_t st, int64_t* launches) {
  k_join_prep<<<grid_for(p.M, 256, 152 * 16), 256, 0, st>>>(p);
  ++*launches;
}

}  // namespace fig
