// SVD of R (§8.2): sigma(A) = sigma(R) and V(A) = V(R); PCA (§8.3) takes the leading
// columns of V.  R is N x N, so a one-sided (Hestenes) Jacobi SVD in FP64 in one
// thread block suffices: columns of W = R are rotated pairwise until orthogonal;
// sigma_j = ||W_j|| and V accumulates the rotations.  The paper used LAPACK's
// divide and conquer on the CPU; one-sided Jacobi is chosen here for its high relative
// accuracy and because every pair of a round-robin round can be rotated in parallel.
#include <cooperative_groups.h>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace fig {

constexpr int kSvdThreads = 1024;   // 32 warps: one column pair per warp and round up to N = 64
constexpr int kSvdMaxSweeps = kSvdDefaultSweeps;
constexpr int kSvdMaxPairs = 512;      // N <= 1024 (the library's column limit)

// sigma_j = ||W_j|| (into sig, N doubles of shared memory), sigma descending with ties by
// index, every column of V signed so that its largest entry is positive; with tk.k > 0 also
// the first k columns (PCA components, row-major N x k) and sigma^2.  One thread block.
// With CG, W and V are read from L2 (__ldcg): other thread blocks of a cluster wrote them.
template <bool CG = false>
__device__ void jacobi_finish(const JacobiTask& tk, const double* W, const double* V, double* sig) {
  auto ld = [](const double* a) { return CG ? __ldcg(a) : *a; };
  const int N = tk.N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < N; j += nw) {
    double s2 = 0.0;
    for (int i = lane; i < N; i += 32) {
      const double w = ld(W + (int64_t)j * N + i);
      s2 = fma(w, w, s2);
    }
    s2 = warp_sum(s2);
    if (lane == 0) sig[j] = sqrt(s2);
  }
  __syncthreads();
  // descending order, ties by index; every column signed so its largest entry is positive;
  // with tk.k > 0 also the first k columns (PCA components, row-major N x k) and sigma^2
  for (int j = warp; j < N; j += nw) {
    const double sj = sig[j];
    int rank = 0;
    for (int k = lane; k < N; k += 32) rank += (sig[k] > sj || (sig[k] == sj && k < j)) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const double* vj = V + (int64_t)j * N;
    double best = -1.0;
    int arg = 0;
    for (int i = lane; i < N; i += 32) {
      const double a = fabs(ld(vj + i));
      if (a > best) { best = a; arg = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
      if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
    }
    const double sgn = ld(vj + arg) < 0.0 ? -1.0 : 1.0;
    if (lane == 0) tk.sigma[rank] = sj;
    for (int i = lane; i < N; i += 32) tk.Vout[(int64_t)i * N + rank] = sgn * ld(vj + i);
    if (rank < tk.k) {
      if (lane == 0) tk.eig[rank] = sj * sj;
      for (int i = lane; i < N; i += 32) tk.comp[(int64_t)i * tk.k + rank] = sgn * ld(vj + i);
    }
  }
}

// One SVD in one thread block: W = R (column j at W + j N), V = I; round-robin rounds of
// disjoint column pairs until a sweep rotates no pair.  The block issues one FP64
// instruction per warp every ~16 cycles at best, so a round is split into three phases
// that keep the FP64 instruction count low: (1) one warp per pair forms w_p . w_q (the
// squared column norms are carried: recomputed at every sweep start, updated exactly by
// each rotation, |w_p'|^2 = |w_p|^2 - t g and |w_q'|^2 = |w_q|^2 + t g); (2) one thread per
// pair forms the rotation (zeta = (|w_q|^2 - |w_p|^2) / 2g, t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t) instead of every lane of a warp;
// (3) one warp per pair applies it to W and V.
__device__ void jacobi_run(const JacobiTask& tk, double* smem, bool use_smem) {
  __shared__ int rotations;
  __shared__ double pg[kSvdMaxPairs];        // w_p . w_q of each pair of the round
  __shared__ double2 pcs[kSvdMaxPairs];      // its rotation (c, s); c = 2 marks "no rotation"
  const int N = tk.N;
  double* W = use_smem ? smem : tk.W;
  double* V = use_smem ? W + (int64_t)N * N : tk.V;
  double* nrm = smem + (use_smem ? 2 * (int64_t)N * N : 0);   // squared column norms
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int idx = tid; idx < N * N; idx += blockDim.x) {
    const int j = idx / N, i = idx - j * N;
    W[idx] = tk.R[(int64_t)i * tk.ldr + j];
    V[idx] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  const int npad = N + (N & 1);
  const int npairs = npad / 2;
  // pair pi of round r: positions pi and npad-1-pi of the round-robin (circle) schedule,
  // position 0 holding column 0 and position k >= 1 column 1 + (k - 1 + r) mod (npad - 1)
  auto pair_of = [&](int pi, int r, int& p, int& q) {
    const int pb = npad - 1 - pi;
    const int a = pi == 0 ? 0 : 1 + (pi - 1 + r) % (npad - 1);
    const int b = 1 + (pb - 1 + r) % (npad - 1);
    p = a < b ? a : b;
    q = a < b ? b : a;
  };
  int sweep = 0;
  for (; sweep < tk.max_sweeps; ++sweep) {
    for (int j = warp; j < N; j += nw) {
      double s2 = 0.0;
      for (int i = lane; i < N; i += 32) s2 = fma(W[(int64_t)j * N + i], W[(int64_t)j * N + i], s2);
      s2 = warp_sum(s2);
      if (lane == 0) nrm[j] = s2;
    }
    if (tid == 0) rotations = 0;
    __syncthreads();
    for (int r = 0; r < npad - 1; ++r) {
      for (int pi = warp; pi < npairs; pi += nw) {
        int p, q;
        pair_of(pi, r, p, q);
        if (q >= N) continue;
        const double* wp = W + (int64_t)p * N;
        const double* wq = W + (int64_t)q * N;
        double ga = 0.0;
        for (int i = lane; i < N; i += 32) ga = fma(wp[i], wq[i], ga);
        ga = warp_sum(ga);
        if (lane == 0) pg[pi] = ga;
      }
      __syncthreads();
      for (int pi = tid; pi < npairs; pi += blockDim.x) {
        int p, q;
        pair_of(pi, r, p, q);
        double2 cs = make_double2(2.0, 0.0);
        if (q < N) {
          const double ga = pg[pi], al = nrm[p], be = nrm[q];
          if (fabs(ga) > 1e-15 * sqrt(al * be) && fabs(ga) > 1e-300) {
            const double zeta = (be - al) / (2.0 * ga);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + t * t);
            cs = make_double2(c, c * t);
            nrm[p] = al - t * ga;
            nrm[q] = be + t * ga;
            atomicAdd(&rotations, 1);
          }
        }
        pcs[pi] = cs;
      }
      __syncthreads();
      for (int pi = warp; pi < npairs; pi += nw) {
        const double2 cs = pcs[pi];
        if (cs.x > 1.5) continue;
        int p, q;
        pair_of(pi, r, p, q);
        const double c = cs.x, s = cs.y;
        double* wp = W + (int64_t)p * N;
        double* wq = W + (int64_t)q * N;
        double* vp = V + (int64_t)p * N;
        double* vq = V + (int64_t)q * N;
        for (int i = lane; i < N; i += 32) {
          const double x = wp[i], y = wq[i];
          wp[i] = c * x - s * y;
          wq[i] = s * x + c * y;
          const double u = vp[i], w = vq[i];
          vp[i] = c * u - s * w;
          vq[i] = s * u + c * w;
        }
      }
      __syncthreads();
    }
    const int rot = rotations;
    __syncthreads();
    if (rot == 0) break;
  }
  if (sweep == tk.max_sweeps && tid == 0) set_error(tk.err, FIGARO_ERR_TIMEOUT);
  jacobi_finish(tk, W, V, smem + (use_smem ? 2 * (int64_t)N * N : 0));
}

__global__ void __launch_bounds__(kSvdThreads) k_jacobi(JacobiTask tk, int use_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  jacobi_run(tk, reinterpret_cast<double*>(smem_raw), use_smem != 0);
}

// Many SVDs in one launch, one thread block per task; a task uses the shared buffer for W
// and V when they fit in smem_bytes.
__global__ void __launch_bounds__(kSvdThreads) k_jacobi_batch(const JacobiTask* tasks, size_t smem_bytes) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const JacobiTask tk = tasks[blockIdx.x];
  jacobi_run(tk, reinterpret_cast<double*>(smem_raw), jacobi_smem(tk.N) <= smem_bytes);
}

__global__ void k_square(const double* s, double* out, int k) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) out[i] = s[i] * s[i];
}

// One SVD on a cluster of kSvdCluster thread blocks (wide R: W and V do not fit in one
// block's shared memory and live in L2, where one SM's FP64 rate would set the pace): the
// same three-phase rounds, with the pairs, rotations and column norms spread over the
// cluster's warps and threads, W, V and the round's scratch in global memory read through
// L2 (__ldcg), and a cluster barrier (release/acquire) between the phases.  aux holds the
// round's (c, s) and dot products, the column norms and two rotation counters.
constexpr int kSvdCluster = 8;

__global__ void __cluster_dims__(kSvdCluster, 1, 1) __launch_bounds__(kSvdThreads)
    k_jacobi_cluster(JacobiTask tk, double* aux) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cluster = cg::this_cluster();
  const int N = tk.N;
  const int npad = N + (N & 1), npairs = npad / 2;
  double2* pcs = reinterpret_cast<double2*>(aux);            // [kSvdMaxPairs]
  double* pg = aux + 2 * kSvdMaxPairs;                       // [kSvdMaxPairs]
  double* nrm = aux + 3 * kSvdMaxPairs;                      // [N]
  int* rotc = reinterpret_cast<int*>(aux + 3 * kSvdMaxPairs + N);   // two counters
  double* W = tk.W;
  double* V = tk.V;
  const int lane = threadIdx.x & 31;
  const int gt = (int)cluster.block_rank() * blockDim.x + threadIdx.x;
  const int gthreads = kSvdCluster * blockDim.x;
  const int gw = gt >> 5, nwg = gthreads >> 5;
  for (int idx = gt; idx < N * N; idx += gthreads) {
    const int j = idx / N, i = idx - j * N;
    W[idx] = tk.R[(int64_t)i * tk.ldr + j];
    V[idx] = i == j ? 1.0 : 0.0;
  }
  if (gt == 0) rotc[0] = rotc[1] = 0;
  cluster.sync();
  auto pair_of = [&](int pi, int r, int& p, int& q) {
    const int pb = npad - 1 - pi;
    const int a = pi == 0 ? 0 : 1 + (pi - 1 + r) % (npad - 1);
    const int b = 1 + (pb - 1 + r) % (npad - 1);
    p = a < b ? a : b;
    q = a < b ? b : a;
  };
  int sweep = 0;
  for (; sweep < tk.max_sweeps; ++sweep) {
    for (int j = gw; j < N; j += nwg) {
      double s2 = 0.0;
      for (int i = lane; i < N; i += 32) {
        const double w = __ldcg(W + (int64_t)j * N + i);
        s2 = fma(w, w, s2);
      }
      s2 = warp_sum(s2);
      if (lane == 0) nrm[j] = s2;
    }
    cluster.sync();
    // the next sweep's counter: every thread block read it (at the end of the previous
    // sweep) before it reached the barrier above; it is next counted after the next
    // sweep's first barrier.  So every block takes the same break below.
    if (gt == 0) rotc[(sweep + 1) & 1] = 0;
    for (int r = 0; r < npad - 1; ++r) {
      for (int pi = gw; pi < npairs; pi += nwg) {
        int p, q;
        pair_of(pi, r, p, q);
        if (q >= N) continue;
        const double* wp = W + (int64_t)p * N;
        const double* wq = W + (int64_t)q * N;
        double ga = 0.0;
        for (int i = lane; i < N; i += 32) ga = fma(__ldcg(wp + i), __ldcg(wq + i), ga);
        ga = warp_sum(ga);
        if (lane == 0) pg[pi] = ga;
      }
      cluster.sync();
      for (int pi = gt; pi < npairs; pi += gthreads) {
        int p, q;
        pair_of(pi, r, p, q);
        double2 cs = make_double2(2.0, 0.0);
        if (q < N) {
          const double ga = __ldcg(pg + pi), al = __ldcg(nrm + p), be = __ldcg(nrm + q);
          if (fabs(ga) > 1e-15 * sqrt(al * be) && fabs(ga) > 1e-300) {
            const double zeta = (be - al) / (2.0 * ga);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + t * t);
            cs = make_double2(c, c * t);
            nrm[p] = al - t * ga;
            nrm[q] = be + t * ga;
            atomicAdd(rotc + (sweep & 1), 1);
          }
        }
        pcs[pi] = cs;
      }
      cluster.sync();
      for (int pi = gw; pi < npairs; pi += nwg) {
        const double2 cs = __ldcg(pcs + pi);
        if (cs.x > 1.5) continue;
        int p, q;
        pair_of(pi, r, p, q);
        const double c = cs.x, s = cs.y;
        double* wp = W + (int64_t)p * N;
        double* wq = W + (int64_t)q * N;
        double* vp = V + (int64_t)p * N;
        double* vq = V + (int64_t)q * N;
        for (int i = lane; i < N; i += 32) {
          const double x = __ldcg(wp + i), y = __ldcg(wq + i);
          wp[i] = c * x - s * y;
          wq[i] = s * x + c * y;
          const double u = __ldcg(vp + i), w = __ldcg(vq + i);
          vp[i] = c * u - s * w;
          vq[i] = s * u + c * w;
        }
      }
      cluster.sync();
    }
    const int rot = __ldcg(rotc + (sweep & 1));
    if (rot == 0) break;
  }
  if (sweep == tk.max_sweeps && gt == 0) set_error(tk.err, FIGARO_ERR_TIMEOUT);
  if (cluster.block_rank() == 0) jacobi_finish<true>(tk, W, V, reinterpret_cast<double*>(smem_raw));
}

cudaError_t svd_set_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, kJacobiSmemCap);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_jacobi_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, kJacobiSmemCap);
  return e;
}

void jacobi_svd(const double* R, int64_t ldr, int N, double* W, double* V, double* sigma, double* Vout,
                int* err, cudaStream_t st, int64_t* launches, int max_sweeps, double* aux) {
  JacobiTask tk{R, ldr, N, W, V, sigma, Vout, err, max_sweeps > 0 ? max_sweeps : kSvdMaxSweeps, nullptr, nullptr, 0};
  size_t smem = jacobi_smem(N);
  const int use_smem = smem <= kJacobiSmemCap;
  if (!use_smem && aux) {                      // wide R: one cluster of thread blocks
    k_jacobi_cluster<<<kSvdCluster, kSvdThreads, (size_t)N * sizeof(double), st>>>(tk, aux);
    ++*launches;
    return;
  }
  if (!use_smem) smem = (size_t)N * sizeof(double);
  k_jacobi<<<1, kSvdThreads, smem, st>>>(tk, use_smem);
  ++*launches;
}

void jacobi_svd_batch(const JacobiTask* tasks_dev, int n, int max_n, cudaStream_t st, int64_t* launches) {
  if (n <= 0) return;
  size_t smem = jacobi_smem(max_n);
  if (smem > kJacobiSmemCap) smem = kJacobiSmemCap;
  k_jacobi_batch<<<n, kSvdThreads, smem, st>>>(tasks_dev, smem);
  ++*launches;
}

// ------------------------------------------------------------------ centred PCA
// Column sums of the join matrix, relation by relation: sum over the tuples t of c(t) y_t
// (c(t) = Phi_circ of t's group, Fig. 4) = sum over the groups g of Phi_circ(g) S(g), with
// the group sums S(g) = head(g) sqrt(rows).  One block per column, threads over groups
// in a fixed order (deterministic).
__global__ void __launch_bounds__(1024) k_join_colsum(const double* heads, int64_t ldh, const int32_t* goff,
                                                      const double* hrow, const uint64_t* phic, const int32_t* sizes,
                                                      double* out) {
  __shared__ double red[33];
  const int a = blockIdx.x;
  const int64_t G = sizes[0];
  double s = 0.0;
  for (int64_t g = threadIdx.x; g < G; g += blockDim.x) {
    const double rows = (double)(goff[g + 1] - goff[g]);
    s = fma((double)phic[g], heads[(int64_t)a * ldh + g] * rows * hrow[g], s);
  }
  s = block_sum<double>(s, red);
  if (threadIdx.x == 0) out[a] = s;
}

// |J| = sum over the root's groups of full_join_size (exact in uint64).
__global__ void k_join_size(const uint64_t* full, const int32_t* sizes, unsigned long long* out) {
  __shared__ unsigned long long red[32];
  const int64_t G = sizes[0];
  unsigned long long s = 0;
  for (int64_t g = threadIdx.x; g < G; g += blockDim.x) s += full[g];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

// C = R^T R - colsum colsum^T / |J| (N x N, row-major), the scatter matrix of the centred
// join rows.
__global__ void k_center_gram(const double* R, int N, const double* colsum, const unsigned long long* join_size,
                              double* C) {
  const double inv = *join_size ? 1.0 / (double)*join_size : 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)N * N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const int kmax = i < j ? i : j;
    double s = 0.0;
    for (int k = 0; k <= kmax; ++k) s = fma(R[(int64_t)k * N + i], R[(int64_t)k * N + j], s);
    C[idx] = s - colsum[i] * colsum[j] * inv;
  }
}

void join_colsum(const double* heads, int64_t ldh, const int32_t* goff, const double* hrow, const uint64_t* phic,
                 const int32_t* sizes, int n, double* out, cudaStream_t st, int64_t* launches) {
  if (n <= 0) return;
  k_join_colsum<<<n, 1024, 0, st>>>(heads, ldh, goff, hrow, phic, sizes, out);
  ++*launches;
}

void join_size(const uint64_t* full, const int32_t* sizes, unsigned long long* out, cudaStream_t st,
               int64_t* launches) {
  k_join_size<<<1, 1024, 0, st>>>(full, sizes, out);
  ++*launches;
}

void center_gram(const double* R, int N, const double* colsum, const unsigned long long* join_size, double* C,
                 cudaStream_t st, int64_t* launches) {
  k_center_gram<<<grid_for((int64_t)N * N, 256, 152), 256, 0, st>>>(R, N, colsum, join_size, C);
  ++*launches;
}

void square_values(const double* s, double* out, int k, cudaStream_t st, int64_t* launches) {
  k_square<<<1, 256, 0, st>>>(s, out, k);
  ++*launches;
}

}  // namespace fig

// ------------------------------------------------------------------ allocation-free variant
// figaro_svd_from_r_static: the same Jacobi kernel, with its W and V work arrays in one
// fixed device array owned by this library instead of memory the caller or a plan
// allocates.  Some callers cannot allocate device memory at the moment they need an SVD
// (a process whose device memory is fully reserved by its own pool, a latency-critical
// loop where an allocation's implicit synchronisation is not allowed); they still pass
// R, sigma and V themselves.

namespace fig {

constexpr int kStaticSvdMaxN = 256;
// W (N x N) + V (N x N) for N <= 256, followed by one error word: 1 MiB + 256 bytes,
// held on every device that loads this library until the process exits.
static __device__ __align__(256) double g_svd_static_scratch[2 * kStaticSvdMaxN * kStaticSvdMaxN + 32];

// Device address of the static array on the current device.  Host code only holds a
// host-side stand-in for the symbol, which must not be passed to a kernel.  The address
// is looked up on every call (a cheap host query; the call waits for its stream anyway),
// so it stays valid if the module is loaded again, e.g. after cudaDeviceReset.
static int static_scratch(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_svd_static_scratch);
  if (e != cudaSuccess || !p)
    return record_error(FIGARO_ERR_CUDA, "figaro_svd_from_r_static: cudaGetSymbolAddress failed");
  *out = static_cast<double*>(p);
  return FIGARO_OK;
}

}  // namespace fig

extern "C" int figaro_svd_from_r_static(const double* R, int64_t ldr, int32_t n, double* sigma, double* V,
                                        void* stream) {
  using namespace fig;
  clear_error();
  if (!R || !sigma || !V || n < 1 || ldr < n)
    return record_error(FIGARO_ERR_INVALID_ARG, "figaro_svd_from_r_static: null pointer, n < 1 or ldr < n");
  if (n > kStaticSvdMaxN)
    return record_error(FIGARO_ERR_UNSUPPORTED, "figaro_svd_from_r_static: n above 256");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The call ends by waiting for its stream, which a stream under capture does not allow
  // (the wait would invalidate the caller's capture): refuse before enqueueing anything.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess)
    return record_error(FIGARO_ERR_CUDA, "figaro_svd_from_r_static: cudaStreamIsCapturing failed");
  if (cap != cudaStreamCaptureStatusNone)
    return record_error(FIGARO_ERR_UNSUPPORTED, "figaro_svd_from_r_static: stream is being captured");
  double* base = nullptr;
  int rc = static_scratch(&base);
  if (rc != FIGARO_OK) return rc;
  double* W = base;
  double* Vw = base + (int64_t)n * n;
  int* err = reinterpret_cast<int*>(base + 2 * kStaticSvdMaxN * kStaticSvdMaxN);
  // an error left by an earlier, unrelated launch on this thread is not this call's
  (void)cudaGetLastError();
  // the error word keeps the previous call's value: clear it first
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess)
    return record_error(FIGARO_ERR_CUDA, "figaro_svd_from_r_static: clearing the error word failed");
  const size_t smem = (size_t)n * sizeof(double);
  const JacobiTask tk{R, ldr, n, W, Vw, sigma, V, err, kSvdMaxSweeps, nullptr, nullptr, 0};
  k_jacobi<<<1, kSvdThreads, smem, st>>>(tk, 0);
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess)
    return record_error(FIGARO_ERR_CUDA, cudaGetErrorString(le));
  int host_err = 0;
  if (cudaMemcpyAsync(&host_err, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return record_error(FIGARO_ERR_CUDA, "figaro_svd_from_r_static: reading the error word failed");
  le = cudaStreamSynchronize(st);
  if (le != cudaSuccess) return record_error(FIGARO_ERR_CUDA, cudaGetErrorString(le));
  if (host_err != FIGARO_OK)
    return record_error(host_err, "figaro_svd_from_r_static: the Jacobi kernel reported an error");
  return FIGARO_OK;
}
