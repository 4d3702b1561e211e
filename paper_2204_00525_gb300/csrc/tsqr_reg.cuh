// Register-resident warp Householder QR of TSQR tiles (n <= 32), shared by the
// translation units that instantiate it (one per element type, to build in parallel).
#pragma once

#include "kernels.cuh"

namespace fig {

__device__ __forceinline__ int64_t block_rows(const TsqrBlock& b) {
  if (b.kind == BLK_FIXED) return b.M;
  const int32_t G = b.sizes[0], P = b.sizes[1];
  switch (b.kind) {
    case BLK_TAILS: return b.fused ? b.M : b.M - G;
    case BLK_GEN: return (int64_t)G - P;
    default: return G;
  }
}

// Tiles of one level: the leaf cuts `rows` into tiles of b.tile rows; a tree level stacks
// b.fan triangles of the level below.
__device__ __forceinline__ int64_t level_tiles(const TsqrBlock& b, int64_t rows, int64_t div_in, bool leaf) {
  if (leaf) return (rows + b.tile - 1) / b.tile;
  const int64_t nt_in = (rows + div_in - 1) / div_in;
  return (nt_in + b.fan - 1) / b.fan;
}

// A tree level whose input is a single triangle only copies it (one warp).
__device__ __forceinline__ bool copy_single(const TsqrBlock& b, int64_t rows, int64_t div_in, const double* tri_in,
                                            double* tri_out) {
  if (!tri_in) return false;
  const int64_t nt_in = (rows + div_in - 1) / div_in;
  if (nt_in != 1) return false;
  if (blockIdx.x == 0 && threadIdx.x < 32)
    for (int i = threadIdx.x; i < b.n * b.n; i += 32) tri_out[i] = tri_in[i];
  return true;
}

// ------------------------------------------------------------------ Householder scalars
// Scalars of one Householder step: the reflector maps x = (alpha, a_{k+1..m-1,k}) with
// sigma = sum_{i>k} a_ik^2 to (beta, 0, ..., 0): nu = ||x||, beta = -sign(alpha) nu,
// v0 = alpha - beta (v = (v0, a_{k+1..m-1,k}) unnormalised) and
// tau = 2 / (v^T v) = 1 / (nu (nu + |alpha|)), returned as the product tau * tau2 of two
// factors: a column that holds only rounding residue (a tile with fewer independent rows
// than columns, reflected again at every later step) shrinks towards the format's smallest
// numbers, where 1 / (nu (nu + |alpha|)) overflows although 1 / nu and 1 / (nu + |alpha|)
// do not; the caller scales by both.
template <typename E>
struct HhScalars {
  __device__ static void get(E alpha, E sigma, E& beta, E& v0, E& tau, E& tau2) {
    const E nu = sqrt(fma(alpha, alpha, sigma));
    beta = alpha >= E(0) ? -nu : nu;
    v0 = alpha - beta;
    tau = E(1) / nu;
    tau2 = E(1) / (nu + fabs(alpha));
  }
};

// Double precision: FP64 instructions issue about once per 70 cycles per warp here, so the
// square root and the reciprocal are formed by Newton-Raphson iterations from float
// hardware approximations (relative error below 2^-22): y <- y (3/2 - t y^2 / 2) for
// 1 / sqrt(t) and r <- r (2 - d r) for 1 / d, two steps each (quadratic convergence; a
// measured sweep gives at most 4e-16 relative error for nu and 1e-15 for tau).  The
// float seeds are moved between the formats by exponent arithmetic on the bit patterns
// (conversions, comparisons and sign tests would each take an FP64 issue slot), which
// is exact for the normal values of the range tested first; outside it (|t| beyond
// 2^+-100) the plain operations are used, with tau in two factors.
static __device__ __noinline__ void hh_scalars_wide(double alpha, double sigma, double& nu, double& tau,
                                                    double& tau2) {
  nu = sqrt(fma(alpha, alpha, sigma));
  tau = 1.0 / nu;
  tau2 = 1.0 / (nu + fabs(alpha));
}

// float nearest below a positive normal double whose exponent is within float range
__device__ __forceinline__ float f32_of_f64_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const unsigned e = (hi >> 20) & 0x7FFu;
  const unsigned mant = ((hi & 0xFFFFFu) << 3) | (unsigned)((b >> 29) & 7ull);
  return __uint_as_float(((e - 1023u + 127u) << 23) | mant);
}

// the double equal to a positive normal float
__device__ __forceinline__ double f64_of_f32_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long e = (u >> 23) & 0xFFu;
  const unsigned long long m = u & 0x7FFFFFu;
  return __longlong_as_double((long long)(((e - 127ull + 1023ull) << 52) | (m << 29)));
}

// |x| in [2^-100, 2^100), by the exponent field
__device__ __forceinline__ bool f64_mid_range(double x) {
  const unsigned e = ((unsigned)((unsigned long long)__double_as_longlong(x) >> 52)) & 0x7FFu;
  return e >= 1023u - 100u && e < 1023u + 100u;
}

template <>
struct HhScalars<double> {
  __device__ static void get(double alpha, double sigma, double& beta, double& v0, double& tau, double& tau2) {
    const double t = fma(alpha, alpha, sigma);
    double nu;
    tau2 = 1.0;
    if (f64_mid_range(t)) {
      double y = f64_of_f32_bits(rsqrtf(f32_of_f64_bits(t)));
      const double ht = 0.5 * t;
      y = y * fma(-ht * y, y, 1.5);
      y = y * fma(-ht * y, y, 1.5);
      nu = t * y;
      const double d = nu * (nu + fabs(alpha));
      double r = f64_of_f32_bits(__frcp_rn(f32_of_f64_bits(d)));
      r = r * fma(-d, r, 2.0);
      tau = r * fma(-d, r, 2.0);
    } else {
      hh_scalars_wide(alpha, sigma, nu, tau, tau2);
    }
    beta = __double_as_longlong(alpha) >= 0 ? -nu : nu;     // sign bit: no FP64 compare
    v0 = alpha - beta;
  }
};

// x == 0 (either sign) without an FP64 compare
__device__ __forceinline__ bool f64_is_zero(double x) { return ((unsigned long long)__double_as_longlong(x) << 1) == 0ull; }
__device__ __forceinline__ bool f64_is_zero(float x) { return x == 0.0f; }

// ------------------------------------------------------------------ multi-value warp sum
// Sum NW per-lane values over the warp by recursive halving: at the level with lane
// offset o the lane keeps half of its values (the upper half if lane & o) and adds the
// partner's copy of that half.  After log2(NW) levels every lane holds one value, summed
// over NW lanes; plain butterflies finish the sum over 32 lanes.  Value index t ends in
// the lanes whose bits 4, 3, ... spell t (most significant first).  NW - 1 + 5 - log2(NW)
// additions instead of 5 NW.
template <typename E, int NW>
__device__ __forceinline__ E warp_multi_sum(E (&v)[NW], int lane) {
  int cnt = NW;
  int o = 16;
#pragma unroll
  for (int lvl = 0; (1 << lvl) < NW; ++lvl) {
    const int half = cnt >> 1;
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int t = 0; t < NW / 2; ++t) {
      if (t < half) {
        const E send = upper ? v[t] : v[t + half];
        const E keep = upper ? v[t + half] : v[t];
        v[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    cnt = half;
    o >>= 1;
  }
  E r = v[0];
  for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

template <int NW>
__device__ __forceinline__ int lane_of_value(int t) {
  int lane = 0, o = 16;
#pragma unroll
  for (int bit = NW >> 1; bit > 0; bit >>= 1, o >>= 1)
    if (t & bit) lane |= o;
  return lane;
}

// ------------------------------------------------------------------ register path (n <= 32)
// Lane l holds rows l, l + 32, ..., l + 32 (RPL - 1) of the tile, all N columns (N = the
// column count padded to the instantiated size; padded columns are zero and stay zero).
// Step k: d_j = sum_{i>k} a_ik a_ij for j = k..N-1 (d_k = sigma) in one pass and one
// multi-value reduction; then beta = -sign(alpha) ||x||, v_k = alpha - beta,
// tau = 2 / (v^T v) = 1 / (||x|| (||x|| + |alpha|)), w_j = tau (v_k a_kj + d_j) and
// a_ij -= w_j a_ik (i > k), a_kj -= w_j v_k, a_kk = beta.
template <int N>
struct RegCfg {
  static constexpr int RPL = N <= 8 ? 8 : N <= 16 ? 64 / N : 2;   // rows per lane
  static constexpr int TW = 32 * RPL;                              // rows per tile
};

template <int C>
struct Pow2 {
  static constexpr int v = C <= 1 ? 1 : C <= 2 ? 2 : C <= 4 ? 4 : C <= 8 ? 8 : C <= 16 ? 16 : 32;
};

template <int P2>
struct Log2 {
  static constexpr int v = P2 <= 1 ? 0 : P2 <= 2 ? 1 : P2 <= 4 ? 2 : P2 <= 8 ? 3 : P2 <= 16 ? 4 : 5;
};

// One step.  After the multi-value sum, the lanes holding value t (t >= 1) form
// w_t = tau (v0 a_Kt + d_t) together (one FMA and one multiply for all columns), and row
// K joins the update of the rows below with x_K = v0, so every column costs RPL FMAs.
template <typename E, int N, int RPL, int K>
__device__ __forceinline__ void reg_hh_step(E (&a)[RPL][N], int m, int lane) {
  constexpr int C = N - K;
  constexpr int P2 = Pow2<C>::v;
  E x[RPL];
#pragma unroll
  for (int r = 0; r < RPL; ++r) {
    const int i = lane + 32 * r;
    x[r] = (i > K && i < m) ? a[r][K] : E(0);
  }
  E d[P2];
#pragma unroll
  for (int t = 0; t < P2; ++t) d[t] = E(0);
#pragma unroll
  for (int r = 0; r < RPL; ++r)
#pragma unroll
    for (int t = 0; t < C; ++t) d[t] = fma(x[r], a[r][K + t], d[t]);
  const E mine = warp_multi_sum<E, P2>(d, lane);
  const E sig = __shfl_sync(0xffffffffu, mine, lane_of_value<P2>(0));
  if (f64_is_zero(sig)) return;              // uniform: column already reduced below K
  constexpr int kr = K / 32, kl = K % 32;    // lane and slot holding row K
  const E alpha = __shfl_sync(0xffffffffu, a[kr][K], kl);
  E beta, v0, tau, tau2;
  HhScalars<E>::get(alpha, sig, beta, v0, tau, tau2);
  const int my_t = lane >> (5 - Log2<P2>::v);   // the value this lane holds
  E akt = E(0);
#pragma unroll
  for (int t = 1; t < C; ++t) {
    const E v = __shfl_sync(0xffffffffu, a[kr][K + t], kl);
    if (my_t == t) akt = v;
  }
  const E w_mine = tau * fma(v0, akt, mine) * tau2;
  if (lane == kl) x[kr] = v0;
#pragma unroll
  for (int t = 1; t < C; ++t) {
    const E w = __shfl_sync(0xffffffffu, w_mine, lane_of_value<P2>(t));
#pragma unroll
    for (int r = 0; r < RPL; ++r) a[r][K + t] = fma(-w, x[r], a[r][K + t]);
  }
  if (lane == kl) a[kr][K] = beta;
}

template <typename E, int N, int RPL, int K>
struct RegQR {
  __device__ __forceinline__ static void run(E (&a)[RPL][N], int m, int lane) {
    if (K >= m) return;
    reg_hh_step<E, N, RPL, K>(a, m, lane);
    RegQR<E, N, RPL, K + 1>::run(a, m, lane);
  }
};
template <typename E, int N, int RPL>
struct RegQR<E, N, RPL, N> {
  __device__ __forceinline__ static void run(E (&)[RPL][N], int, int) {}
};

// Every level (leaf or tree) of a block with <= 32 columns runs two kernels: this one (one
// warp per tile) works only when the level has at least b.warp_min tiles; the
// block-per-tile kernel takes the levels with fewer tiles, where the latency of one
// warp's QR would dominate.  (The live tile count is known only on the device.)
// Two warps per block: with ~190 registers per thread, 64-thread blocks pack 10 warps on
// an SM where 128-thread blocks fit 8 (every FP64 instruction keeps its SM sub-partition
// busy for tens of cycles, so resident warps are what keeps the FP64 pipe fed).
constexpr int kRegThreads = 64;

template <typename E, int N>
__global__ void __launch_bounds__(kRegThreads) k_tsqr_reg(TsqrBlock b, const double* tri_in, double* tri_out,
                                                  int64_t div_in) {
  constexpr int RPL = RegCfg<N>::RPL, TW = RegCfg<N>::TW;
  const int lane = threadIdx.x & 31;
  const int n = b.n;
  const int64_t rows = block_rows(b);
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nt_in = tri_in ? (rows + div_in - 1) / div_in : 0;
  const int64_t n_tiles = level_tiles(b, rows, div_in, tri_in == nullptr);
  if (n_tiles < b.warp_min) return;                   // the block-per-tile kernel takes it
  for (int64_t t = gw; t < n_tiles; t += nw) {
    E a[RPL][N];
    int m;
    if (!tri_in) {
      const int64_t r0 = t * TW;
      m = (int)((rows - r0) < TW ? (rows - r0) : TW);
      // uniform branch on the source type: no conversion of the unused source is issued
      if (b.ptr32) {
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          const int i = lane + 32 * r;
#pragma unroll
          for (int c = 0; c < N; ++c) a[r][c] = (i < m && c < n) ? (E)b.ptr32[(int64_t)c * b.ld + r0 + i] : E(0);
        }
      } else {
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          const int i = lane + 32 * r;
#pragma unroll
          for (int c = 0; c < N; ++c) a[r][c] = (i < m && c < n) ? (E)b.ptr[(int64_t)c * b.ld + r0 + i] : E(0);
        }
      }
    } else {
      const int64_t first = t * b.fan;
      const int cnt = (int)((nt_in - first) < b.fan ? (nt_in - first) : b.fan);
      m = cnt * n;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        const int i = lane + 32 * r;
        const int f = i / n, rr = i - f * n;
#pragma unroll
        for (int c = 0; c < N; ++c)
          a[r][c] = (i < m && c < n) ? (E)tri_in[(first + f) * n * n + (int64_t)c * n + rr] : E(0);
      }
    }
    RegQR<E, N, RPL, 0>::run(a, m, lane);
    double* tri = tri_out + t * n * n;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      const int i = lane + 32 * r;
      if (i < n) {
#pragma unroll
        for (int c = 0; c < N; ++c)
          if (c < n) tri[(int64_t)c * n + i] = (c >= i && i < m) ? (double)a[r][c] : 0.0;
      }
    }
  }
}

template <typename E, int N>
void launch_reg(const TsqrBlock& b, const double* tri_in, double* tri_out, int64_t div_in, int64_t tiles,
                cudaStream_t st) {
  // persistent: as many blocks as are resident at once (registers decide), so that
  // no second, partial wave of blocks runs at low occupancy
  static int resident = 0;
  if (resident == 0) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tsqr_reg<E, N>, kRegThreads, 0);
    resident = (per_sm > 0 && sms > 0) ? per_sm * sms : 152 * 4;
  }
  constexpr int wpb = kRegThreads / 32;
  int64_t blocks = (tiles + wpb - 1) / wpb;
  if (blocks > resident) blocks = resident;
  if (blocks < 1) blocks = 1;
  k_tsqr_reg<E, N><<<(unsigned)blocks, kRegThreads, 0, st>>>(b, tri_in, tri_out, div_in);
}

// Dispatch on the padded column count b.nreg; defined in tsqr_reg_f64.cu / tsqr_reg_f32.cu.
template <typename E>
void launch_reg_n(const TsqrBlock& b, const double* tri_in, double* tri_out, int64_t div_in, int64_t tiles,
                  cudaStream_t st);

template <>
void launch_reg_n<double>(const TsqrBlock&, const double*, double*, int64_t, int64_t, cudaStream_t);
template <>
void launch_reg_n<float>(const TsqrBlock&, const double*, double*, int64_t, int64_t, cudaStream_t);

template <typename E>
void launch_reg_dispatch(const TsqrBlock& b, const double* tri_in, double* tri_out, int64_t div_in,
                         int64_t tiles, cudaStream_t st) {
  switch (b.nreg) {
    case 2: launch_reg<E, 2>(b, tri_in, tri_out, div_in, tiles, st); break;
    case 4: launch_reg<E, 4>(b, tri_in, tri_out, div_in, tiles, st); break;
    case 6: launch_reg<E, 6>(b, tri_in, tri_out, div_in, tiles, st); break;
    case 8: launch_reg<E, 8>(b, tri_in, tri_out, div_in, tiles, st); break;
    case 10: launch_reg<E, 10>(b, tri_in, tri_out, div_in, tiles, st); break;
    case 12: launch_reg<E, 12>(b, tri_in, tri_out, div_in, tiles, st); break;
    case 14: launch_reg<E, 14>(b, tri_in, tri_out, div_in, tiles, st); break;
    case 16: launch_reg<E, 16>(b, tri_in, tri_out, div_in, tiles, st); break;
    case 20: launch_reg<E, 20>(b, tri_in, tri_out, div_in, tiles, st); break;
    case 24: launch_reg<E, 24>(b, tri_in, tri_out, div_in, tiles, st); break;
    case 28: launch_reg<E, 28>(b, tri_in, tri_out, div_in, tiles, st); break;
    default: launch_reg<E, 32>(b, tri_in, tri_out, div_in, tiles, st); break;
  }
}

}  // namespace fig
