// Float TSQR leaf of wide blocks on the 5th-generation tensor cores (mixed path, §7
// post-processing).  A thread block keeps the n x n triangle T of the rows it has folded
// and brings every next chunk X of 128 rows into it by Householder QR of [T; X], panel by
// panel of 16 columns (the fold of the float32 path; 33 <= n <= 112):
//
//   panel    the 16 reflectors of columns p0 .. p0+15 from [T rows p0..; X panel], held in
//            registers by four warps (thread = row of X), one named barrier per column;
//            reflector q maps (T_qq, x_q) to (beta, 0); in normalised form its vector is
//            (1, x_q / v0_q) and tau' = tau v0_q^2 (as in the FP64 fold);
//   P        = X^T X_v on the tensor cores: 128 x 16 x 128 (tcgen05.mma M = 128 over the
//            columns of X, N = 16 panel columns, K = 128 rows), accumulator in TMEM.  Its
//            panel rows are the Gram matrix x_r^T x_q of the reflectors, its trailing rows
//            X_trail^T X_v;
//   Tw       the compact-WY factor, H_0 ... H_15 = I - Y Tw Y^T, column by column from
//            tau' and the Gram matrix;
//   W'       = Tw^T (T[panel rows, trailing] + diag(1/v0) P_trail^T); T's panel rows -= W';
//   update   X_trail -= X_v diag(1/v0) W' on the tensor cores: 128 x c x 16, accumulator in
//            TMEM, subtracted from X by the epilogue.
//
// Operands are bf16 triples: every float x is held as x0 + x1 + x2 (each rounded to
// bfloat16, the remainders exact in float), and each product keeps the six terms of order
// <= 2 (a0 b0, a0 b1, a1 b0, a1 b1, a0 b2, a2 b0), summed in the f32 accumulator: the
// dropped terms are below 2^-23 of the product, float-level accuracy.  X itself is stored
// only as its three bf16 parts, in the tensor core's K-major layout (columns of X as rows of
// the operand, rows of X along K); the panel and the epilogue read x = x0 + x1 + x2.
//
// Every wait on the tensor core is bounded: on expiry the kernel sets FIGARO_ERR_TIMEOUT,
// waits once more (bounded) for the operations in flight, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "tc.cuh"
#include "tsqr_reg.cuh"

namespace fig {

constexpr int kTcThreads = 256;              // 8 warps; warps 0-3 factor the panels
constexpr int kTcRows = 128;                 // rows per chunk (M of the update product)
constexpr int kTcWin = 128;                  // columns of X held (M of the P product)
constexpr int kTcMaxN = 112;
constexpr int kTcB = 16;                     // panel width
constexpr uint32_t kXLbo = 144;              // X: K-adjacent core matrices (padded: no bank conflicts)
constexpr uint32_t kXSbo = 16 * kXLbo;       // X: 8-column groups (128 rows = 16 core matrices)
constexpr uint32_t kXSplit = 16 * kXSbo;     // one bf16 part of X, 128 columns: 36,864 B
constexpr uint32_t kVLbo = 128, kVSbo = 256; // X_v (128 rows x 16) and W'' (<= 128 columns x 16)
constexpr uint32_t kVSplit = 16 * kVSbo;     // 4,096 B
constexpr int kPsLd = 17;
constexpr uint32_t kTmemCols = 128;          // P at columns 0-15, the update at 16 ..
constexpr int kTcWaitIters = 1 << 22;

// byte offsets of the shared-memory regions
constexpr uint32_t kOffX = 0;
constexpr uint32_t kOffA = kOffX + 3 * kXSplit;
constexpr uint32_t kOffB = kOffA + 3 * kVSplit;
constexpr uint32_t kOffPs = kOffB + 3 * kVSplit;
constexpr uint32_t kOffRed = kOffPs + kTcWin * kPsLd * 4;
constexpr uint32_t kOffTau = kOffRed + 2 * 4 * 16 * 4;
constexpr uint32_t kOffRv = kOffTau + 16 * 4;
constexpr uint32_t kOffTw = kOffRv + 16 * 4;
constexpr uint32_t kOffMisc = kOffTw + 16 * 16 * 4;   // mbarrier (8 B), TMEM slot, abort flag
constexpr uint32_t kOffT = kOffMisc + 64;

size_t fold_tc_smem(int n) { return (size_t)kOffT + (size_t)n * n * sizeof(float); }
bool fold_tc_fits(int n) { return n > 32 && n <= kTcMaxN && fold_tc_smem(n) <= 200 * 1024; }

__device__ __forceinline__ uint32_t x_off(int col, int row) {
  return (uint32_t)(col & 7) * 16u + (uint32_t)(row & 7) * 2u + (uint32_t)(row >> 3) * kXLbo + (uint32_t)(col >> 3) * kXSbo;
}
__device__ __forceinline__ uint32_t v_off(int r, int q) {     // (row or column r, panel index q)
  return (uint32_t)(r & 7) * 16u + (uint32_t)(q & 7) * 2u + (uint32_t)(q >> 3) * kVLbo + (uint32_t)(r >> 3) * kVSbo;
}

__device__ __forceinline__ float bf(const unsigned char* base, uint32_t off) {
  return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(base + off));
}
__device__ __forceinline__ void put_bf(unsigned char* base, uint32_t off, __nv_bfloat16 v) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = v;
}

// x = x0 + x1 + x2, each part rounded to bfloat16 (the remainders are exact in float)
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

__device__ __forceinline__ float x_get(const unsigned char* sm, int col, int row) {
  const uint32_t o = kOffX + x_off(col, row);
  return bf(sm, o) + (bf(sm, o + kXSplit) + bf(sm, o + 2 * kXSplit));
}
__device__ __forceinline__ void x_put(unsigned char* sm, int col, int row, float x) {
  __nv_bfloat16 a, b, c;
  split3(x, a, b, c);
  const uint32_t o = kOffX + x_off(col, row);
  put_bf(sm, o, a);
  put_bf(sm, o + kXSplit, b);
  put_bf(sm, o + 2 * kXSplit, c);
}

// Two consecutive rows (2r, 2r + 1) of one column share a 32-bit word of every part.
__device__ __forceinline__ float2 x_get2(const unsigned char* sm, int col, int row_even) {
  const uint32_t o = kOffX + x_off(col, row_even);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(sm + o));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(sm + o + kXSplit));
  const float2 c = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(sm + o + 2 * kXSplit));
  return make_float2(a.x + (b.x + c.x), a.y + (b.y + c.y));
}
__device__ __forceinline__ void split3x2(float2 x, __nv_bfloat162& a, __nv_bfloat162& b, __nv_bfloat162& c) {
  a = __float22bfloat162_rn(x);
  const float2 fa = __bfloat1622float2(a);
  const float2 r1 = make_float2(x.x - fa.x, x.y - fa.y);
  b = __float22bfloat162_rn(r1);
  const float2 fb = __bfloat1622float2(b);
  c = __float22bfloat162_rn(make_float2(r1.x - fb.x, r1.y - fb.y));
}
__device__ __forceinline__ void x_put2(unsigned char* sm, int col, int row_even, float2 x) {
  __nv_bfloat162 a, b, c;
  split3x2(x, a, b, c);
  const uint32_t o = kOffX + x_off(col, row_even);
  *reinterpret_cast<__nv_bfloat162*>(sm + o) = a;
  *reinterpret_cast<__nv_bfloat162*>(sm + o + kXSplit) = b;
  *reinterpret_cast<__nv_bfloat162*>(sm + o + 2 * kXSplit) = c;
}

// Sixteen consecutive K values of one operand row (3 parts, 16-byte stores): the row's K
// values 0-7 are 16 contiguous bytes, 8-15 the next core matrix (kVLbo further).
__device__ __forceinline__ void put_row16(unsigned char* base, uint32_t off, const float (&w)[16]) {
  uint32_t p[3][8];
#pragma unroll
  for (int q = 0; q < 16; q += 2) {
    __nv_bfloat162 a, b, c;
    split3x2(make_float2(w[q], w[q + 1]), a, b, c);
    p[0][q / 2] = *reinterpret_cast<uint32_t*>(&a);
    p[1][q / 2] = *reinterpret_cast<uint32_t*>(&b);
    p[2][q / 2] = *reinterpret_cast<uint32_t*>(&c);
  }
#pragma unroll
  for (int part = 0; part < 3; ++part) {
    *reinterpret_cast<uint4*>(base + off + part * kVSplit) = make_uint4(p[part][0], p[part][1], p[part][2], p[part][3]);
    *reinterpret_cast<uint4*>(base + off + part * kVSplit + kVLbo) =
        make_uint4(p[part][4], p[part][5], p[part][6], p[part][7]);
  }
}

// Sum over the warp of sixteen values per lane: lane l (l even) returns the total of value
// ((l >> 4) & 1) * 8 + ((l >> 3) & 1) * 4 + ((l >> 2) & 1) * 2 + ((l >> 1) & 1) (recursive
// halving: each exchange sends the half the partner keeps).
__device__ __forceinline__ float warp_sum16(const float (&v)[16], int lane) {
  float a8[8], a4[4], a2[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4, h2 = lane & 2;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const float mine = h16 ? v[8 + m] : v[m], other = h16 ? v[m] : v[8 + m];
    a8[m] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const float mine = h8 ? a8[4 + m] : a8[m], other = h8 ? a8[m] : a8[4 + m];
    a4[m] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
  }
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const float mine = h4 ? a4[2 + m] : a4[m], other = h4 ? a4[m] : a4[2 + m];
    a2[m] = mine + __shfl_xor_sync(0xffffffffu, other, 4);
  }
  const float mine = h2 ? a2[1] : a2[0], other = h2 ? a2[0] : a2[1];
  float a1 = mine + __shfl_xor_sync(0xffffffffu, other, 2);
  a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
  return a1;
}
__device__ __forceinline__ int sum16_index(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

__device__ __forceinline__ void bar_panel() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// The panel: reflectors of columns p0 .. p0+b-1 (b <= 16) of [T; X] by warps 0-3, thread t
// holding row t of the panel in registers.  Per column k: the column's sum of squares and
// its dot products with the later panel columns are summed over the warps through shared
// memory (double-buffered, one named barrier); lane j of every warp sums value j and forms
// w'_j, which the warp exchanges by shuffles; lane j of warp 0 writes entry j of row k of T
// one step later, once every thread has read it.
// The reflector columns are stored back into X and, row-major, as the update's A operand.
__device__ void tc_panel(unsigned char* sm, float* T, int n, int p0, int b) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  float* red = reinterpret_cast<float*>(sm + kOffRed);   // [2][4][16]
  float* tau = reinterpret_cast<float*>(sm + kOffTau);
  float* rvs = reinterpret_cast<float*>(sm + kOffRv);
  float x[kTcB];
#pragma unroll
  for (int q = 0; q < kTcB; ++q) x[q] = q < b ? x_get(sm, p0 + q, t) : 0.f;
  float tpend = 0.f;                 // warp 0, lane j: entry j of the previous step's T row
  int buf = 0;
  // one copy of the step body (a rolled loop keeps the kernel small for the instruction
  // cache); the registers are addressed statically through predicated selects
#pragma unroll 1
  for (int k = 0; k < b; ++k) {
    float xk = 0.f;
#pragma unroll
    for (int j = 0; j < kTcB; ++j)
      if (j == k) xk = x[j];
    // every product is formed; only value 0 (the sum of squares) and the dots with the
    // later panel columns (j > k, j < b) are read below
    float v[kTcB];
    v[0] = xk * xk;
#pragma unroll
    for (int j = 1; j < kTcB; ++j) v[j] = xk * x[j];
    const float s = warp_sum16(v, lane);
    if ((lane & 1) == 0) red[(buf * 4 + warp) * 16 + sum16_index(lane)] = s;
    bar_panel();
    // lane j < 16 sums value j over the four warps: sigma (j = 0) and the dots d_j (j > k)
    const float* rb = red + buf * 64;
    const int jl = lane & 15;
    const float tot = (rb[jl] + rb[16 + jl]) + (rb[32 + jl] + rb[48 + jl]);
    const float sigma = __shfl_sync(0xffffffffu, tot, 0);
    // warp 0 writes the previous step's row of T, now that every thread has read it
    if (warp == 0 && k > 0 && lane >= k - 1 && lane < b) T[(p0 + k - 1) * n + p0 + lane] = tpend;
    const float alpha = T[(p0 + k) * n + p0 + k];
    float beta = alpha, taup = 0.f, rv = 0.f;        // a zero column: nothing to reflect
    if (sigma != 0.f) {
      const float nu = sqrtf(fmaf(alpha, alpha, sigma));
      beta = alpha >= 0.f ? -nu : nu;
      const float v0 = alpha - beta;
      taup = fabsf(v0) / nu;
      rv = 1.f / v0;
    }
    // lane j (k < j < b): w'_j = tau' (T_kj + d_j / v0) and the new T_kj
    float wl = 0.f;
    if (lane > k && lane < b) {
      const float tkj = T[(p0 + k) * n + p0 + lane];
      wl = taup * fmaf(rv, tot, tkj);
      tpend = tkj - wl;
    }
    if (lane == k) tpend = beta;
    const float xs = rv * xk;
#pragma unroll
    for (int j = 0; j < kTcB; ++j)                      // x_j -= w'_j x_k / v0 (w' = 0 off k < j < b)
      x[j] = fmaf(-__shfl_sync(0xffffffffu, wl, j), xs, x[j]);
    if (t == 0) {
      tau[k] = taup;
      rvs[k] = rv;
    }
    buf ^= 1;
  }
  bar_panel();                                        // every thread has read T's last row
  if (warp == 0 && lane == b - 1) T[(p0 + b - 1) * n + p0 + lane] = tpend;
  // reflector columns: back into X, and row-major (row t) as the update's A operand
#pragma unroll
  for (int q = 0; q < kTcB; ++q) {
    if (q >= b) x[q] = 0.f;
    if (q < b) x_put(sm, p0 + q, t, x[q]);
  }
  put_row16(sm + kOffA, v_off(t, 0), x);
}

// X[:, p0 + 16 ch + e] -= D2[:, 16 ch + e] for the chunks ch in [ch0, ch1) and columns
// below c (the pending update, TMEM columns 16 ..), on the 32 rows of sub-partition `sub`
// (a warp reads only its sub-partition's lanes).  Lanes 2r and 2r + 1 hold rows 2r and
// 2r + 1: the even lane updates the even columns of both rows, the odd lane the odd ones
// (one 32-bit word per part).
__device__ __forceinline__ void tc_apply(unsigned char* sm, uint32_t tmem, int sub, int lane, int p0, int ch0,
                                         int ch1, int c) {
  const bool odd = lane & 1;
  const int row0 = (32 * sub + lane) & ~1;
  for (int ch = ch0; ch < ch1; ++ch) {
    float v[16];
    tc::ld16(tmem + ((uint32_t)(32 * sub) << 16) + 16 + 16 * ch, v);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const float other = __shfl_xor_sync(0xffffffffu, v[e], 1);
      const int jj = 16 * ch + e;
      if (((e & 1) != 0) == odd && jj < c) {
        const int col = p0 + jj;
        const float2 d = odd ? make_float2(other, v[e]) : make_float2(v[e], other);
        const float2 xv = x_get2(sm, col, row0);
        x_put2(sm, col, row0, make_float2(xv.x - d.x, xv.y - d.y));
      }
    }
  }
}

// Folds the block's rows into one triangle per unit of b.seg chunks of 128 rows, like the
// leaf of k_tsqr_fold (same units, so that its tree levels follow unchanged).
__global__ void __launch_bounds__(kTcThreads, 1) k_tsqr_fold_tc(TsqrBlock b, double* tri_out, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int n = b.n;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  float* T = reinterpret_cast<float*>(sm + kOffT);
  float* Ps = reinterpret_cast<float*>(sm + kOffPs);
  float* Tw = reinterpret_cast<float*>(sm + kOffTw);
  const float* rvs = reinterpret_cast<const float*>(sm + kOffRv);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kOffMisc);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffMisc + 8);
  int* abort_flag = reinterpret_cast<int*>(sm + kOffMisc + 12);
  if (t == 0) {
    tc::mbar_init(mbar, 1);
    *abort_flag = 0;
  }
  if (warp == 0) tc::alloc(tslot, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  bool in_flight = false;

  const int64_t rows = block_rows(b);
  const int64_t chunks = (rows + kTcRows - 1) / kTcRows;
  int64_t seg = (chunks + b.fold_g0 - 1) / b.fold_g0;
  if (seg > b.seg) seg = b.seg;
  if (seg < 1) seg = 1;
  int64_t units = (chunks + seg - 1) / seg;
  if (units < 1) units = 1;                   // an empty block still leaves a (zero) triangle
  const uint32_t base = tc::smem_addr(sm);
  const uint32_t id_p = tc::idesc_bf16(128, kTcB);
  const int pa[6] = {0, 0, 1, 1, 0, 2}, pb[6] = {0, 1, 0, 1, 2, 0};

  for (int64_t u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
    for (int i = t; i < n * n; i += kTcThreads) T[i] = 0.f;
    const int64_t q1 = (u + 1) * seg < chunks ? (u + 1) * seg : chunks;
    for (int64_t q = u * seg; q < q1 && !*abort_flag; ++q) {
      // ---- the chunk into X (three bf16 parts); rows past the block and columns past n are 0
      const int64_t r0 = q * kTcRows;
      const int m = (int)((rows - r0) < kTcRows ? (rows - r0) : kTcRows);
      __syncthreads();
      constexpr int kPairs = kTcWin * kTcRows / 2;     // (column, row pair)
      for (int base_idx = 0; base_idx < kPairs; base_idx += kTcThreads * 8) {
        float2 v[8];                                    // sixteen loads in flight, then the stores
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int idx = base_idx + e * kTcThreads + t;
          const int c = idx / (kTcRows / 2), i = 2 * (idx - c * (kTcRows / 2));
          v[e] = make_float2(0.f, 0.f);
          if (c < n) {
            const int64_t g = (int64_t)c * b.ld + r0 + i;
            if (i < m) v[e].x = b.ptr32 ? b.ptr32[g] : (float)b.ptr[g];
            if (i + 1 < m) v[e].y = b.ptr32 ? b.ptr32[g + 1] : (float)b.ptr[g + 1];
          }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int idx = base_idx + e * kTcThreads + t;
          const int c = idx / (kTcRows / 2);
          x_put2(sm, c, 2 * (idx - c * (kTcRows / 2)), v[e]);
        }
      }
      __syncthreads();
      int cprev = 0;                                    // columns of the pending update in D2
      for (int p0 = 0; p0 < n; p0 += kTcB) {
        const int bw = (n - p0) < kTcB ? (n - p0) : kTcB;
        const int c = n - p0 - bw;                      // trailing columns
        // The previous panel's update X[:, p0 ..] -= D2 is applied with look-ahead: warps
        // 0-3 first take its first 16 columns (this panel: each warp its own 32 rows, so a
        // warp only waits for itself), then factor the panel while warps 4-7 apply the rest.
        if (warp < 4) {
          if (cprev > 0) tc_apply(sm, tmem, warp, lane, p0, 0, 1, cprev);
          __syncwarp();
          tc_panel(sm, T, n, p0, bw);
        } else if (cprev > 16) {
          tc_apply(sm, tmem, warp - 4, lane, p0, 1, (cprev + 15) / 16, cprev);
        }
        cprev = 0;
        if (c <= 0) {
          __syncthreads();
          break;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        // ---- P = X^T X_v: 128 x 16, K = 128 rows in 8 steps of 16, six products each
        if (t == 0) {
          tc::fence_after_sync();
          const uint64_t ad0 = tc::desc(base + kOffX, kXLbo, kXSbo);
          const uint64_t bd0 = tc::desc(base + kOffX + (p0 >> 3) * kXSbo, kXLbo, kXSbo);
          for (int kk = 0; kk < kTcRows / 16; ++kk)
            for (int pr = 0; pr < 6; ++pr)            // the address field (bits 0-13, 16-byte units) advances
              tc::mma_bf16(tmem, ad0 + ((pa[pr] * kXSplit + kk * 2 * kXLbo) >> 4),
                           bd0 + ((pb[pr] * kXSplit + kk * 2 * kXLbo) >> 4), id_p, (kk | pr) != 0);
          tc::commit(mbar);
        }
        in_flight = true;
        if (!tc::mbar_wait(mbar, phase, kTcWaitIters)) {
          set_error(err, FIGARO_ERR_TIMEOUT);
          *abort_flag = 1;
        }
        __syncthreads();
        if (*abort_flag) break;
        in_flight = false;
        phase ^= 1;
        tc::fence_after_sync();
        if (warp < 4) {                                 // row j of P = column j of X
          float v[16];
          tc::ld16(tmem + ((uint32_t)(32 * warp) << 16), v);
          const int j = 32 * warp + lane;
          if (j >= p0 && j < n)
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) Ps[j * kPsLd + qq] = v[qq];
        }
        tc::fence_before_sync();
        __syncthreads();
        // G'[r][q] = y_r^T y_q = (x_r^T x_q) / (v0_r v0_q) for r < q: Tw^-1 = diag(1/tau') + G'
        {
          const int r = t >> 4, q = t & 15;
          Tw[t] = (r < q && q < bw) ? Ps[(p0 + q) * kPsLd + r] * rvs[r] * rvs[q] : 0.f;
        }
        __syncthreads();
        // ---- W' = Tw^T W per trailing column by forward substitution with Tw^-T:
        // W'_q = tau'_q (W_q - sum_{r<q} G'[r][q] W'_r), W = T[panel rows, j] + diag(1/v0) P[:, j];
        // T's panel rows -= W'; W'' = diag(1/v0) W' is the update's B operand
        const int cpad = (c + 15) & ~15;
        unsigned char* B2 = sm + kOffB;
        const float* taus = reinterpret_cast<const float*>(sm + kOffTau);
        for (int jj = t; jj < cpad; jj += kTcThreads) {
          const int j = p0 + bw + jj;
          float w[kTcB];
          if (jj < c) {
#pragma unroll
            for (int qq = 0; qq < kTcB; ++qq) {
              float acc = qq < bw ? fmaf(rvs[qq], Ps[j * kPsLd + qq], T[(p0 + qq) * n + j]) : 0.f;
#pragma unroll
              for (int r = 0; r < qq; ++r) acc = fmaf(-Tw[r * kTcB + qq], w[r], acc);
              w[qq] = qq < bw ? taus[qq] * acc : 0.f;
            }
#pragma unroll
            for (int qq = 0; qq < kTcB; ++qq)
              if (qq < bw) {
                T[(p0 + qq) * n + j] -= w[qq];
                w[qq] *= rvs[qq];
              }
          } else {
#pragma unroll
            for (int qq = 0; qq < kTcB; ++qq) w[qq] = 0.f;
          }
          put_row16(B2, v_off(jj, 0), w);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        // ---- X_trail -= X_v W'': 128 x cpad, K = 16, six products, applied by the next panel
        if (t == 0) {
          tc::fence_after_sync();
          const uint32_t id_u = tc::idesc_bf16(128, cpad);
          for (int pr = 0; pr < 6; ++pr) {
            const uint64_t ad = tc::desc(base + kOffA + pa[pr] * kVSplit, kVLbo, kVSbo);
            const uint64_t bd = tc::desc(base + kOffB + pb[pr] * kVSplit, kVLbo, kVSbo);
            tc::mma_bf16(tmem + 16, ad, bd, id_u, pr != 0);
          }
          tc::commit(mbar);
        }
        in_flight = true;
        if (!tc::mbar_wait(mbar, phase, kTcWaitIters)) {
          set_error(err, FIGARO_ERR_TIMEOUT);
          *abort_flag = 1;
        }
        __syncthreads();
        if (*abort_flag) break;
        in_flight = false;
        phase ^= 1;
        tc::fence_after_sync();
        cprev = c;
      }
    }
    if (*abort_flag) break;
    __syncthreads();
    double* tri = tri_out + u * (int64_t)n * n;
    for (int idx = t; idx < n * n; idx += kTcThreads) {
      const int cc = idx / n, r = idx - cc * n;
      tri[idx] = r <= cc ? (double)T[r * n + cc] : 0.0;
    }
    __syncthreads();                                  // T is read above before the next unit zeroes it
  }
  // a timed-out product may still be running: wait once more (bounded) before freeing TMEM
  if (in_flight) tc::mbar_wait(mbar, phase, kTcWaitIters);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, kTmemCols);
}

void launch_fold_tc(const TsqrBlock& b, double* tri_out, int* err, cudaStream_t st) {
  int64_t grid = (b.bound + kTcRows - 1) / kTcRows;
  grid = (grid + b.seg - 1) / b.seg;
  if (grid > 152) grid = 152;
  if (grid < 1) grid = 1;
  k_tsqr_fold_tc<<<(unsigned)grid, kTcThreads, fold_tc_smem(b.n), st>>>(b, tri_out, err);
}

cudaError_t fold_tc_set_attributes() {
  return cudaFuncSetAttribute(k_tsqr_fold_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace fig
