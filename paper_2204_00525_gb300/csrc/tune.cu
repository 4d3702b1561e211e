// TSQR tile autotuner (options.autotune): the planner's rules fix every block's leaf tile,
// chunk height, blocks per SM, chunks per leaf triangle and tree fan from its width,
// precision and the shared-memory budget; with autotune, figaro_plan instead times a small
// set of candidate plans for each block on synthetic rows of the block's width and row
// bound (at most 2^30 cells and rows x width^2 <= 2^37, so that one timed run stays within
// about a third of a second in FP64 at any width; uniform values from a counter-based
// generator) and keeps the fastest, the rule's own plan among them.  Only the speed
// depends on the choice: every candidate is an exact Householder TSQR of the same rows (on
// the float path the chunks per leaf triangle stay at most 16, the bound that keeps its
// error within the stated one).
// Results are cached per (precision, leaf kind, width, power-of-two row bucket) for the
// life of the process, so plans of equal shapes (a batch's instances) are tuned once.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kernels.cuh"

namespace fig {

// splitmix64 of (seed + i * golden), its top 53 bits scaled to [-1, 1)
__global__ void k_tune_fill(double* d, float* f, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double x = (double)(z >> 11) * (1.0 / 4503599627370496.0) - 1.0;   // 2^52
    d[i] = x;
    if (f) f[i] = (float)x;
  }
}

constexpr int64_t kTuneCellsCap = int64_t(1) << 30;   // 8 GiB of float64 rows at most
constexpr int64_t kTuneMacCap = int64_t(1) << 37;     // rows x n^2 of one timed run
constexpr int64_t kFarAway = int64_t(1) << 40;   // warp_min that leaves every level to the block kernel

// Candidate overrides for block b (the all-zero override, the rule's plan, first).
static std::vector<TsqrTune> tune_candidates(const TsqrBlock& rule, bool mixed) {
  std::vector<TsqrTune> c;
  c.push_back(TsqrTune{0, 0, 0, 0});
  if (rule.nreg) {
    const int alt_fan = rule.nreg <= 16 ? (rule.fan / 2 >= 2 ? rule.fan / 2 : 0) : 12;
    const int64_t mins[] = {2, 152, 152 * 4, kFarAway};
    for (int64_t wm : mins) {
      if (wm != rule.warp_min) c.push_back(TsqrTune{0, 0, 0, wm});
      if (alt_fan) c.push_back(TsqrTune{0, 0, alt_fan, wm});
    }
    if (rule.nreg > 16) c.push_back(TsqrTune{0, 0, 3, 0});
  } else if (rule.fold && rule.fold_tc5) {
    const int segs[] = {0, 8, 4};
    for (int s : segs) {
      if (s) c.push_back(TsqrTune{0, s, 0, 0});
      c.push_back(TsqrTune{0, s, 4, 0});
    }
  } else if (rule.fold) {
    if (mixed) {
      c.push_back(TsqrTune{64, 0, 0, 0});
      c.push_back(TsqrTune{0, 8, 0, 0});
      c.push_back(TsqrTune{64, 8, 0, 0});
    } else {
      const int budgets[] = {0, 100, 64};
      for (int kib : budgets) {
        if (kib) c.push_back(TsqrTune{kib, 0, 0, 0});
        c.push_back(TsqrTune{kib, 0, 2, 0});
      }
    }
  }
  return c;
}

using TuneKey = std::tuple<bool, bool, bool, int, int>;
static std::mutex g_tune_mu;
static std::map<TuneKey, TsqrTune> g_tune_cache;

TsqrTune tsqr_autotune(const TsqrBlock& b, bool mixed, bool givens, bool tcgen05) {
  const TsqrTune none{0, 0, 0, 0};
  if (b.n < 1 || b.fused) return none;
  if (cudaPeekAtLastError() != cudaSuccess) return none;   // an earlier error stays for the caller
  int64_t cap = kTuneCellsCap / b.n;
  if (cap > kTuneMacCap / ((int64_t)b.n * b.n)) cap = kTuneMacCap / ((int64_t)b.n * b.n);
  const int64_t rows = b.bound < cap ? (b.bound > 0 ? b.bound : 1) : cap;
  int bucket = 0;
  while ((int64_t(1) << bucket) < rows) ++bucket;
  const TuneKey key{mixed, givens, tcgen05, b.n, bucket};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) return it->second;
  }
  // the block as a fixed block of `rows` synthetic rows
  TsqrBlock base = b;
  base.kind = BLK_FIXED;
  base.M = rows;
  base.bound = rows;
  base.ld = rows;
  base.fused = false;
  base.prio = false;
  TsqrBlock rule = base;
  tsqr_plan_block(rule, mixed, givens, tcgen05);
  if (!rule.nreg && !rule.fold) return none;          // the block-per-tile path: nothing to choose
  std::vector<TsqrTune> cand = tune_candidates(rule, mixed);
  std::vector<TsqrBlock> plans;
  int64_t tri_max = 0, scr_max = 0;
  for (const TsqrTune& t : cand) {
    TsqrBlock p = base;
    tsqr_plan_block(p, mixed, givens, tcgen05, &t);
    tri_max = std::max(tri_max, tsqr_tri_elems(p));
    scr_max = std::max(scr_max, tsqr_scratch_elems(p, mixed));
    plans.push_back(p);
  }
  double* data = nullptr;
  float* data32 = nullptr;
  double* tri = nullptr;
  double* scratch = nullptr;
  int* err = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const int64_t cells = rows * (int64_t)b.n;
  bool ok = cudaMalloc(&data, sizeof(double) * cells) == cudaSuccess &&
            (!mixed || cudaMalloc(&data32, sizeof(float) * cells) == cudaSuccess) &&
            cudaMalloc(&tri, sizeof(double) * 2 * tri_max) == cudaSuccess &&
            (scr_max == 0 || cudaMalloc(&scratch, sizeof(double) * scr_max) == cudaSuccess) &&
            cudaMalloc(&err, sizeof(int)) == cudaSuccess &&
            cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  TsqrTune best = none;
  if (ok) {
    k_tune_fill<<<grid_for(cells, 256, 152 * 8), 256, 0, st>>>(data, data32, cells, 0x5eedull + (uint64_t)b.n);
    ok = cudaGetLastError() == cudaSuccess && cudaMemsetAsync(err, 0, sizeof(int), st) == cudaSuccess;
    double best_ms = -1.0;
    for (size_t i = 0; ok && i < plans.size(); ++i) {
      TsqrBlock p = plans[i];
      p.ptr = data;
      p.ptr32 = data32;
      p.tri[0] = tri;
      p.tri[1] = tri + tri_max;
      p.scratch = scratch;
      p.err = err;
      int64_t launches = 0;
      float ms = 0.f, total = 0.f;
      for (int rep = 0; rep < 3 && ok; ++rep) {      // one warm-up, two timed runs
        ok = cudaEventRecord(e0, st) == cudaSuccess;
        tsqr_leaf(p, mixed, st, &launches);
        tsqr_reduce(p, mixed, st, &launches);
        ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (rep > 0) total += ms;
      }
      // a launch the device refused (its configuration) disqualifies the candidate only;
      // an error that persists fails the event calls above and ends the tuning
      const bool ran = cudaGetLastError() == cudaSuccess;
      if (ok && ran && (best_ms < 0.0 || total < best_ms)) {
        best_ms = total;
        best = cand[i];
      }
    }
    int h_err = 0;
    if (ok) ok = cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && h_err == 0;
  }
  if (!ok) {
    cudaGetLastError();
    best = none;                                      // measurement failed: keep the rule
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(data);
  cudaFree(data32);
  cudaFree(tri);
  cudaFree(scratch);
  cudaFree(err);
  if (ok) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  return best;
}

}  // namespace fig
