// Host-only check of the TSQR planner (no CUDA runtime call is made).  For every block
// width 1..1024, row counts from 1 to 9M, both precisions and both float leaves:
//  - every autotuner candidate planned from the rule-planned block (as the tuner and the
//    plan builder do) equals the same candidate planned from a zeroed block, so no field of
//    an earlier plan survives into a plan of another path;
//  - the dynamic shared memory of every leaf and tree launch of the plan fits the limit
//    that the library sets for that kernel, and tile and fan are valid.
// Exit status 0 when every plan passes; the first failures are printed.
#include <cstdio>

#include "tsqr.cu"
#include "tune.cu"

using namespace fig;

static bool same_plan(const TsqrBlock& a, const TsqrBlock& b) {
  return a.tile == b.tile && a.fan == b.fan && a.levels == b.levels && a.top == b.top && a.nreg == b.nreg &&
         a.warp_min == b.warp_min && a.givens == b.givens && a.fold == b.fold && a.fold_tsmem == b.fold_tsmem &&
         a.seg == b.seg && a.fold_g0 == b.fold_g0 && a.fold_tc == b.fold_tc && a.fold_tc5 == b.fold_tc5 &&
         a.fused == b.fused && a.fold_res == b.fold_res;
}

int main() {
  int bad = 0, checked = 0;
  const int64_t rows_list[] = {1, 60, 2940, 100000, 9000000};
  for (int mixed = 0; mixed < 2; ++mixed)
    for (int tc5 = 0; tc5 < 2; ++tc5)
      for (int n = 1; n <= 1024; ++n)
        for (int64_t rows : rows_list) {
          const size_t esz = mixed ? sizeof(float) : sizeof(double);
          TsqrBlock base{};
          base.n = n;
          base.kind = BLK_FIXED;
          base.M = base.bound = base.ld = rows;
          TsqrBlock rule = base;
          tsqr_plan_block(rule, mixed, false, tc5);
          for (const TsqrTune& t : tune_candidates(rule, mixed)) {
            TsqrBlock again = rule, fresh = base;
            tsqr_plan_block(again, mixed, false, tc5, &t);
            tsqr_plan_block(fresh, mixed, false, tc5, &t);
            ++checked;
            if (!same_plan(again, fresh)) {
              if (bad < 20) printf("re-planned block differs: n=%d rows=%lld mixed=%d tcgen05=%d\n", n, (long long)rows,
                                   mixed, tc5);
              ++bad;
            }
            size_t smem = 0, cap = kSmemCap;
            if (fresh.fold && fresh.fold_tc5) {
              smem = fold_tc_smem(n);
              cap = 200 * 1024;
            } else if (fresh.fold) {
              smem = fold_smem(fresh, esz);
            } else if (!fresh.nreg) {
              for (int tree = 0; tree < 2; ++tree) {
                size_t s = cta_smem(cta_lda(fresh, tree), n, esz);
                if (s > kSmemCap) s = kRedElems * esz;     // the tile in a global slot
                if (s > smem) smem = s;
              }
            }
            if (smem > cap || fresh.tile < 1 || fresh.fan < 2) {
              if (bad < 20)
                printf("launch out of limits: n=%d rows=%lld mixed=%d tcgen05=%d smem=%zu tile=%d fan=%d\n", n,
                       (long long)rows, mixed, tc5, smem, fresh.tile, fresh.fan);
              ++bad;
            }
          }
        }
  printf("%d plans checked, %d failed\n", checked, bad);
  return bad != 0;
}
