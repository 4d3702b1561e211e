/* CPU FiGaRo: R of the join matrix A[:, Y] over an acyclic join, on the host cores.
 *
 * TEST INFRASTRUCTURE AND CPU BASELINE ONLY.  Only tests/, __graft_entry__ (build) and the
 * CPU legs of bench.py (cpu_baseline, --impl reference) may load this library.  It shares
 * no code with the CUDA path; its R is checked against the Python oracle by the
 * -m "not gpu" tests.
 *
 * What it computes, in the paper's order: Alg. 3 (compute-counts: rows_per_key,
 * Theta_down, Phi_down bottom-up; full_join_size, Phi_up, Phi_circ top-down, exact
 * 64-bit integers), Alg. 4 (heads_and_tails with the Def. of head and tail,
 * process_and_join_children, project_away_join_attributes with Alg. 2's generalized
 * head and tail, the root's Data) and the §7 post-processing (Householder QR of every
 * R0 block on its own columns, then of the stack of the block triangles), R normalised
 * to a non-negative diagonal (§2 "Output").  OpenMP parallelises the sorts (relations),
 * the per-group loops of Alg. 3 and Alg. 4 and the row tiles of the QRs.
 */
#ifndef FIGARO_CPU_H
#define FIGARO_CPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CFIG_OK = 0,
  CFIG_ERR_INVALID = 1,       /* not a tree, too many keys, negative sizes, null pointers */
  CFIG_ERR_NOT_REDUCED = 2,   /* a tuple has no join partner (the paper assumes fully reduced input) */
  CFIG_ERR_OVERFLOW = 3,      /* a count does not fit in 64 bits */
  CFIG_ERR_NOMEM = 4,         /* a host allocation failed */
  CFIG_ERR_NOT_SORTED = 5     /* presorted was set but a relation is not in join-key order */
};

#define CFIG_MAX_KEYS 8

/* One relation S_i: n_keys join-key columns tagged with global attribute ids (the natural
 * join equates equal ids) and n_data FP64 data columns, column-major with leading
 * dimension ld >= n_rows.  All pointers are host memory owned by the caller. */
typedef struct {
  int64_t n_rows;
  int32_t n_keys;
  const int32_t* key_attr;     /* [n_keys] */
  const int64_t* const* keys;  /* n_keys arrays of n_rows values */
  int32_t n_data;
  const double* data;          /* column c of row r at data[c * ld + r] */
  int64_t ld;
} cfig_relation;

/* R (n_cols x n_cols, row-major, n_cols = sum of n_data) of the join given by the
 * relations and the join tree parent[] (parent[root] = -1).  Columns of R are the
 * relations' data columns in relation order.  presorted = 1 takes every relation as
 * already sorted in join-key order (attributes shared with the parent first, then the
 * others, each part by ascending attribute id; ties in any order) and checks it;
 * n_threads <= 0 uses OpenMP's default.  seconds (optional, [4]) receives the wall time
 * of sort + grouping, Alg. 3, Alg. 4 and the post-processing.  Returns a CFIG_* status. */
int cfig_figaro_r(int32_t n_rel, const cfig_relation* rels, const int32_t* parent, int32_t presorted,
                  int32_t n_threads, double* R, double* seconds);

/* Number of OpenMP threads a call with n_threads <= 0 uses. */
int cfig_max_threads(void);

#ifdef __cplusplus
}
#endif

#endif
