/* CPU FiGaRo (see figaro_cpu.h): Alg. 3, Alg. 4 with Alg. 2, and the §7 post-processing
 * in C with OpenMP.  Test infrastructure and CPU baseline only. */
#include "figaro_cpu.h"

#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ per-relation state */
typedef struct {
  const cfig_relation* rel;
  int parent;
  int n_child;
  int* child;                  /* children in relation order */
  int n_sort;                  /* X_i in sort order: X_p first, then the rest (ascending ids) */
  int sort_col[CFIG_MAX_KEYS]; /* key column of each sorted attribute */
  int sort_attr[CFIG_MAX_KEYS];
  int n_xp;                    /* leading attributes shared with the parent */
  int64_t* order;              /* rows in sorted order */
  int64_t G;                   /* groups: distinct x_i */
  int64_t* gstart;             /* [G + 1] */
  int64_t* gkey;               /* [G * n_sort] */
  int64_t P;                   /* parent groups: distinct x_p (consecutive groups) */
  int64_t* pstart;             /* [P + 1] first group of every parent group */
  int64_t* g2p;                /* [G] */
  int64_t** cidx;              /* per child j: [G] parent group of S_j holding x_ij */
  /* Alg. 3 (Fig. 4), exact */
  uint64_t *rows, *theta, *full, *circ;   /* per group */
  uint64_t *down, *up;                    /* per parent group */
  /* columns of the subtree of S_i (global ids, ascending) and the own columns' offset */
  int n_sub, own_off;
  int* sub_cols;
} Rel;

typedef struct {
  int n_rel, root, n_cols;
  const int32_t* parent;
  Rel* r;
  int* col_off;                /* global offset of every relation's columns */
  volatile int status;
} Ctx;

static void set_status(Ctx* c, int s) {
#pragma omp critical(cfig_status)
  if (c->status == CFIG_OK) c->status = s;
}

static int cmp_rows(const Rel* R, int64_t a, int64_t b) {
  for (int k = 0; k < R->n_sort; ++k) {
    const int64_t x = R->rel->keys[R->sort_col[k]][a], y = R->rel->keys[R->sort_col[k]][b];
    if (x != y) return x < y ? -1 : 1;
  }
  return 0;
}

/* ------------------------------------------------------------------ sort (§5 order)
 * Stable merge sort of the row indices by the key tuple in sort order: rows with equal
 * keys keep their input order.  The halves of large ranges are sorted as OpenMP tasks. */
static void merge_sort(const Rel* R, int64_t* a, int64_t* tmp, int64_t n) {
  if (n < 32) {
    for (int64_t i = 1; i < n; ++i) {
      const int64_t v = a[i];
      int64_t j = i - 1;
      while (j >= 0 && cmp_rows(R, a[j], v) > 0) {
        a[j + 1] = a[j];
        --j;
      }
      a[j + 1] = v;
    }
    return;
  }
  const int64_t h = n / 2;
  if (n > 65536) {
#pragma omp task
    merge_sort(R, a, tmp, h);
#pragma omp task
    merge_sort(R, a + h, tmp + h, n - h);
#pragma omp taskwait
  } else {
    merge_sort(R, a, tmp, h);
    merge_sort(R, a + h, tmp + h, n - h);
  }
  int64_t i = 0, j = h, k = 0;
  while (i < h && j < n) tmp[k++] = cmp_rows(R, a[j], a[i]) < 0 ? a[j++] : a[i++];
  while (i < h) tmp[k++] = a[i++];
  while (j < n) tmp[k++] = a[j++];
  memcpy(a, tmp, (size_t)n * sizeof(int64_t));
}

static int sort_and_group(Ctx* c, int i, int presorted) {
  Rel* R = &c->r[i];
  const int64_t M = R->rel->n_rows;
  R->order = (int64_t*)malloc((size_t)(M > 0 ? M : 1) * sizeof(int64_t));
  if (!R->order) return CFIG_ERR_NOMEM;
  for (int64_t t = 0; t < M; ++t) R->order[t] = t;
  if (presorted) {
    for (int64_t t = 1; t < M; ++t)
      if (cmp_rows(R, t - 1, t) > 0) return CFIG_ERR_NOT_SORTED;
  } else if (M > 1) {
    int64_t* tmp = (int64_t*)malloc((size_t)M * sizeof(int64_t));
    if (!tmp) return CFIG_ERR_NOMEM;
    merge_sort(R, R->order, tmp, M);
    free(tmp);
  }
  /* groups: runs of equal x_i; parent groups: runs of equal x_p */
  int64_t G = 0;
  for (int64_t t = 0; t < M; ++t)
    if (t == 0 || cmp_rows(R, R->order[t - 1], R->order[t]) != 0) ++G;
  R->G = G;
  R->gstart = (int64_t*)malloc((size_t)(G + 1) * sizeof(int64_t));
  R->gkey = (int64_t*)malloc((size_t)(G * R->n_sort + 1) * sizeof(int64_t));
  R->g2p = (int64_t*)malloc((size_t)(G + 1) * sizeof(int64_t));
  R->pstart = (int64_t*)malloc((size_t)(G + 1) * sizeof(int64_t));
  if (!R->gstart || !R->gkey || !R->g2p || !R->pstart) return CFIG_ERR_NOMEM;
  int64_t g = 0;
  for (int64_t t = 0; t < M; ++t) {
    if (t == 0 || cmp_rows(R, R->order[t - 1], R->order[t]) != 0) {
      R->gstart[g] = t;
      for (int k = 0; k < R->n_sort; ++k) R->gkey[g * R->n_sort + k] = R->rel->keys[R->sort_col[k]][R->order[t]];
      ++g;
    }
  }
  R->gstart[G] = M;
  int64_t P = 0;
  for (g = 0; g < G; ++g) {
    int newp = g == 0;
    for (int k = 0; k < R->n_xp && !newp; ++k)
      newp = R->gkey[g * R->n_sort + k] != R->gkey[(g - 1) * R->n_sort + k];
    if (newp) R->pstart[P++] = g;
    R->g2p[g] = P - 1;
  }
  R->pstart[P] = G;
  R->P = P;
  return CFIG_OK;
}

/* Parent group of child j whose x_p equals group g's projection on the attributes that
 * S_i shares with S_j (binary search over S_j's sorted parent groups), or -1. */
static int64_t find_in_child(const Rel* Ri, int64_t g, const Rel* Rj, const int* pos) {
  int64_t lo = 0, hi = Rj->P - 1;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) / 2;
    const int64_t* key = Rj->gkey + Rj->pstart[mid] * Rj->n_sort;
    int cmp = 0;
    for (int k = 0; k < Rj->n_xp && !cmp; ++k) {
      const int64_t x = Ri->gkey[g * Ri->n_sort + pos[k]], y = key[k];
      cmp = x < y ? -1 : (x > y ? 1 : 0);
    }
    if (cmp == 0) return mid;
    if (cmp < 0) hi = mid - 1; else lo = mid + 1;
  }
  return -1;
}

/* ------------------------------------------------------------------ Alg. 3 (compute-counts)
 * pass 1, bottom-up: Theta_down_i(x_i) = rows_per_key_i(x_i) * prod over the children j of
 * Phi_down_j(x_ij); Phi_down_i(x_p) = sum of Theta_down_i over the x_i projecting to x_p.
 * pass 2, top-down: full_join_size_i(x_i) = Theta_down_i(x_i) * Phi_up_i(x_p) (1 at the
 * root); every child j accumulates full_join_size_i into Phi_up_j(x_ij), which is divided
 * by Phi_down_j(x_ij) before S_j is visited; Phi_circ_i(x_i) = full / rows_per_key. */
static void count_pass1(Ctx* c, int i) {
  Rel* R = &c->r[i];
  for (int q = 0; q < R->n_child; ++q) count_pass1(c, R->child[q]);
  if (c->status != CFIG_OK) return;
  const int64_t G = R->G, P = R->P;
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < G; ++g) {
    uint64_t th = (uint64_t)(R->gstart[g + 1] - R->gstart[g]);
    R->rows[g] = th;
    for (int q = 0; q < R->n_child; ++q) {
      const int64_t k = R->cidx[q][g];
      if (k < 0) {
        set_status(c, CFIG_ERR_NOT_REDUCED);
        th = 0;
        break;
      }
      if (__builtin_mul_overflow(th, c->r[R->child[q]].down[k], &th)) set_status(c, CFIG_ERR_OVERFLOW);
    }
    R->theta[g] = th;
  }
  if (R->parent >= 0) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
      uint64_t s = 0;
      for (int64_t g = R->pstart[p]; g < R->pstart[p + 1]; ++g)
        if (__builtin_add_overflow(s, R->theta[g], &s)) set_status(c, CFIG_ERR_OVERFLOW);
      R->down[p] = s;
    }
  }
}

static void count_pass2(Ctx* c, int i) {
  Rel* R = &c->r[i];
  const int64_t G = R->G;
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < G; ++g) {
    uint64_t f = R->theta[g];
    if (R->parent >= 0 && __builtin_mul_overflow(f, R->up[R->g2p[g]], &f)) set_status(c, CFIG_ERR_OVERFLOW);
    R->full[g] = f;
    R->circ[g] = f / R->rows[g];
    if (f == 0) set_status(c, CFIG_ERR_NOT_REDUCED);
  }
  if (c->status != CFIG_OK) return;
  for (int q = 0; q < R->n_child; ++q) {
    Rel* Rj = &c->r[R->child[q]];
    for (int64_t p = 0; p < Rj->P; ++p) Rj->up[p] = 0;
    for (int64_t g = 0; g < G; ++g) {
      uint64_t* u = &Rj->up[R->cidx[q][g]];
      if (__builtin_add_overflow(*u, R->full[g], u)) set_status(c, CFIG_ERR_OVERFLOW);
    }
    for (int64_t p = 0; p < Rj->P; ++p) {
      if (Rj->down[p] == 0) {
        set_status(c, CFIG_ERR_NOT_REDUCED);
        continue;
      }
      Rj->up[p] /= Rj->down[p];
    }
  }
  for (int q = 0; q < R->n_child; ++q) count_pass2(c, R->child[q]);
}

/* ------------------------------------------------------------------ Alg. 4
 * R0 is kept as blocks: all rows appended to Out with the same column support (the tails
 * of one relation; the generalized tails of one node; the root's Data), column-major. */
typedef struct {
  int64_t rows;
  int n;
  const int* cols;             /* global column of each of the block's columns */
  double* a;                   /* rows x n, leading dimension rows */
} Block;

typedef struct {
  Block* b;
  int nb;
} Out;

/* What S_i returns to its parent: Data (rows x n_sub, row-major) and scales, one row per
 * x_p (the parent groups of S_i). */
typedef struct {
  double* data;
  double* scales;
} Ret;

static int position_of(const int* cols, int n, int col) {
  for (int k = 0; k < n; ++k)
    if (cols[k] == col) return k;
  return -1;
}

static int figaro_node(Ctx* c, int i, Out* out, Ret* ret) {
  Rel* R = &c->r[i];
  const cfig_relation* rel = R->rel;
  const int64_t G = R->G, M = rel->n_rows;
  const int ns = R->n_sub, ni = rel->n_data;
  double* Data = (double*)calloc((size_t)(G > 0 ? G : 1) * (size_t)(ns > 0 ? ns : 1), sizeof(double));
  double* scales = (double*)malloc((size_t)(G > 0 ? G : 1) * sizeof(double));
  if (!Data || !scales) return CFIG_ERR_NOMEM;

  /* heads_and_tails: for every x_i, the tails of S_i^{x_i} (Def. of head and tail, row
   * j >= 1 of a group of m rows a_0..a_{m-1}: (sqrt(j) a_j - S_j / sqrt(j)) / sqrt(j + 1),
   * S_j = a_0 + ... + a_{j-1}) scaled by sqrt(Phi_circ_i(x_i)) go to Out;
   * Data[x_i : Y_i] = H(S_i^{x_i}) = S_m / sqrt(m), scales[x_i] = sqrt(m). */
  {
    Block* b = &out->b[out->nb++];
    b->rows = M - G;
    b->n = ni;
    b->cols = R->sub_cols + R->own_off;
    b->a = (double*)malloc((size_t)(b->rows > 0 ? b->rows : 1) * (size_t)(ni > 0 ? ni : 1) * sizeof(double));
    if (!b->a) return CFIG_ERR_NOMEM;
    double* T = b->a;
    const int64_t ldt = b->rows;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t g = 0; g < G; ++g) {
      const int64_t s = R->gstart[g], m = R->gstart[g + 1] - s;
      const double w = sqrt((double)R->circ[g]);
      for (int col = 0; col < ni; ++col) {
        const double* y = rel->data + (int64_t)col * rel->ld;
        double S = 0.0;
        for (int64_t j = 0; j < m; ++j) {
          const double a = y[R->order[s + j]];
          if (j > 0) {
            const double sj = sqrt((double)j);
            T[(int64_t)col * ldt + (s - g) + (j - 1)] = w * ((sj * a - S / sj) / sqrt((double)j + 1.0));
          }
          S += a;
        }
        Data[g * ns + R->own_off + col] = S / sqrt((double)m);
      }
      scales[g] = sqrt((double)m);
    }
  }

  /* process_and_join_children: Data[x_i : Y_k] = Data_j[x_ij : Y_k] * scales[x_i] *
   * prod over the other children j' of scales_j'[x_ij'] for S_k in the subtree of S_j;
   * then Data[x_i : Y_i] and scales[x_i] are multiplied by prod_j scales_j[x_ij]. */
  if (R->n_child > 0) {
    Ret* cr = (Ret*)calloc((size_t)R->n_child, sizeof(Ret));
    int** cpos = (int**)calloc((size_t)R->n_child, sizeof(int*));
    if (!cr || !cpos) return CFIG_ERR_NOMEM;
    for (int q = 0; q < R->n_child; ++q) {
      const int j = R->child[q];
      int rc = figaro_node(c, j, out, &cr[q]);
      if (rc != CFIG_OK) return rc;
      const Rel* Rj = &c->r[j];
      cpos[q] = (int*)malloc((size_t)(Rj->n_sub > 0 ? Rj->n_sub : 1) * sizeof(int));
      if (!cpos[q]) return CFIG_ERR_NOMEM;
      for (int k = 0; k < Rj->n_sub; ++k) cpos[q][k] = position_of(R->sub_cols, ns, Rj->sub_cols[k]);
    }
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < G; ++g) {
      double all = 1.0;
      for (int q = 0; q < R->n_child; ++q) all *= cr[q].scales[R->cidx[q][g]];
      for (int q = 0; q < R->n_child; ++q) {
        const Rel* Rj = &c->r[R->child[q]];
        const int64_t k = R->cidx[q][g];
        double other = 1.0;
        for (int q2 = 0; q2 < R->n_child; ++q2)
          if (q2 != q) other *= cr[q2].scales[R->cidx[q2][g]];
        const double f = scales[g] * other;
        for (int col = 0; col < Rj->n_sub; ++col) Data[g * ns + cpos[q][col]] = cr[q].data[k * Rj->n_sub + col] * f;
      }
      for (int col = 0; col < ni; ++col) Data[g * ns + R->own_off + col] *= all;
      scales[g] *= all;
    }
    for (int q = 0; q < R->n_child; ++q) {
      free(cr[q].data);
      free(cr[q].scales);
      free(cpos[q]);
    }
    free(cr);
    free(cpos);
  }

  if (R->parent < 0) {
    /* root: Out.append(Data) */
    Block* b = &out->b[out->nb++];
    b->rows = G;
    b->n = ns;
    b->cols = R->sub_cols;
    b->a = (double*)malloc((size_t)(G > 0 ? G : 1) * (size_t)(ns > 0 ? ns : 1) * sizeof(double));
    if (!b->a) return CFIG_ERR_NOMEM;
    for (int64_t g = 0; g < G; ++g)
      for (int col = 0; col < ns; ++col) b->a[(int64_t)col * G + g] = Data[g * ns + col];
    free(Data);
    free(scales);
    return CFIG_OK;
  }
  if (R->n_child == 0) {
    /* a leaf: every join attribute of a leaf is shared with its parent (X_i = X_p), so
     * its groups are its parent groups and Data is returned as it is */
    ret->data = Data;
    ret->scales = scales;
    return CFIG_OK;
  }

  /* project_away_join_attributes: for every x_p, the x_i projecting to it are the
   * consecutive groups a..b-1; Out gets sqrt(Phi_up_i(x_p)) T(Data[a..b-1], scales[a..b-1])
   * (Alg. 2: a running ssum_v = sum of v_t^2 and sum_A = sum of v_t A_t; row j is
   * (sqrt(ssum_v) A_{j+1} - v_{j+1} sum_A / sqrt(ssum_v)) / sqrt(ssum_v + v_{j+1}^2)), the
   * parent receives H(Data[a..b-1], scales[a..b-1]) = sum_A / ||v|| and sqrt(Phi_down_i(x_p)). */
  const int64_t P = R->P;
  Block* b = &out->b[out->nb++];
  b->rows = G - P;
  b->n = ns;
  b->cols = R->sub_cols;
  b->a = (double*)malloc((size_t)(b->rows > 0 ? b->rows : 1) * (size_t)(ns > 0 ? ns : 1) * sizeof(double));
  ret->data = (double*)malloc((size_t)(P > 0 ? P : 1) * (size_t)(ns > 0 ? ns : 1) * sizeof(double));
  ret->scales = (double*)malloc((size_t)(P > 0 ? P : 1) * sizeof(double));
  if (!b->a || !ret->data || !ret->scales) return CFIG_ERR_NOMEM;
  double* T = b->a;
  const int64_t ldt = b->rows;
#pragma omp parallel
  {
    double* sumA = (double*)malloc((size_t)(ns > 0 ? ns : 1) * sizeof(double));
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < P; ++p) {
      if (!sumA) {
        set_status(c, CFIG_ERR_NOMEM);
        continue;
      }
      const int64_t a0 = R->pstart[p], a1 = R->pstart[p + 1];
      const double w = sqrt((double)R->up[p]);
      for (int col = 0; col < ns; ++col) sumA[col] = 0.0;
      double ssum = 0.0;
      for (int64_t g = a0; g < a1; ++g) {
        const double v = scales[g];
        if (g > a0) {
          const double sq = sqrt(ssum), den = sqrt(ssum + v * v);
          const int64_t row = (a0 - p) + (g - a0 - 1);
          for (int col = 0; col < ns; ++col)
            T[(int64_t)col * ldt + row] = w * ((sq * Data[g * ns + col] - v * sumA[col] / sq) / den);
        }
        ssum += v * v;
        for (int col = 0; col < ns; ++col) sumA[col] += v * Data[g * ns + col];
      }
      const double nv = sqrt(ssum);
      for (int col = 0; col < ns; ++col) ret->data[p * ns + col] = sumA[col] / nv;
      ret->scales[p] = sqrt((double)R->down[p]);
    }
    free(sumA);
  }
  free(Data);
  free(scales);
  return c->status;
}

/* ------------------------------------------------------------------ §7 post-processing
 * Householder QR in place of the m x n column-major A (leading dimension lda): for each
 * column k, the reflector H = I - tau v v^T with v = (1, x_{k+1..} / v0), v0 = alpha - beta,
 * beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta maps x = A[k:, k] to beta e_1 and
 * is applied to the later columns.  On return the upper triangle of A[0:min(m,n), :] is R
 * (the entries below it are left as they are). */
static void householder_qr(double* A, int64_t m, int n, int64_t lda) {
  const int64_t kmax = m < n ? m : n;
  for (int64_t k = 0; k < kmax; ++k) {
    double* x = A + k * lda;
    double sigma = 0.0;
    for (int64_t i = k + 1; i < m; ++i) sigma += x[i] * x[i];
    if (sigma == 0.0) continue;              /* nothing below the diagonal: H = I */
    const double alpha = x[k];
    const double nu = sqrt(alpha * alpha + sigma);
    const double beta = alpha >= 0.0 ? -nu : nu;
    const double v0 = alpha - beta;
    const double tau = (beta - alpha) / beta;
    for (int64_t i = k + 1; i < m; ++i) x[i] /= v0;
    x[k] = beta;
    for (int j = (int)k + 1; j < n; ++j) {
      double* y = A + (int64_t)j * lda;
      double w = y[k];
      for (int64_t i = k + 1; i < m; ++i) w += x[i] * y[i];
      w *= tau;
      y[k] -= w;
      for (int64_t i = k + 1; i < m; ++i) y[i] -= w * x[i];
    }
  }
}

/* R (n x n, column-major, zeros below the diagonal) of the rows x n column-major block A
 * (leading dimension lda): a tree of Householder QRs over row tiles of `tile` rows, the
 * tiles of a level in parallel, each level stacking the previous level's triangles. */
static int tsqr(const double* A, int64_t rows, int n, int64_t lda, double* Rout) {
  memset(Rout, 0, (size_t)n * n * sizeof(double));
  if (rows <= 0 || n <= 0) return CFIG_OK;
  const int64_t tile = (4 * (int64_t)n > 1024) ? 4 * (int64_t)n : 1024;
  const double* src = A;
  int64_t src_rows = rows, src_ld = lda;
  double* level = NULL;
  int status = CFIG_OK;
  for (;;) {
    const int64_t tiles = (src_rows + tile - 1) / tile;
    /* each tile leaves min(tile rows, n) rows of its triangle */
    int64_t out_rows = 0;
    for (int64_t t = 0; t < tiles; ++t) {
      const int64_t tr = (t + 1) * tile < src_rows ? tile : src_rows - t * tile;
      out_rows += tr < n ? tr : n;
    }
    if (tiles == 1) {
      double* buf = (double*)malloc((size_t)src_rows * n * sizeof(double));
      if (!buf) { status = CFIG_ERR_NOMEM; break; }
      for (int col = 0; col < n; ++col) memcpy(buf + (int64_t)col * src_rows, src + (int64_t)col * src_ld,
                                               (size_t)src_rows * sizeof(double));
      householder_qr(buf, src_rows, n, src_rows);
      const int64_t r = src_rows < n ? src_rows : n;
      for (int col = 0; col < n; ++col)
        for (int64_t i = 0; i < r && i <= col; ++i) Rout[(int64_t)col * n + i] = buf[(int64_t)col * src_rows + i];
      free(buf);
      break;
    }
    double* next = (double*)calloc((size_t)out_rows * n, sizeof(double));
    if (!next) { status = CFIG_ERR_NOMEM; break; }
#pragma omp parallel
    {
      double* buf = (double*)malloc((size_t)tile * n * sizeof(double));
#pragma omp for schedule(dynamic, 1)
      for (int64_t t = 0; t < tiles; ++t) {
        if (!buf) continue;
        const int64_t r0 = t * tile;
        const int64_t tr = r0 + tile < src_rows ? tile : src_rows - r0;
        /* the first output row of tile t: the earlier tiles are all full (tile >= n rows) */
        const int64_t o0 = t * (int64_t)n;
        for (int col = 0; col < n; ++col)
          memcpy(buf + (int64_t)col * tr, src + (int64_t)col * src_ld + r0, (size_t)tr * sizeof(double));
        householder_qr(buf, tr, n, tr);
        const int64_t r = tr < n ? tr : n;
        for (int col = 0; col < n; ++col)
          for (int64_t i = 0; i < r && i <= col; ++i) next[(int64_t)col * out_rows + o0 + i] = buf[(int64_t)col * tr + i];
      }
      if (!buf) status = CFIG_ERR_NOMEM;
      free(buf);
    }
    free(level);
    level = next;
    src = next;
    src_rows = out_rows;
    src_ld = out_rows;
    if (status != CFIG_OK) break;
  }
  free(level);
  return status;
}

/* ------------------------------------------------------------------ entry point */
static void free_ctx(Ctx* c) {
  if (!c->r) return;
  for (int i = 0; i < c->n_rel; ++i) {
    Rel* R = &c->r[i];
    free(R->child); free(R->order); free(R->gstart); free(R->gkey); free(R->pstart); free(R->g2p);
    if (R->cidx)
      for (int q = 0; q < R->n_child; ++q) free(R->cidx[q]);
    free(R->cidx);
    free(R->rows); free(R->theta); free(R->full); free(R->circ); free(R->down); free(R->up);
    free(R->sub_cols);
  }
  free(c->r);
  free(c->col_off);
}

int cfig_max_threads(void) { return omp_get_max_threads(); }

static int in_subtree(const int32_t* parent, int n_rel, int node, int top) {
  for (int v = node, steps = 0; v >= 0 && steps <= n_rel; v = parent[v], ++steps)
    if (v == top) return 1;
  return 0;
}

int cfig_figaro_r(int32_t n_rel, const cfig_relation* rels, const int32_t* parent, int32_t presorted,
                  int32_t n_threads, double* R_out, double* seconds) {
  if (n_rel < 1 || !rels || !parent || !R_out) return CFIG_ERR_INVALID;
  if (n_threads > 0) omp_set_num_threads(n_threads);
  Ctx c;
  memset(&c, 0, sizeof(c));
  c.n_rel = n_rel;
  c.parent = parent;
  c.root = -1;
  c.status = CFIG_OK;
  /* the join tree: one root, every node reaches it */
  for (int i = 0; i < n_rel; ++i) {
    if (parent[i] < -1 || parent[i] >= n_rel || parent[i] == i) return CFIG_ERR_INVALID;
    if (parent[i] < 0) {
      if (c.root >= 0) return CFIG_ERR_INVALID;
      c.root = i;
    }
    if (rels[i].n_rows < 0 || rels[i].n_keys < 0 || rels[i].n_keys > CFIG_MAX_KEYS || rels[i].n_data < 0)
      return CFIG_ERR_INVALID;
    if (rels[i].n_data > 0 && (!rels[i].data || rels[i].ld < rels[i].n_rows)) return CFIG_ERR_INVALID;
  }
  if (c.root < 0) return CFIG_ERR_INVALID;
  for (int i = 0; i < n_rel; ++i)
    if (!in_subtree(parent, n_rel, i, c.root)) return CFIG_ERR_INVALID;
  c.r = (Rel*)calloc((size_t)n_rel, sizeof(Rel));
  c.col_off = (int*)calloc((size_t)n_rel + 1, sizeof(int));
  if (!c.r || !c.col_off) { free_ctx(&c); return CFIG_ERR_NOMEM; }
  for (int i = 0; i < n_rel; ++i) c.col_off[i + 1] = c.col_off[i] + rels[i].n_data;
  c.n_cols = c.col_off[n_rel];
  const int N = c.n_cols;
  int status = CFIG_OK;
  double t0 = omp_get_wtime(), t1, t2, t3, t4;

  /* per relation: children, sort order of the key attributes, subtree columns */
  for (int i = 0; i < n_rel && status == CFIG_OK; ++i) {
    Rel* R = &c.r[i];
    R->rel = &rels[i];
    R->parent = parent[i];
    R->child = (int*)malloc((size_t)n_rel * sizeof(int));
    R->sub_cols = (int*)malloc((size_t)(N > 0 ? N : 1) * sizeof(int));
    if (!R->child || !R->sub_cols) { status = CFIG_ERR_NOMEM; break; }
    for (int j = 0; j < n_rel; ++j)
      if (parent[j] == i) R->child[R->n_child++] = j;
    /* X_p (attributes shared with the parent) first, then the rest, ascending ids */
    int used[CFIG_MAX_KEYS] = {0};
    for (int pass = 0; pass < 2; ++pass) {
      for (;;) {
        int best = -1;
        for (int k = 0; k < rels[i].n_keys; ++k) {
          if (used[k]) continue;
          int shared = 0;
          if (parent[i] >= 0)
            for (int k2 = 0; k2 < rels[parent[i]].n_keys; ++k2)
              if (rels[parent[i]].key_attr[k2] == rels[i].key_attr[k]) shared = 1;
          if ((pass == 0) != (shared == 1)) continue;
          if (best < 0 || rels[i].key_attr[k] < rels[i].key_attr[best]) best = k;
        }
        if (best < 0) break;
        used[best] = 1;
        R->sort_col[R->n_sort] = best;
        R->sort_attr[R->n_sort] = rels[i].key_attr[best];
        ++R->n_sort;
        if (pass == 0) ++R->n_xp;
      }
    }
    for (int j = 0; j < n_rel; ++j)
      if (in_subtree(parent, n_rel, j, i))
        for (int col = 0; col < rels[j].n_data; ++col) R->sub_cols[R->n_sub++] = c.col_off[j] + col;
    R->own_off = 0;
    while (R->own_off < R->n_sub && R->sub_cols[R->own_off] != c.col_off[i]) ++R->own_off;
  }

  /* sort and group every relation (relations and the halves of large sorts as tasks) */
  if (status == CFIG_OK) {
    int* st = (int*)calloc((size_t)n_rel, sizeof(int));
    if (!st) status = CFIG_ERR_NOMEM;
    else {
#pragma omp parallel
#pragma omp single
      for (int i = 0; i < n_rel; ++i) {
#pragma omp task firstprivate(i)
        st[i] = sort_and_group(&c, i, presorted);
      }
      for (int i = 0; i < n_rel; ++i)
        if (st[i] != CFIG_OK && status == CFIG_OK) status = st[i];
      free(st);
    }
  }
  /* the parent group of every child that each group of S_i joins with */
  for (int i = 0; i < n_rel && status == CFIG_OK; ++i) {
    Rel* R = &c.r[i];
    R->cidx = (int64_t**)calloc((size_t)(R->n_child > 0 ? R->n_child : 1), sizeof(int64_t*));
    R->rows = (uint64_t*)malloc((size_t)(R->G + 1) * sizeof(uint64_t));
    R->theta = (uint64_t*)malloc((size_t)(R->G + 1) * sizeof(uint64_t));
    R->full = (uint64_t*)malloc((size_t)(R->G + 1) * sizeof(uint64_t));
    R->circ = (uint64_t*)malloc((size_t)(R->G + 1) * sizeof(uint64_t));
    R->down = (uint64_t*)calloc((size_t)(R->P + 1), sizeof(uint64_t));
    R->up = (uint64_t*)calloc((size_t)(R->P + 1), sizeof(uint64_t));
    if (!R->cidx || !R->rows || !R->theta || !R->full || !R->circ || !R->down || !R->up) {
      status = CFIG_ERR_NOMEM;
      break;
    }
    for (int q = 0; q < R->n_child; ++q) {
      const Rel* Rj = &c.r[R->child[q]];
      int pos[CFIG_MAX_KEYS];
      for (int k = 0; k < Rj->n_xp; ++k) {
        pos[k] = -1;
        for (int k2 = 0; k2 < R->n_sort; ++k2)
          if (R->sort_attr[k2] == Rj->sort_attr[k]) pos[k] = k2;
        if (pos[k] < 0) status = CFIG_ERR_INVALID;
      }
      R->cidx[q] = (int64_t*)malloc((size_t)(R->G + 1) * sizeof(int64_t));
      if (!R->cidx[q]) status = CFIG_ERR_NOMEM;
      if (status != CFIG_OK) break;
      const int64_t G = R->G;
#pragma omp parallel for schedule(static)
      for (int64_t g = 0; g < G; ++g) R->cidx[q][g] = find_in_child(R, g, Rj, pos);
    }
  }
  t1 = omp_get_wtime();

  /* Alg. 3 */
  if (status == CFIG_OK) {
    count_pass1(&c, c.root);
    if (c.status == CFIG_OK) count_pass2(&c, c.root);
    status = c.status;
  }
  t2 = omp_get_wtime();

  /* Alg. 4 */
  Out out;
  out.nb = 0;
  out.b = (Block*)calloc((size_t)2 * n_rel + 1, sizeof(Block));
  if (!out.b && status == CFIG_OK) status = CFIG_ERR_NOMEM;
  if (status == CFIG_OK) status = figaro_node(&c, c.root, &out, NULL);
  t3 = omp_get_wtime();

  /* §7: the triangle of every block, stacked at its global columns, then the stack's R */
  if (status == CFIG_OK) {
    int64_t srows = 0;
    for (int k = 0; k < out.nb; ++k) srows += out.b[k].rows > 0 ? out.b[k].n : 0;
    double* stack = (double*)calloc((size_t)(srows > 0 ? srows : 1) * (size_t)(N > 0 ? N : 1), sizeof(double));
    double* tri = (double*)malloc((size_t)(N > 0 ? N : 1) * (size_t)(N > 0 ? N : 1) * sizeof(double));
    if (!stack || !tri) status = CFIG_ERR_NOMEM;
    int64_t off = 0;
    for (int k = 0; k < out.nb && status == CFIG_OK; ++k) {
      const Block* b = &out.b[k];
      if (b->rows <= 0 || b->n == 0) continue;
      status = tsqr(b->a, b->rows, b->n, b->rows, tri);
      for (int col = 0; col < b->n; ++col)
        for (int r = 0; r < b->n; ++r) stack[(int64_t)b->cols[col] * srows + off + r] = tri[(int64_t)col * b->n + r];
      off += b->n;
    }
    if (status == CFIG_OK) status = tsqr(stack, srows, N, srows, tri);
    if (status == CFIG_OK) {
      /* §2 "Output": row k multiplied by the sign of R_kk (zero counts as positive) */
      for (int i = 0; i < N; ++i) {
        const double s = tri[(int64_t)i * N + i] < 0.0 ? -1.0 : 1.0;
        for (int j = 0; j < N; ++j) R_out[(int64_t)i * N + j] = j >= i ? s * tri[(int64_t)j * N + i] : 0.0;
      }
    }
    free(stack);
    free(tri);
  }
  t4 = omp_get_wtime();
  if (out.b)
    for (int k = 0; k < out.nb; ++k) free(out.b[k].a);
  free(out.b);
  free_ctx(&c);
  if (seconds) {
    seconds[0] = t1 - t0;
    seconds[1] = t2 - t1;
    seconds[2] = t3 - t2;
    seconds[3] = t4 - t3;
  }
  return status;
}
