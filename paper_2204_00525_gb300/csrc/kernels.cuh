// Kernel parameter structs and launcher declarations (internal).
#pragma once

#include "common.cuh"

namespace fig {

// ------------------------------------------------------------------ keys.cu
struct PackParams {
  int n_keys;
  int key_type;
  const void* cols[kMaxKeys];   // key columns in packing order
  long long kmin[kMaxKeys];
  int shift[kMaxKeys];
  int bits[kMaxKeys];
};

// Device buffers of one relation (node of the join tree).  Sizes in brackets are
// allocation bounds; G (groups of X_i) and P (groups of X_p) live in sizes[0..1].
struct NodeBuf {
  uint64_t* key[2];     // [M] packed keys (ping-pong for the sort)
  int32_t* perm[2];     // [M] permutation (ping-pong)
  uint64_t* skey;       // sorted keys (points into key[])
  int32_t* sperm;       // sorted permutation (points into perm[]), null if identity
  int32_t* row_gid;     // [M] group of every sorted row
  int32_t* goff;        // [M+1] group offsets
  uint64_t* gkey;       // [M] group keys
  int32_t* g2p;         // [M] parent group of every group
  int32_t* pgoff;       // [M+1] parent-group offsets (in groups)
  uint64_t* pkey;       // [M] parent-group keys (X_p part)
  int32_t* sizes;       // [4] G, P
  int32_t* itmp;        // [M] scan output scratch
  int32_t* scan_tmp_i;  // scan tile sums
  uint64_t* scan_tmp_u; // scan tile sums (uint64)
  // counts (§5)
  uint64_t* theta;      // [M] Theta_down per group
  uint64_t* full;       // [M] full_join_size per group
  uint64_t* phic;       // [M] Phi_circ per group
  uint64_t* phid;       // [M] Phi_down per parent group
  double* sq_phid;      // [M] sqrt(Phi_down) per parent group (the scales passed to the parent)
  uint64_t* phiu;       // [M] Phi_up per parent group
  uint64_t* theta_incl; // [M] inclusive prefix of theta over groups
  double* sq_phic;      // [M] sqrt(Phi_circ) per group
  double* hrow;         // [M] 1/sqrt(rows) per group
  int32_t* q;           // [n_children * M] index of x_ij among the child's parent groups
  // generalized head/tail inputs (internal nodes)
  double* fac;          // [M * (1 + n_children)] scale factors per group
  double* vw;           // [M * 3] v, W, gamma per group
  double* hf;           // [M] 1 / sqrt(Phi_down) per parent group
  double* sdata;        // [lds x N_i] the data in sorted row order (lds = M rounded up to 8)
  int64_t lds;
  // outputs
  double* heads;        // [M x N_i] col-major, ld M
  double* tails;        // [M x N_i] col-major, ld M  (rows M - G used)
  float* tails32;       // optional float copy for the mixed TSQR
  float* tails32lo;     // refined mixed path: the low float of each double-float tail
  double* data2;        // [M x N_sub] col-major: generalized heads for the parent
  double* gtails;       // [M x N_sub] col-major: generalized tails
  double* rootrows;     // [M x N] col-major (root only)
  // scan tile aggregates
  uint8_t* tflag;       // [n_tiles * max(N_i, N_sub)]
  uint8_t* ttail;       // [n_tiles]: the relation pass's tile holds a tail row (a row after its group's first)
  double* tsum;
  double* tcarry;
  double* ltcarry;      // tile carries of the relation pass (a fused leaf reads them while the
                        // generalized pass of the same node uses tflag/tsum/tcarry)
  uint8_t* lflag;       // [n_tiles * N_sub * 32]: lane exclusive partials of the generalized pass
  double* lsum;
  uint8_t* llflag;      // [n_tiles * N_i * 32]: those of the relation pass (a fused leaf reads
  double* llsum;        //   them while the generalized pass runs)
  int2* coldesc;        // [N_sub] (source kind, source column) for the join
};

void launch_minmax(const void* col, int key_type, int64_t n, long long* dmin, long long* dmax,
                   cudaStream_t st);
void launch_pack(const PackParams& p, int64_t n, uint64_t* key, int32_t* perm, int* err,
                 cudaStream_t st, int64_t* launches);
int64_t radix_tiles(int64_t n);
int64_t radix_hist_elems(int64_t n);
cudaError_t keys_set_attributes();
int radix_sort(uint64_t* key[2], int32_t* perm[2], int64_t n, int bits, int32_t* hist, int32_t* scan_tmp,
               cudaStream_t st, int64_t* launches);
void segment(NodeBuf& b, int64_t n, int rest_bits, cudaStream_t st, int64_t* launches);
void check_sorted(const uint64_t* key, int64_t n, int* err, cudaStream_t st, int64_t* launches);

// ------------------------------------------------------------------ counts.cu
struct ChildLink {
  int n_attr;
  int src_shift[kMaxKeys];   // field position in the parent's packed key
  int bits[kMaxKeys];
  int dst_shift[kMaxKeys];   // field position in the child's X_p key
  const uint64_t* pkey;      // child's parent-group keys [P_c], strictly increasing
  const int32_t* sizes;      // child's sizes (P_c = sizes[1])
  const uint64_t* phid;      // child's Phi_down [P_c]
  double* sq_phid;           // child's sqrt(Phi_down) [P_c] (written with the division below)
  uint64_t* phiu;            // child's Phi_up [P_c] (accumulated, then divided)
  int32_t* q;                // [G_i] out
  const double* data;        // child's table of heads passed up (leaf: heads, else data2)
  int64_t ld;                // its leading dimension
};

struct CountParams {
  int n_child;
  ChildLink ch[kMaxChildren];
  int is_root;
  int require_reduced;
  int64_t M;
  const uint64_t* gkey;
  const int32_t* goff;
  const int32_t* g2p;
  const int32_t* pgoff;
  const int32_t* sizes;
  uint64_t* theta;
  uint64_t* full;
  uint64_t* phic;
  uint64_t* phid;
  const uint64_t* phiu;
  const uint64_t* theta_incl;
  double* sq_phic;
  double* hrow;
  double* fac;
  double* vw;
  double* hf;
};

void counts_clear(NodeBuf& b, int64_t bound, cudaStream_t st, int64_t* launches);
void counts_pass1(const CountParams& p, cudaStream_t st, int* err, int64_t* launches);
void counts_pass2(const CountParams& p, cudaStream_t st, int* err, int64_t* launches);
void counts_finalize_child(const ChildLink& c, int64_t bound, cudaStream_t st, int64_t* launches);
void join_prep(const CountParams& p, cudaStream_t st, int64_t* launches);

// ------------------------------------------------------------------ heads.cu
constexpr int kHtItems = 8;
constexpr int kHtTile = 32 * kHtItems;   // elements per warp tile
inline int64_t ht_tiles(int64_t n) { return (n + kHtTile - 1) / kHtTile; }

struct LeafParams {
  int64_t M;
  int N;
  const double* data;
  int64_t rs, cs;            // element (input row r, column c) at data[r * rs + c * cs]
  const int32_t* perm;       // sorted position -> input row; null means identity
  double* sdata;             // with perm: the data in sorted order, written by the first pass
  int64_t lds;               //   and read back by the last (leading dimension lds, a multiple of 8)
  const int32_t* row_gid;
  const int32_t* goff;
  const double* sq_phic;
  const double* hrow;
  const double2* beta;       // {beta_p, p beta_p}, beta_p = 1 / sqrt(p (p + 1)), every position p < M
  int64_t beta_len;
  double* tails;
  int64_t ldt;
  float* tails32;            // mixed precision: float tails (leading dimension ldt) instead of tails
  float* tails32lo;          // with tails32, optional: the low parts (tail = tails32 + tails32lo)
  int sorted_ready;          // 1: sdata already holds the data in sorted order (k_rows_gather)
  int mixed;                 // mixed precision: double-float prefix sums, float tails
  double* heads;
  int64_t ldh;
  uint8_t* tflag;
  double* tsum;
  double* tcarry;
  uint8_t* lflag;
  double* lsum;
  uint8_t* ttail;            // per tile: 1 if it holds a tail row (set by the first pass); null: unknown
  int64_t n_tiles;
};

struct GenParams {
  int N;                     // N_sub
  int n_child;
  int64_t M;                 // allocation bound of groups
  const int32_t* sizes;      // G at [0], P at [1]
  const int32_t* g2p;
  const int32_t* pgoff;
  const double* heads;       // own heads [G x N_i], ld ldh
  int64_t ldh;
  const double* fac;
  const double* vw;
  const double* hf;
  const int32_t* q;          // [n_child * M]
  const double* cdata[kMaxChildren];
  int64_t cld[kMaxChildren];
  const double* crow[kMaxChildren];   // row-major copies of cdata (row stride cnp)
  int cnp[kMaxChildren];
  const double* jdata;       // the node's joined Data [G x N_sub], ld ldj (k_gen_gather)
  int64_t ldj;
  const int2* coldesc;
  double* gtails;            // [G - P x N_sub], ld M
  float* gtails32;           // mixed path (not refined): float generalized tails instead, ld M
  double* data2;             // [P x N_sub], ld M
  double* rootrows;          // root only: [G x N], ld M
  uint8_t* tflag;
  double* tsum;
  double* tcarry;
  uint8_t* lflag;
  double* lsum;
  int64_t n_tiles;
  int is_root;
};

void beta_table(double2* beta, int64_t len, cudaStream_t st);
// Row moves for the gathers: a row-major copy of a column-major table (rows beyond *live,
// if given, are skipped), and the sorted copy out[c][e] = rows[perm[e]][c].
cudaError_t rows_of_set_attributes();   // the slab copy's shared memory (up to 133 KB)
void rows_of(const double* src, int64_t ld, int64_t bound, const int32_t* live, int cols, double* dst, int np,
             cudaStream_t st, int64_t* launches);
void rows_gather(const double* rows, int64_t rs, const int32_t* perm, int64_t M, int cols, double* out,
                 int64_t ldo, cudaStream_t st, int64_t* launches);
inline int row_pitch(int cols) { return (cols + 1) & ~1; }
// Whole-row gathers move about 4 x 8 N bytes per row (copy in, copy out, gather in, sorted
// copy out) against N sectors of 32 bytes for the plain gather, part of which hit L2 while
// the table is not much larger than L2: they pay for tables of 1 GiB and more.
inline bool row_gather_pays(int64_t rows, int cols) { return cols > 0 && (double)rows * cols * 8.0 >= 1073741824.0; }
// Heads of a relation (first pass, tile carries, the fix-up of groups that cross a tile
// start) and, for tails blocks that are stored, the tails (last pass).
void leaf_heads(const LeafParams& p, cudaStream_t st, int64_t* launches);
void leaf_tails(const LeafParams& p, cudaStream_t st, int64_t* launches);
void gen_heads_tails(const GenParams& p, cudaStream_t st, int64_t* launches);

// ------------------------------------------------------------------ tsqr.cu
enum BlockKind : int { BLK_TAILS = 0, BLK_GEN = 1, BLK_ROOT = 2, BLK_FIXED = 3 };

struct TsqrBlock {
  const double* ptr;         // col-major, leading dimension ld
  const float* ptr32;        // mixed-precision tails: float rows in place of ptr
  int64_t ld;
  int n;                     // columns
  int kind;
  int64_t M;
  const int32_t* sizes;      // rows = M - G (tails), G - P (gen), G (root), M (fixed)
  int64_t bound;             // allocation bound of rows
  int tile;                  // leaf tile rows
  int fan;                   // triangles merged per reduce tile
  int levels;                // reduce levels after the leaf
  double* tri[2];            // ping-pong triangle buffers [bound tiles x n x n]
  int top;                   // buffer holding the last level
  int nreg;                  // register (warp-per-tile) path: padded column count; 0 = not used
  int64_t warp_min;          // register path: levels with at least this many tiles (else block-per-tile)
  bool prio;                 // on the critical path: its stream gets the high priority
  bool givens;               // leaf by per-thread Givens rotations on b.tile-row chunks
  const int* cols;           // device [n]: global column of each block column
  void* scratch;             // block path: global tile slots when a tile exceeds shared memory;
                             // fold path: one n x n triangle per thread block when T is not in shared memory
  bool fold;                 // n > 32: streamed fold (b.tile = chunk rows, b.seg chunks per leaf triangle)
  bool fold_tsmem;           // fold path: the running triangle lives in shared memory
  int64_t seg;               // fold path: at most this many chunks folded into one leaf triangle
  int64_t fold_g0;           // fold path: thread blocks of the leaf launch
  bool fold_tc;              // fold path, float leaf: panels with tensor-core trailing updates
  bool fold_tc5;             // fold path, float leaf on tcgen05 (k_tsqr_fold_tc, 128-row chunks)
  int* err;                  // the plan's device error word (bounded waits report TIMEOUT)
  bool fused;                // tails block formed inside its leaf kernel (tails_qr): rows = M sorted rows
  int fold_res;              // fold path: most thread blocks of a launch (T slots when T is global)
};

// A TSQR plan override chosen by the autotuner; 0 keeps the planner's rule for that field.
struct TsqrTune {
  int fold_budget_kib;       // fold path: shared memory of a thread block (chunk height, blocks per SM)
  int seg_cap;               // fold path: at most this many chunks folded into one leaf triangle
  int fan;                   // tree levels: triangles reduced per unit
  int64_t warp_min;          // register path: levels with at least this many tiles take the warp kernel
};

// tsqr_tc.cu: the float leaf on the 5th-generation tensor cores
size_t fold_tc_smem(int n);
bool fold_tc_fits(int n);
void launch_fold_tc(const TsqrBlock& b, double* tri_out, int* err, cudaStream_t st);
cudaError_t fold_tc_set_attributes();

void tsqr_plan_block(TsqrBlock& b, bool mixed, bool givens = false, bool tcgen05 = false,
                     const TsqrTune* tune = nullptr);
// The fastest of the candidate plans of block b (its width, kind and row bound) measured on
// synthetic rows (at most 2^30 cells) at plan time; results are kept per (precision, leaf,
// width, row bucket) for the process.  Returns the override (zero: the rule's plan won).
TsqrTune tsqr_autotune(const TsqrBlock& b, bool mixed, bool givens, bool tcgen05);
// tails_qr_f64.cu: the tails of a relation with <= 32 data columns formed in registers and
// triangularised by the leaf (the block's tri[0]), after leaf_heads has made the carries
void tails_qr(const LeafParams& p, const TsqrBlock& b, cudaStream_t st, int64_t* launches);
int64_t tsqr_tri_elems(const TsqrBlock& b);
int64_t tsqr_scratch_elems(const TsqrBlock& b, bool mixed);
void tsqr_leaf(const TsqrBlock& b, bool mixed, cudaStream_t st, int64_t* launches);
void tsqr_reduce(TsqrBlock& b, bool mixed, cudaStream_t st, int64_t* launches);
void tsqr_final(const TsqrBlock* blocks_dev, int n_blocks, TsqrBlock& stack_blk, double* R, int64_t ldr,
                cudaStream_t st, int64_t* launches);
double tsqr_leaf_flops(int64_t rows, int n);
cudaError_t tsqr_set_attributes();

// ------------------------------------------------------------------ svd.cu
// One Jacobi SVD: R (row-major, ldr), work arrays W and V (N x N each, used when they do not
// fit in shared memory), sigma[N] descending, Vout (row-major N x N), the error word, the
// sweep limit; with k > 0 also the first k columns of Vout (comp, row-major N x k) and
// sigma^2 (eig[k]).
struct JacobiTask {
  const double* R;
  int64_t ldr;
  int N;
  double* W;
  double* V;
  double* sigma;
  double* Vout;
  int* err;
  int max_sweeps;
  double* comp;
  double* eig;
  int k;
};
constexpr size_t kJacobiSmemCap = 200 * 1024;
constexpr int kSvdDefaultSweeps = 40;     // svd_max_sweeps = 0
__host__ __device__ inline size_t jacobi_smem(int N) { return (2 * (size_t)N * N + N) * sizeof(double); }
cudaError_t svd_set_attributes();
// every task's SVD in one launch (one thread block each); max_n = the largest N
void jacobi_svd_batch(const JacobiTask* tasks_dev, int n, int max_n, cudaStream_t st, int64_t* launches);
// aux (jacobi_aux_elems doubles, or null): the scratch of the cluster version used for R
// too wide for one block's shared memory
void jacobi_svd(const double* R, int64_t ldr, int N, double* W, double* V, double* sigma,
                double* Vout, int* err, cudaStream_t st, int64_t* launches, int max_sweeps,
                double* aux = nullptr);
inline int64_t jacobi_aux_elems(int N) { return 3 * 512 + N + 2; }
void square_values(const double* s, double* out, int k, cudaStream_t st, int64_t* launches);

// figaro_last_error's message for entry points outside api.cu: record_error sets it and
// returns `code`; clear_error empties it at the start of a call.
int record_error(int code, const char* msg);
void clear_error();
void join_colsum(const double* heads, int64_t ldh, const int32_t* goff, const double* hrow, const uint64_t* phic,
                 const int32_t* sizes, int n, double* out, cudaStream_t st, int64_t* launches);
void join_size(const uint64_t* full, const int32_t* sizes, unsigned long long* out, cudaStream_t st,
               int64_t* launches);
void center_gram(const double* R, int N, const double* colsum, const unsigned long long* join_size, double* C,
                 cudaStream_t st, int64_t* launches);

// ------------------------------------------------------------------ refine.cu
cudaError_t refine_set_attributes();
int64_t gram_partial_elems(const TsqrBlock& b);
void gram_block(const TsqrBlock& b, const float* lo32, double* partial, cudaStream_t st, int64_t* launches);
void gram_add(const TsqrBlock& b, const double* partial, double* G, int N, cudaStream_t st, int64_t* launches);
void refine_r(double* R, int64_t ldr, const double* G, int N, double* W1, double* W2, int* ok, cudaStream_t st,
              int64_t* launches);

// ------------------------------------------------------------------ grad.cu
// One relation's view for the gradient kernels (see grad.cu).
struct GradNode {
  int N, Ni, col_off, n_child, is_root;
  int64_t M;
  const int32_t* sizes;      // G, P
  const int32_t* goff;
  const int32_t* g2p;
  const int32_t* row_gid;
  const int32_t* perm;       // sorted position -> input row (null: identity)
  const double* heads;       // finished heads S(g) / sqrt(rows), [col][g], ld ldh
  int64_t ldh;
  const double* hrow;        // 1 / sqrt(rows)
  const uint64_t* phic;      // Phi_circ per group
  const uint64_t* phiu;      // Phi_up per parent group (not the root)
  const int32_t* q;          // [child][M]: index of the group's key among the child's X_p keys
  const uint64_t* cphid[kMaxChildren];   // children's Phi_down
  const double* cup[kMaxChildren];       // children's up messages [col][x], ld cld
  int64_t cld[kMaxChildren];
  const uint8_t* colkind;    // [N]: 0 own column, 1 + c child c's subtree, 255 the rest
  double* up;                // own up message [col][x_p], ld ldu
  int64_t ldu;
  const double* dn;          // own down message [col][x_p], ld ldd (not the root)
  int64_t ldd;
  const double* W;           // N x N row-major
  double* phi;               // [a][g], ld M
  const double* data;        // the relation's data: element (row r, column b) at r * rs + b * cs
  int64_t rs, cs;
  const double* sdata;       // the forward's copy of the data in sorted order (or null), ld lds
  int64_t lds;
  double* grad;              // output, column-major, ld ldg (input row order)
  int64_t ldg;
};

void grad_w(const double* R, int64_t ldr, const double* Rbar, int64_t ldb, int N, double* W, double* T1, double* T2,
            int* err, cudaStream_t st);
void grad_clear(double* a, int64_t ld, const int32_t* sizes, int N, int64_t bound, cudaStream_t st);
void grad_up(const GradNode& g, int64_t bound, cudaStream_t st);
void grad_down(const GradNode& g, int j, double* dn_child, int64_t ld_child, int64_t bound, cudaStream_t st);
void grad_rows(const GradNode& g, int64_t bound, cudaStream_t st);

// ------------------------------------------------------------------ shared device helpers
// X <- R^-1 X for upper-triangular R (row-major, ld ldr) and a row-major N x N X, by one
// block: row i is final after its division, then the rows above lose R[i2][i] times it.
__device__ inline void tri_solve_upper_rows(const double* R, int64_t ldr, double* X, int N) {
  // X <- R^-1 X for upper-triangular R (X row-major N x N), all columns at once
  const int t = threadIdx.x, nt = blockDim.x;
  for (int i = N - 1; i >= 0; --i) {
    const double ri = 1.0 / R[(int64_t)i * ldr + i];
    for (int c = t; c < N; c += nt) X[(int64_t)i * N + c] *= ri;
    __syncthreads();
    for (int64_t idx = t; idx < (int64_t)i * N; idx += nt) {
      const int i2 = (int)(idx / N), c = (int)(idx % N);
      X[(int64_t)i2 * N + c] = fma(-R[(int64_t)i2 * ldr + i], X[(int64_t)i * N + c], X[(int64_t)i2 * N + c]);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ proj.cu
constexpr int kMaxRel = 32;       // relations a projection can enumerate

struct ProjNode {
  int n_child;
  int child[kMaxChildren];   // positions of the children in the node array
  int64_t M;
  const int32_t* sizes;
  const int32_t* goff;
  const int32_t* pgoff;
  const uint64_t* theta;       // Theta_down per group
  const uint64_t* theta_incl;  // its inclusive prefix over the groups
  const uint64_t* phid;        // Phi_down per X_p group
  const int32_t* q;            // [child][M]
  const int32_t* perm;
  const double* P;             // [input row][k] projected rows, or null (no data columns)
};

void tri_inverse(const double* R, int64_t ldr, int N, double* X, int* err, cudaStream_t st);
void scale_v(const double* V, const double* sigma, int N, int k, bool divide, double* X, int* err, cudaStream_t st);
void proj_rows(const double* data, int64_t rs, int64_t cs, int64_t M, int Ni, const double* X, int64_t ldx,
               int col_off, int k, double* P, cudaStream_t st);
void project(const ProjNode* nodes, int r, int k, uint64_t total, double* out, int64_t ldo, cudaStream_t st);

}  // namespace fig

