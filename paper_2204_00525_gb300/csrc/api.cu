// C ABI (include/figaro.h): validation, planning, workspace and the per-call pipeline.
//
// figaro_plan checks the database and join tree (§2), fixes the key packing and sizes
// one device arena from the bounds of the Theorem of §6 (R0 has at most sum M_i rows;
// groups never outnumber rows).  Every compute call then enqueues, on one stream and
// without host synchronisation until a final error-word read:
//   pack + radix sort + segmentation of every relation        (§5 sort assumption)
//   Alg. 3 pass 1 (post-order) and pass 2 (pre-order)         (§5)
//   heads_and_tails of every relation                         (Alg. 4, Alg. 2)
//   process_and_join_children + project_away, root Data       (Alg. 4, post-order)
//   TSQR of the R0 blocks and the final QR                    (§7)
//   Jacobi SVD of R for figaro_svd / figaro_pca               (§8.2-8.3)
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace fig {

static thread_local std::string g_last_error;

static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

// The same record for entry points defined in other translation units.
int record_error(int code, const char* msg) { return fail(code, msg ? msg : ""); }
void clear_error() { g_last_error.clear(); }

#define FIG_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(FIGARO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

constexpr int kStages = 8;

struct Node {
  int id = 0, parent = -1;
  std::vector<int> children;
  bool leaf = true, root = false;
  int64_t M = 0;
  int K = 0, N = 0, key_type = 0, layout = 0;
  int64_t ld = 0;
  std::vector<int> key_attr;
  std::vector<const void*> key_ptr;     // as given by the caller
  const double* data = nullptr;         // as given by the caller
  std::vector<void*> dkey;              // device copies (host-memory mode)
  double* ddata = nullptr;              // device copy (host-memory mode)
  double* rowin = nullptr;              // row-major copy of the data for the sorted gather
  double* crow = nullptr;               // row-major copy of the table passed to the parent
  int crow_pitch = 0;
  float* gtails32 = nullptr;            // mixed path (not refined): float generalized tails
  double* jdata = nullptr;              // joined Data of process_and_join_children (internal)
  int64_t ldj = 0;
  // packing: X_p attributes (ascending id) in the high bits, then the rest
  std::vector<int> pack_attr, pack_col, shift;
  int bits = 0, rest_bits = 0;
  // columns
  int col_off = 0, N_sub = 0;
  std::vector<int> sub_cols;
  std::vector<int2> coldesc;
  NodeBuf b{};
  int64_t n_tiles = 0;
  ChildLink link[kMaxChildren]{};      // one per child (filled for the parent's passes)
  int32_t* radix_hist = nullptr;        // per relation: the sorts run concurrently
  int32_t* radix_tmp = nullptr;
  int blk_tails = -1, blk_gen = -1;     // R0 blocks fed by this relation (index into blocks)
  // gradients (options.gradients): messages over the join tree, per-group shares
  int64_t pbound = 1;                   // bound on the number of X_p groups
  double* g_up = nullptr;               // [N][pbound]
  double* g_dn = nullptr;               // [N][pbound]
  double* g_phi = nullptr;              // [N_i][M]
  uint8_t* g_colkind = nullptr;         // [N]
  std::vector<uint8_t> colkind;
};

}  // namespace fig

struct figaro_plan_s {
  std::vector<fig::Node> nodes;
  int root = 0, N = 0;
  figaro_options opt{};
  cudaStream_t st = nullptr;
  int device = 0;
  std::vector<int> post, pre;
  std::vector<long long> amin;
  std::vector<int> abits;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  int* err_dev = nullptr;
  int* err_host = nullptr;             // pinned: [0] error word, [4 + 4 i ..] sizes of node i
  double2* beta = nullptr;
  int64_t beta_len = 0;
  std::vector<fig::TsqrBlock> blocks;
  fig::TsqrBlock* blocks_dev = nullptr;
  int stack_rows = 0;
  double* stack = nullptr;
  fig::TsqrBlock stack_blk{};          // the stacked block triangles (final QR)
  std::vector<cudaStream_t> side;      // one stream per R0 block: the TSQR chains run concurrently
  std::vector<cudaEvent_t> side_done;
  std::vector<cudaStream_t> nstream;   // one stream per relation: sort, segmentation, heads/tails
  cudaStream_t copy_st = nullptr;      // host-memory mode: input copies, keys first
  std::vector<cudaEvent_t> ev_keys, ev_data, ev_seg, ev_leaf, ev_gen;
  cudaEvent_t ev_counts = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph_exec = nullptr;  // captured R pipeline (see run_r)
  cudaStream_t exec = nullptr;           // the plan's own stream: the graph runs here
  cudaEvent_t join_in = nullptr, join_out = nullptr;
  bool graph_failed = false;
  int64_t graph_launches = 0;
  std::vector<cudaEvent_t> leaf_ev;    // stage timing: start/end of every block's leaf kernel
  std::vector<double> block_leaf_ms;   // stage timing: leaf time per block since the last reset
  std::vector<int64_t> block_rows;     // rows of every block in the last call
  double* Rtmp = nullptr;
  double* svdW = nullptr;
  double* svdV = nullptr;
  double* svdAux = nullptr;             // the cluster Jacobi's scratch (wide R)
  double* sig = nullptr;
  double* Vtmp = nullptr;
  double* hostbuf_dev = nullptr;        // staging for host-memory outputs
  int64_t launches = 0;
  cudaEvent_t ev[fig::kStages + 1]{};
  double stage_ms[fig::kStages]{};
  int64_t stage_launch[fig::kStages]{};
  int64_t input_cells = 0, input_bytes = 0;
  double leaf_flops = 0.0;
  int64_t r0_rows = 0;
  // refinement of the mixed R (FIGARO_PREC_MIXED_REFINED)
  std::vector<double*> gram_partial;   // per block: per-CTA partial Gram matrices
  std::vector<const float*> block_lo32; // per block: low floats of its rows (tails blocks)
  std::vector<fig::LeafParams> block_lp; // per block: the relation's pass parameters (fused tails blocks)
  double* gram = nullptr;              // A^T A (N x N)
  double* refine_w = nullptr;          // two N x N work arrays
  int* refine_ok = nullptr;            // device: 1 when the last refinement was applied
  int refined = 0;
  double* grad_w = nullptr;            // gradients: W and two N x N work arrays
  double* colsum = nullptr;            // centred PCA: column sums of A, |J|, scatter matrix
  unsigned long long* jsize = nullptr;
  double* scatter = nullptr;
  bool pending = false;                // figaro_qr_r_async issued, figaro_plan_sync not yet
};

struct figaro_batch_s {
  std::vector<figaro_plan_t> plans;
  cudaStream_t st = nullptr;           // the batch graph runs here
  cudaGraphExec_t exec = nullptr;
  int* status_dev = nullptr;           // [n] every instance's error word, gathered
  int* status_host = nullptr;          // pinned copy
  fig::JacobiTask* tasks_dev = nullptr; // the PCA instances' SVDs, one batched launch
  int64_t launches = 0;
};

namespace fig {

// ------------------------------------------------------------------ arena
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(int64_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += (size_t)(count > 0 ? count : 1) * sizeof(T);
    return p;
  }
};

static int bits_for(unsigned long long range) {
  int b = 0;
  while (b < 64 && (range >> b) != 0ull) ++b;
  return b;
}

// Lays out every device buffer of the plan; with a.base == nullptr only measures.
static void layout(figaro_plan_s& P, Arena& a) {
  const bool mixed = P.opt.precision != FIGARO_PREC_FP64;
  const bool refine = P.opt.precision == FIGARO_PREC_MIXED_REFINED;
  int64_t maxM = 1;
  for (auto& n : P.nodes) maxM = std::max(maxM, n.M);
  P.err_dev = a.take<int>(4);
  P.beta_len = maxM + 1;                 // every position of every group: no fallback path
  P.beta = a.take<double2>(P.beta_len);
  for (auto& n : P.nodes) {
    NodeBuf& b = n.b;
    const int64_t M = n.M;
    const int nch = (int)n.children.size();
    const int64_t rh = radix_hist_elems(M);
    n.radix_hist = a.take<int32_t>(2 * rh);
    n.radix_tmp = a.take<int32_t>(scan_tmp_elems(rh));
    if (P.opt.mem == FIGARO_MEM_HOST) {
      for (int k = 0; k < n.K; ++k)
        n.dkey[k] = n.key_type == FIGARO_KEY_I32 ? (void*)a.take<int32_t>(M) : (void*)a.take<int64_t>(M);
      n.ddata = a.take<double>(n.layout == FIGARO_COL_MAJOR ? n.ld * n.N : M * n.ld);
    }
    b.key[0] = a.take<uint64_t>(M);
    b.key[1] = a.take<uint64_t>(M);
    b.perm[0] = a.take<int32_t>(M);
    b.perm[1] = a.take<int32_t>(M);
    b.row_gid = a.take<int32_t>(M);
    b.goff = a.take<int32_t>(M + 1);
    b.gkey = a.take<uint64_t>(M);
    b.g2p = a.take<int32_t>(M);
    b.pgoff = a.take<int32_t>(M + 1);
    b.pkey = a.take<uint64_t>(M);
    b.sizes = a.take<int32_t>(4);
    b.itmp = a.take<int32_t>(M);
    b.scan_tmp_i = a.take<int32_t>(scan_tmp_elems(M));
    b.scan_tmp_u = a.take<uint64_t>(scan_tmp_elems(M));
    b.theta = a.take<uint64_t>(M);
    b.full = a.take<uint64_t>(M);
    b.phic = a.take<uint64_t>(M);
    b.phid = a.take<uint64_t>(M);
    b.sq_phid = a.take<double>(M);
    b.phiu = a.take<uint64_t>(M);
    b.theta_incl = a.take<uint64_t>(M);
    b.sq_phic = a.take<double>(M);
    b.hrow = a.take<double>(M);
    b.q = a.take<int32_t>((int64_t)std::max(nch, 1) * M);
    b.fac = a.take<double>(M * (1 + nch));
    b.vw = a.take<double>(3 * M);
    b.hf = a.take<double>(M);
    b.lds = (M + 7) & ~int64_t(7);
    b.sdata = a.take<double>(b.lds * std::max(n.N, 1));
    b.heads = a.take<double>(M * std::max(n.N, 1));
    // a tails block formed inside its leaf kernel is never stored
    const bool fused = n.blk_tails >= 0 && P.blocks[n.blk_tails].fused;
    b.tails = fused ? nullptr : a.take<double>(M * std::max(n.N, 1));
    b.tails32 = (mixed && !fused) ? a.take<float>(M * std::max(n.N, 1)) : nullptr;
    b.tails32lo = refine ? a.take<float>(M * std::max(n.N, 1)) : nullptr;
    if (!n.leaf && !n.root) {
      b.data2 = a.take<double>(M * n.N_sub);
      b.gtails = a.take<double>(M * n.N_sub);
      n.gtails32 = (mixed && !refine) ? a.take<float>(M * n.N_sub) : nullptr;
      n.ldj = (M + 7) & ~int64_t(7);
      n.jdata = a.take<double>(n.ldj * std::max(n.N_sub, 1));
    }
    if (!n.root) {                        // the parent gathers whole rows of this table
      n.crow_pitch = row_pitch(std::max(n.leaf ? n.N : n.N_sub, 1));
      n.crow = a.take<double>(M * n.crow_pitch);
    }
    // the sorted copy of a large table is gathered by whole rows: column-major data gets a
    // row-major copy first
    n.rowin = (!P.opt.presorted && n.layout == FIGARO_COL_MAJOR && row_gather_pays(M, n.N))
                  ? a.take<double>(M * row_pitch(n.N)) : nullptr;
    if (n.root) b.rootrows = a.take<double>(M * n.N_sub);
    n.n_tiles = ht_tiles(M);
    const int wide = std::max(std::max(n.N, n.N_sub), 1);
    b.tflag = a.take<uint8_t>(n.n_tiles * wide);
    b.ttail = a.take<uint8_t>(n.n_tiles);
    b.tsum = a.take<double>(n.n_tiles * wide);
    b.tcarry = a.take<double>(n.n_tiles * wide);
    b.ltcarry = a.take<double>(n.n_tiles * std::max(n.N, 1));
    b.lflag = a.take<uint8_t>(n.n_tiles * std::max(n.N_sub, 1) * 32);
    b.lsum = a.take<double>(n.n_tiles * std::max(n.N_sub, 1) * 32);
    b.llflag = a.take<uint8_t>(n.n_tiles * std::max(n.N, 1) * 32);
    b.llsum = a.take<double>(n.n_tiles * std::max(n.N, 1) * 32);
    b.coldesc = a.take<int2>(std::max(n.N_sub, 1));
    if (P.opt.gradients) {
      n.g_up = a.take<double>((int64_t)P.N * n.pbound);
      n.g_dn = a.take<double>((int64_t)P.N * n.pbound);
      n.g_phi = a.take<double>(M * std::max(n.N, 1));
      n.g_colkind = a.take<uint8_t>(P.N);
    }
  }
  for (auto& blk : P.blocks) {
    blk.tri[0] = a.take<double>(tsqr_tri_elems(blk));
    blk.tri[1] = a.take<double>(tsqr_tri_elems(blk));
    blk.cols = a.take<int>(blk.n);
    const int64_t sc = tsqr_scratch_elems(blk, mixed);
    blk.scratch = sc ? a.take<double>(sc) : nullptr;
  }
  {
    const int64_t sc = tsqr_scratch_elems(P.stack_blk, false);
    P.stack_blk.scratch = sc ? a.take<double>(sc) : nullptr;
  }
  P.blocks_dev = a.take<TsqrBlock>((int64_t)P.blocks.size());
  P.stack = a.take<double>((int64_t)P.stack_rows * P.N);
  P.stack_blk.ptr = P.stack;
  P.stack_blk.tri[0] = a.take<double>(tsqr_tri_elems(P.stack_blk));
  P.stack_blk.tri[1] = a.take<double>(tsqr_tri_elems(P.stack_blk));
  const int64_t NN = (int64_t)P.N * P.N;
  P.Rtmp = a.take<double>(NN);
  if (P.opt.gradients) P.grad_w = a.take<double>(3 * NN);
  P.colsum = a.take<double>(P.N);
  P.jsize = a.take<unsigned long long>(1);
  P.scatter = a.take<double>(NN);
  P.gram_partial.assign(P.blocks.size(), nullptr);
  if (refine) {
    for (size_t bi = 0; bi < P.blocks.size(); ++bi) P.gram_partial[bi] = a.take<double>(gram_partial_elems(P.blocks[bi]));
    P.gram = a.take<double>(NN);
    P.refine_w = a.take<double>(2 * NN);
    P.refine_ok = a.take<int>(1);
  }
  P.svdW = a.take<double>(NN);
  P.svdV = a.take<double>(NN);
  P.svdAux = a.take<double>(jacobi_aux_elems(P.N));
  P.sig = a.take<double>(P.N);
  P.Vtmp = a.take<double>(NN);
  P.hostbuf_dev = a.take<double>(NN + P.N);
}

// ------------------------------------------------------------------ validation + planning
static int build(figaro_plan_s& P, const figaro_join_tree* tree) {
  const int r = tree->n_rel;
  if (r < 1 || !tree->rels || !tree->parent) return fail(FIGARO_ERR_INVALID_ARG, "empty database");
  P.nodes.resize(r);
  int roots = 0;
  for (int i = 0; i < r; ++i) {
    const figaro_relation& R = tree->rels[i];
    Node& n = P.nodes[i];
    n.id = i;
    n.parent = tree->parent[i];
    if (n.parent < -1 || n.parent >= r || n.parent == i)
      return fail(FIGARO_ERR_INVALID_TREE, "parent index out of range in relation " + std::to_string(i));
    if (n.parent < 0) { ++roots; P.root = i; }
    if (R.n_rows < 1 || R.n_rows > 0x7fffffffLL)
      return fail(FIGARO_ERR_INVALID_ARG, "n_rows must be in [1, 2^31-1] (relation " + std::to_string(i) + ")");
    if (R.n_keys < 0 || R.n_keys > kMaxKeys)
      return fail(R.n_keys < 0 ? FIGARO_ERR_INVALID_ARG : FIGARO_ERR_UNSUPPORTED, "n_keys must be in [0, 8]");
    if (R.n_data < 0) return fail(FIGARO_ERR_INVALID_ARG, "n_data < 0");
    if (R.key_type != FIGARO_KEY_I64 && R.key_type != FIGARO_KEY_I32) return fail(FIGARO_ERR_INVALID_ARG, "key_type");
    if (R.layout != FIGARO_COL_MAJOR && R.layout != FIGARO_ROW_MAJOR) return fail(FIGARO_ERR_INVALID_ARG, "layout");
    if (R.n_keys > 0 && (!R.key_attr || !R.key_cols)) return fail(FIGARO_ERR_INVALID_ARG, "null key arrays");
    if (R.n_data > 0 && !R.data) return fail(FIGARO_ERR_INVALID_ARG, "null data");
    if (R.layout == FIGARO_COL_MAJOR ? R.ld < R.n_rows : R.ld < R.n_data)
      return fail(FIGARO_ERR_INVALID_ARG, "leading dimension too small (relation " + std::to_string(i) + ")");
    n.M = R.n_rows;
    n.K = R.n_keys;
    n.N = R.n_data;
    n.key_type = R.key_type;
    n.layout = R.layout;
    n.ld = R.ld;
    n.data = R.data;
    for (int k = 0; k < n.K; ++k) {
      if (R.key_attr[k] < 0) return fail(FIGARO_ERR_INVALID_ARG, "negative attribute id");
      if (!R.key_cols[k]) return fail(FIGARO_ERR_INVALID_ARG, "null key column");
      for (int kk = 0; kk < k; ++kk)
        if (R.key_attr[kk] == R.key_attr[k]) return fail(FIGARO_ERR_INVALID_ARG, "repeated attribute in a relation");
      n.key_attr.push_back(R.key_attr[k]);
      n.key_ptr.push_back(R.key_cols[k]);
    }
    n.dkey.assign(n.K, nullptr);
    P.input_cells += n.M * (n.N + n.K);
    P.input_bytes += n.M * (8 * (int64_t)n.N + (n.key_type == FIGARO_KEY_I32 ? 4 : 8) * (int64_t)n.K);
  }
  if (roots != 1) return fail(FIGARO_ERR_INVALID_TREE, "the join tree must have exactly one root");
  for (int i = 0; i < r; ++i)
    if (P.nodes[i].parent >= 0) P.nodes[P.nodes[i].parent].children.push_back(i);
  for (auto& n : P.nodes) {
    if ((int)n.children.size() > kMaxChildren) return fail(FIGARO_ERR_UNSUPPORTED, "more than 8 children");
    n.leaf = n.children.empty();
    n.root = n.parent < 0;
  }
  // connectivity and acyclicity: a DFS from the root must reach every node once
  {
    std::vector<int> seen(r, 0), stack{P.root};
    while (!stack.empty()) {
      int u = stack.back();
      stack.pop_back();
      if (seen[u]++) return fail(FIGARO_ERR_INVALID_TREE, "parent[] has a cycle");
      P.pre.push_back(u);
      for (int c : P.nodes[u].children) stack.push_back(c);
    }
    for (int i = 0; i < r; ++i)
      if (!seen[i]) return fail(FIGARO_ERR_INVALID_TREE, "parent[] is not connected");
    // post-order: reverse of a pre-order that visits children after the parent works
    // as long as every child precedes its parent, which the reverse guarantees.
    P.post.assign(P.pre.rbegin(), P.pre.rend());
  }
  // attributes: at least two holders, holders connected in the tree (§2 join tree)
  int max_attr = -1;
  for (auto& n : P.nodes)
    for (int a : n.key_attr) max_attr = std::max(max_attr, a);
  P.amin.assign(max_attr + 1, 0);
  P.abits.assign(max_attr + 1, 0);
  for (int a = 0; a <= max_attr; ++a) {
    int holders = 0, tops = 0;
    for (auto& n : P.nodes) {
      bool has = std::find(n.key_attr.begin(), n.key_attr.end(), a) != n.key_attr.end();
      if (!has) continue;
      ++holders;
      bool parent_has = n.parent >= 0 && std::find(P.nodes[n.parent].key_attr.begin(),
                                                   P.nodes[n.parent].key_attr.end(), a) !=
                                             P.nodes[n.parent].key_attr.end();
      if (!parent_has) ++tops;
    }
    if (holders == 1)
      return fail(FIGARO_ERR_INVALID_TREE, "attribute " + std::to_string(a) + " occurs in one relation only");
    if (holders > 1 && tops != 1)
      return fail(FIGARO_ERR_INVALID_TREE, "relations holding attribute " + std::to_string(a) +
                                               " are not connected in the join tree");
  }
  // columns of A[:, Y]
  int off = 0;
  for (auto& n : P.nodes) {
    n.col_off = off;
    off += n.N;
  }
  P.N = off;
  if (P.N < 1 || P.N > 1024) return fail(FIGARO_ERR_UNSUPPORTED, "total data columns must be in [1, 1024]");
  for (int i : P.post) {
    Node& n = P.nodes[i];
    std::vector<int> cols;
    for (int c = 0; c < n.N; ++c) cols.push_back(n.col_off + c);
    for (int c : n.children) cols.insert(cols.end(), P.nodes[c].sub_cols.begin(), P.nodes[c].sub_cols.end());
    std::sort(cols.begin(), cols.end());
    n.sub_cols = cols;
    n.N_sub = (int)cols.size();
    for (int gc : cols) {
      if (gc >= n.col_off && gc < n.col_off + n.N) {
        n.coldesc.push_back(make_int2(0, gc - n.col_off));
        continue;
      }
      for (int jj = 0; jj < (int)n.children.size(); ++jj) {
        const auto& sc = P.nodes[n.children[jj]].sub_cols;
        auto it = std::find(sc.begin(), sc.end(), gc);
        if (it != sc.end()) {
          n.coldesc.push_back(make_int2(1 + jj, (int)(it - sc.begin())));
          break;
        }
      }
    }
    // every global column: 0 own, 1 + c in child c's subtree, 255 outside the subtree
    n.colkind.assign(P.N, 255);
    for (int c = 0; c < n.N; ++c) n.colkind[n.col_off + c] = 0;
    for (int jj = 0; jj < (int)n.children.size(); ++jj)
      for (int gc : P.nodes[n.children[jj]].sub_cols) n.colkind[gc] = (uint8_t)(1 + jj);
  }
  return FIGARO_OK;
}

static int scan_key_ranges(figaro_plan_s& P) {
  const int na = (int)P.amin.size();
  std::vector<long long> lo(na, LLONG_MAX), hi(na, LLONG_MIN);
  std::vector<std::pair<int, int>> cols;
  for (auto& n : P.nodes)
    for (int k = 0; k < n.K; ++k) cols.push_back({n.id, k});
  if (cols.empty()) return FIGARO_OK;
  if (P.opt.mem == FIGARO_MEM_HOST) {
    for (auto [i, k] : cols) {
      const Node& n = P.nodes[i];
      int a = n.key_attr[k];
      for (int64_t r = 0; r < n.M; ++r) {
        long long v = n.key_type == FIGARO_KEY_I32 ? (long long)static_cast<const int32_t*>(n.key_ptr[k])[r]
                                                   : static_cast<const long long*>(n.key_ptr[k])[r];
        lo[a] = std::min(lo[a], v);
        hi[a] = std::max(hi[a], v);
      }
    }
  } else {
    long long* d = nullptr;
    FIG_CUDA(cudaMalloc(&d, 2 * sizeof(long long) * cols.size()));
    std::vector<long long> init(2 * cols.size());
    for (size_t c = 0; c < cols.size(); ++c) { init[2 * c] = LLONG_MAX; init[2 * c + 1] = LLONG_MIN; }
    cudaError_t e = cudaMemcpyAsync(d, init.data(), init.size() * sizeof(long long), cudaMemcpyHostToDevice, P.st);
    for (size_t c = 0; c < cols.size() && e == cudaSuccess; ++c) {
      const Node& n = P.nodes[cols[c].first];
      launch_minmax(n.key_ptr[cols[c].second], n.key_type, n.M, d + 2 * c, d + 2 * c + 1, P.st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(init.data(), d, init.size() * sizeof(long long), cudaMemcpyDeviceToHost, P.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P.st);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(d);
    if (e != cudaSuccess) return fail(FIGARO_ERR_CUDA, std::string("key range scan: ") + cudaGetErrorString(e));
    for (size_t c = 0; c < cols.size(); ++c) {
      int a = P.nodes[cols[c].first].key_attr[cols[c].second];
      lo[a] = std::min(lo[a], init[2 * c]);
      hi[a] = std::max(hi[a], init[2 * c + 1]);
    }
  }
  for (int a = 0; a < na; ++a) {
    if (lo[a] > hi[a]) continue;
    P.amin[a] = lo[a];
    P.abits[a] = bits_for((unsigned long long)(hi[a] - lo[a]));
  }
  // packing of every relation
  for (auto& n : P.nodes) {
    std::vector<int> xp, rest;
    for (int a : n.key_attr) {
      bool shared = false;
      if (n.parent >= 0) {
        const auto& pa = P.nodes[n.parent].key_attr;
        shared = std::find(pa.begin(), pa.end(), a) != pa.end();
      }
      (shared ? xp : rest).push_back(a);
    }
    std::sort(xp.begin(), xp.end());
    std::sort(rest.begin(), rest.end());
    n.pack_attr = xp;
    n.pack_attr.insert(n.pack_attr.end(), rest.begin(), rest.end());
    int total = 0;
    for (int a : n.pack_attr) total += P.abits[a];
    if (total > 64)
      return fail(FIGARO_ERR_UNSUPPORTED, "packed key of relation " + std::to_string(n.id) + " needs " +
                                              std::to_string(total) + " bits (> 64)");
    n.bits = total;
    n.rest_bits = 0;
    for (int a : rest) n.rest_bits += P.abits[a];
    const int xp_bits = total - n.rest_bits;   // distinct X_p values <= 2^xp_bits
    n.pbound = n.root ? 1 : (xp_bits >= 40 ? n.M : std::min<int64_t>(n.M, int64_t(1) << xp_bits));
    if (n.pbound < 1) n.pbound = 1;
    int cur = total;
    n.shift.clear();
    n.pack_col.clear();
    for (int a : n.pack_attr) {
      cur -= P.abits[a];
      n.shift.push_back(cur);
      n.pack_col.push_back((int)(std::find(n.key_attr.begin(), n.key_attr.end(), a) - n.key_attr.begin()));
    }
  }
  return FIGARO_OK;
}

static int shift_of(const Node& n, int a) {
  for (size_t k = 0; k < n.pack_attr.size(); ++k)
    if (n.pack_attr[k] == a) return n.shift[k];
  return -1;
}

static void make_links(figaro_plan_s& P) {
  for (auto& n : P.nodes) {
    for (int jj = 0; jj < (int)n.children.size(); ++jj) {
      Node& c = P.nodes[n.children[jj]];
      ChildLink& L = n.link[jj];
      L = ChildLink{};
      int na = 0;
      for (int a : c.pack_attr) {
        if (shift_of(c, a) < c.rest_bits) continue;   // not in the child's X_p
        L.src_shift[na] = shift_of(n, a);
        L.bits[na] = P.abits[a];
        L.dst_shift[na] = shift_of(c, a) - c.rest_bits;
        ++na;
      }
      L.n_attr = na;
      L.pkey = c.b.pkey;
      L.sizes = c.b.sizes;
      L.phid = c.b.phid;
      L.sq_phid = c.b.sq_phid;
      L.phiu = c.b.phiu;
      L.q = n.b.q + (int64_t)jj * n.M;
      L.data = c.leaf ? c.b.heads : c.b.data2;
      L.ld = c.M;
    }
  }
}

static void make_blocks(figaro_plan_s& P) {
  const bool mixed = P.opt.precision != FIGARO_PREC_FP64;
  const bool givens = P.opt.leaf == FIGARO_LEAF_GIVENS, tc5 = P.opt.leaf != FIGARO_LEAF_MMA_SYNC;
  // the planner's rule, or the autotuner's fastest candidate (options.autotune)
  auto plan_block = [&](TsqrBlock& t) {
    tsqr_plan_block(t, mixed, givens, tc5);
    if (P.opt.autotune && !t.fused) {
      const TsqrTune tune = tsqr_autotune(t, mixed, givens, tc5);
      tsqr_plan_block(t, mixed, givens, tc5, &tune);
    }
  };
  P.blocks.clear();
  P.stack_rows = 0;
  for (auto& n : P.nodes) {
    n.blk_tails = n.blk_gen = -1;
    if (n.N > 0) {
      n.blk_tails = (int)P.blocks.size();
      TsqrBlock t{};
      t.n = n.N;
      t.kind = BLK_TAILS;
      t.M = n.M;
      t.bound = n.M;
      // formed inside the leaf where tsqr_plan_block allows it (<= 32 columns, Householder)
      t.fused = P.opt.precision != FIGARO_PREC_MIXED_REFINED && P.opt.fuse_tails;
      plan_block(t);
      P.blocks.push_back(t);
      P.stack_rows += t.n;
    }
    if (!n.leaf && !n.root && n.N_sub > 0) {
      n.blk_gen = (int)P.blocks.size();
      TsqrBlock t{};
      t.n = n.N_sub;
      t.kind = BLK_GEN;
      t.prio = true;
      t.M = n.M;
      t.bound = n.M;
      plan_block(t);
      P.blocks.push_back(t);
      P.stack_rows += t.n;
    }
    if (n.root) {
      n.blk_gen = (int)P.blocks.size();
      TsqrBlock t{};
      t.n = n.N_sub;
      t.kind = BLK_ROOT;
      t.prio = true;
      t.M = n.M;
      t.bound = n.M;
      plan_block(t);
      P.blocks.push_back(t);
      P.stack_rows += t.n;
    }
  }
  TsqrBlock s{};
  s.n = P.N;
  s.kind = BLK_FIXED;
  s.M = P.stack_rows;
  s.bound = P.stack_rows;
  s.ld = P.stack_rows;
  tsqr_plan_block(s, false);
  P.stack_blk = s;
}

// block pointers that depend on the arena
static void bind_blocks(figaro_plan_s& P) {
  for (auto& blk : P.blocks) blk.err = P.err_dev;
  P.stack_blk.err = P.err_dev;
  size_t bi = 0;
  P.block_lo32.assign(P.blocks.size(), nullptr);
  P.block_lp.assign(P.blocks.size(), fig::LeafParams{});
  for (auto& n : P.nodes) {
    if (n.N > 0) {
      P.block_lo32[bi] = n.b.tails32lo;
      P.blocks[bi].ptr = n.b.tails;
      P.blocks[bi].ptr32 = n.b.tails32;
      P.blocks[bi].ld = n.M;
      P.blocks[bi].sizes = n.b.sizes;
      ++bi;
    }
    if (!n.leaf && !n.root && n.N_sub > 0) {
      P.blocks[bi].ptr = n.b.gtails;
      P.blocks[bi].ptr32 = n.gtails32;
      P.blocks[bi].ld = n.M;
      P.blocks[bi].sizes = n.b.sizes;
      ++bi;
    }
    if (n.root) {
      P.blocks[bi].ptr = n.b.rootrows;
      P.blocks[bi].ld = n.M;
      P.blocks[bi].sizes = n.b.sizes;
      ++bi;
    }
  }
}

static std::vector<int> block_cols(const figaro_plan_s& P, size_t bi) {
  size_t k = 0;
  for (auto& n : P.nodes) {
    if (n.N > 0) {
      if (k++ == bi) {
        std::vector<int> c;
        for (int j = 0; j < n.N; ++j) c.push_back(n.col_off + j);
        return c;
      }
    }
    if (!n.leaf && !n.root && n.N_sub > 0)
      if (k++ == bi) return n.sub_cols;
    if (n.root)
      if (k++ == bi) return n.sub_cols;
  }
  return {};
}

// ------------------------------------------------------------------ per-call pipeline
struct StageClock {
  figaro_plan_s& P;
  int64_t l0 = 0;
  int s = -1;
  explicit StageClock(figaro_plan_s& p) : P(p) {}
  void start(int stage) {
    s = stage;
    l0 = P.launches;
    if (P.opt.stage_timing) cudaEventRecord(P.ev[stage], P.st);
  }
  void stop() {
    if (P.opt.stage_timing) cudaEventRecord(P.ev[s + 1], P.st);
    P.stage_launch[s] += P.launches - l0;
  }
};

// The pipeline as a dependency graph over streams:
//   copies (host-memory mode)  keys of every relation, then the data in post-order
//   relation i                 pack + sort + segmentation       (needs its keys)
//   main                       Alg. 3 counts                      (needs every segmentation)
//   relation i                 heads and tails                    (needs counts and its data)
//   block stream               TSQR of relation i's tails block   (needs its heads and tails)
//   main                       join + project-away, post-order    (needs the heads of the node
//                                                                  and of its leaf children)
//   block stream               TSQR of each generalized-tail / root block (after its join)
//   main                       final QR of the stacked triangles  (needs every block)
// With stage timing everything runs in that order on the main stream instead, the TSQR
// chains last, so that each stage's event times cover only its own kernels.
static int enqueue_r(figaro_plan_s& P, double* R, int64_t ldr) {
  cudaStream_t st = P.st;
  const bool mixed = P.opt.precision != FIGARO_PREC_FP64;
  const bool refine = P.opt.precision == FIGARO_PREC_MIXED_REFINED;
  const bool serial = P.opt.stage_timing != 0;
  const bool host = P.opt.mem == FIGARO_MEM_HOST;
  const int r = (int)P.nodes.size();
  P.launches = 0;
  auto nst = [&](int i) { return serial ? st : P.nstream[i]; };
  auto rec = [&](cudaEvent_t e, cudaStream_t s) { return serial ? cudaSuccess : cudaEventRecord(e, s); };
  auto wait = [&](cudaStream_t s, cudaEvent_t e) { return serial ? cudaSuccess : cudaStreamWaitEvent(s, e, 0); };
  FIG_CUDA(cudaMemsetAsync(P.err_dev, 0, sizeof(int), st));
  if (refine) FIG_CUDA(cudaMemsetAsync(P.gram, 0, sizeof(double) * P.N * P.N, st));
  FIG_CUDA(rec(P.fork, st));
  if (host) {
    cudaStream_t cs = serial ? st : P.copy_st;
    FIG_CUDA(wait(cs, P.fork));
    for (int i = 0; i < r; ++i) {
      Node& n = P.nodes[i];
      for (int k = 0; k < n.K; ++k)
        FIG_CUDA(cudaMemcpyAsync(n.dkey[k], n.key_ptr[k], n.M * (n.key_type == FIGARO_KEY_I32 ? 4 : 8),
                                 cudaMemcpyHostToDevice, cs));
      FIG_CUDA(rec(P.ev_keys[i], cs));
    }
    for (int i : P.post) {
      Node& n = P.nodes[i];
      if (n.N > 0) {
        const int64_t elems = n.layout == FIGARO_COL_MAJOR ? n.ld * (n.N - 1) + n.M : n.ld * (n.M - 1) + n.N;
        FIG_CUDA(cudaMemcpyAsync(n.ddata, n.data, elems * sizeof(double), cudaMemcpyHostToDevice, cs));
      }
      FIG_CUDA(rec(P.ev_data[i], cs));
    }
  }
  // TSQR of one R0 block: on its own stream after `ready`, or in place when serial
  auto run_block = [&](int bi, cudaEvent_t ready) -> int {
    cudaStream_t s = serial ? st : P.side[bi];
    FIG_CUDA(wait(s, ready));
    if (serial) FIG_CUDA(cudaEventRecord(P.leaf_ev[2 * bi], s));
    const int64_t l0 = P.launches;
    if (P.blocks[bi].fused) tails_qr(P.block_lp[bi], P.blocks[bi], s, &P.launches);
    else tsqr_leaf(P.blocks[bi], mixed, s, &P.launches);
    P.stage_launch[5] += P.launches - l0;
    if (serial) FIG_CUDA(cudaEventRecord(P.leaf_ev[2 * bi + 1], s));
    tsqr_reduce(P.blocks[bi], mixed, s, &P.launches);
    if (refine) gram_block(P.blocks[bi], P.block_lo32[bi], P.gram_partial[bi], s, &P.launches);
    FIG_CUDA(rec(P.side_done[bi], s));
    return FIGARO_OK;
  };
  StageClock clk(P);
  // ---- stage 0: pack + sort
  clk.start(0);
  for (int i = 0; i < r; ++i) {
    Node& n = P.nodes[i];
    cudaStream_t s = nst(i);
    FIG_CUDA(wait(s, host ? P.ev_keys[i] : P.fork));
    PackParams pp{};
    pp.n_keys = (int)n.pack_attr.size();
    pp.key_type = n.key_type;
    for (int k = 0; k < pp.n_keys; ++k) {
      const int col = n.pack_col[k];
      pp.cols[k] = host ? n.dkey[col] : n.key_ptr[col];
      pp.kmin[k] = P.amin[n.pack_attr[k]];
      pp.shift[k] = n.shift[k];
      pp.bits[k] = P.abits[n.pack_attr[k]];
    }
    const bool sort = !P.opt.presorted && n.bits > 0;
    launch_pack(pp, n.M, n.b.key[0], sort ? n.b.perm[0] : nullptr, P.err_dev, s, &P.launches);
    if (sort) {
      int cur = radix_sort(n.b.key, n.b.perm, n.M, n.bits, n.radix_hist, n.radix_tmp, s, &P.launches);
      n.b.skey = n.b.key[cur];
      n.b.sperm = n.b.perm[cur];
    } else {
      if (P.opt.presorted) check_sorted(n.b.key[0], n.M, P.err_dev, s, &P.launches);
      n.b.skey = n.b.key[0];
      n.b.sperm = nullptr;
    }
  }
  clk.stop();
  // ---- stage 1: segmentation
  clk.start(1);
  for (int i = 0; i < r; ++i) {
    segment(P.nodes[i].b, P.nodes[i].M, P.nodes[i].rest_bits, nst(i), &P.launches);
    counts_clear(P.nodes[i].b, P.nodes[i].M, nst(i), &P.launches);
    FIG_CUDA(rec(P.ev_seg[i], nst(i)));
    FIG_CUDA(wait(st, P.ev_seg[i]));
  }
  clk.stop();
  // ---- stage 2: counts (Alg. 3)
  clk.start(2);
  make_links(P);
  auto count_params = [&](Node& n) {
    CountParams c{};
    c.n_child = (int)n.children.size();
    for (int j = 0; j < c.n_child; ++j) c.ch[j] = n.link[j];
    c.is_root = n.root;
    c.require_reduced = P.opt.require_reduced;
    c.M = n.M;
    c.gkey = n.b.gkey;
    c.goff = n.b.goff;
    c.g2p = n.b.g2p;
    c.pgoff = n.b.pgoff;
    c.sizes = n.b.sizes;
    c.theta = n.b.theta;
    c.full = n.b.full;
    c.phic = n.b.phic;
    c.phid = n.b.phid;
    c.phiu = n.b.phiu;
    c.theta_incl = n.b.theta_incl;
    c.sq_phic = n.b.sq_phic;
    c.hrow = n.b.hrow;
    c.fac = n.b.fac;
    c.vw = n.b.vw;
    c.hf = n.b.hf;
    return c;
  };
  for (int i : P.post) counts_pass1(count_params(P.nodes[i]), st, P.err_dev, &P.launches);
  for (int i : P.pre) {
    Node& n = P.nodes[i];
    counts_pass2(count_params(n), st, P.err_dev, &P.launches);
    for (int j = 0; j < (int)n.children.size(); ++j)
      counts_finalize_child(n.link[j], P.nodes[n.children[j]].M, st, &P.launches);
  }
  for (auto& n : P.nodes) {
    if (n.leaf && !n.root) continue;
    if (!n.root) {
      ScanSrc src{SCAN_PLAIN_U64, n.b.theta, 0};
      scan_inclusive<uint64_t>(src, n.b.theta_incl, n.M, n.b.sizes, n.b.scan_tmp_u, st, &P.launches);
    }
    join_prep(count_params(n), st, &P.launches);
  }
  FIG_CUDA(rec(P.ev_counts, st));
  clk.stop();
  // ---- stage 3: heads and tails of every relation; each tails block's TSQR follows at once
  clk.start(3);
  for (int i = 0; i < r; ++i) {
    Node& n = P.nodes[i];
    cudaStream_t s = nst(i);
    FIG_CUDA(wait(s, P.ev_counts));
    if (host) FIG_CUDA(wait(s, P.ev_data[i]));
    LeafParams lp{};
    lp.M = n.M;
    lp.N = n.N;
    lp.data = host ? n.ddata : n.data;
    lp.rs = n.layout == FIGARO_COL_MAJOR ? 1 : n.ld;
    lp.cs = n.layout == FIGARO_COL_MAJOR ? n.ld : 1;
    lp.perm = n.b.sperm;
    lp.sdata = n.b.sperm ? n.b.sdata : nullptr;
    lp.lds = n.b.lds;
    lp.row_gid = n.b.row_gid;
    lp.goff = n.b.goff;
    lp.sq_phic = n.b.sq_phic;
    lp.hrow = n.b.hrow;
    lp.beta = P.beta;
    lp.beta_len = P.beta_len;
    const bool fused = n.blk_tails >= 0 && P.blocks[n.blk_tails].fused;
    lp.mixed = mixed;
    lp.tails = n.b.tails;
    lp.tails32 = mixed ? n.b.tails32 : nullptr;
    lp.tails32lo = refine ? n.b.tails32lo : nullptr;
    lp.ldt = n.M;
    lp.heads = n.b.heads;
    lp.ldh = n.M;
    lp.tflag = n.b.tflag;
    lp.ttail = n.b.ttail;
    lp.tsum = n.b.tsum;
    lp.tcarry = n.b.ltcarry;
    // lane partials for the stored tails pass and for a fused leaf with the first pass's
    // lanes (8 rows each: blocks of <= 8 columns); wider fused leaves scan their lanes
    lp.lflag = (fused && P.blocks[n.blk_tails].nreg > 8) ? nullptr : n.b.llflag;
    lp.lsum = n.b.llsum;
    lp.n_tiles = n.n_tiles;
    if (n.b.sperm && row_gather_pays(n.M, n.N)) {   // the sorted copy, by whole rows
      if (n.layout == FIGARO_COL_MAJOR) {
        rows_of(lp.data, n.ld, n.M, nullptr, n.N, n.rowin, row_pitch(n.N), s, &P.launches);
        rows_gather(n.rowin, row_pitch(n.N), n.b.sperm, n.M, n.N, n.b.sdata, n.b.lds, s, &P.launches);
      } else {
        rows_gather(lp.data, n.ld, n.b.sperm, n.M, n.N, n.b.sdata, n.b.lds, s, &P.launches);
      }
      lp.sorted_ready = 1;
    }
    leaf_heads(lp, s, &P.launches);
    if (fused) P.block_lp[n.blk_tails] = lp;
    else leaf_tails(lp, s, &P.launches);
    FIG_CUDA(rec(P.ev_leaf[i], s));
    if (!serial && n.blk_tails >= 0) {
      const int rc = run_block(n.blk_tails, P.ev_leaf[i]);
      if (rc != FIGARO_OK) return rc;
    }
  }
  clk.stop();
  // ---- stage 4: join children, project away, root rows (post-order)
  clk.start(4);
  for (int i : P.post) {
    Node& n = P.nodes[i];
    if (n.leaf && !n.root) continue;
    FIG_CUDA(wait(st, P.ev_leaf[i]));
    for (int c : n.children) FIG_CUDA(wait(st, P.ev_leaf[c]));
    GenParams gp{};
    gp.N = n.N_sub;
    gp.n_child = (int)n.children.size();
    gp.M = n.M;
    gp.sizes = n.b.sizes;
    gp.g2p = n.b.g2p;
    gp.pgoff = n.b.pgoff;
    gp.heads = n.b.heads;
    gp.ldh = n.M;
    gp.fac = n.b.fac;
    gp.vw = n.b.vw;
    gp.hf = n.b.hf;
    gp.q = n.b.q;
    for (int j = 0; j < gp.n_child; ++j) {
      Node& c = P.nodes[n.children[j]];
      gp.cdata[j] = n.link[j].data;
      gp.cld[j] = n.link[j].ld;
      // whole rows of the child's table are gathered from a row-major copy of it
      rows_of(n.link[j].data, n.link[j].ld, c.M, c.b.sizes + 1, c.leaf ? c.N : c.N_sub, c.crow, c.crow_pitch, st,
              &P.launches);
      gp.crow[j] = c.crow;
      gp.cnp[j] = c.crow_pitch;
    }
    gp.jdata = n.jdata;
    gp.ldj = n.ldj;
    gp.coldesc = n.b.coldesc;
    gp.gtails = n.b.gtails;
    gp.gtails32 = n.gtails32;
    gp.data2 = n.b.data2;
    gp.rootrows = n.b.rootrows;
    gp.tflag = n.b.tflag;
    gp.tsum = n.b.tsum;
    gp.tcarry = n.b.tcarry;
    gp.lflag = n.b.lflag;
    gp.lsum = n.b.lsum;
    gp.n_tiles = n.n_tiles;
    gp.is_root = n.root;
    if (gp.N > 0) gen_heads_tails(gp, st, &P.launches);
    FIG_CUDA(rec(P.ev_gen[i], st));
    if (!serial && n.blk_gen >= 0) {
      const int rc = run_block(n.blk_gen, P.ev_gen[i]);
      if (rc != FIGARO_OK) return rc;
    }
  }
  clk.stop();
  // ---- stages 5-6: with stage timing the TSQR chains run here, one after another (stage 5
  // sums the leaf launches, stage 6 is the wall time of the whole TSQR section); then the
  // final QR of the stacked block triangles on the main stream.
  clk.start(6);
  for (size_t bi = 0; bi < P.blocks.size(); ++bi) {
    if (serial) {
      const int rc = run_block((int)bi, nullptr);
      if (rc != FIGARO_OK) return rc;
    } else {
      FIG_CUDA(cudaStreamWaitEvent(st, P.side_done[bi], 0));
    }
  }
  if (refine)
    for (size_t bi = 0; bi < P.blocks.size(); ++bi) gram_add(P.blocks[bi], P.gram_partial[bi], P.gram, P.N, st, &P.launches);
  tsqr_final(P.blocks_dev, (int)P.blocks.size(), P.stack_blk, R, ldr, st, &P.launches);
  if (refine)
    refine_r(R, ldr, P.gram, P.N, P.refine_w, P.refine_w + (int64_t)P.N * P.N, P.refine_ok, st, &P.launches);
  clk.stop();
  FIG_CUDA(cudaGetLastError());
  return FIGARO_OK;
}

// The whole R pipeline depends on the data only through device-side sizes, so it is
// captured once into a CUDA graph (writing into the plan's R buffer) and replayed on every
// later call; the ~100 small launches of a step then cost no host time.  Stage timing and
// any capture failure (e.g. pageable host inputs) fall back to direct launches.
static int run_r(figaro_plan_s& P, double* R, int64_t ldr) {
  if (P.opt.stage_timing || P.graph_failed) return enqueue_r(P, R, ldr);
  cudaStream_t user = P.st;
  if (!P.graph_exec) {
    // capture on the plan's own stream (the caller's may be the uncapturable legacy stream)
    cudaGraph_t g = nullptr;
    int rc = FIGARO_OK;
    P.st = P.exec;
    cudaError_t e = cudaStreamBeginCapture(P.exec, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = enqueue_r(P, P.Rtmp, P.N);
      e = cudaStreamEndCapture(P.exec, &g);
    }
    P.st = user;
    if (e == cudaSuccess && rc == FIGARO_OK) e = cudaGraphInstantiate(&P.graph_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || rc != FIGARO_OK) {
      cudaGetLastError();
      P.graph_exec = nullptr;
      P.graph_failed = true;
      g_last_error.clear();
      return enqueue_r(P, R, ldr);
    }
    P.graph_launches = P.launches;
  }
  FIG_CUDA(cudaEventRecord(P.join_in, user));
  FIG_CUDA(cudaStreamWaitEvent(P.exec, P.join_in, 0));
  FIG_CUDA(cudaGraphLaunch(P.graph_exec, P.exec));
  FIG_CUDA(cudaEventRecord(P.join_out, P.exec));
  FIG_CUDA(cudaStreamWaitEvent(user, P.join_out, 0));
  P.launches = P.graph_launches;
  if (R != P.Rtmp)
    FIG_CUDA(cudaMemcpy2DAsync(R, ldr * sizeof(double), P.Rtmp, P.N * sizeof(double), P.N * sizeof(double), P.N,
                               cudaMemcpyDeviceToDevice, user));
  return FIGARO_OK;
}

static int finish(figaro_plan_s& P, int stages_used) {
  FIG_CUDA(cudaMemcpyAsync(P.err_host, P.err_dev, sizeof(int), cudaMemcpyDeviceToHost, P.st));
  if (P.refine_ok) FIG_CUDA(cudaMemcpyAsync(P.err_host + 1, P.refine_ok, sizeof(int), cudaMemcpyDeviceToHost, P.st));
  for (size_t i = 0; i < P.nodes.size(); ++i)
    FIG_CUDA(cudaMemcpyAsync(P.err_host + 4 + 4 * i, P.nodes[i].b.sizes, 4 * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, P.st));
  FIG_CUDA(cudaStreamSynchronize(P.st));
  FIG_CUDA(cudaGetLastError());
  if (P.opt.stage_timing) {
    for (int s = 0; s < stages_used; ++s) {
      if (s == 5) continue;                      // stage 5 is measured per block below
      float ms = 0.f;
      const int from = s == 6 ? 6 : s;           // stage 6 starts at its own event
      if (cudaEventElapsedTime(&ms, P.ev[from], P.ev[s + 1]) == cudaSuccess) P.stage_ms[s] += ms;
    }
    P.block_leaf_ms.resize(P.blocks.size(), 0.0);
    for (size_t bi = 0; bi < P.blocks.size(); ++bi) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, P.leaf_ev[2 * bi], P.leaf_ev[2 * bi + 1]) == cudaSuccess) {
        P.stage_ms[5] += ms;
        P.block_leaf_ms[bi] += ms;
      }
    }
  }
  // bookkeeping for figaro_plan_get_info: R0 rows and TSQR leaf flops of this call
  P.r0_rows = 0;
  P.leaf_flops = 0.0;
  P.refined = P.refine_ok ? P.err_host[1] : 0;
  P.block_rows.assign(P.blocks.size(), 0);
  for (size_t i = 0; i < P.nodes.size(); ++i) {
    const Node& n = P.nodes[i];
    const int64_t G = P.err_host[4 + 4 * i], Pg = P.err_host[4 + 4 * i + 1];
    if (n.blk_tails >= 0) P.block_rows[n.blk_tails] = n.M - G;
    if (n.blk_gen >= 0) P.block_rows[n.blk_gen] = n.root ? G : G - Pg;
  }
  for (size_t i = 0; i < P.nodes.size(); ++i) {
    const Node& n = P.nodes[i];
    const int64_t G = P.err_host[4 + 4 * i], Pg = P.err_host[4 + 4 * i + 1];
    if (n.N > 0) { P.r0_rows += n.M - G; P.leaf_flops += tsqr_leaf_flops(n.M - G, n.N); }
    if (!n.leaf && !n.root && n.N_sub > 0) { P.r0_rows += G - Pg; P.leaf_flops += tsqr_leaf_flops(G - Pg, n.N_sub); }
    if (n.root) { P.r0_rows += G; P.leaf_flops += tsqr_leaf_flops(G, n.N_sub); }
  }
  const int e = *P.err_host;
  if (e != 0) return fail(e, std::string("device reported: ") + figaro_error_string(e));
  return FIGARO_OK;
}

}  // namespace fig

using namespace fig;

extern "C" {

void figaro_default_options(figaro_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = FIGARO_PREC_FP64;
  opt->mem = FIGARO_MEM_DEVICE;
}

const char* figaro_error_string(int s) {
  switch (s) {
    case FIGARO_OK: return "FIGARO_OK";
    case FIGARO_ERR_INVALID_ARG: return "FIGARO_ERR_INVALID_ARG";
    case FIGARO_ERR_INVALID_TREE: return "FIGARO_ERR_INVALID_TREE";
    case FIGARO_ERR_NOT_REDUCED: return "FIGARO_ERR_NOT_REDUCED";
    case FIGARO_ERR_OVERFLOW: return "FIGARO_ERR_OVERFLOW";
    case FIGARO_ERR_NOMEM: return "FIGARO_ERR_NOMEM";
    case FIGARO_ERR_TIMEOUT: return "FIGARO_ERR_TIMEOUT";
    case FIGARO_ERR_CUDA: return "FIGARO_ERR_CUDA";
    case FIGARO_ERR_KEY_RANGE: return "FIGARO_ERR_KEY_RANGE";
    case FIGARO_ERR_NOT_SORTED: return "FIGARO_ERR_NOT_SORTED";
    case FIGARO_ERR_UNSUPPORTED: return "FIGARO_ERR_UNSUPPORTED";
    case FIGARO_ERR_SINGULAR: return "FIGARO_ERR_SINGULAR";
    default: return "FIGARO_ERR_UNKNOWN";
  }
}

const char* figaro_last_error(void) { return g_last_error.c_str(); }

int figaro_plan_destroy(figaro_plan_t p) {
  if (!p) return FIGARO_OK;
  if (p->arena) cudaStreamSynchronize(p->st);
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : p->side_done)
    if (e) cudaEventDestroy(e);
  for (auto& e : p->leaf_ev)
    if (e) cudaEventDestroy(e);
  if (p->fork) cudaEventDestroy(p->fork);
  if (p->join_in) cudaEventDestroy(p->join_in);
  if (p->join_out) cudaEventDestroy(p->join_out);
  if (p->exec) cudaStreamDestroy(p->exec);
  for (auto& s : p->side)
    if (s) cudaStreamDestroy(s);
  for (auto& s : p->nstream)
    if (s) cudaStreamDestroy(s);
  if (p->copy_st) cudaStreamDestroy(p->copy_st);
  for (auto* v : {&p->ev_keys, &p->ev_data, &p->ev_seg, &p->ev_leaf, &p->ev_gen})
    for (auto& e : *v)
      if (e) cudaEventDestroy(e);
  if (p->ev_counts) cudaEventDestroy(p->ev_counts);
  if (p->err_host) cudaFreeHost(p->err_host);
  if (p->arena) cudaFree(p->arena);
  delete p;
  return FIGARO_OK;
}

int figaro_plan(const figaro_join_tree* tree, const figaro_options* opt, void* stream, figaro_plan_t* out) {
  g_last_error.clear();
  if (!out) return fail(FIGARO_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!tree) return fail(FIGARO_ERR_INVALID_ARG, "tree is null");
  auto* P = new (std::nothrow) figaro_plan_s();
  if (!P) return fail(FIGARO_ERR_NOMEM, "host allocation");
  if (opt) P->opt = *opt; else figaro_default_options(&P->opt);
  if ((P->opt.precision != FIGARO_PREC_FP64 && P->opt.precision != FIGARO_PREC_MIXED &&
       P->opt.precision != FIGARO_PREC_MIXED_REFINED) ||
      (P->opt.leaf != FIGARO_LEAF_HOUSEHOLDER && P->opt.leaf != FIGARO_LEAF_GIVENS &&
       P->opt.leaf != FIGARO_LEAF_TCGEN05 && P->opt.leaf != FIGARO_LEAF_MMA_SYNC)) {
    delete P;
    return fail(FIGARO_ERR_INVALID_ARG, "precision");
  }
  if (P->opt.mem != FIGARO_MEM_DEVICE && P->opt.mem != FIGARO_MEM_HOST) {
    delete P;
    return fail(FIGARO_ERR_INVALID_ARG, "mem");
  }
  if (P->opt.autotune != 0 && P->opt.autotune != 1) {
    delete P;
    return fail(FIGARO_ERR_INVALID_ARG, "autotune");
  }
  if (P->opt.fuse_tails != 0 && P->opt.fuse_tails != 1) {
    delete P;
    return fail(FIGARO_ERR_INVALID_ARG, "fuse_tails");
  }
  if (P->opt.workspace_limit_mib < 0 || P->opt.svd_max_sweeps < 0) {
    delete P;
    return fail(FIGARO_ERR_INVALID_ARG, "workspace_limit_mib or svd_max_sweeps negative");
  }
  P->st = static_cast<cudaStream_t>(stream);
  int rc = build(*P, tree);
  if (rc == FIGARO_OK) {
    // per-function shared-memory limits, raised once to the largest size any launch uses
    cudaError_t e = keys_set_attributes();
    if (e == cudaSuccess) e = tsqr_set_attributes();
    if (e == cudaSuccess) e = svd_set_attributes();
    if (e == cudaSuccess) e = rows_of_set_attributes();
    if (e == cudaSuccess) e = refine_set_attributes();
    if (e != cudaSuccess) {
      delete P;
      return fail(FIGARO_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    }
  }
  if (rc != FIGARO_OK) { delete P; return rc; }
  if (cudaGetDevice(&P->device) != cudaSuccess) {
    delete P;
    return fail(FIGARO_ERR_CUDA, "no CUDA device");
  }
  rc = scan_key_ranges(*P);
  if (rc != FIGARO_OK) { delete P; return rc; }
  make_blocks(*P);
  Arena measure;
  layout(*P, measure);
  P->arena_bytes = measure.off + 256;
  if (P->opt.workspace_limit_mib > 0 && P->arena_bytes > ((size_t)P->opt.workspace_limit_mib << 20)) {
    const size_t need = P->arena_bytes;
    P->arena_bytes = 0;
    figaro_plan_destroy(P);
    return fail(FIGARO_ERR_NOMEM, "device workspace of " + std::to_string(need) + " bytes exceeds workspace_limit_mib");
  }
  if (cudaMalloc(&P->arena, P->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    P->arena = nullptr;
    figaro_plan_destroy(P);
    return fail(FIGARO_ERR_NOMEM, "device workspace of " + std::to_string(P->arena_bytes) + " bytes");
  }
  Arena real;
  real.base = P->arena;
  layout(*P, real);
  bind_blocks(*P);
  auto bail = [&](cudaError_t e, const char* what) {
    figaro_plan_destroy(P);
    return fail(FIGARO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e = cudaMallocHost(&P->err_host, sizeof(int) * (4 + 4 * P->nodes.size()));
  if (e != cudaSuccess) return bail(e, "cudaMallocHost");
  for (auto& ev : P->ev) {
    e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return bail(e, "cudaEventCreate");
  }
  e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->join_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->join_out, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(e, "cudaEventCreate");
  // The tails blocks' TSQR streams get the lowest priority (long FP64 work that fills the
  // gaps); the relation and main streams and the generalized-tail / root blocks, which
  // form the dependency chain to R, get the highest.
  int prio_lo = 0, prio_hi = 0;
  e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&P->exec, cudaStreamNonBlocking, prio_hi);
  if (e != cudaSuccess) return bail(e, "plan streams");
  P->side.assign(P->blocks.size(), nullptr);
  P->side_done.assign(P->blocks.size(), nullptr);
  for (size_t bi = 0; bi < P->blocks.size(); ++bi) {
    e = cudaStreamCreateWithPriority(&P->side[bi], cudaStreamNonBlocking, P->blocks[bi].prio ? prio_hi : prio_lo);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->side_done[bi], cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(e, "side streams");
  }
  const size_t r = P->nodes.size();
  P->nstream.assign(r, nullptr);
  for (auto* v : {&P->ev_keys, &P->ev_data, &P->ev_seg, &P->ev_leaf, &P->ev_gen}) v->assign(r, nullptr);
  for (size_t i = 0; i < r && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithPriority(&P->nstream[i], cudaStreamNonBlocking, prio_hi);
    for (auto* v : {&P->ev_keys, &P->ev_data, &P->ev_seg, &P->ev_leaf, &P->ev_gen})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&(*v)[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&P->copy_st, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_counts, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(e, "relation streams");
  P->leaf_ev.assign(2 * P->blocks.size(), nullptr);
  for (auto& ev : P->leaf_ev) {
    e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return bail(e, "cudaEventCreate");
  }
  // static tables: column descriptors, block column maps, block list, beta table
  for (auto& n : P->nodes) {
    if (!n.coldesc.empty()) {
      e = cudaMemcpyAsync(n.b.coldesc, n.coldesc.data(), n.coldesc.size() * sizeof(int2), cudaMemcpyHostToDevice, P->st);
      if (e != cudaSuccess) return bail(e, "upload column map");
    }
    if (n.g_colkind) {
      e = cudaMemcpyAsync(n.g_colkind, n.colkind.data(), n.colkind.size(), cudaMemcpyHostToDevice, P->st);
      if (e != cudaSuccess) return bail(e, "upload column kinds");
    }
  }
  std::vector<std::vector<int>> cols(P->blocks.size());
  for (size_t bi = 0; bi < P->blocks.size(); ++bi) {
    cols[bi] = block_cols(*P, bi);
    e = cudaMemcpyAsync(const_cast<int*>(P->blocks[bi].cols), cols[bi].data(), cols[bi].size() * sizeof(int),
                        cudaMemcpyHostToDevice, P->st);
    if (e != cudaSuccess) return bail(e, "upload block columns");
  }
  e = cudaMemcpyAsync(P->blocks_dev, P->blocks.data(), P->blocks.size() * sizeof(TsqrBlock), cudaMemcpyHostToDevice,
                      P->st);
  if (e != cudaSuccess) return bail(e, "upload blocks");
  beta_table(P->beta, P->beta_len, P->st);
  e = cudaStreamSynchronize(P->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return bail(e, "plan setup");
  *out = P;
  return FIGARO_OK;
}

int figaro_qr_r(figaro_plan_t p, double* R, int64_t ldr) {
  g_last_error.clear();
  if (!p || !R) return fail(FIGARO_ERR_INVALID_ARG, "null plan or R");
  if (ldr < p->N) return fail(FIGARO_ERR_INVALID_ARG, "ldr < N");
  const bool host = p->opt.mem == FIGARO_MEM_HOST;
  double* Rd = host ? p->Rtmp : R;
  int64_t ld = host ? p->N : ldr;
  int rc = run_r(*p, Rd, ld);
  if (rc != FIGARO_OK) return rc;
  if (host)
    FIG_CUDA(cudaMemcpy2DAsync(R, ldr * sizeof(double), Rd, ld * sizeof(double), p->N * sizeof(double), p->N,
                               cudaMemcpyDeviceToHost, p->st));
  return finish(*p, 7);
}

int figaro_qr_r_async(figaro_plan_t p, double* R, int64_t ldr) {
  g_last_error.clear();
  if (!p || !R) return fail(FIGARO_ERR_INVALID_ARG, "null plan or R");
  if (ldr < p->N) return fail(FIGARO_ERR_INVALID_ARG, "ldr < N");
  const bool host = p->opt.mem == FIGARO_MEM_HOST;
  double* Rd = host ? p->Rtmp : R;
  int64_t ld = host ? p->N : ldr;
  int rc = run_r(*p, Rd, ld);
  if (rc != FIGARO_OK) return rc;
  if (host)
    FIG_CUDA(cudaMemcpy2DAsync(R, ldr * sizeof(double), Rd, ld * sizeof(double), p->N * sizeof(double), p->N,
                               cudaMemcpyDeviceToHost, p->st));
  p->pending = true;
  return FIGARO_OK;
}

int figaro_plan_sync(figaro_plan_t p) {
  g_last_error.clear();
  if (!p) return fail(FIGARO_ERR_INVALID_ARG, "null plan");
  if (!p->pending) return FIGARO_OK;
  p->pending = false;
  return finish(*p, 7);
}

static int run_svd(figaro_plan_s& P, double* R_out) {
  int rc = run_r(P, P.Rtmp, P.N);
  if (rc != FIGARO_OK) return rc;
  StageClock clk(P);
  clk.start(7);
  jacobi_svd(P.Rtmp, P.N, P.N, P.svdW, P.svdV, P.sig, P.Vtmp, P.err_dev, P.st, &P.launches, P.opt.svd_max_sweeps,
             P.svdAux);
  clk.stop();
  if (R_out) {
    const bool host = P.opt.mem == FIGARO_MEM_HOST;
    FIG_CUDA(cudaMemcpyAsync(R_out, P.Rtmp, (size_t)P.N * P.N * sizeof(double),
                             host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, P.st));
  }
  return FIGARO_OK;
}

int figaro_svd(figaro_plan_t p, double* sigma, double* V, double* R) {
  g_last_error.clear();
  if (!p || !sigma || !V) return fail(FIGARO_ERR_INVALID_ARG, "null argument");
  int rc = run_svd(*p, R);
  if (rc != FIGARO_OK) return rc;
  const cudaMemcpyKind kind = p->opt.mem == FIGARO_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  FIG_CUDA(cudaMemcpyAsync(sigma, p->sig, p->N * sizeof(double), kind, p->st));
  FIG_CUDA(cudaMemcpyAsync(V, p->Vtmp, (size_t)p->N * p->N * sizeof(double), kind, p->st));
  return finish(*p, 8);
}

int figaro_pca(figaro_plan_t p, int32_t k, double* components, double* eigvals) {
  g_last_error.clear();
  if (!p || !components || !eigvals) return fail(FIGARO_ERR_INVALID_ARG, "null argument");
  if (k < 1 || k > p->N) return fail(FIGARO_ERR_INVALID_ARG, "k must be in [1, N]");
  int rc = run_svd(*p, nullptr);
  if (rc != FIGARO_OK) return rc;
  const bool host = p->opt.mem == FIGARO_MEM_HOST;
  const cudaMemcpyKind kind = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  FIG_CUDA(cudaMemcpy2DAsync(components, k * sizeof(double), p->Vtmp, p->N * sizeof(double), k * sizeof(double), p->N,
                             kind, p->st));
  double* ev = host ? p->hostbuf_dev : eigvals;
  square_values(p->sig, ev, k, p->st, &p->launches);
  if (host) FIG_CUDA(cudaMemcpyAsync(eigvals, ev, k * sizeof(double), cudaMemcpyDeviceToHost, p->st));
  return finish(*p, 8);
}

// ------------------------------------------------------------------ batches of instances
namespace fig {
__global__ void k_gather_status(int* const* words, int n, int* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = *words[i];
}
}  // namespace fig

int figaro_batch_destroy(figaro_batch_t b) {
  if (!b) return FIGARO_OK;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->status_dev) cudaFree(b->status_dev);
  if (b->status_host) cudaFreeHost(b->status_host);
  if (b->tasks_dev) cudaFree(b->tasks_dev);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
  return FIGARO_OK;
}

int figaro_batch_create(int32_t n, const figaro_plan_t* plans, double* const* R, double* const* components,
                        double* const* eigvals, const int32_t* k, figaro_batch_t* out) {
  using namespace fig;
  g_last_error.clear();
  if (!out || n < 1 || !plans || !R) return fail(FIGARO_ERR_INVALID_ARG, "null argument or n < 1");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    const figaro_plan_t p = plans[i];
    if (!p || !R[i]) return fail(FIGARO_ERR_INVALID_ARG, "null plan or R of instance " + std::to_string(i));
    if (p->opt.mem != FIGARO_MEM_DEVICE || p->opt.stage_timing)
      return fail(FIGARO_ERR_UNSUPPORTED, "batched plans need device memory and no stage timing");
    const int ki = k ? k[i] : 0;
    if (ki < 0 || ki > p->N || (ki > 0 && (!components || !eigvals || !components[i] || !eigvals[i])))
      return fail(FIGARO_ERR_INVALID_ARG, "PCA outputs of instance " + std::to_string(i));
    for (int j = 0; j < i; ++j)
      if (plans[j] == p) return fail(FIGARO_ERR_INVALID_ARG, "a plan appears twice in the batch");
  }
  auto* B = new (std::nothrow) figaro_batch_s();
  if (!B) return fail(FIGARO_ERR_NOMEM, "host allocation");
  B->plans.assign(plans, plans + n);
  auto bail = [&](cudaError_t e, const char* what) {
    figaro_batch_destroy(B);
    return fail(FIGARO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e = cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&B->status_dev, sizeof(int) * (n + 1) + sizeof(int*) * n);
  if (e == cudaSuccess) e = cudaMallocHost(&B->status_host, sizeof(int) * n);
  if (e != cudaSuccess) return bail(e, "batch setup");
  int** words = reinterpret_cast<int**>(B->status_dev + n + (n & 1));
  {
    std::vector<int*> w(n);
    for (int i = 0; i < n; ++i) w[i] = plans[i]->err_dev;
    e = cudaMemcpy(words, w.data(), sizeof(int*) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(e, "batch setup");
  }
  // the SVD + top-k components of every instance with k > 0: one thread block each, all in
  // one launch after every instance's R
  std::vector<JacobiTask> tasks;
  int max_n = 0;
  for (int i = 0; i < n; ++i) {
    figaro_plan_s& P = *plans[i];
    const int ki = k ? k[i] : 0;
    if (ki <= 0) continue;
    tasks.push_back(JacobiTask{P.Rtmp, P.N, P.N, P.svdW, P.svdV, P.sig, P.Vtmp, P.err_dev,
                               P.opt.svd_max_sweeps > 0 ? P.opt.svd_max_sweeps : kSvdDefaultSweeps, components[i], eigvals[i], ki});
    max_n = std::max(max_n, P.N);
  }
  if (!tasks.empty()) {
    e = cudaMalloc(&B->tasks_dev, sizeof(JacobiTask) * tasks.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(B->tasks_dev, tasks.data(), sizeof(JacobiTask) * tasks.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bail(e, "batch setup");
  }
  // one capture: every plan's pipeline on its own streams, forked from and joined to the
  // batch stream, so the instances are independent branches of one graph
  cudaEvent_t fork = nullptr;
  e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(e, "batch event");
  std::vector<cudaStream_t> saved(n);
  cudaGraph_t g = nullptr;
  int rc = FIGARO_OK;
  e = cudaStreamBeginCapture(B->st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(fork, B->st);
  for (int i = 0; i < n && e == cudaSuccess && rc == FIGARO_OK; ++i) {
    figaro_plan_s& P = *plans[i];
    saved[i] = P.st;
    P.st = P.exec;
    e = cudaStreamWaitEvent(P.exec, fork, 0);
    if (e != cudaSuccess) break;
    rc = enqueue_r(P, P.Rtmp, P.N);
    if (rc == FIGARO_OK && e == cudaSuccess)
      e = cudaMemcpyAsync(R[i], P.Rtmp, (size_t)P.N * P.N * sizeof(double), cudaMemcpyDeviceToDevice, P.exec);
    B->launches += P.launches;
    if (rc == FIGARO_OK && e == cudaSuccess) e = cudaEventRecord(P.join_out, P.exec);
    if (rc == FIGARO_OK && e == cudaSuccess) e = cudaStreamWaitEvent(B->st, P.join_out, 0);
  }
  if (e == cudaSuccess && rc == FIGARO_OK) {
    jacobi_svd_batch(B->tasks_dev, (int)tasks.size(), max_n, B->st, &B->launches);
    k_gather_status<<<1, 256, 0, B->st>>>(words, n, B->status_dev);
    ++B->launches;
    e = cudaMemcpyAsync(B->status_host, B->status_dev, sizeof(int) * n, cudaMemcpyDeviceToHost, B->st);
  }
  cudaError_t e_end = cudaStreamEndCapture(B->st, &g);
  for (int i = 0; i < n; ++i)
    if (saved[i]) plans[i]->st = saved[i];
  cudaEventDestroy(fork);
  if (e == cudaSuccess) e = e_end;
  if (e == cudaSuccess && rc == FIGARO_OK) e = cudaGraphInstantiate(&B->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (rc != FIGARO_OK) {
    cudaGetLastError();
    figaro_batch_destroy(B);
    return rc;
  }
  if (e != cudaSuccess) return bail(e, "batch graph");
  *out = B;
  return FIGARO_OK;
}

int figaro_batch_run(figaro_batch_t b, int32_t* status) {
  g_last_error.clear();
  if (!b) return fail(FIGARO_ERR_INVALID_ARG, "null batch");
  FIG_CUDA(cudaGraphLaunch(b->exec, b->st));
  FIG_CUDA(cudaStreamSynchronize(b->st));
  FIG_CUDA(cudaGetLastError());
  int first = FIGARO_OK;
  for (size_t i = 0; i < b->plans.size(); ++i) {
    if (status) status[i] = b->status_host[i];
    if (first == FIGARO_OK && b->status_host[i] != FIGARO_OK) first = b->status_host[i];
  }
  if (first != FIGARO_OK) return fail(first, "an instance of the batch failed (see the status array)");
  return FIGARO_OK;
}

int64_t figaro_batch_launches(figaro_batch_t b) { return b ? b->launches : -1; }

// ------------------------------------------------------------------ projections A X
// Theta_down prefixes of every relation (the forward forms them only for inner nodes) and
// |J| = the root's last prefix, copied to the host.
static int join_rows(figaro_plan_s& P, uint64_t* total) {
  using namespace fig;
  cudaStream_t st = P.st;
  for (auto& n : P.nodes) {
    ScanSrc src{SCAN_PLAIN_U64, n.b.theta, 0};
    scan_inclusive<uint64_t>(src, n.b.theta_incl, n.M, n.b.sizes, n.b.scan_tmp_u, st, &P.launches);
  }
  int32_t G = 0;
  const Node& root = P.nodes[P.root];
  FIG_CUDA(cudaMemcpyAsync(&G, root.b.sizes, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  FIG_CUDA(cudaStreamSynchronize(st));
  *total = 0;
  if (G > 0) {
    FIG_CUDA(cudaMemcpyAsync(total, root.b.theta_incl + (G - 1), sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    FIG_CUDA(cudaStreamSynchronize(st));
  }
  return FIGARO_OK;
}

int figaro_join_size(figaro_plan_t p, uint64_t* rows) {
  g_last_error.clear();
  if (!p || !rows) return fail(FIGARO_ERR_INVALID_ARG, "null argument");
  return join_rows(*p, rows);
}

int figaro_project(figaro_plan_t p, int32_t mode, const double* R, int64_t ldr, const double* X, int64_t ldx,
                   int32_t k, double* out, int64_t ldo, int64_t max_rows, int64_t* rows) {
  using namespace fig;
  g_last_error.clear();
  if (!p || !R) return fail(FIGARO_ERR_INVALID_ARG, "null plan or R");
  figaro_plan_s& P = *p;
  const int N = P.N;
  if (mode < FIGARO_PROJ_X || mode > FIGARO_PROJ_SCORES) return fail(FIGARO_ERR_INVALID_ARG, "mode");
  if (mode == FIGARO_PROJ_Q) k = N;
  if (k < 1 || (mode != FIGARO_PROJ_X && k > N)) return fail(FIGARO_ERR_INVALID_ARG, "k");
  if (mode == FIGARO_PROJ_X && (!X || ldx < k)) return fail(FIGARO_ERR_INVALID_ARG, "X or ldx");
  if (ldr < N || ldo < k) return fail(FIGARO_ERR_INVALID_ARG, "ldr or ldo");
  if (P.opt.mem != FIGARO_MEM_DEVICE) return fail(FIGARO_ERR_UNSUPPORTED, "projections need device memory");
  if ((int)P.nodes.size() > kMaxRel) return fail(FIGARO_ERR_UNSUPPORTED, "more than 32 relations");
  uint64_t total = 0;
  int rc = join_rows(P, &total);
  if (rc != FIGARO_OK) return rc;
  if (rows) *rows = (int64_t)total;
  if (total > (uint64_t)(max_rows < 0 ? 0 : max_rows))
    return fail(FIGARO_ERR_UNSUPPORTED, "the join has " + std::to_string(total) + " rows, more than max_rows");
  if (!out) return fail(FIGARO_ERR_INVALID_ARG, "null out");
  cudaStream_t st = P.st;
  FIG_CUDA(cudaMemsetAsync(P.err_dev, 0, sizeof(int), st));
  // X for the mode, N x k row-major, in the plan's scratch
  const double* Xd = X;
  int64_t ldxd = ldx;
  if (mode != FIGARO_PROJ_X) {
    if (mode == FIGARO_PROJ_Q) {
      tri_inverse(R, ldr, N, P.scatter, P.err_dev, st);
    } else {
      jacobi_svd(R, ldr, N, P.svdW, P.svdV, P.sig, P.Vtmp, P.err_dev, st, &P.launches, P.opt.svd_max_sweeps,
                 P.svdAux);
      scale_v(P.Vtmp, P.sig, N, k, mode == FIGARO_PROJ_U, P.scatter, P.err_dev, st);
    }
    Xd = P.scatter;
    ldxd = mode == FIGARO_PROJ_Q ? N : k;
  }
  // every relation's rows times its block of X
  std::vector<double*> Pk(P.nodes.size(), nullptr);
  auto release = [&]() {
    for (double* q : Pk)
      if (q) cudaFree(q);
  };
  for (size_t i = 0; i < P.nodes.size(); ++i) {
    Node& n = P.nodes[i];
    if (n.N == 0 || n.M == 0) continue;
    if (cudaMalloc(&Pk[i], sizeof(double) * n.M * k) != cudaSuccess) {
      cudaGetLastError();
      release();
      return fail(FIGARO_ERR_NOMEM, "projection buffers");
    }
    proj_rows(n.data, n.layout == FIGARO_COL_MAJOR ? 1 : n.ld, n.layout == FIGARO_COL_MAJOR ? n.ld : 1, n.M, n.N,
              Xd, ldxd, n.col_off, k, Pk[i], st);
  }
  // the nodes in pre-order
  std::vector<int> pos(P.nodes.size(), -1);
  for (size_t v = 0; v < P.pre.size(); ++v) pos[P.pre[v]] = (int)v;
  std::vector<ProjNode> pn(P.pre.size());
  for (size_t v = 0; v < P.pre.size(); ++v) {
    Node& n = P.nodes[P.pre[v]];
    ProjNode& q = pn[v];
    q.n_child = (int)n.children.size();
    for (int c = 0; c < q.n_child; ++c) q.child[c] = pos[n.children[c]];
    q.M = n.M;
    q.sizes = n.b.sizes;
    q.goff = n.b.goff;
    q.pgoff = n.b.pgoff;
    q.theta = n.b.theta;
    q.theta_incl = n.b.theta_incl;
    q.phid = n.b.phid;
    q.q = n.b.q;
    q.perm = n.b.sperm;
    q.P = Pk[P.pre[v]];
  }
  ProjNode* pn_dev = nullptr;
  cudaError_t e = cudaMalloc(&pn_dev, sizeof(ProjNode) * pn.size());
  if (e == cudaSuccess) e = cudaMemcpyAsync(pn_dev, pn.data(), sizeof(ProjNode) * pn.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && total > 0) {
    project(pn_dev, (int)pn.size(), k, total, out, ldo, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(P.err_host, P.err_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (pn_dev) cudaFree(pn_dev);
  release();
  if (e != cudaSuccess) return fail(FIGARO_ERR_CUDA, std::string("figaro_project: ") + cudaGetErrorString(e));
  if (P.err_host[0] != FIGARO_OK) return fail(P.err_host[0], "figaro_project: singular R or Sigma");
  return FIGARO_OK;
}

int figaro_pca_centered(figaro_plan_t p, int32_t k, double* components, double* eigvals) {
  using namespace fig;
  g_last_error.clear();
  if (!p || !components || !eigvals) return fail(FIGARO_ERR_INVALID_ARG, "null argument");
  if (k < 1 || k > p->N) return fail(FIGARO_ERR_INVALID_ARG, "k must be in [1, N]");
  figaro_plan_s& P = *p;
  int rc = run_r(P, P.Rtmp, P.N);
  if (rc != FIGARO_OK) return rc;
  cudaStream_t st = P.st;
  for (auto& n : P.nodes)
    join_colsum(n.b.heads, n.M, n.b.goff, n.b.hrow, n.b.phic, n.b.sizes, n.N, P.colsum + n.col_off, st, &P.launches);
  join_size(P.nodes[P.root].b.full, P.nodes[P.root].b.sizes, P.jsize, st, &P.launches);
  center_gram(P.Rtmp, P.N, P.colsum, P.jsize, P.scatter, st, &P.launches);
  jacobi_svd(P.scatter, P.N, P.N, P.svdW, P.svdV, P.sig, P.Vtmp, P.err_dev, st, &P.launches, P.opt.svd_max_sweeps,
             P.svdAux);
  const bool host = P.opt.mem == FIGARO_MEM_HOST;
  const cudaMemcpyKind kind = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  FIG_CUDA(cudaMemcpy2DAsync(components, k * sizeof(double), P.Vtmp, P.N * sizeof(double), k * sizeof(double), P.N,
                             kind, st));
  FIG_CUDA(cudaMemcpyAsync(eigvals, P.sig, k * sizeof(double), kind, st));
  return finish(P, 8);
}

int figaro_backward(figaro_plan_t p, const double* R, int64_t ldr, const double* Rbar, int64_t ldb,
                    double* const* grads, const int64_t* ldg) {
  using namespace fig;
  g_last_error.clear();
  if (!p || !R || !Rbar || !grads || !ldg) return fail(FIGARO_ERR_INVALID_ARG, "null argument");
  if (ldr < p->N || ldb < p->N) return fail(FIGARO_ERR_INVALID_ARG, "ldr or ldb < N");
  if (!p->opt.gradients) return fail(FIGARO_ERR_UNSUPPORTED, "plan made without gradients = 1");
  if (p->opt.mem != FIGARO_MEM_DEVICE) return fail(FIGARO_ERR_UNSUPPORTED, "gradients need device memory");
  const int r = (int)p->nodes.size();
  for (int i = 0; i < r; ++i)
    if (p->nodes[i].N > 0 && (!grads[i] || ldg[i] < p->nodes[i].M))
      return fail(FIGARO_ERR_INVALID_ARG, "gradient buffer of relation " + std::to_string(i));
  figaro_plan_s& P = *p;
  cudaStream_t st = P.st;
  const int N = P.N;
  const int64_t NN = (int64_t)N * N;
  FIG_CUDA(cudaMemsetAsync(P.err_dev, 0, sizeof(int), st));
  grad_w(R, ldr, Rbar, ldb, N, P.grad_w, P.grad_w + NN, P.grad_w + 2 * NN, P.err_dev, st);
  auto view = [&](int i) {
    Node& n = P.nodes[i];
    GradNode g{};
    g.N = N;
    g.Ni = n.N;
    g.col_off = n.col_off;
    g.n_child = (int)n.children.size();
    g.is_root = n.root;
    g.M = n.M;
    g.sizes = n.b.sizes;
    g.goff = n.b.goff;
    g.g2p = n.b.g2p;
    g.row_gid = n.b.row_gid;
    g.perm = n.b.sperm;
    g.heads = n.b.heads;
    g.ldh = n.M;
    g.hrow = n.b.hrow;
    g.phic = n.b.phic;
    g.phiu = n.b.phiu;
    g.q = n.b.q;
    for (int c = 0; c < g.n_child; ++c) {
      const Node& ch = P.nodes[n.children[c]];
      g.cphid[c] = ch.b.phid;
      g.cup[c] = ch.g_up;
      g.cld[c] = ch.pbound;
    }
    g.colkind = n.g_colkind;
    g.up = n.g_up;
    g.ldu = n.pbound;
    g.dn = n.g_dn;
    g.ldd = n.pbound;
    g.W = P.grad_w;
    g.phi = n.g_phi;
    g.data = n.data;
    g.rs = n.layout == FIGARO_COL_MAJOR ? 1 : n.ld;
    g.cs = n.layout == FIGARO_COL_MAJOR ? n.ld : 1;
    g.sdata = n.b.sperm ? n.b.sdata : nullptr;      // written by the forward whenever it sorted
    g.lds = n.b.lds;
    g.grad = grads[i];
    g.ldg = ldg[i];
    return g;
  };
  for (int i = 0; i < r; ++i) {
    Node& n = P.nodes[i];
    grad_clear(n.g_up, n.pbound, n.b.sizes, N, n.pbound, st);
    grad_clear(n.g_dn, n.pbound, n.b.sizes, N, n.pbound, st);
  }
  for (int i : P.post)
    if (!P.nodes[i].root) grad_up(view(i), P.nodes[i].M, st);
  for (int i : P.pre) {
    Node& n = P.nodes[i];
    for (int j = 0; j < (int)n.children.size(); ++j) {
      Node& ch = P.nodes[n.children[j]];
      grad_down(view(i), j, ch.g_dn, ch.pbound, n.M, st);
    }
  }
  for (int i = 0; i < r; ++i)
    if (P.nodes[i].N > 0) grad_rows(view(i), P.nodes[i].M, st);
  FIG_CUDA(cudaGetLastError());
  FIG_CUDA(cudaMemcpyAsync(P.err_host, P.err_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  FIG_CUDA(cudaStreamSynchronize(st));
  if (P.err_host[0] != FIGARO_OK)
    return fail(P.err_host[0], P.err_host[0] == FIGARO_ERR_SINGULAR ? "R has a zero diagonal entry"
                                                                    : "device error in figaro_backward");
  return FIGARO_OK;
}

int figaro_plan_get_info(figaro_plan_t p, figaro_plan_info* info) {
  if (!p || !info) return fail(FIGARO_ERR_INVALID_ARG, "null argument");
  info->n_rel = (int32_t)p->nodes.size();
  info->n_cols = p->N;
  info->input_cells = p->input_cells;
  info->input_bytes = p->input_bytes;
  info->workspace_bytes = (int64_t)p->arena_bytes;
  info->r0_rows = p->r0_rows;
  info->launches = p->launches;
  info->tsqr_leaf_flops = p->leaf_flops;
  info->refined = p->refined;
  info->reserved = 0;
  return FIGARO_OK;
}

int figaro_stage_times(figaro_plan_t p, double* ms, int64_t* counts, int32_t n) {
  if (!p) return -FIGARO_ERR_INVALID_ARG;
  for (int s = 0; s < n && s < kStages; ++s) {
    if (ms) ms[s] = p->stage_ms[s];
    if (counts) counts[s] = p->stage_launch[s];
  }
  return kStages;
}

int figaro_reset_stage_times(figaro_plan_t p) {
  if (!p) return FIGARO_ERR_INVALID_ARG;
  for (int s = 0; s < kStages; ++s) {
    p->stage_ms[s] = 0.0;
    p->stage_launch[s] = 0;
  }
  for (auto& v : p->block_leaf_ms) v = 0.0;
  return FIGARO_OK;
}

int figaro_block_times(figaro_plan_t p, int32_t max, double* leaf_ms, int32_t* n_cols, int64_t* rows) {
  if (!p || max < 0) return -FIGARO_ERR_INVALID_ARG;
  const int nb = (int)p->blocks.size();
  for (int b = 0; b < nb && b < max; ++b) {
    if (leaf_ms) leaf_ms[b] = b < (int)p->block_leaf_ms.size() ? p->block_leaf_ms[b] : 0.0;
    if (n_cols) n_cols[b] = p->blocks[b].n;
    if (rows) rows[b] = b < (int)p->block_rows.size() ? p->block_rows[b] : 0;
  }
  return nb;
}

int64_t figaro_debug_read(figaro_plan_t p, int32_t rel, int32_t what, void* dst, int64_t bytes) {
  if (!p || rel < 0 || rel >= (int)p->nodes.size()) return -FIGARO_ERR_INVALID_ARG;
  const Node& n = p->nodes[rel];
  int32_t sz[4] = {0, 0, 0, 0};
  if (cudaStreamSynchronize(p->st) != cudaSuccess ||
      cudaMemcpy(sz, n.b.sizes, sizeof(sz), cudaMemcpyDeviceToHost) != cudaSuccess)
    return -FIGARO_ERR_CUDA;
  const int64_t G = sz[0], Pg = sz[1];
  auto copy2d = [&](const void* src, int64_t rows, int64_t cols, int64_t ld, size_t esz) -> int64_t {
    const int64_t need = rows * cols * (int64_t)esz;
    if (dst && bytes >= need && need > 0)
      if (cudaMemcpy2D(dst, rows * esz, src, ld * esz, rows * esz, cols, cudaMemcpyDeviceToHost) != cudaSuccess)
        return -FIGARO_ERR_CUDA;
    return need;
  };
  switch (what) {
    case FIGARO_DBG_SIZES: {
      int64_t v[8] = {n.M, G, Pg, n.M - G, (!n.leaf && !n.root) ? G - Pg : 0, n.root ? G : 0, n.K, n.N_sub};
      if (dst && bytes >= (int64_t)sizeof(v)) std::memcpy(dst, v, sizeof(v));
      return sizeof(v);
    }
    case FIGARO_DBG_PERM: {
      if (!n.b.sperm) {   // identity
        if (dst && bytes >= n.M * 4)
          for (int64_t r = 0; r < n.M; ++r) static_cast<int32_t*>(dst)[r] = (int32_t)r;
        return n.M * 4;
      }
      return copy2d(n.b.sperm, n.M, 1, n.M, 4);
    }
    case FIGARO_DBG_GROUP_OFF: return copy2d(n.b.goff, G + 1, 1, G + 1, 4);
    case FIGARO_DBG_COUNTS: {
      const int64_t need = 4 * G * 8;
      if (dst && bytes >= need) {
        std::vector<int32_t> off(G + 1);
        std::vector<uint64_t> th(G), fu(G), ci(G);
        if (cudaMemcpy(off.data(), n.b.goff, (G + 1) * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(th.data(), n.b.theta, G * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(fu.data(), n.b.full, G * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(ci.data(), n.b.phic, G * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
          return -FIGARO_ERR_CUDA;
        uint64_t* o = static_cast<uint64_t*>(dst);
        for (int64_t g = 0; g < G; ++g) {
          o[4 * g] = (uint64_t)(off[g + 1] - off[g]);
          o[4 * g + 1] = th[g];
          o[4 * g + 2] = fu[g];
          o[4 * g + 3] = ci[g];
        }
      }
      return need;
    }
    case FIGARO_DBG_PCOUNTS: {
      const int64_t need = 2 * Pg * 8;
      if (dst && bytes >= need) {
        std::vector<uint64_t> d(Pg), u(Pg);
        if (cudaMemcpy(d.data(), n.b.phid, Pg * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(u.data(), n.b.phiu, Pg * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
          return -FIGARO_ERR_CUDA;
        uint64_t* o = static_cast<uint64_t*>(dst);
        for (int64_t q = 0; q < Pg; ++q) { o[2 * q] = d[q]; o[2 * q + 1] = u[q]; }
      }
      return need;
    }
    case FIGARO_DBG_TAILS:
      if (!n.b.tails) return -FIGARO_ERR_INVALID_ARG;   // formed in the leaf, never stored
      return copy2d(n.b.tails, n.M - G, n.N, n.M, 8);
    case FIGARO_DBG_HEADS: return copy2d(n.b.heads, G, n.N, n.M, 8);
    case FIGARO_DBG_GEN_TAILS:
      if (n.leaf || n.root) return 0;
      return copy2d(n.b.gtails, G - Pg, n.N_sub, n.M, 8);
    case FIGARO_DBG_DATA:
      if (n.leaf || n.root) return 0;
      return copy2d(n.b.data2, Pg, n.N_sub, n.M, 8);
    case FIGARO_DBG_ROOT_ROWS:
      if (!n.root) return 0;
      return copy2d(n.b.rootrows, G, n.N_sub, n.M, 8);
    default: return -FIGARO_ERR_INVALID_ARG;
  }
}

}  // extern "C"
