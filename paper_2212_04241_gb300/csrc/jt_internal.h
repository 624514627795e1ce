// Internal structures shared by the host compiler, the runtime and the kernels.
#pragma once

#include <array>
#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/jt.h"

namespace jt {

// ---------------------------------------------------------------------------
// Device descriptors (plain old data, copied to the device once per plan)
// ---------------------------------------------------------------------------

// A clique for the collect pass.  Its table is laid out with the upward
// separator's variables outermost, so entry e = s*R + u with s the separator
// entry (segment) and u the row inside the segment.
struct DClique {
  int64_t psi_row;    // first row of this clique inside a tile's psi region
  int64_t nsep;       // |S_up| (1 for the root)
  int64_t R;          // |C| / |S_up|
  int64_t base_off;   // offset into the FP32 base-table pool
  int64_t sep_row;    // first row of its upward message inside a tile's sep region
  int32_t map_begin;  // collect maps [map_begin, map_end)
  int32_t map_end;
  int32_t parent;     // -1 for the root
  int32_t is_root;    // 1 for a component root: the tree root, or a clique
                      // whose separator towards its parent is empty
  int32_t comp_begin; // component roots: the other cliques of the component,
  int32_t comp_end;   //   [comp_begin, comp_end) in the comp_cliques list
  int32_t comp_base_exp;  // component roots: sum of the component's base-table exponents
  int32_t sev_begin;  // evidence applied to its upward message as it is
  int32_t sev_end;    //   written: MAP_SEP_EVIDENCE maps [sev_begin, sev_end)
  int32_t slice_begin;  // sliced plan: the clique's variables of the observed
  int32_t slice_end;    //   set, MAP_SLICE maps [slice_begin, slice_end)
  int64_t bmap_A;     // sliced plan: base-table entry of table entry s*R+u
  int64_t bmap_B;     //   = A[s] + B[u] (int32 pool offsets); unused otherwise
};

// A linear index map over a clique's entries: idx(s*R + u) = A[s] + B[u].
//   kind MAP_CHILD: idx is the entry of child clique `src`'s upward message
//   kind MAP_EVIDENCE: idx is the digit (state) of variable `src` at the
//     entry; the entry is zeroed for the cases that observed another state
//   kind MAP_SEP_EVIDENCE: the same over the entries s of the clique's
//     upward message only (A[s] is the digit, B unused), applied to the
//     message entry when it is written
//   kind MAP_SLICE (sliced plan): variable `src` of the observed set in the
//     clique; A_off is its stride in the full base table
enum { MAP_CHILD = 0, MAP_EVIDENCE = 1, MAP_SEP_EVIDENCE = 2, MAP_SLICE = 3 };
struct DMap {
  int64_t A_off;      // int32 pool offset, nsep entries
  int64_t B_off;      // int32 pool offset, R entries
  int64_t src_row;    // MAP_CHILD: child's sep_row; evidence maps: the variable's posterior row
  int32_t kind;
  int32_t src;        // child clique / variable
};

// A distribute target: for t in [0, T),
//   value(t) = sum_{u < U} X[A[t] + B[u]] * Y[sA[t] + sB[u]]
// src_sep == 0: X = psi of `clique`, Y = its upward ratio rho (a component
//   root uses 2^-k instead);
// src_sep == 1: X = phi* and Y = rho of the separator above `clique` (their
//   product is that separator's calibrated marginal; sA = A, sB = B).
//   kind TASK_CHILD: writes rho_child[t] = value(t) / phistar_child[t]
//   kind TASK_POSTERIOR: writes the unnormalised marginal of variable dst
//
// Fused pair (sec_b > 0): the task also computes a second marginal of the
// same table (the "secondary", another child separator or posterior
// variable T2 of the clique) from the same rows, so the table is read once
// for both.  With F = T1 and T2's common variables, the primary's targets
// are enumerated F-block by F-block (t = f * sec_a + t', f over F's
// entries, t' over T1 \ F's), and the rows u of a target with T2 \ T1's
// variables outermost.  Within one F-block (sec_a consecutive targets) the
// rows touch exactly sec_b secondary targets, k = Ku[u]; the warp sums
// them in shared memory and writes target (f, k) at row
// sec_dst_row + OSf[f] + OSk[k] (the secondary's own enumeration) when the
// F-block ends.  The primary's target t is written at row
// dst_row + OP[t] (its enumeration before the reordering).  The secondary
// task itself is marked absorbed and gets no work items.
enum { TASK_CHILD = 0, TASK_POSTERIOR = 1 };
constexpr int64_t kFusedRowBytes = 6144;  // shared memory per warp for a fused pair's secondary sums
constexpr int64_t kFusedMaxRows = 4096;   // a fused primary target has at most this many rows
constexpr int64_t kFusedTerms = 256;      // rows summed per secondary target before a partial is written
constexpr int64_t kFusedMinRows = 128;    // a pair is fused only where items hold at least this many rows
struct DTask {
  int64_t T, U;
  int64_t A_off, B_off, sA_off, sB_off;  // int32 pool offsets
  int64_t dst_row;    // TASK_CHILD: child's sep_row; TASK_POSTERIOR: row in the posterior region
  int32_t clique;     // source clique
  int32_t kind;
  int32_t dst;        // child clique / variable
  int32_t src_sep;
  // fused pair (sec_b == 0: none); the fused items use their own tables
  // (the fields above stay the task's plain enumeration, used when a work
  // shape gives the pair plain items)
  int64_t fA_off, fB_off, fsA_off, fsB_off;  // A, B, sA, sB of the reordered enumeration
  int64_t op_off;     // OP[t]: primary target t's row offset (int32 pool; -1: t itself)
  int64_t ku_off;     // Ku[u]: secondary target of row u inside the F-block
  int64_t osf_off;    // OSf[f]
  int64_t osk_off;    // OSk[k]
  int64_t sec_dst_row;
  int32_t sec_a;      // primary targets per F-block
  int32_t sec_b;      // secondary targets per F-block
  int32_t sec_kind;   // TASK_CHILD / TASK_POSTERIOR
  int32_t sec_dst;    // child clique / variable
  int32_t sec_task;   // index of the partner task
  int32_t absorbed;   // 1: the partner of a fused pair (gets no items while the pair is fused)
};

// One warp's work item in a layer launch (the same list serves every tile).
//   split == 0: the warp owns segments [t0, t0+nt)
//   split == 1: the warp owns rows [u0, u0+nu) of segment t0; when the
//               segment has several pieces, the warp writes a partial sum
//               and the last piece to finish combines them in piece order
struct DItem {
  int64_t t0, nt;
  int64_t u0, nu;
  int32_t task;       // clique (collect) or task (distribute)
  int32_t split;
  int32_t npieces;
  int32_t piece;
  int32_t group;      // split group (counter index), -1 if npieces == 1
  int32_t partial;    // partial-sum slot of this piece
  int32_t fused;      // 1: a fused pair's item (the task's primary and secondary marginals)
};

// Plain FP64 path: descriptor of a mixed-radix mapping from the entries of a
// source table onto a target table (one thread per source entry).
struct DPlainMap {
  int64_t size;       // source entries
  int64_t var_off;    // offset into the int64 plain pool: nv triples (card, src stride, dst stride)
  int32_t nv;
  int32_t pad;
};

// ---------------------------------------------------------------------------
// Host plan
// ---------------------------------------------------------------------------

struct HostClique {
  // Layout of the clique's tables (psi, messages, maps).  In a plan
  // specialised to an observed set O (every case observes the variables of
  // O), the tables leave O's variables out ("sliced"); the base table keeps
  // the full layout (fvars...) and each case reads the slice of its states.
  std::vector<int> vars;        // layout order: upward separator first
  std::vector<int> card;
  std::vector<int64_t> stride;  // stride of vars[i] in this table (last fastest)
  int64_t size = 1;
  std::vector<int> fvars;       // full layout of the base table (= vars when nothing is sliced)
  std::vector<int64_t> fstride;
  int64_t fsize = 1;
  int n_up = 0;                 // number of upward-separator variables
  int64_t nsep = 1, R = 1;
  int parent = -1, depth = 0;
  std::vector<int> children;
  std::vector<int> homed;       // variables whose CPT this clique holds
  std::vector<int> ev_clique;   // batched path: evidence gathered per clique entry
  std::vector<int> ev_sep;      // batched path: evidence applied to the upward message
  std::vector<int> owned;       // variables whose posterior this clique's table provides
  std::vector<int> owned_sep;   // variables whose posterior its upward separator provides
};

struct Level {
  // collect and distribute work of one tree layer
  int64_t c_item_begin = 0, c_item_end = 0;   // into collect_items
  int64_t d_item_begin = 0, d_item_end = 0;   // into distribute_items
  int c_max_maps = 0;                          // most maps of a clique in the layer
};

struct Plan {
  // network
  int n = 0;
  std::vector<int> card;
  std::vector<int> pptr, par;
  std::vector<double> cpt;
  std::vector<int64_t> cpt_off;
  std::vector<int64_t> post_off;  // per variable, offset into a posterior row
  int64_t sum_card = 0;

  // tree
  std::vector<HostClique> cl;
  int root = 0;
  int height = 0;
  std::vector<int> bfs;           // BFS order from the root
  std::vector<int> assign;        // CPT v -> clique
  std::vector<int> post_src;      // variable -> smallest clique containing it
  int64_t sum_cl = 0, max_cl = 0, sum_sep = 0;
  int64_t sum_base = 0;           // entries of the base tables (full layouts)
  std::vector<int32_t> slice_var; // sliced plan: 1 for the variables of the observed set
  int n_sliced = 0;

  // device-side description (host copies)
  std::vector<DClique> dcl;
  std::vector<DMap> dmap;
  std::vector<DTask> dtask;
  std::vector<DItem> citems, ditems;
  std::vector<Level> levels;      // index = depth
  std::vector<int32_t> ipool;     // int32 index tables
  std::vector<float> base32;
  std::vector<double> base64;
  int64_t sep_rows = 0;           // rows of a tile's sep region (sum of nsep incl. root)
  int64_t n_groups = 0, n_partials = 0;
  int32_t base_exp_sum = 0;       // sum of the FP32 base-table power-of-two exponents
  // variables of each component tree, listed under its root clique (CSR)
  std::vector<int32_t> comp_ptr;  // [n_cliques + 1]
  std::vector<int32_t> comp_vars; // [n]
  std::vector<int32_t> comp_cliques;  // non-root cliques of each component, grouped by component
  std::vector<int32_t> comp_roots;    // component root cliques
  std::vector<int32_t> comp_owner;    // per comp_cliques entry: its component (index into comp_roots)
  std::vector<int32_t> comp_var_owner;  // per comp_vars entry: its component (index into comp_roots)
  std::vector<int32_t> pgroup_ptr;    // consecutive variable groups of <= 16 posterior columns
  // dataflow schedule (see DevPlan)
  std::vector<int64_t> c_flow_pref, c_flow_begin, d_flow_pref, d_flow_begin;
  std::vector<uint32_t> c_need, d_need;
  std::vector<int32_t> c_notify;

  // plain path
  std::vector<DPlainMap> pmap;
  std::vector<int64_t> ppool;
  std::vector<int> p_child_map;   // per clique: child entries -> its separator
  std::vector<int> p_parent_map;  // per clique: parent entries -> its separator
  std::vector<int> p_post_map;    // per variable: owner entries -> the variable
  std::vector<int> p_root_map;    // root entries -> scalar (size 1)
  std::vector<int> p_init_map;    // per clique: entries -> (unused dst), digit decode
  std::vector<int64_t> p_base_off;  // per clique, offset in base64 / plain psi
  std::vector<int64_t> p_sep_off;   // per clique, offset in plain sep arrays

  // pruned plan (query set): the tree is built on the kept variables only;
  // evidence and posterior rows keep the full network's layout
  int io_n = 0;                       // variables of a row of evidence (full network)
  int64_t io_sum_card = 0;            // columns of a posterior row (full network)
  int n_pruned = 0;                   // barren variables removed
  std::vector<int32_t> io_var;        // kept variable -> its id in the full network
  std::vector<int32_t> io_dropped;    // ids of the removed variables
  std::vector<int32_t> io_post_col;   // kept posterior column -> full-row column
  std::vector<int32_t> io_nan_cols;   // full-row columns of the removed variables

  // rows per work item used in each size bucket, and the entries there
  std::array<int32_t, JT_SIZE_BUCKETS> c_bucket_rows{}, d_bucket_rows{};
  std::array<int64_t, JT_SIZE_BUCKETS> c_bucket_entries{}, d_bucket_entries{};

  jt_compile_opts opts{};
  int cpt_per_thread = 4;
  int recompute = 0;              // 1: no stored clique tables; distribute recomputes them
  int sec_rows = 0;               // largest sec_b of the fused tasks (shared-memory rows per warp)
  int tile = 128;
  int rows_per_cta = 2048;
};

// compile.cpp
jt_status build_plan(int32_t n, const int32_t *card, const int32_t *pptr, const int32_t *par,
                     const double *cpt, const jt_compile_opts &opts, Plan &P, std::string &err);
// the work lists of a built plan (items of both passes, flow layers,
// producer counts) for the work-shape options of opts (items_per_tile*,
// rows_per_cta, *_rows_by_bucket, stall_clique)
jt_status emit_work(Plan &P, const jt_compile_opts &opts, std::string &err);
// build_plan on the network pruned to opts.query_set (build_plan when none)
jt_status build_plan_pruned(int32_t n, const int32_t *card, const int32_t *pptr, const int32_t *par,
                            const double *cpt, const jt_compile_opts &opts, Plan &P, std::string &err);

void set_error(const std::string &msg);
// size bucket of a table of `rows` entries: floor(log2(rows)), capped
int size_bucket(int64_t rows);

// Runs the body of a C entry point: a C++ exception (a failed host
// allocation, a thread that cannot start) becomes a status, never an abort.
template <class F>
jt_status guarded(F &&body) {
  try {
    return body();
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    return JT_ENOMEM;
  } catch (const std::exception &e) {
    set_error(std::string("host error: ") + e.what());
    return JT_EINVAL;
  }
}

// cpu_layers.cpp: the multi-core CPU comparator (jt_infer_cpu)
jt_status cpu_layers_infer(const Plan &P, int32_t n_cases, const int32_t *ev, double *log_pe, double *post,
                           int32_t *status, int threads);

}  // namespace jt
