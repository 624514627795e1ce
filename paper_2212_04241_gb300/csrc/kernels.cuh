// Device-side views of a plan and of a batch arena, shared by the kernels and the runtime.
#pragma once

#include <cuda_runtime.h>

#include "jt_internal.h"

namespace jt {

constexpr int kWarps = 8;               // warps (independent work items) per block of a layer launch
constexpr int kThreads = 32 * kWarps;

struct DevPlan {
  const DClique *cl;
  const DMap *maps;
  const DTask *tasks;
  const DItem *citems;
  const DItem *ditems;
  const int32_t *ipool;
  const float *base32;
  const int32_t *card;       // [n]
  const int64_t *post_off;   // [n]
  const int32_t *comp_ptr;   // [n_cliques + 1] variables of the component rooted at a clique
  const int32_t *comp_vars;  // [n]
  const int32_t *comp_cliques;  // non-root cliques of each component
  const int32_t *comp_roots;    // [n_comp] component root cliques
  const int32_t *comp_owner;    // per comp_cliques entry: its component
  const int32_t *comp_var_owner;  // per comp_vars entry: its component
  int32_t n_comp_vars;          // entries of comp_vars
  int32_t n_comp_cliques;       // entries of comp_cliques
  const int32_t *pgroup_ptr;    // [n_pgroups + 1] variable groups of the posterior kernel
  // dataflow schedule: per pass, the items of each flow layer (collect:
  // deepest layer first; distribute: root first) and the producers a
  // clique's units wait for on their tile
  const int64_t *c_flow_pref;   // [n_flow_layers + 1] items before each flow layer
  const int64_t *c_flow_begin;  // [n_flow_layers] first item of each flow layer
  const int64_t *d_flow_pref;
  const int64_t *d_flow_begin;
  const uint32_t *c_need;       // [n_cliques] collect items of the children that send a message
  const int32_t *c_notify;      // [n_cliques] parent that receives the clique's message, or -1
  const uint32_t *d_need;       // [n_cliques] items of the parent's task that writes the clique's ratio
  const int32_t *slice_var;     // sliced plan: [n] 1 for the observed set; nullptr otherwise
  int32_t n_flow_layers;
  uint64_t wait_limit_ns;       // bound of a dataflow wait
  int32_t n_comp;
  int32_t n_pgroups;
  int32_t n_vars;
  int32_t n_cliques;
  int32_t root;
  int32_t rescale;           // 1: messages scaled by 2^-k (k per case and message)
  int32_t recompute;         // 1: no stored clique tables; the distribute pass recomputes them
  int32_t max_maps;          // most maps of a clique (the warp's shared-memory map layout)
  int32_t msg_prefetch;      // 1: collect requests each batch's child-message rows into L2 when it starts
  int32_t sec_rows;          // shared-memory rows (W floats) per warp of the distribute kernels (fused pairs)
  int64_t fused_items;       // fused items in the work lists (0: the plain distribute kernels)
  int64_t psi_rows;          // rows of one tile's psi region (sum |C|)
  int64_t sep_rows;          // rows of one tile's message regions
  int64_t post_rows;         // rows of one tile's posterior region (sum card)
  int64_t n_partials;
  int64_t n_groups;
  // plan pruned to a query set: rows of evidence and posteriors keep the
  // full network's layout (identity maps when nothing was pruned)
  const int32_t *io_var;       // [n_vars] evidence column of each kept variable; nullptr: identity
  const int32_t *io_dropped;   // [n_dropped] evidence columns that must stay unobserved
  const int32_t *io_post_col;  // [post_rows] output column of each posterior column; nullptr: identity
  const int32_t *io_nan_cols;  // [n_nan_cols] output columns of removed variables (NaN)
  int64_t io_post_rows;        // output columns per case
  int32_t io_n;                // evidence columns per case
  int32_t n_dropped;
  int32_t n_nan_cols;
};

// Per-batch device memory.  Row-major [tile][row][W] for the FP32 tables,
// W = 32 * cases-per-thread consecutive evidence cases in a row.
struct DevArena {
  float *psi;          // collect-pass clique tables
  float *phistar;      // collect messages (raw sums), one block of rows per clique
  float *rho;          // distribute ratios phi** / phi*, same layout as phistar
  float *post;         // unnormalised posterior marginals
  float *partial;      // partial sums of split segments [tile][slot][W]
  uint32_t *maxbits;   // [tile][clique][W] bit pattern of max psi (>= 0)
  uint32_t *counters;  // [tile][group] pieces finished
  int32_t *ev;         // [tile][var][W] evidence, -1 = unobserved
  int32_t *bad;        // [tile * W] 1 = invalid evidence
  uint32_t *ready;     // [tile][2][clique] dataflow counters (collect, distribute)
  unsigned long long *queue;  // dataflow unit counters: [0] collect pass, [16] distribute pass
  uint32_t *errflag;   // one word per arena: nonzero after a bounded device wait expired
  int32_t tiles;       // tiles in this chunk
};

// launchers (kernels.cu)
void launch_evidence(int cpt, const int32_t *d_ev_in, int32_t n_cases, const DevPlan &P,
                     const DevArena &A, cudaStream_t s);
void launch_collect(int cpt, const DevPlan &P, const DevArena &A, int64_t item_begin,
                    int64_t n_items, int max_maps, cudaStream_t s);
void launch_distribute(int cpt, const DevPlan &P, const DevArena &A, int64_t item_begin,
                       int64_t n_items, cudaStream_t s);
void launch_finalize(int cpt, const DevPlan &P, const DevArena &A, int32_t n_cases,
                     int64_t root_sep_row, double *d_log_pe, double *d_post, int32_t *d_status,
                     cudaStream_t s);
size_t collect_smem_bytes(int cpt, int max_maps);        // block (capped at kCollectSmemLimit)
size_t collect_warp_smem_bytes(int cpt, int max_maps);   // one warp
constexpr size_t kCollectSmemLimit = 220 * 1024;
// raise the dynamic shared-memory limit of the collect kernels (once per
// plan; `sliced`: the instantiation for plans specialised to an observed set)
cudaError_t configure_collect_smem(int cpt, bool sliced, size_t bytes);
// the log P(e) kernel keeps one word per component tree in shared memory
size_t logpe_smem_bytes(int n_comp);
cudaError_t configure_logpe_smem(int n_comp);
// the posterior kernel stages a case tile's outputs and inputs in shared memory
size_t posterior_smem_bytes(int W);
cudaError_t configure_posterior_smem();
constexpr int kMaxTilesPerChunk = 16384;
// dataflow schedule: one persistent launch per pass (blocks = SMs x resident blocks per SM)
void launch_collect_flow(int cpt, const DevPlan &P, const DevArena &A, int blocks, int max_maps, cudaStream_t s);
void launch_distribute_flow(int cpt, const DevPlan &P, const DevArena &A, int blocks, cudaStream_t s);
int flow_blocks_per_sm(int cpt, bool sliced, int max_maps);  // the collect pass
// the distribute pass, in the plan's mode (plain, fused items, recomputed tables)
int distribute_flow_blocks_per_sm(int cpt, const DevPlan &P);
// explicit (item, tile) unit lists: one launch per pass over tiles at
// different layers (iteration-level batching of the serving loop)
void launch_collect_units(int cpt, const DevPlan &P, const DevArena &A, const int2 *units, int n_units, int max_maps,
                          cudaStream_t s);
void launch_distribute_units(int cpt, const DevPlan &P, const DevArena &A, const int2 *units, int n_units,
                             cudaStream_t s);
// dynamic shared memory of a distribute block (fused pairs' secondary sums)
size_t distribute_smem_bytes(int cpt, int sec_rows);
// a warp's shared memory for a clique's maps when recomputing its rows
size_t recompute_warp_smem_bytes(int cpt, int max_maps);
cudaError_t configure_distribute_smem(int cpt, int sec_rows, int max_maps);

// plain FP64 path
void launch_plain_init(double *psi, const double *base, const DPlainMap &m, const int64_t *pool,
                       const int32_t *d_ev, cudaStream_t s);
void launch_plain_marg(const double *src, double *dst, const DPlainMap &m, const int64_t *pool,
                       cudaStream_t s);
void launch_plain_extend(double *x, const double *y, const DPlainMap &m, const int64_t *pool,
                         cudaStream_t s);
void launch_plain_divide(double *num, const double *den, int64_t n, cudaStream_t s);
void launch_plain_finalize(const double *pe, const double *marg, const int32_t *d_ev,
                           const int32_t *card, const int64_t *post_off, int32_t n_vars,
                           double *d_log_pe, double *d_post, int32_t *d_status, cudaStream_t s);

}  // namespace jt
