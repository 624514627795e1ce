// C ABI: plan lifetime, table arena, layer scheduling (CUDA graphs), the
// batched and plain inference drivers.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <exception>
#include <map>
#include <mutex>
#include <new>
#include <string>

#include "kernels.cuh"
#include "runtime.h"

namespace jt {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

#define JT_CUDA_TRY(expr)                                                     \
  do {                                                                        \
    cudaError_t _e = (expr);                                                  \
    if (_e != cudaSuccess) {                                                  \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));          \
      return JT_ECUDA;                                                        \
    }                                                                         \
  } while (0)

static size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// arena
// ---------------------------------------------------------------------------
ArenaLayout arena_layout(const Plan &P) {
  ArenaLayout L{};
  const size_t W = (size_t)P.tile;
  // recomputed clique tables: no psi region (its base pointer still anchors
  // the message offsets of the kernels)
  L.psi = P.recompute ? 0 : align_up(sizeof(float) * W * (size_t)P.sum_cl);
  L.sep = align_up(sizeof(float) * W * (size_t)P.sep_rows);
  L.post = align_up(sizeof(float) * W * (size_t)P.sum_card);
  L.partial = align_up(sizeof(float) * W * (size_t)std::max<int64_t>(1, P.n_partials));
  L.maxbits = align_up(sizeof(uint32_t) * W * P.cl.size());
  L.counters = align_up(sizeof(uint32_t) * (size_t)std::max<int64_t>(1, P.n_groups));
  L.ev = align_up(sizeof(int32_t) * W * (size_t)P.n);
  L.bad = align_up(sizeof(int32_t) * W);
  L.ready = align_up(sizeof(uint32_t) * 2 * P.cl.size());
  L.per_tile = L.psi + 2 * L.sep + L.post + L.partial + L.maxbits + L.counters + L.ev + L.bad + L.ready;
  return L;
}

void arena_free(Arena &a) {
  for (auto &kv : a.graphs) cudaGraphExecDestroy(kv.second);
  a.graphs.clear();
  if (a.mem && a.owns) cudaFree(a.mem);
  a.mem = nullptr;
  a.bytes = 0;
  a.alloc_bytes = 0;
  a.tiles = 0;
}

static void arena_bind(const Plan &P, Arena &a, char *mem, int tiles) {
  const ArenaLayout L = arena_layout(P);
  size_t off = 0;
  auto take = [&](size_t per_tile) {
    char *p = mem + off;
    off += per_tile * (size_t)tiles;
    return p;
  };
  a.da.psi = reinterpret_cast<float *>(take(L.psi));
  a.da.phistar = reinterpret_cast<float *>(take(L.sep));
  a.da.rho = reinterpret_cast<float *>(take(L.sep));
  a.da.post = reinterpret_cast<float *>(take(L.post));
  a.da.partial = reinterpret_cast<float *>(take(L.partial));
  a.da.maxbits = reinterpret_cast<uint32_t *>(take(L.maxbits));
  a.da.counters = reinterpret_cast<uint32_t *>(take(L.counters));
  a.da.ev = reinterpret_cast<int32_t *>(take(L.ev));
  a.da.bad = reinterpret_cast<int32_t *>(take(L.bad));
  a.da.ready = reinterpret_cast<uint32_t *>(take(L.ready));
  a.da.errflag = reinterpret_cast<uint32_t *>(mem + off);
  a.da.queue = reinterpret_cast<unsigned long long *>(mem + off + ArenaLayout::kQueueOffset);
  off += ArenaLayout::kTail;
  a.da.tiles = tiles;
  a.mem = mem;
  a.bytes = off;
  a.tiles = tiles;
}

jt_status arena_alloc(const Plan &P, Arena &a, int tiles) {
  arena_free(a);
  const ArenaLayout L = arena_layout(P);
  void *mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, L.bytes(tiles));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("arena cudaMalloc: ") + cudaGetErrorString(e));
    return JT_ENOMEM;
  }
  a.owns = true;
  arena_bind(P, a, static_cast<char *>(mem), tiles);
  a.alloc_bytes = L.bytes(tiles);
  // counters start at zero; every combining warp resets its own counter.
  // cudaMemset runs on the legacy default stream, which does not order the
  // library's non-blocking streams: wait for it before any batch can use
  // the arena (fresh memory may hold another arena's old data)
  JT_CUDA_TRY(cudaMemset(a.da.counters, 0, L.counters * (size_t)tiles));
  JT_CUDA_TRY(cudaMemset(a.da.errflag, 0, sizeof(uint32_t)));
  JT_CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));
  return JT_OK;
}

jt_status arena_wrap(const Plan &P, Arena &a, void *mem, size_t bytes, int tiles) {
  arena_free(a);
  const ArenaLayout L = arena_layout(P);
  if (L.bytes(tiles) > bytes) {
    set_error("arena buffer too small");
    return JT_ENOMEM;
  }
  a.owns = false;
  arena_bind(P, a, static_cast<char *>(mem), tiles);
  a.alloc_bytes = bytes;
  return JT_OK;
}

void enqueue_collect_layer(const jt_plan *pl, const DevArena &A, int L, cudaStream_t s) {
  const Plan &P = pl->P;
  const Level &lv = P.levels[L];
  launch_collect(P.cpt_per_thread, pl->dp, A, lv.c_item_begin, lv.c_item_end - lv.c_item_begin, lv.c_max_maps, s);
}

void enqueue_distribute_layer(const jt_plan *pl, const DevArena &A, int L, cudaStream_t s) {
  const Plan &P = pl->P;
  const Level &lv = P.levels[L];
  launch_distribute(P.cpt_per_thread, pl->dp, A, lv.d_item_begin, lv.d_item_end - lv.d_item_begin, s);
}

// Enqueue the two passes of one chunk in Section 2's BFS layer order
// (collect from the deepest layer up, distribute from the root down): one
// launch per layer, or one dataflow launch per pass.
void enqueue_passes(const jt_plan *pl, const DevArena &A, cudaStream_t s) {
  const Plan &P = pl->P;
  const ArenaLayout L = arena_layout(P);
  cudaMemsetAsync(A.maxbits, 0, L.maxbits * (size_t)A.tiles, s);
  // split-sum counters start every chunk at zero: the last piece of a group
  // resets its counter, but a pass whose bounded wait expired may leave a
  // group short of its last piece, and the next chunk must not inherit it
  cudaMemsetAsync(A.counters, 0, L.counters * (size_t)A.tiles, s);
  if (P.opts.schedule == JT_SCHEDULE_LAYERS) {
    for (int l = P.height; l >= 0; --l) enqueue_collect_layer(pl, A, l, s);
    for (int l = 0; l <= P.height; ++l) enqueue_distribute_layer(pl, A, l, s);
    return;
  }
  // dataflow: fresh per-tile counters and unit counters for this chunk
  cudaMemsetAsync(A.ready, 0, L.ready * (size_t)A.tiles, s);
  cudaMemsetAsync(A.queue, 0, ArenaLayout::kTail - ArenaLayout::kQueueOffset, s);
  int max_maps = 0;
  for (const Level &lv : P.levels) max_maps = std::max(max_maps, lv.c_max_maps);
  launch_collect_flow(P.cpt_per_thread, pl->dp, A, pl->flow_collect_blocks, max_maps, s);
  launch_distribute_flow(P.cpt_per_thread, pl->dp, A, pl->flow_distribute_blocks, s);
}

static jt_status graph_for(jt_plan *pl, Arena &a, int tiles, cudaGraphExec_t *out) {
  auto it = a.graphs.find(tiles);
  if (it != a.graphs.end()) { *out = it->second; return JT_OK; }
  DevArena A = a.da;
  A.tiles = tiles;
  cudaGraph_t g = nullptr;
  JT_CUDA_TRY(cudaStreamBeginCapture(pl->capture_stream, cudaStreamCaptureModeThreadLocal));
  enqueue_passes(pl, A, pl->capture_stream);
  cudaError_t e = cudaStreamEndCapture(pl->capture_stream, &g);
  if (e != cudaSuccess) {
    set_error(std::string("graph capture: ") + cudaGetErrorString(e));
    return JT_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    set_error(std::string("graph instantiate: ") + cudaGetErrorString(e));
    return JT_ECUDA;
  }
  a.graphs[tiles] = ex;
  *out = ex;
  return JT_OK;
}

jt_status run_chunk(jt_plan *pl, Arena &a, const int32_t *d_ev, int32_t nc, double *d_lp,
                    double *d_post, int32_t *d_st, cudaStream_t s) {
  const Plan &P = pl->P;
  const int W = P.tile;
  const int tiles = (nc + W - 1) / W;
  if (tiles <= 0) return JT_OK;
  if (tiles > a.tiles) { set_error("chunk larger than arena"); return JT_EINVAL; }
  DevArena A = a.da;
  A.tiles = tiles;
  JT_CUDA_TRY(cudaMemsetAsync(A.bad, 0, arena_layout(P).bad * (size_t)tiles, s));
  launch_evidence(P.cpt_per_thread, d_ev, nc, pl->dp, A, s);
  if (P.opts.use_graphs) {
    cudaGraphExec_t ex;
    jt_status st = graph_for(pl, a, tiles, &ex);
    if (st != JT_OK) return st;
    JT_CUDA_TRY(cudaGraphLaunch(ex, s));
  } else {
    enqueue_passes(pl, A, s);
  }
  launch_finalize(P.cpt_per_thread, pl->dp, A, nc, P.dcl[P.root].sep_row, d_lp, d_post, d_st, s);
  JT_CUDA_TRY(cudaGetLastError());
  return JT_OK;
}

jt_status check_arena_flag(Arena &a) {
  uint32_t f = 0;
  JT_CUDA_TRY(cudaMemcpy(&f, a.da.errflag, sizeof(f), cudaMemcpyDeviceToHost));
  if (f) {
    cudaMemset(a.da.errflag, 0, sizeof(uint32_t));
    cudaStreamSynchronize(cudaStreamLegacy);  // cleared before the next batch is issued
    set_error("a bounded device wait for work on the same case tile expired");
    return JT_ETIMEOUT;
  }
  return JT_OK;
}

int budget_tiles(const jt_plan *pl, int64_t budget_bytes) {
  const ArenaLayout L = arena_layout(pl->P);
  if (budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    budget_bytes = std::min<int64_t>(224LL << 30, (int64_t)(0.7 * (double)fr));
  }
  return (int)std::min<int64_t>((budget_bytes - (int64_t)ArenaLayout::kTail) / (int64_t)L.per_tile,
                                kMaxTilesPerChunk);
}

// Make the plan's default arena hold at least min(need, budget) tiles.
static jt_status ensure_default_arena(jt_plan *pl, int need_tiles) {
  int want = need_tiles;
  if (pl->budget_tiles_cache <= 0) pl->budget_tiles_cache = budget_tiles(pl, pl->P.opts.arena_bytes);
  want = std::min(want, pl->budget_tiles_cache);
  if (want <= 0) {
    set_error("arena budget is smaller than one case tile");
    return JT_ENOMEM;
  }
  if (pl->arena.tiles >= want) return JT_OK;
  return arena_alloc(pl->P, pl->arena, want);
}

}  // namespace jt

using namespace jt;

// ---------------------------------------------------------------------------
// plan lifetime
// ---------------------------------------------------------------------------
extern "C" void jt_default_opts(jt_compile_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->root_rule = JT_ROOT_MIN_HEIGHT;
  o->host_only = 0;
  o->cases_per_thread = 0;
  o->rows_per_cta = 0;
  o->max_clique_entries = 0;
  o->arena_bytes = 0;
  o->use_graphs = 1;
  o->rescale = 1;
  o->fuse_distribute = 1;
}

template <class T>
static size_t put(std::vector<char> &blob, const std::vector<T> &v) {
  size_t off = align_up(blob.size());
  blob.resize(off + align_up(sizeof(T) * std::max<size_t>(1, v.size())), 0);
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), sizeof(T) * v.size());
  return off;
}

// The work lists (items of both passes, flow layers, producer counts) live
// in their own device block so that retile can replace them.
static jt_status upload_work(jt_plan *pl) {
  Plan &P = pl->P;
  std::vector<char> blob;
  const size_t o_ci = put(blob, P.citems), o_di = put(blob, P.ditems);
  const size_t o_cfp = put(blob, P.c_flow_pref), o_cfb = put(blob, P.c_flow_begin);
  const size_t o_dfp = put(blob, P.d_flow_pref), o_dfb = put(blob, P.d_flow_begin);
  const size_t o_cn = put(blob, P.c_need), o_cno = put(blob, P.c_notify), o_dn = put(blob, P.d_need);
  if (pl->d_work) {
    cudaFree(pl->d_work);
    pl->d_work = nullptr;
  }
  JT_CUDA_TRY(cudaMalloc(&pl->d_work, blob.size()));
  pl->work_bytes = blob.size();
  JT_CUDA_TRY(cudaMemcpy(pl->d_work, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  JT_CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));  // see upload_plan
  char *b = static_cast<char *>(pl->d_work);
  DevPlan &D = pl->dp;
  D.citems = reinterpret_cast<const DItem *>(b + o_ci);
  D.ditems = reinterpret_cast<const DItem *>(b + o_di);
  D.c_flow_pref = reinterpret_cast<const int64_t *>(b + o_cfp);
  D.c_flow_begin = reinterpret_cast<const int64_t *>(b + o_cfb);
  D.d_flow_pref = reinterpret_cast<const int64_t *>(b + o_dfp);
  D.d_flow_begin = reinterpret_cast<const int64_t *>(b + o_dfb);
  D.c_need = reinterpret_cast<const uint32_t *>(b + o_cn);
  D.c_notify = reinterpret_cast<const int32_t *>(b + o_cno);
  D.d_need = reinterpret_cast<const uint32_t *>(b + o_dn);
  D.n_partials = std::max<int64_t>(1, P.n_partials);
  D.n_groups = std::max<int64_t>(1, P.n_groups);
  D.fused_items = 0;
  for (const DItem &it : P.ditems) D.fused_items += it.fused;
  // the distribute grid fills the GPU once at its kernel's occupancy
  int sms = 0;
  JT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device));
  pl->flow_distribute_blocks = sms * distribute_flow_blocks_per_sm(P.cpt_per_thread, D);
  return JT_OK;
}

static jt_status upload_plan(jt_plan *pl) {
  Plan &P = pl->P;
  // the kernels index evidence and posterior rows with these sizes
  const bool rows_ok = P.n_pruned > 0
                           ? (P.io_n > P.n && P.io_sum_card > P.sum_card && (int)P.io_var.size() == P.n &&
                              (int64_t)P.io_post_col.size() == P.sum_card && (int)P.io_dropped.size() == P.io_n - P.n &&
                              (int64_t)P.io_nan_cols.size() == P.io_sum_card - P.sum_card)
                           : (P.io_n == P.n && P.io_sum_card == P.sum_card);
  if (!rows_ok) {
    set_error("internal: inconsistent evidence or posterior row layout");
    return JT_EINVAL;
  }
  std::vector<char> blob;
  std::vector<int32_t> card32(P.card.begin(), P.card.end());
  const size_t o_cl = put(blob, P.dcl), o_map = put(blob, P.dmap), o_task = put(blob, P.dtask);
  const size_t o_ip = put(blob, P.ipool);
  const size_t o_b32 = put(blob, P.base32), o_card = put(blob, card32), o_po = put(blob, P.post_off);
  const size_t o_cp = put(blob, P.comp_ptr), o_cv = put(blob, P.comp_vars), o_cc = put(blob, P.comp_cliques);
  const size_t o_cr = put(blob, P.comp_roots), o_pg = put(blob, P.pgroup_ptr), o_co = put(blob, P.comp_owner);
  const size_t o_sv = put(blob, P.slice_var);
  const size_t o_cvo = put(blob, P.comp_var_owner);
  const size_t o_iv = put(blob, P.io_var), o_id = put(blob, P.io_dropped);
  const size_t o_ipc = put(blob, P.io_post_col), o_inc = put(blob, P.io_nan_cols);
  JT_CUDA_TRY(cudaMalloc(&pl->d_static, blob.size()));
  pl->static_bytes = blob.size();
  JT_CUDA_TRY(cudaMemcpy(pl->d_static, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  // a host-to-device cudaMemcpy may return before its last bytes land, and
  // the legacy stream does not order the plan's non-blocking streams
  JT_CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));
  char *b = static_cast<char *>(pl->d_static);
  DevPlan &D = pl->dp;
  D.cl = reinterpret_cast<const DClique *>(b + o_cl);
  D.maps = reinterpret_cast<const DMap *>(b + o_map);
  D.tasks = reinterpret_cast<const DTask *>(b + o_task);
  D.ipool = reinterpret_cast<const int32_t *>(b + o_ip);
  D.base32 = reinterpret_cast<const float *>(b + o_b32);
  D.card = reinterpret_cast<const int32_t *>(b + o_card);
  D.post_off = reinterpret_cast<const int64_t *>(b + o_po);
  D.comp_ptr = reinterpret_cast<const int32_t *>(b + o_cp);
  D.comp_vars = reinterpret_cast<const int32_t *>(b + o_cv);
  D.comp_cliques = reinterpret_cast<const int32_t *>(b + o_cc);
  D.comp_roots = reinterpret_cast<const int32_t *>(b + o_cr);
  D.comp_owner = reinterpret_cast<const int32_t *>(b + o_co);
  D.comp_var_owner = reinterpret_cast<const int32_t *>(b + o_cvo);
  D.n_comp_vars = (int32_t)P.comp_vars.size();
  D.n_comp_cliques = (int32_t)P.comp_cliques.size();
  D.n_comp = (int32_t)P.comp_roots.size();
  D.pgroup_ptr = reinterpret_cast<const int32_t *>(b + o_pg);
  D.slice_var = P.n_sliced > 0 ? reinterpret_cast<const int32_t *>(b + o_sv) : nullptr;
  const bool pruned = P.n_pruned > 0;
  D.io_var = pruned ? reinterpret_cast<const int32_t *>(b + o_iv) : nullptr;
  D.io_dropped = pruned ? reinterpret_cast<const int32_t *>(b + o_id) : nullptr;
  D.io_post_col = pruned ? reinterpret_cast<const int32_t *>(b + o_ipc) : nullptr;
  D.io_nan_cols = pruned ? reinterpret_cast<const int32_t *>(b + o_inc) : nullptr;
  D.io_post_rows = P.io_sum_card;
  D.io_n = P.io_n;
  D.n_dropped = (int32_t)P.io_dropped.size();
  D.n_nan_cols = (int32_t)P.io_nan_cols.size();
  D.sec_rows = P.sec_rows;
  D.recompute = P.recompute;
  D.msg_prefetch = P.opts.collect_prefetch ? 1 : 0;
  int max_maps = 0;
  for (const Level &lv : P.levels) max_maps = std::max(max_maps, lv.c_max_maps);
  D.max_maps = max_maps;
  if (P.recompute && recompute_warp_smem_bytes(P.cpt_per_thread, max_maps) * kWarps > kCollectSmemLimit) {
    set_error("recompute_psi: a clique has too many maps for the distribute blocks' shared memory");
    return JT_ETOOBIG;
  }
  // before the work lists: their upload sizes the distribute grid by the
  // kernel's occupancy at its shared memory
  JT_CUDA_TRY(configure_distribute_smem(P.cpt_per_thread, P.sec_rows, max_maps));
  jt_status wst = upload_work(pl);
  if (wst != JT_OK) return wst;
  D.n_flow_layers = P.height + 1;
  D.rescale = P.opts.rescale;
  D.wait_limit_ns = 1000ull * (uint64_t)(P.opts.wait_limit_us > 0 ? P.opts.wait_limit_us : 2000000);
  D.n_pgroups = (int32_t)P.pgroup_ptr.size() - 1;
  D.n_vars = P.n;
  D.n_cliques = (int32_t)P.cl.size();
  D.root = P.root;
  D.psi_rows = P.sum_cl;
  D.sep_rows = P.sep_rows;
  D.post_rows = P.sum_card;
  D.n_partials = std::max<int64_t>(1, P.n_partials);
  D.n_groups = std::max<int64_t>(1, P.n_groups);
  const size_t smem = collect_smem_bytes(P.cpt_per_thread, max_maps);
  if (collect_warp_smem_bytes(P.cpt_per_thread, max_maps) > kCollectSmemLimit) {
    set_error("a clique has too many child messages and evidence variables for one warp's shared memory");
    return JT_ETOOBIG;
  }
  JT_CUDA_TRY(configure_collect_smem(P.cpt_per_thread, P.n_sliced > 0, smem));
  if (logpe_smem_bytes((int)P.comp_roots.size()) > 220 * 1024) {
    set_error("the network splits into too many independent component trees for the log P(e) kernel");
    return JT_ETOOBIG;
  }
  JT_CUDA_TRY(configure_logpe_smem((int)P.comp_roots.size()));
  JT_CUDA_TRY(configure_posterior_smem());
  int sms = 0;
  JT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device));
  pl->flow_collect_blocks = sms * flow_blocks_per_sm(P.cpt_per_thread, P.n_sliced > 0, max_maps);
  return JT_OK;
}

namespace jt {
jt_status retile(jt_plan *pl, const jt_compile_opts &shape) {
  Plan &P = pl->P;
  jt_compile_opts o = P.opts;
  o.items_per_tile = shape.items_per_tile;
  o.items_per_tile_distribute = shape.items_per_tile_distribute;
  o.rows_per_cta = shape.rows_per_cta;
  std::memcpy(o.collect_rows_by_bucket, shape.collect_rows_by_bucket, sizeof(o.collect_rows_by_bucket));
  std::memcpy(o.distribute_rows_by_bucket, shape.distribute_rows_by_bucket, sizeof(o.distribute_rows_by_bucket));
  std::string err;
  jt_status st = emit_work(P, o, err);
  if (st != JT_OK) {
    set_error(err);
    return st;
  }
  P.opts = o;
  // captured graphs hold the old work lists' addresses
  for (auto &kv : pl->arena.graphs) cudaGraphExecDestroy(kv.second);
  pl->arena.graphs.clear();
  st = upload_work(pl);
  if (st != JT_OK) return st;
  pl->budget_tiles_cache = 0;
  if (pl->arena.mem) {
    const ArenaLayout L = arena_layout(P);
    if (pl->arena.owns && L.bytes(pl->arena.tiles) <= pl->arena.alloc_bytes) {
      // the new layout fits the allocation: rebind in place
      char *mem = static_cast<char *>(pl->arena.mem);
      const size_t alloc = pl->arena.alloc_bytes;
      arena_bind(P, pl->arena, mem, pl->arena.tiles);
      pl->arena.alloc_bytes = alloc;
      JT_CUDA_TRY(cudaMemset(pl->arena.da.errflag, 0, sizeof(uint32_t)));
      JT_CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));
    } else {
      arena_free(pl->arena);
    }
  }
  return JT_OK;
}
}  // namespace jt

extern "C" jt_status jt_compile(int32_t n_vars, const int32_t *card, const int32_t *parent_ptr,
                                const int32_t *parents, const double *cpt, const jt_compile_opts *opts,
                                jt_plan **out) {
  if (!out) { set_error("out is NULL"); return JT_EINVAL; }
  *out = nullptr;
  jt_compile_opts o;
  if (opts) o = *opts; else jt_default_opts(&o);
  jt_plan *pl = new (std::nothrow) jt_plan();
  if (!pl) return JT_ENOMEM;
  std::string err;
  jt_status st;
  try {
    st = build_plan_pruned(n_vars, card, parent_ptr, parents, cpt, o, pl->P, err);
  } catch (const std::bad_alloc &) {
    st = JT_ENOMEM;
    err = "host allocation failed while compiling";
  }
  if (st != JT_OK) {
    set_error(err);
    delete pl;
    return st;
  }
  pl->host_only = o.host_only != 0;
  if (!pl->host_only) {
    if (cudaGetDevice(&pl->device) != cudaSuccess) {
      cudaGetLastError();
      set_error("no CUDA device");
      delete pl;
      return JT_ECUDA;
    }
    if (cudaStreamCreateWithFlags(&pl->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&pl->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      set_error("stream creation failed");
      jt_plan_free(pl);
      return JT_ECUDA;
    }
    st = upload_plan(pl);
    if (st != JT_OK) {
      jt_plan_free(pl);
      return st;
    }
  }
  *out = pl;
  return JT_OK;
}

static void free_io(jt_plan *pl) {
  if (pl->d_io) cudaFree(pl->d_io);
  if (pl->h_io) cudaFreeHost(pl->h_io);
  pl->d_io = pl->h_io = nullptr;
  pl->io_cases = 0;
}

extern "C" void jt_plan_free(jt_plan *pl) {
  if (!pl) return;
  if (!pl->host_only) {
    arena_free(pl->arena);
    free_io(pl);
    if (pl->d_plain) cudaFree(pl->d_plain);
    if (pl->d_static) cudaFree(pl->d_static);
    if (pl->d_work) cudaFree(pl->d_work);
    if (pl->stream) cudaStreamDestroy(pl->stream);
    if (pl->capture_stream) cudaStreamDestroy(pl->capture_stream);
  }
  delete pl;
}

extern "C" jt_status jt_plan_info(const jt_plan *pl, jt_plan_info_t *o) {
  if (!pl || !o) { set_error("null argument"); return JT_EINVAL; }
  const Plan &P = pl->P;
  std::memset(o, 0, sizeof(*o));
  o->n_vars = P.io_n;
  o->n_cliques = (int32_t)P.cl.size();
  o->n_levels = P.height + 1;
  o->root = P.root;
  o->sum_clique_entries = P.sum_cl;
  o->max_clique_entries = P.max_cl;
  o->sum_sep_entries = P.sum_sep;
  o->sum_card = P.io_sum_card;
  o->tile_cases = P.tile;
  o->chunk_cases = pl->arena.tiles * P.tile;
  o->arena_bytes = (int64_t)pl->arena.bytes;
  o->static_device_bytes = (int64_t)pl->static_bytes;
  o->collect_items = (int64_t)P.citems.size();
  o->distribute_items = (int64_t)P.ditems.size();
  o->algorithmic_bytes_per_case = 8.0 * (double)P.sum_cl + 16.0 * (double)P.sum_sep + 4.0 * P.io_n +
                                  8.0 * (double)P.io_sum_card + 8.0;
  int k = 3;  // evidence + log P(e) + posteriors
  if (P.opts.schedule == JT_SCHEDULE_LAYERS) {
    for (const Level &lv : P.levels) {
      k += lv.c_item_end > lv.c_item_begin;
      k += lv.d_item_end > lv.d_item_begin;
    }
  } else {
    k += 2;  // one dataflow launch per pass
  }
  o->kernels_per_chunk = k;
  o->sliced_vars = P.n_sliced;
  o->pruned_vars = P.n_pruned;
  o->separator_evidence_vars = 0;
  for (const HostClique &C : P.cl) o->separator_evidence_vars += (int32_t)C.ev_sep.size();
  o->budget_chunk_cases = 0;
  if (!pl->host_only) {
    const int t = pl->budget_tiles_cache > 0 ? pl->budget_tiles_cache : budget_tiles(pl, P.opts.arena_bytes);
    o->budget_chunk_cases = t > 0 ? t * P.tile : 0;
  }
  for (int b = 0; b < JT_SIZE_BUCKETS; ++b) {
    o->collect_rows_by_bucket[b] = P.c_bucket_rows[b];
    o->distribute_rows_by_bucket[b] = P.d_bucket_rows[b];
    o->collect_entries_by_bucket[b] = P.c_bucket_entries[b];
    o->distribute_entries_by_bucket[b] = P.d_bucket_entries[b];
  }
  return JT_OK;
}

extern "C" jt_status jt_debug_stall(jt_plan *pl, int32_t enabled) {
  if (!pl || pl->host_only) { set_error("bad plan"); return JT_EINVAL; }
  const Plan &P = pl->P;
  if (P.opts.stall_clique <= 0) { set_error("the plan was compiled without stall_clique"); return JT_EINVAL; }
  std::lock_guard<std::mutex> lk(pl->mu);
  JT_CUDA_TRY(cudaSetDevice(pl->device));
  const int k = P.opts.stall_clique - 1;
  // the host copy counts the missing producer; the device copy is the one
  // the collect pass reads
  const uint32_t need = P.c_need[k] - (enabled ? 0u : 1u);
  JT_CUDA_TRY(cudaMemcpy(const_cast<uint32_t *>(pl->dp.c_need) + k, &need, sizeof(need), cudaMemcpyHostToDevice));
  JT_CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));
  return JT_OK;
}

extern "C" jt_status jt_plan_clique(const jt_plan *pl, int32_t c, int32_t *n_vars, int32_t *vars,
                                    int32_t *parent, int32_t *depth) {
  if (!pl || c < 0 || c >= (int32_t)pl->P.cl.size()) { set_error("bad clique id"); return JT_EINVAL; }
  const HostClique &C = pl->P.cl[c];
  if (n_vars) *n_vars = (int32_t)C.vars.size();
  // variable ids of the full network (a pruned plan renumbers its kept variables)
  if (vars)
    for (size_t i = 0; i < C.vars.size() && i < 64; ++i)
      vars[i] = pl->P.n_pruned > 0 ? pl->P.io_var[C.vars[i]] : C.vars[i];
  if (parent) *parent = C.parent;
  if (depth) *depth = C.depth;
  return JT_OK;
}

extern "C" const char *jt_status_string(jt_status s) {
  switch (s) {
    case JT_OK: return "ok";
    case JT_EINVAL: return "invalid argument";
    case JT_ECYCLE: return "parent graph has a cycle";
    case JT_ETOOBIG: return "clique table too large";
    case JT_ENOMEM: return "out of memory";
    case JT_ECUDA: return "CUDA error";
    case JT_ETIMEOUT: return "device wait timed out";
    case JT_EBUSY: return "not ready";
    case JT_ENOTFOUND: return "not found";
  }
  return "unknown status";
}

extern "C" const char *jt_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// batched inference
// ---------------------------------------------------------------------------
static cudaStream_t pick_stream(jt_plan *pl, void *s) {
  return s ? static_cast<cudaStream_t>(s) : pl->stream;
}

static jt_status jt_infer_device_impl(jt_plan *pl, int32_t n_cases, const int32_t *d_ev, double *d_lp,
                                     double *d_post, int32_t *d_st, void *stream) {
  if (!pl || n_cases < 0) { set_error("bad plan or n_cases"); return JT_EINVAL; }
  if (pl->host_only) { set_error("plan compiled with host_only"); return JT_EINVAL; }
  if (n_cases == 0) return JT_OK;
  if (!d_ev || !d_lp || !d_post || !d_st) { set_error("null buffer"); return JT_EINVAL; }
  std::lock_guard<std::mutex> lk(pl->mu);
  JT_CUDA_TRY(cudaSetDevice(pl->device));
  const int W = pl->P.tile;
  jt_status st = ensure_default_arena(pl, (n_cases + W - 1) / W);
  if (st != JT_OK) return st;
  cudaStream_t s = pick_stream(pl, stream);
  const int64_t chunk = (int64_t)pl->arena.tiles * W;
  for (int64_t b = 0; b < n_cases; b += chunk) {
    const int32_t nc = (int32_t)std::min<int64_t>(chunk, n_cases - b);
    st = run_chunk(pl, pl->arena, d_ev + b * pl->P.io_n, nc, d_lp + b, d_post + b * pl->P.io_sum_card, d_st + b, s);
    if (st != JT_OK) return st;
  }
  return JT_OK;
}

extern "C" jt_status jt_infer_device(jt_plan *pl, int32_t n_cases, const int32_t *d_ev, double *d_lp,
                                     double *d_post, int32_t *d_st, void *stream) {
  return guarded([&] { return jt_infer_device_impl(pl, n_cases, d_ev, d_lp, d_post, d_st, stream); });
}

static jt_status ensure_io(jt_plan *pl, int cases) {
  if (pl->io_cases >= cases) return JT_OK;
  free_io(pl);
  const Plan &P = pl->P;
  pl->io_ev = align_up(sizeof(int32_t) * (size_t)cases * P.io_n);
  pl->io_lp = align_up(sizeof(double) * (size_t)cases);
  pl->io_post = align_up(sizeof(double) * (size_t)cases * P.io_sum_card);
  pl->io_st = align_up(sizeof(int32_t) * (size_t)cases);
  const size_t bytes = pl->io_ev + pl->io_lp + pl->io_post + pl->io_st;
  JT_CUDA_TRY(cudaMalloc(&pl->d_io, bytes));
  JT_CUDA_TRY(cudaHostAlloc(&pl->h_io, bytes, cudaHostAllocDefault));
  pl->io_cases = cases;
  return JT_OK;
}

static jt_status jt_infer_impl(jt_plan *pl, int32_t n_cases, const int32_t *ev, double *lp, double *post,
                              int32_t *cst, void *stream) {
  if (!pl || n_cases < 0) { set_error("bad plan or n_cases"); return JT_EINVAL; }
  if (pl->host_only) { set_error("plan compiled with host_only"); return JT_EINVAL; }
  if (n_cases == 0) return JT_OK;
  if (!ev || !lp || !post || !cst) { set_error("null buffer"); return JT_EINVAL; }
  std::lock_guard<std::mutex> lk(pl->mu);
  JT_CUDA_TRY(cudaSetDevice(pl->device));
  const Plan &P = pl->P;
  const int W = P.tile;
  jt_status st = ensure_default_arena(pl, (n_cases + W - 1) / W);
  if (st != JT_OK) return st;
  const int chunk = pl->arena.tiles * W;
  st = ensure_io(pl, std::min<int>(chunk, n_cases));
  if (st != JT_OK) return st;
  cudaStream_t s = pick_stream(pl, stream);
  char *d = static_cast<char *>(pl->d_io), *h = static_cast<char *>(pl->h_io);
  int32_t *d_ev = reinterpret_cast<int32_t *>(d), *h_ev = reinterpret_cast<int32_t *>(h);
  double *d_lp = reinterpret_cast<double *>(d + pl->io_ev), *h_lp = reinterpret_cast<double *>(h + pl->io_ev);
  double *d_po = reinterpret_cast<double *>(d + pl->io_ev + pl->io_lp);
  double *h_po = reinterpret_cast<double *>(h + pl->io_ev + pl->io_lp);
  int32_t *d_st = reinterpret_cast<int32_t *>(d + pl->io_ev + pl->io_lp + pl->io_post);
  int32_t *h_st = reinterpret_cast<int32_t *>(h + pl->io_ev + pl->io_lp + pl->io_post);
  // Page-locked caller buffers are copied directly (asynchronously, one
  // synchronisation at the end); pageable ones through the plan's pinned
  // staging buffer.
  auto pinned = [](const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return a.type == cudaMemoryTypeHost;
  };
  if (pinned(ev) && pinned(lp) && pinned(post) && pinned(cst)) {
    for (int64_t b = 0; b < n_cases; b += chunk) {
      const int32_t nc = (int32_t)std::min<int64_t>(chunk, n_cases - b);
      JT_CUDA_TRY(cudaMemcpyAsync(d_ev, ev + b * P.io_n, sizeof(int32_t) * (size_t)nc * P.io_n, cudaMemcpyHostToDevice, s));
      st = run_chunk(pl, pl->arena, d_ev, nc, d_lp, d_po, d_st, s);
      if (st != JT_OK) return st;
      JT_CUDA_TRY(cudaMemcpyAsync(lp + b, d_lp, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
      JT_CUDA_TRY(cudaMemcpyAsync(post + b * P.io_sum_card, d_po, sizeof(double) * (size_t)nc * P.io_sum_card,
                                  cudaMemcpyDeviceToHost, s));
      JT_CUDA_TRY(cudaMemcpyAsync(cst + b, d_st, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, s));
    }
    JT_CUDA_TRY(cudaStreamSynchronize(s));
    return check_arena_flag(pl->arena);
  }
  for (int64_t b = 0; b < n_cases; b += chunk) {
    const int32_t nc = (int32_t)std::min<int64_t>(chunk, n_cases - b);
    std::memcpy(h_ev, ev + b * P.io_n, sizeof(int32_t) * (size_t)nc * P.io_n);
    JT_CUDA_TRY(cudaMemcpyAsync(d_ev, h_ev, sizeof(int32_t) * (size_t)nc * P.io_n, cudaMemcpyHostToDevice, s));
    st = run_chunk(pl, pl->arena, d_ev, nc, d_lp, d_po, d_st, s);
    if (st != JT_OK) return st;
    JT_CUDA_TRY(cudaMemcpyAsync(h_lp, d_lp, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
    JT_CUDA_TRY(cudaMemcpyAsync(h_po, d_po, sizeof(double) * (size_t)nc * P.io_sum_card, cudaMemcpyDeviceToHost, s));
    JT_CUDA_TRY(cudaMemcpyAsync(h_st, d_st, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, s));
    JT_CUDA_TRY(cudaStreamSynchronize(s));
    st = check_arena_flag(pl->arena);
    if (st != JT_OK) return st;
    std::memcpy(lp + b, h_lp, sizeof(double) * nc);
    std::memcpy(post + b * P.io_sum_card, h_po, sizeof(double) * (size_t)nc * P.io_sum_card);
    std::memcpy(cst + b, h_st, sizeof(int32_t) * nc);
  }
  return JT_OK;
}

extern "C" jt_status jt_infer(jt_plan *pl, int32_t n_cases, const int32_t *ev, double *lp, double *post,
                              int32_t *cst, void *stream) {
  return guarded([&] { return jt_infer_impl(pl, n_cases, ev, lp, post, cst, stream); });
}

// ---------------------------------------------------------------------------
// plain FP64 per-case path
// ---------------------------------------------------------------------------
static jt_status ensure_plain(jt_plan *pl) {
  if (pl->d_plain) return JT_OK;
  const Plan &P = pl->P;
  int64_t maxsep = 1;
  for (auto &C : P.cl) maxsep = std::max(maxsep, C.nsep);
  std::vector<char> blob;
  std::vector<int32_t> card32(P.card.begin(), P.card.end());
  const size_t o_b = put(blob, P.base64), o_pp = put(blob, P.ppool), o_card = put(blob, card32),
               o_po = put(blob, P.post_off);
  const size_t o_psi = align_up(blob.size());
  const size_t o_sep = o_psi + align_up(sizeof(double) * P.sum_cl);
  const size_t o_tmp = o_sep + align_up(sizeof(double) * P.sep_rows);
  const size_t o_marg = o_tmp + align_up(sizeof(double) * maxsep);
  const size_t o_pe = o_marg + align_up(sizeof(double) * P.sum_card);
  const size_t o_ev = o_pe + align_up(sizeof(double));
  const size_t total = o_ev + align_up(sizeof(int32_t) * P.n);
  void *mem = nullptr;
  if (cudaMalloc(&mem, total) != cudaSuccess) {
    cudaGetLastError();
    set_error("plain path workspace allocation failed");
    return JT_ENOMEM;
  }
  JT_CUDA_TRY(cudaMemcpy(mem, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  JT_CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));  // see upload_plan
  char *b = static_cast<char *>(mem);
  pl->d_plain = mem;
  pl->pw.base = reinterpret_cast<double *>(b + o_b);
  pl->pw.pool = reinterpret_cast<int64_t *>(b + o_pp);
  pl->pw.card = reinterpret_cast<int32_t *>(b + o_card);
  pl->pw.post_off = reinterpret_cast<int64_t *>(b + o_po);
  pl->pw.psi = reinterpret_cast<double *>(b + o_psi);
  pl->pw.sep = reinterpret_cast<double *>(b + o_sep);
  pl->pw.tmp = reinterpret_cast<double *>(b + o_tmp);
  pl->pw.marg = reinterpret_cast<double *>(b + o_marg);
  pl->pw.pe = reinterpret_cast<double *>(b + o_pe);
  pl->pw.ev = reinterpret_cast<int32_t *>(b + o_ev);
  return JT_OK;
}

static jt_status plain_case(jt_plan *pl, const int32_t *h_ev, double *d_lp, double *d_post, int32_t *d_st,
                            cudaStream_t s) {
  const Plan &P = pl->P;
  const PlainWork &w = pl->pw;
  JT_CUDA_TRY(cudaMemcpyAsync(w.ev, h_ev, sizeof(int32_t) * P.n, cudaMemcpyHostToDevice, s));
  const int m = (int)P.cl.size();
  // initialisation + reduction (evidence), one launch per clique
  for (int c = 0; c < m; ++c)
    launch_plain_init(w.psi + P.p_base_off[c], w.base + P.p_base_off[c], P.pmap[P.p_init_map[c]], w.pool, w.ev, s);
  // collect: children before parents
  for (int q = m - 1; q >= 1; --q) {
    const int c = P.bfs[q], p = P.cl[c].parent;
    double *sep = w.sep + P.p_sep_off[c];
    JT_CUDA_TRY(cudaMemsetAsync(sep, 0, sizeof(double) * P.cl[c].nsep, s));
    launch_plain_marg(w.psi + P.p_base_off[c], sep, P.pmap[P.p_child_map[c]], w.pool, s);
    launch_plain_extend(w.psi + P.p_base_off[p], sep, P.pmap[P.p_parent_map[c]], w.pool, s);
  }
  JT_CUDA_TRY(cudaMemsetAsync(w.pe, 0, sizeof(double), s));
  launch_plain_marg(w.psi + P.p_base_off[P.root], w.pe, P.pmap[P.p_root_map[0]], w.pool, s);
  // distribute: parents before children
  for (int q = 1; q < m; ++q) {
    const int c = P.bfs[q], p = P.cl[c].parent;
    const int64_t ns = P.cl[c].nsep;
    JT_CUDA_TRY(cudaMemsetAsync(w.tmp, 0, sizeof(double) * ns, s));
    launch_plain_marg(w.psi + P.p_base_off[p], w.tmp, P.pmap[P.p_parent_map[c]], w.pool, s);
    launch_plain_divide(w.tmp, w.sep + P.p_sep_off[c], ns, s);
    launch_plain_extend(w.psi + P.p_base_off[c], w.tmp, P.pmap[P.p_child_map[c]], w.pool, s);
  }
  JT_CUDA_TRY(cudaMemsetAsync(w.marg, 0, sizeof(double) * P.sum_card, s));
  for (int v = 0; v < P.n; ++v) {
    if (h_ev[v] >= 0) continue;
    const int c = P.post_src[v];
    launch_plain_marg(w.psi + P.p_base_off[c], w.marg + P.post_off[v], P.pmap[P.p_post_map[v]], w.pool, s);
  }
  launch_plain_finalize(w.pe, w.marg, w.ev, w.card, w.post_off, P.n, d_lp, d_post, d_st, s);
  JT_CUDA_TRY(cudaGetLastError());
  return JT_OK;
}

extern "C" jt_status jt_infer_cpu(const jt_plan *pl, int32_t n_cases, const int32_t *ev, double *lp,
                                  double *post, int32_t *cst, int32_t n_threads) {
  if (!pl || n_cases < 0) { set_error("bad plan or n_cases"); return JT_EINVAL; }
  if (n_cases == 0) return JT_OK;
  if (!ev || !lp || !post || !cst) { set_error("null buffer"); return JT_EINVAL; }
  try {
    return cpu_layers_infer(pl->P, n_cases, ev, lp, post, cst, std::min<int32_t>(n_threads, 1024));
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed in the CPU comparator");
    return JT_ENOMEM;
  } catch (const std::exception &e) {
    set_error(std::string("CPU comparator: ") + e.what());
    return JT_EINVAL;
  }
}

static jt_status jt_infer_plain_impl(jt_plan *pl, int32_t n_cases, const int32_t *ev, double *lp,
                                    double *post, int32_t *cst, void *stream) {
  if (!pl || n_cases < 0) { set_error("bad plan or n_cases"); return JT_EINVAL; }
  if (pl->host_only) { set_error("plan compiled with host_only"); return JT_EINVAL; }
  if (pl->P.n_sliced > 0 || pl->P.n_pruned > 0) {
    set_error("the plain path runs unspecialised plans only");
    return JT_EINVAL;
  }
  if (n_cases == 0) return JT_OK;
  if (!ev || !lp || !post || !cst) { set_error("null buffer"); return JT_EINVAL; }
  std::lock_guard<std::mutex> lk(pl->mu);
  JT_CUDA_TRY(cudaSetDevice(pl->device));
  jt_status st = ensure_plain(pl);
  if (st != JT_OK) return st;
  const Plan &P = pl->P;
  const int batch = 256;
  st = ensure_io(pl, std::min<int>(batch, n_cases));
  if (st != JT_OK) return st;
  cudaStream_t s = pick_stream(pl, stream);
  char *d = static_cast<char *>(pl->d_io);
  double *d_lp = reinterpret_cast<double *>(d + pl->io_ev);
  double *d_po = reinterpret_cast<double *>(d + pl->io_ev + pl->io_lp);
  int32_t *d_st = reinterpret_cast<int32_t *>(d + pl->io_ev + pl->io_lp + pl->io_post);
  for (int64_t b = 0; b < n_cases; b += batch) {
    const int nb = (int)std::min<int64_t>(batch, n_cases - b);
    for (int i = 0; i < nb; ++i) {
      const int32_t *e = ev + (b + i) * P.n;
      bool badev = false;
      for (int v = 0; v < P.n; ++v)
        if (e[v] < -1 || e[v] >= P.card[v]) badev = true;
      if (badev) {
        // flagged on the host; the device outputs of this slot are overwritten below
        continue;
      }
      st = plain_case(pl, e, d_lp + i, d_po + (size_t)i * P.sum_card, d_st + i, s);
      if (st != JT_OK) return st;
    }
    JT_CUDA_TRY(cudaMemcpyAsync(lp + b, d_lp, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    JT_CUDA_TRY(cudaMemcpyAsync(post + b * P.sum_card, d_po, sizeof(double) * (size_t)nb * P.sum_card,
                                cudaMemcpyDeviceToHost, s));
    JT_CUDA_TRY(cudaMemcpyAsync(cst + b, d_st, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
    JT_CUDA_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < nb; ++i) {
      const int32_t *e = ev + (b + i) * P.n;
      bool badev = false;
      for (int v = 0; v < P.n; ++v)
        if (e[v] < -1 || e[v] >= P.card[v]) badev = true;
      if (badev) {
        lp[b + i] = std::nan("");
        cst[b + i] = JT_CASE_BAD_EVIDENCE;
        for (int64_t k = 0; k < P.sum_card; ++k) post[(b + i) * P.sum_card + k] = std::nan("");
      }
    }
  }
  return JT_OK;
}

extern "C" jt_status jt_infer_plain(jt_plan *pl, int32_t n_cases, const int32_t *ev, double *lp,
                                    double *post, int32_t *cst, void *stream) {
  return guarded([&] { return jt_infer_plain_impl(pl, n_cases, ev, lp, post, cst, stream); });
}

// ---------------------------------------------------------------------------
// instrumented run (per-kernel timing with CUDA events)
// ---------------------------------------------------------------------------
static jt_status jt_profile_impl(jt_plan *pl, int32_t n_cases, const int32_t *d_ev, double *d_lp,
                                double *d_post, int32_t *d_st, void *stream, double *out) {
  if (!pl || n_cases <= 0 || !out) { set_error("bad argument"); return JT_EINVAL; }
  if (pl->host_only) { set_error("plan compiled with host_only"); return JT_EINVAL; }
  std::lock_guard<std::mutex> lk(pl->mu);
  JT_CUDA_TRY(cudaSetDevice(pl->device));
  const Plan &P = pl->P;
  const int W = P.tile;
  jt_status st = ensure_default_arena(pl, (n_cases + W - 1) / W);
  if (st != JT_OK) return st;
  cudaStream_t s = pick_stream(pl, stream);
  const int64_t chunk = (int64_t)pl->arena.tiles * W;
  std::vector<cudaEvent_t> ev;
  auto mark = [&]() {
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, s);
    ev.push_back(e);
    return (int)ev.size() - 1;
  };
  struct Span { int a, b, kind; };
  std::vector<Span> spans;
  const int start = mark();
  for (int64_t b = 0; b < n_cases; b += chunk) {
    const int32_t nc = (int32_t)std::min<int64_t>(chunk, n_cases - b);
    DevArena A = pl->arena.da;
    A.tiles = (nc + W - 1) / W;
    JT_CUDA_TRY(cudaMemsetAsync(A.bad, 0, arena_layout(P).bad * (size_t)A.tiles, s));
    JT_CUDA_TRY(cudaMemsetAsync(A.counters, 0, arena_layout(P).counters * (size_t)A.tiles, s));
    int e0 = mark();
    launch_evidence(P.cpt_per_thread, d_ev + b * P.io_n, nc, pl->dp, A, s);
    spans.push_back({e0, mark(), 2});
    if (P.opts.schedule != JT_SCHEDULE_LAYERS) {
      // dataflow: one span per pass (the counters are reset inside the first)
      int max_maps = 0;
      for (const Level &lv : P.levels) max_maps = std::max(max_maps, lv.c_max_maps);
      JT_CUDA_TRY(cudaMemsetAsync(A.maxbits, 0, arena_layout(P).maxbits * (size_t)A.tiles, s));
      JT_CUDA_TRY(cudaMemsetAsync(A.ready, 0, arena_layout(P).ready * (size_t)A.tiles, s));
      JT_CUDA_TRY(cudaMemsetAsync(A.queue, 0, ArenaLayout::kTail - ArenaLayout::kQueueOffset, s));
      int a = mark();
      launch_collect_flow(P.cpt_per_thread, pl->dp, A, pl->flow_collect_blocks, max_maps, s);
      spans.push_back({a, mark(), 0});
      a = mark();
      launch_distribute_flow(P.cpt_per_thread, pl->dp, A, pl->flow_distribute_blocks, s);
      spans.push_back({a, mark(), 1});
    } else {
    JT_CUDA_TRY(cudaMemsetAsync(A.maxbits, 0, arena_layout(P).maxbits * (size_t)A.tiles, s));
    for (int L = P.height; L >= 0; --L) {
      const Level &lv = P.levels[L];
      if (lv.c_item_end == lv.c_item_begin) continue;
      int a = mark();
      launch_collect(P.cpt_per_thread, pl->dp, A, lv.c_item_begin, lv.c_item_end - lv.c_item_begin,
                     lv.c_max_maps, s);
      spans.push_back({a, mark(), 0});
    }
    for (int L = 0; L <= P.height; ++L) {
      const Level &lv = P.levels[L];
      if (lv.d_item_end == lv.d_item_begin) continue;
      int a = mark();
      enqueue_distribute_layer(pl, A, L, s);
      spans.push_back({a, mark(), 1});
    }
    }
    int f0 = mark();
    launch_finalize(P.cpt_per_thread, pl->dp, A, nc, P.dcl[P.root].sep_row, d_lp + b,
                    d_post + b * P.io_sum_card, d_st + b, s);
    spans.push_back({f0, mark(), 2});
  }
  const int stop = mark();
  JT_CUDA_TRY(cudaGetLastError());
  JT_CUDA_TRY(cudaStreamSynchronize(s));
  st = check_arena_flag(pl->arena);
  if (st != JT_OK) return st;
  for (int k = 0; k < 6; ++k) out[k] = 0;
  for (const Span &sp : spans) {
    float ms = 0;
    cudaEventElapsedTime(&ms, ev[sp.a], ev[sp.b]);
    out[sp.kind] += ms;
    if (sp.kind < 2) out[3 + sp.kind] += 1;
  }
  float tot = 0;
  cudaEventElapsedTime(&tot, ev[start], ev[stop]);
  out[5] = tot;
  for (auto e : ev) cudaEventDestroy(e);
  return JT_OK;
}

extern "C" jt_status jt_profile(jt_plan *pl, int32_t n_cases, const int32_t *d_ev, double *d_lp,
                                double *d_post, int32_t *d_st, void *stream, double *out) {
  return guarded([&] { return jt_profile_impl(pl, n_cases, d_ev, d_lp, d_post, d_st, stream, out); });
}

// ---------------------------------------------------------------------------
// autotuner: time candidate tile shapes on the caller's batch size
// ---------------------------------------------------------------------------
// Two stages, both timed with jt_profile on the caller's batch size (one
// warm-up run, then the best of two): (1) per tile width (cases per thread
// 4 and 8) the work-item target of each pass over {96 .. 1536} items per
// tile and layer; (2) on the best width, per table-size bucket (in order of
// the rows the bucket holds, those with at least 2 % of a pass's rows, at
// most eight), the rows of one warp work item over powers of two from 32
// to 4096, each pass keeping its own best value per bucket (coordinate
// descent; a change is kept when it is at least 1 % faster).  Only the
// work lists are rebuilt between candidates (retile), not the plan.
static jt_status jt_autotune_impl(int32_t n_vars, const int32_t *card, const int32_t *parent_ptr,
                                 const int32_t *parents, const double *cpt, const jt_compile_opts *base,
                                 int32_t n_cases, jt_compile_opts *best, double *best_ns_per_case) {
  if (!best || n_cases <= 0 || n_vars <= 0 || !card) { set_error("bad argument"); return JT_EINVAL; }
  jt_compile_opts b;
  if (base) b = *base; else jt_default_opts(&b);
  b.host_only = 0;
  const int cpts[] = {4, 8};
  const int items[] = {96, 192, 384, 768, 1536};
  int64_t sum_card = 0;
  for (int v = 0; v < n_vars; ++v) sum_card += card[v];
  int32_t *d_ev = nullptr;
  double *d_lp = nullptr, *d_post = nullptr;
  int32_t *d_st = nullptr;
  if (cudaMalloc(&d_ev, sizeof(int32_t) * (size_t)n_cases * n_vars) != cudaSuccess ||
      cudaMalloc(&d_lp, sizeof(double) * n_cases) != cudaSuccess ||
      cudaMalloc(&d_post, sizeof(double) * (size_t)n_cases * sum_card) != cudaSuccess ||
      cudaMalloc(&d_st, sizeof(int32_t) * n_cases) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_ev); cudaFree(d_lp); cudaFree(d_post); cudaFree(d_st);
    set_error("autotune buffers");
    return JT_ENOMEM;
  }
  // all variables unobserved: the timing does not depend on the evidence values
  cudaMemset(d_ev, 0xff, sizeof(int32_t) * (size_t)n_cases * n_vars);
  cudaStreamSynchronize(cudaStreamLegacy);  // filled before the plans' streams read it
  auto time_plan = [&](jt_plan *pl, double &c_ms, double &d_ms) -> jt_status {
    double out[6];
    c_ms = d_ms = -1;
    for (int r = 0; r < 3; ++r) {
      jt_status st = jt_profile(pl, n_cases, d_ev, d_lp, d_post, d_st, pl->stream, out);
      if (st != JT_OK) return st;
      if (r > 0) {  // the first run warms up
        c_ms = (c_ms < 0) ? out[0] : std::min(c_ms, out[0]);
        d_ms = (d_ms < 0) ? out[1] : std::min(d_ms, out[1]);
      }
    }
    return JT_OK;
  };
  auto shape_of = [](const jt_compile_opts &o) { return o; };
  jt_status result = JT_OK;
  double best_total = -1;
  jt_compile_opts best_o = b;
  int best_cw = 0;
  // stage 1: tile width x work-item target per pass
  for (int ci = 0; result == JT_OK && ci < 2; ++ci) {
    if (base && base->cases_per_thread != 0 && ci > 0) break;  // the caller fixed the tile width
    const int cw = (base && base->cases_per_thread != 0) ? base->cases_per_thread : cpts[ci];
    jt_compile_opts o = b;
    o.cases_per_thread = cw;
    o.rows_per_cta = 0;
    std::memset(o.collect_rows_by_bucket, 0, sizeof(o.collect_rows_by_bucket));
    std::memset(o.distribute_rows_by_bucket, 0, sizeof(o.distribute_rows_by_bucket));
    jt_plan *pl = nullptr;
    jt_status st = jt_compile(n_vars, card, parent_ptr, parents, cpt, &o, &pl);
    if (st != JT_OK) { result = st; break; }
    double best_c = -1, best_d = -1;
    int item_c = 192, item_d = 192;
    for (int ii = 0; st == JT_OK && ii < (int)(sizeof(items) / sizeof(items[0])); ++ii) {
      jt_compile_opts sh = shape_of(o);
      sh.items_per_tile = items[ii];
      sh.items_per_tile_distribute = items[ii];
      double c_ms, d_ms;
      st = retile(pl, sh);
      if (st == JT_OK) st = time_plan(pl, c_ms, d_ms);
      if (st != JT_OK) break;
      if (best_c < 0 || c_ms < best_c) { best_c = c_ms; item_c = items[ii]; }
      if (best_d < 0 || d_ms < best_d) { best_d = d_ms; item_d = items[ii]; }
    }
    jt_plan_free(pl);
    if (st != JT_OK) { result = st; break; }
    if (best_total < 0 || best_c + best_d < best_total) {
      best_total = best_c + best_d;
      best_o = o;
      best_o.items_per_tile = item_c;
      best_o.items_per_tile_distribute = item_d;
      best_cw = cw;
    }
  }
  // stage 2: rows per work item per table-size bucket, on the best width
  if (result == JT_OK && best_cw > 0) {
    jt_plan *pl = nullptr;
    jt_status st = jt_compile(n_vars, card, parent_ptr, parents, cpt, &best_o, &pl);
    double cur_c = -1, cur_d = -1;
    if (st == JT_OK) st = time_plan(pl, cur_c, cur_d);
    if (st == JT_OK) {
      const Plan &P = pl->P;
      int64_t ctot = 0, dtot = 0;
      for (int k = 0; k < JT_SIZE_BUCKETS; ++k) { ctot += P.c_bucket_entries[k]; dtot += P.d_bucket_entries[k]; }
      std::vector<std::pair<double, int>> order;
      for (int k = 0; k < JT_SIZE_BUCKETS; ++k) {
        const double w = std::max(ctot ? (double)P.c_bucket_entries[k] / ctot : 0.0,
                                  dtot ? (double)P.d_bucket_entries[k] / dtot : 0.0);
        if (w >= 0.02) order.push_back({-w, k});
      }
      std::sort(order.begin(), order.end());
      if (order.size() > 8) order.resize(8);
      // starting point: the per-layer values of stage 1 (table entries 0)
      jt_compile_opts sh = best_o;
      const std::array<int64_t, JT_SIZE_BUCKETS> ce = P.c_bucket_entries, de = P.d_bucket_entries;
      const int cand[] = {32, 64, 128, 256, 512, 1024, 2048, 4096};
      for (const auto &wk : order) {
        const int k = wk.second;
        const bool tune_c = ctot && (double)ce[k] / ctot >= 0.02, tune_d = dtot && (double)de[k] / dtot >= 0.02;
        int keep_c = sh.collect_rows_by_bucket[k], keep_d = sh.distribute_rows_by_bucket[k];
        for (int r : cand) {
          if (r > (int64_t(2) << k)) break;  // an item cannot outgrow the bucket's tables
          jt_compile_opts t = sh;
          if (tune_c) t.collect_rows_by_bucket[k] = r;
          if (tune_d) t.distribute_rows_by_bucket[k] = r;
          double c_ms, d_ms;
          st = retile(pl, t);
          if (st == JT_OK) st = time_plan(pl, c_ms, d_ms);
          if (st != JT_OK) break;
          if (tune_c && c_ms < 0.99 * cur_c) { cur_c = c_ms; keep_c = r; }
          if (tune_d && d_ms < 0.99 * cur_d) { cur_d = d_ms; keep_d = r; }
        }
        if (st != JT_OK) break;
        sh.collect_rows_by_bucket[k] = keep_c;
        sh.distribute_rows_by_bucket[k] = keep_d;
      }
      if (st == JT_OK) {
        best_o = sh;
        best_total = cur_c + cur_d;
      }
    }
    if (pl) jt_plan_free(pl);
    if (st != JT_OK) result = st;
  }
  // stage 3: the tuned shape with fused distribute pairs turned the other
  // way (fused items need the distribute kernel that runs at fewer blocks
  // per SM), and with recomputed clique tables; which one wins depends on
  // the network
  if (result == JT_OK && best_cw > 0) {
    jt_compile_opts alts[3] = {best_o, best_o, best_o};
    alts[0].fuse_distribute = best_o.fuse_distribute ? 0 : 1;
    alts[1].recompute_psi = best_o.recompute_psi ? 0 : 1;
    alts[2].collect_prefetch = best_o.collect_prefetch ? 0 : 1;
    for (const jt_compile_opts &alt : alts) {
      jt_plan *pl = nullptr;
      jt_status st = jt_compile(n_vars, card, parent_ptr, parents, cpt, &alt, &pl);
      double c_ms = -1, d_ms = -1;
      if (st == JT_OK) st = time_plan(pl, c_ms, d_ms);
      if (pl) jt_plan_free(pl);
      if (st == JT_ETOOBIG || st == JT_ENOMEM) continue;  // this variant does not fit: keep the others
      if (st != JT_OK) { result = st; break; }
      if (c_ms + d_ms < 0.99 * best_total) {
        best_o = alt;
        best_total = c_ms + d_ms;
      }
    }
  }
  cudaFree(d_ev);
  cudaFree(d_lp);
  cudaFree(d_post);
  cudaFree(d_st);
  if (result != JT_OK) return result;
  *best = best_o;
  if (best_ns_per_case) *best_ns_per_case = best_total * 1e6 / n_cases;
  return JT_OK;
}

extern "C" jt_status jt_autotune(int32_t n_vars, const int32_t *card, const int32_t *parent_ptr,
                                 const int32_t *parents, const double *cpt, const jt_compile_opts *base,
                                 int32_t n_cases, jt_compile_opts *best, double *best_ns_per_case) {
  return guarded([&] {
    return jt_autotune_impl(n_vars, card, parent_ptr, parents, cpt, base, n_cases, best, best_ns_per_case);
  });
}
