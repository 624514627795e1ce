// Serving loop: continuous batching of single-case requests over resident plans.
//
// One worker thread owns the device side.  Requests queue per plan; the
// worker repeatedly (1) retires finished batches -- copies their results to
// the request records and releases their stream and staging buffers -- and
// (2) admits new batches: for a plan with pending requests it takes up to
// max_batch of them (FIFO), picks an idle slot of that plan or carves a new
// one out of the server's device pool if the pool has room (evicting idle
// slots of other plans, least recently used first, when it has not), and
// enqueues the H2D copy, the batched inference chunk and the D2H copy on
// one of the server's streams.  Batches of different plans, and several
// batches of the same plan, are in flight at once and overlap on the GPU;
// requests that arrive meanwhile are admitted as soon as a stream and pool
// bytes free up.  A case's result does not depend on its batch: every case
// occupies one lane of a tile and its reductions run in a fixed order.
//
// Every device and pinned host buffer and every stream is created by
// jt_server_create and jt_server_add_plan: the pool (one device allocation
// of the server's arena budget, sub-allocated first-fit with coalescing),
// 2 x max_inflight streams (default and highest priority) and events, and
// per plan max_inflight pairs of staging buffers.  The worker itself
// allocates nothing.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <unordered_map>
#include <vector>

#include "runtime.h"

using namespace jt;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t ticket;
  int plan_id;
  std::vector<int32_t> ev;
  std::vector<int32_t> query;  // empty = all variables
  Clock::time_point t_submit;
};

struct Result {
  bool ready = false;
  double log_pe = 0;
  int32_t status = 0;
  std::vector<double> post;    // full posterior row of the plan
  std::vector<int32_t> query;
  int plan_id = 0;
};

// A batch slot: one plan's per-batch tables in a region of the pool.
struct Slot {
  int plan_id = -1;
  size_t off = 0, bytes = 0;   // region of the pool
  jt::Arena arena;             // bound to the region (graphs captured per tile count)
  bool busy = false;
  int stream = -1, io = -1;    // while busy: the server stream and the plan's staging pair
  uint64_t last_used = 0;
  std::vector<Request> reqs;
};

// Pinned host and device staging buffers of one batch of a plan.
struct Io {
  void *d = nullptr, *h = nullptr;
  bool used = false;
};

// Iteration-level batching of one plan ("rolling" tiles).  The plan's
// tables for R case tiles are resident in a region of the pool; each tile
// holds up to W requests and advances one tree layer per tick: collect
// layers from the deepest to the root, then distribute layers from the
// root, then its finalize kernels.  A tick is two launches over explicit
// (work item, tile) lists -- every active tile's units at that tile's own
// layer -- so a tile admitted now joins the passes of tiles admitted
// earlier at the next tick instead of waiting for them to finish.  A tile's
// phase advances on the host, independent of the GPU's progress, so up to
// kRollDepth ticks are enqueued ahead (each with its own unit-list buffers
// and completion event): the ticks run back to back on the GPU without a
// host round trip between them, and a request arriving meanwhile joins at
// the next tick the host enqueues.  A tile's results are handed back when
// the tick that finalized it has completed.
struct RollTile {
  int phase = -1;            // -1 free; 0..2H+1 the next layer step; kDone finalized
  int64_t done_tick = -1;    // the tick whose completion makes its results readable
  std::vector<Request> reqs;
};
constexpr int kDone = 1 << 30;
constexpr int kRollDepth = 8;  // ticks of one plan enqueued ahead of the GPU

struct Roll {
  size_t off = 0, bytes = 0;   // pool region of the tiles' tables
  jt::Arena arena;
  int R = 0;                   // tiles
  cudaStream_t stream = nullptr;
  cudaEvent_t ev[kRollDepth] = {};
  std::vector<RollTile> tiles;
  void *d_io = nullptr, *h_io = nullptr;  // per tile: evidence, log P(e), posteriors, status
  size_t io_tile = 0, o_lp = 0, o_post = 0, o_st = 0;
  int2 *d_units = nullptr, *h_units = nullptr;  // [tick % kRollDepth][pass][cap]
  size_t cap = 0;
  int64_t ticks = 0;
  std::deque<int64_t> outstanding;  // enqueued ticks not yet seen complete
  int max_maps = 0;
};

struct PlanEntry {
  jt_plan *plan = nullptr;
  std::deque<Request> pending;
  size_t o_lp = 0, o_post = 0, o_st = 0, io_bytes = 0;
  std::vector<Io> io;
  std::vector<int64_t> latencies;
  int64_t completed = 0, batches = 0;
  std::unique_ptr<Roll> roll;  // iteration-level batching (else batch slots)
  int32_t high = 0;            // batches run on the high-priority streams
};

}  // namespace

struct jt_server {
  int64_t budget = 0;
  int max_batch = 256;
  int max_inflight = 8;
  int device = 0;
  char *pool = nullptr;              // device pool of `budget` bytes
  std::map<size_t, size_t> free_;    // free regions of the pool: offset -> bytes
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<char> stream_busy;
  std::vector<PlanEntry> plans;
  std::vector<std::unique_ptr<Slot>> slots;
  std::unordered_map<uint64_t, Result> results;
  uint64_t next_ticket = 1, tick = 0;
  int64_t bytes_in_use = 0, peak_bytes = 0;
  int64_t completed = 0, batches = 0, largest = 0, pending = 0, inflight = 0;
  int64_t slot_creations = 0, slot_evictions = 0;
  std::vector<int64_t> latencies;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread worker;
  size_t rr = 0;  // round-robin cursor over plans
};

namespace {

constexpr size_t kAlign = 256;
size_t al(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit allocation from the pool; false when no free region is large enough.
bool pool_alloc(jt_server *S, size_t bytes, size_t *off) {
  for (auto it = S->free_.begin(); it != S->free_.end(); ++it) {
    if (it->second < bytes) continue;
    *off = it->first;
    const size_t rest = it->second - bytes;
    const size_t roff = it->first + bytes;
    S->free_.erase(it);
    if (rest) S->free_[roff] = rest;
    return true;
  }
  return false;
}

void pool_free(jt_server *S, size_t off, size_t bytes) {
  auto it = S->free_.emplace(off, bytes).first;
  auto next = std::next(it);
  if (next != S->free_.end() && it->first + it->second == next->first) {
    it->second += next->second;
    S->free_.erase(next);
  }
  if (it != S->free_.begin()) {
    auto prev = std::prev(it);
    if (prev->first + prev->second == it->first) {
      prev->second += it->second;
      S->free_.erase(it);
    }
  }
}

size_t slot_arena_bytes(const jt_plan *pl, int max_batch) {
  const Plan &P = pl->P;
  const int tiles = (max_batch + P.tile - 1) / P.tile;
  return al(arena_layout(P).bytes(tiles));
}

// Bind a new slot of plan `pid` to a pool region (no allocation: host
// bookkeeping only).  When the pool has no region large enough, idle slots
// of other plans are evicted, least recently used first -- by a plan
// without any slot, or by one with a full batch of requests waiting behind
// its busy slots; a plan with a slot and a short queue waits for it
// instead, so resident slots are not traded back and forth under light
// load.
Slot *slot_create(jt_server *S, int pid) {
  jt_plan *pl = S->plans[pid].plan;
  const size_t need = slot_arena_bytes(pl, S->max_batch);
  size_t off = 0;
  bool has_slot = false;
  for (auto &sp : S->slots) has_slot = has_slot || sp->plan_id == pid;
  const bool backlog = (int64_t)S->plans[pid].pending.size() >= S->max_batch;
  while (!pool_alloc(S, need, &off)) {
    if (has_slot && !backlog) return nullptr;
    Slot *victim = nullptr;
    size_t vi = 0;
    for (size_t j = 0; j < S->slots.size(); ++j) {
      Slot &o = *S->slots[j];
      if (o.busy || o.plan_id == pid) continue;
      if (!victim || o.last_used < victim->last_used) { victim = &o; vi = j; }
    }
    if (!victim) return nullptr;  // wait for a busy slot to retire
    arena_free(victim->arena);    // the region is not owned: only its graphs are released
    pool_free(S, victim->off, victim->bytes);
    S->bytes_in_use -= (int64_t)victim->bytes;
    S->slots.erase(S->slots.begin() + vi);
    ++S->slot_evictions;
  }
  auto ns = std::make_unique<Slot>();
  ns->plan_id = pid;
  ns->off = off;
  ns->bytes = need;
  const int tiles = (S->max_batch + pl->P.tile - 1) / pl->P.tile;
  if (arena_wrap(pl->P, ns->arena, S->pool + off, need, tiles) != JT_OK) {
    pool_free(S, off, need);
    return nullptr;
  }
  S->bytes_in_use += (int64_t)need;
  S->peak_bytes = std::max(S->peak_bytes, S->bytes_in_use);
  ++S->slot_creations;
  S->slots.push_back(std::move(ns));
  return S->slots.back().get();
}

// Launch one batch on a slot.  Called with S->mu held.
bool slot_launch(jt_server *S, Slot &s, std::vector<Request> &&reqs) {
  PlanEntry &pe = S->plans[s.plan_id];
  jt_plan *pl = pe.plan;
  const Plan &P = pl->P;
  const int nb = (int)reqs.size();
  // streams [0, max_inflight) run at the default priority, the next
  // max_inflight at the highest; fewer than max_inflight batches are in
  // flight, so the plan's class has a free stream
  int si = pe.high ? S->max_inflight : 0;
  while (S->stream_busy[si]) ++si;
  int ii = 0;
  while (pe.io[ii].used) ++ii;      // and a free staging pair of the plan
  S->stream_busy[si] = 1;
  pe.io[ii].used = true;
  s.stream = si;
  s.io = ii;
  cudaStream_t st_ = S->streams[si];
  char *h = static_cast<char *>(pe.io[ii].h), *d = static_cast<char *>(pe.io[ii].d);
  int32_t *h_ev = reinterpret_cast<int32_t *>(h);
  for (int i = 0; i < nb; ++i) std::memcpy(h_ev + (size_t)i * P.n, reqs[i].ev.data(), sizeof(int32_t) * P.n);
  cudaMemcpyAsync(d, h, sizeof(int32_t) * (size_t)nb * P.n, cudaMemcpyHostToDevice, st_);
  // a fresh slot, or one whose last batch hit an expired device wait (its
  // cases reported JT_CASE_INCOMPLETE): the flag starts the batch cleared
  // (the passes clear every other per-chunk counter themselves)
  cudaMemsetAsync(s.arena.da.errflag, 0, sizeof(uint32_t), st_);
  jt_status st;
  {
    std::lock_guard<std::mutex> lk(pl->mu);
    st = run_chunk(pl, s.arena, reinterpret_cast<int32_t *>(d), nb, reinterpret_cast<double *>(d + pe.o_lp),
                   reinterpret_cast<double *>(d + pe.o_post), reinterpret_cast<int32_t *>(d + pe.o_st), st_);
  }
  cudaMemcpyAsync(h + pe.o_lp, d + pe.o_lp, sizeof(double) * nb, cudaMemcpyDeviceToHost, st_);
  cudaMemcpyAsync(h + pe.o_post, d + pe.o_post, sizeof(double) * (size_t)nb * P.sum_card, cudaMemcpyDeviceToHost, st_);
  cudaMemcpyAsync(h + pe.o_st, d + pe.o_st, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, st_);
  cudaEventRecord(S->events[si], st_);
  s.reqs = std::move(reqs);
  s.busy = true;
  s.last_used = ++S->tick;
  ++pe.batches;
  return st == JT_OK;
}

// Copy a finished slot's results to the request records.  S->mu held.
void slot_retire(jt_server *S, Slot &s, bool failed) {
  PlanEntry &pe = S->plans[s.plan_id];
  const Plan &P = pe.plan->P;
  const char *h = static_cast<const char *>(pe.io[s.io].h);
  const double *lp = reinterpret_cast<const double *>(h + pe.o_lp);
  const double *po = reinterpret_cast<const double *>(h + pe.o_post);
  const int32_t *st = reinterpret_cast<const int32_t *>(h + pe.o_st);
  const auto now = Clock::now();
  for (size_t i = 0; i < s.reqs.size(); ++i) {
    Result &r = S->results[s.reqs[i].ticket];
    r.ready = true;
    r.plan_id = s.plan_id;
    r.query = std::move(s.reqs[i].query);
    if (failed) {
      r.status = -1;
      r.log_pe = std::nan("");
      r.post.assign(P.sum_card, std::nan(""));
    } else {
      r.log_pe = lp[i];
      r.status = st[i];
      r.post.assign(po + i * P.sum_card, po + (i + 1) * P.sum_card);
    }
    const int64_t ns = std::chrono::duration_cast<std::chrono::nanoseconds>(now - s.reqs[i].t_submit).count();
    S->latencies.push_back(ns);
    pe.latencies.push_back(ns);
    ++pe.completed;
    ++S->completed;
  }
  S->inflight -= (int64_t)s.reqs.size();
  s.reqs.clear();
  s.busy = false;
  S->stream_busy[s.stream] = 0;
  pe.io[s.io].used = false;
  s.stream = s.io = -1;
}

// A one-tile view of an arena: every per-tile region starts at `tile`.
DevArena tile_view(const DevArena &A, const DevPlan &D, int tile, int W) {
  DevArena v = A;
  const int64_t t = tile;
  v.psi += t * D.psi_rows * W;
  v.phistar += t * D.sep_rows * W;
  v.rho += t * D.sep_rows * W;
  v.post += t * D.post_rows * W;
  v.partial += t * D.n_partials * W;
  v.maxbits += t * D.n_cliques * W;
  v.counters += t * D.n_groups;
  v.ev += t * D.n_vars * W;
  v.bad += t * W;
  v.ready += t * 2 * D.n_cliques;
  v.tiles = 1;
  return v;
}

// Hand back the results of the tiles a completed tick finalized.  S->mu held.
void roll_retire(jt_server *S, int pid, int64_t tick) {
  PlanEntry &pe = S->plans[pid];
  Roll &r = *pe.roll;
  const Plan &P = pe.plan->P;
  const auto now = Clock::now();
  for (int t = 0; t < r.R; ++t) {
    RollTile &T = r.tiles[t];
    if (T.phase != kDone || T.done_tick != tick) continue;
    const char *h = static_cast<const char *>(r.h_io) + (size_t)t * r.io_tile;
    const double *lp = reinterpret_cast<const double *>(h + r.o_lp);
    const double *po = reinterpret_cast<const double *>(h + r.o_post);
    const int32_t *st = reinterpret_cast<const int32_t *>(h + r.o_st);
    for (size_t i = 0; i < T.reqs.size(); ++i) {
      Result &res = S->results[T.reqs[i].ticket];
      res.ready = true;
      res.plan_id = pid;
      res.query = std::move(T.reqs[i].query);
      res.log_pe = lp[i];
      res.status = st[i];
      res.post.assign(po + i * P.sum_card, po + (i + 1) * P.sum_card);
      const int64_t ns = std::chrono::duration_cast<std::chrono::nanoseconds>(now - T.reqs[i].t_submit).count();
      S->latencies.push_back(ns);
      pe.latencies.push_back(ns);
      ++pe.completed;
      ++S->completed;
    }
    S->inflight -= (int64_t)T.reqs.size();
    T.reqs.clear();
    T.phase = -1;
    T.done_tick = -1;
  }
}

// Enqueue one tick of a rolling plan: admit pending requests into free
// tiles, advance every active tile by one layer, finalize the tiles that
// finished their last distribute layer.  S->mu held.
void roll_tick(jt_server *S, int pid) {
  PlanEntry &pe = S->plans[pid];
  Roll &r = *pe.roll;
  jt_plan *pl = pe.plan;
  const Plan &P = pl->P;
  const int W = P.tile, H = P.height;
  const int64_t k = r.ticks++;
  const int par = (int)(k % kRollDepth);
  cudaStream_t st_ = r.stream;
  std::lock_guard<std::mutex> plk(pl->mu);
  // admissions
  for (int t = 0; t < r.R && !pe.pending.empty(); ++t) {
    RollTile &T = r.tiles[t];
    if (T.phase != -1) continue;
    while (!pe.pending.empty() && (int)T.reqs.size() < W) {
      T.reqs.push_back(std::move(pe.pending.front()));
      pe.pending.pop_front();
    }
    const int nc = (int)T.reqs.size();
    S->pending -= nc;
    S->inflight += nc;
    S->largest = std::max<int64_t>(S->largest, nc);
    ++S->batches;
    ++pe.batches;
    char *h = static_cast<char *>(r.h_io) + (size_t)t * r.io_tile;
    char *d = static_cast<char *>(r.d_io) + (size_t)t * r.io_tile;
    int32_t *h_ev = reinterpret_cast<int32_t *>(h);
    for (int i = 0; i < nc; ++i) std::memcpy(h_ev + (size_t)i * P.n, T.reqs[i].ev.data(), sizeof(int32_t) * P.n);
    cudaMemcpyAsync(d, h, sizeof(int32_t) * (size_t)nc * P.n, cudaMemcpyHostToDevice, st_);
    // exactly this tile's entries (the kernels' per-tile strides, not the
    // arena's aligned region sizes: the next tile may be mid-pass)
    const DevArena v = tile_view(r.arena.da, pl->dp, t, W);
    cudaMemsetAsync(v.maxbits, 0, sizeof(uint32_t) * (size_t)pl->dp.n_cliques * W, st_);
    cudaMemsetAsync(v.counters, 0, sizeof(uint32_t) * (size_t)pl->dp.n_groups, st_);
    cudaMemsetAsync(v.bad, 0, sizeof(int32_t) * (size_t)W, st_);
    launch_evidence(P.cpt_per_thread, reinterpret_cast<const int32_t *>(d), nc, pl->dp, v, st_);
    T.phase = 0;
  }
  // this tick's units: every active tile at its own layer
  int2 *hc = r.h_units + (size_t)(2 * par) * r.cap, *hd = r.h_units + (size_t)(2 * par + 1) * r.cap;
  int2 *dc = r.d_units + (size_t)(2 * par) * r.cap, *dd = r.d_units + (size_t)(2 * par + 1) * r.cap;
  int nc = 0, nd = 0;
  for (int t = 0; t < r.R; ++t) {
    const int ph = r.tiles[t].phase;
    if (ph < 0 || ph == kDone) continue;
    if (ph <= H) {
      const Level &lv = P.levels[H - ph];
      for (int64_t i = lv.c_item_begin; i < lv.c_item_end; ++i) hc[nc++] = make_int2((int)i, t);
    } else {
      const Level &lv = P.levels[ph - H - 1];
      for (int64_t i = lv.d_item_begin; i < lv.d_item_end; ++i) hd[nd++] = make_int2((int)i, t);
    }
  }
  if (nc) cudaMemcpyAsync(dc, hc, sizeof(int2) * nc, cudaMemcpyHostToDevice, st_);
  if (nd) cudaMemcpyAsync(dd, hd, sizeof(int2) * nd, cudaMemcpyHostToDevice, st_);
  launch_collect_units(P.cpt_per_thread, pl->dp, r.arena.da, dc, nc, r.max_maps, st_);
  launch_distribute_units(P.cpt_per_thread, pl->dp, r.arena.da, dd, nd, st_);
  // tiles that ran their last distribute layer: finalize and copy back
  for (int t = 0; t < r.R; ++t) {
    RollTile &T = r.tiles[t];
    if (T.phase < 0 || T.phase == kDone) continue;
    if (T.phase < 2 * H + 1) {
      ++T.phase;
      continue;
    }
    const int n = (int)T.reqs.size();
    char *h = static_cast<char *>(r.h_io) + (size_t)t * r.io_tile;
    char *d = static_cast<char *>(r.d_io) + (size_t)t * r.io_tile;
    const DevArena v = tile_view(r.arena.da, pl->dp, t, W);
    launch_finalize(P.cpt_per_thread, pl->dp, v, n, P.dcl[P.root].sep_row, reinterpret_cast<double *>(d + r.o_lp),
                    reinterpret_cast<double *>(d + r.o_post), reinterpret_cast<int32_t *>(d + r.o_st), st_);
    cudaMemcpyAsync(h + r.o_lp, d + r.o_lp, sizeof(double) * n, cudaMemcpyDeviceToHost, st_);
    cudaMemcpyAsync(h + r.o_post, d + r.o_post, sizeof(double) * (size_t)n * P.sum_card, cudaMemcpyDeviceToHost, st_);
    cudaMemcpyAsync(h + r.o_st, d + r.o_st, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st_);
    T.phase = kDone;
    T.done_tick = k;
  }
  cudaEventRecord(r.ev[par], st_);
  r.outstanding.push_back(k);
}

// Retire completed ticks and enqueue the next ones of every rolling plan.
bool roll_step(jt_server *S) {
  bool progress = false;
  for (size_t pid = 0; pid < S->plans.size(); ++pid) {
    PlanEntry &pe = S->plans[pid];
    if (!pe.roll) continue;
    Roll &r = *pe.roll;
    while (!r.outstanding.empty()) {
      const int64_t k = r.outstanding.front();
      const cudaError_t q = cudaEventQuery(r.ev[k % kRollDepth]);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) cudaGetLastError();
      r.outstanding.pop_front();
      roll_retire(S, (int)pid, k);
      progress = true;
    }
    // enqueue ticks while a unit buffer is free and there is work
    while (r.outstanding.size() < (size_t)kRollDepth) {
      bool active = false, free_tile = false;
      for (const RollTile &T : r.tiles) {
        active = active || (T.phase >= 0 && T.phase != kDone);
        free_tile = free_tile || T.phase == -1;
      }
      if (!active && !(free_tile && !pe.pending.empty())) break;
      roll_tick(S, (int)pid);
      progress = true;
    }
  }
  return progress;
}

void worker_main(jt_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    bool progress = roll_step(S);
    if (progress) S->cv_done.notify_all();
    // (1) retire finished batches
    for (auto &sp : S->slots) {
      Slot &s = *sp;
      if (!s.busy) continue;
      cudaError_t q = cudaEventQuery(S->events[s.stream]);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) cudaGetLastError();
      slot_retire(S, s, q != cudaSuccess);
      progress = true;
    }
    if (progress) S->cv_done.notify_all();
    // (2) admit new batches, round-robin over plans
    const size_t np = S->plans.size();
    int busy = 0;
    for (char b : S->stream_busy) busy += b;
    for (size_t k = 0; k < np && busy < S->max_inflight; ++k) {
      const int pid = (int)((S->rr + k) % np);
      PlanEntry &pe = S->plans[pid];
      if (pe.pending.empty() || pe.roll) continue;
      Slot *slot = nullptr;
      for (auto &sp : S->slots)
        if (!sp->busy && sp->plan_id == pid) { slot = sp.get(); break; }
      if (!slot) slot = slot_create(S, pid);
      if (!slot) continue;  // wait for pool bytes
      std::vector<Request> batch;
      while (!pe.pending.empty() && (int)batch.size() < S->max_batch) {
        batch.push_back(std::move(pe.pending.front()));
        pe.pending.pop_front();
      }
      S->pending -= (int64_t)batch.size();
      S->inflight += (int64_t)batch.size();
      S->largest = std::max<int64_t>(S->largest, (int64_t)batch.size());
      ++S->batches;
      if (!slot_launch(S, *slot, std::move(batch))) {
        cudaStreamSynchronize(S->streams[slot->stream]);
        slot_retire(S, *slot, true);
      }
      ++busy;
      progress = true;
    }
    S->rr = np ? (S->rr + 1) % np : 0;
    if (S->stop && S->pending == 0 && S->inflight == 0) break;
    if (!progress) {
      if (S->inflight > 0)
        S->cv_work.wait_for(lk, std::chrono::microseconds(20));
      else
        S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

void roll_release(Roll &r) {
  if (r.stream) cudaStreamSynchronize(r.stream);
  arena_free(r.arena);
  if (r.d_io) cudaFree(r.d_io);
  if (r.h_io) cudaFreeHost(r.h_io);
  if (r.d_units) cudaFree(r.d_units);
  if (r.h_units) cudaFreeHost(r.h_units);
  for (cudaEvent_t e : r.ev) if (e) cudaEventDestroy(e);
  if (r.stream) cudaStreamDestroy(r.stream);
}

void server_release(jt_server *S) {
  for (auto &sp : S->slots) arena_free(sp->arena);
  S->slots.clear();
  for (auto &pe : S->plans) {
    for (Io &io : pe.io) {
      if (io.d) cudaFree(io.d);
      if (io.h) cudaFreeHost(io.h);
    }
    if (pe.roll) roll_release(*pe.roll);
  }
  for (cudaStream_t st : S->streams) if (st) cudaStreamDestroy(st);
  for (cudaEvent_t ev : S->events) if (ev) cudaEventDestroy(ev);
  if (S->pool) cudaFree(S->pool);
}

int64_t percentile(std::vector<int64_t> l, double q) {
  if (l.empty()) return 0;
  const size_t k = (size_t)std::min<double>((double)l.size() - 1, std::floor(q * (double)(l.size() - 1) + 0.5));
  std::nth_element(l.begin(), l.begin() + k, l.end());
  return l[k];
}

}  // namespace

extern "C" jt_status jt_server_create(int64_t arena_bytes, int32_t max_batch, int32_t max_inflight,
                                      jt_server **out) {
  if (!out) { set_error("out is NULL"); return JT_EINVAL; }
  *out = nullptr;
  if (max_batch <= 0 || max_inflight <= 0) { set_error("max_batch and max_inflight must be > 0"); return JT_EINVAL; }
  jt_server *S = new (std::nothrow) jt_server();
  if (!S) { set_error("host allocation failed"); return JT_ENOMEM; }
  S->budget = arena_bytes > 0 ? arena_bytes : (16LL << 30);
  S->max_batch = max_batch;
  S->max_inflight = max_inflight;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    set_error("no CUDA device");
    return JT_ECUDA;
  }
  // the whole budget as one pool, and the streams, now: the worker never allocates
  void *pool = nullptr;
  if (cudaMalloc(&pool, (size_t)S->budget) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    set_error("server pool: cudaMalloc of the arena budget failed");
    return JT_ENOMEM;
  }
  S->pool = static_cast<char *>(pool);
  S->free_[0] = (size_t)S->budget;
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  S->streams.assign(2 * (size_t)max_inflight, nullptr);
  S->events.assign(2 * (size_t)max_inflight, nullptr);
  S->stream_busy.assign(2 * (size_t)max_inflight, 0);
  for (int i = 0; i < 2 * max_inflight; ++i) {
    if (cudaStreamCreateWithPriority(&S->streams[i], cudaStreamNonBlocking, i < max_inflight ? least : greatest) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&S->events[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      server_release(S);
      delete S;
      set_error("server streams");
      return JT_ECUDA;
    }
  }
  try {
    S->worker = std::thread(worker_main, S);
  } catch (const std::exception &e) {
    server_release(S);
    delete S;
    set_error(std::string("server thread: ") + e.what());
    return JT_EINVAL;
  }
  *out = S;
  return JT_OK;
}

static jt_status jt_server_add_plan_impl(jt_server *S, jt_plan *pl, int32_t *plan_id) {
  if (!S || !pl || !plan_id) { set_error("null argument"); return JT_EINVAL; }
  if (pl->host_only) { set_error("plan compiled with host_only"); return JT_EINVAL; }
  if (pl->P.n_pruned > 0) { set_error("the server takes plans that are not pruned to a query set"); return JT_EINVAL; }
  if ((int64_t)slot_arena_bytes(pl, S->max_batch) > S->budget) {
    set_error("one batch of this plan does not fit the server's arena budget");
    return JT_ENOMEM;
  }
  // staging buffers for max_inflight batches of this plan (pinned host +
  // device), allocated here so the worker never allocates
  const Plan &P = pl->P;
  PlanEntry pe;
  pe.plan = pl;
  pe.o_lp = al(sizeof(int32_t) * (size_t)S->max_batch * P.n);
  pe.o_post = al(pe.o_lp + sizeof(double) * S->max_batch);
  pe.o_st = al(pe.o_post + sizeof(double) * (size_t)S->max_batch * P.sum_card);
  pe.io_bytes = al(pe.o_st + sizeof(int32_t) * S->max_batch);
  pe.io.assign(S->max_inflight, Io{});
  for (Io &io : pe.io) {
    if (cudaMalloc(&io.d, pe.io_bytes) != cudaSuccess || cudaHostAlloc(&io.h, pe.io_bytes, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      for (Io &j : pe.io) {
        if (j.d) cudaFree(j.d);
        if (j.h) cudaFreeHost(j.h);
      }
      set_error("server staging buffers");
      return JT_ENOMEM;
    }
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->plans.push_back(std::move(pe));
  *plan_id = (int32_t)S->plans.size() - 1;
  return JT_OK;
}

static jt_status jt_server_add_plan_rolling_impl(jt_server *S, jt_plan *pl, int32_t tiles, int32_t *plan_id) {
  if (!S || !pl || !plan_id || tiles <= 0) { set_error("bad argument"); return JT_EINVAL; }
  if (pl->host_only) { set_error("plan compiled with host_only"); return JT_EINVAL; }
  if (pl->P.n_pruned > 0) { set_error("the server takes plans that are not pruned to a query set"); return JT_EINVAL; }
  const Plan &P = pl->P;
  const int W = P.tile;
  auto r = std::make_unique<Roll>();
  r->R = tiles;
  r->tiles.assign(tiles, RollTile{});
  for (const Level &lv : P.levels) r->max_maps = std::max(r->max_maps, lv.c_max_maps);
  int64_t per_layer = 1;
  for (const Level &lv : P.levels)
    per_layer = std::max({per_layer, lv.c_item_end - lv.c_item_begin, lv.d_item_end - lv.d_item_begin});
  r->cap = (size_t)per_layer * tiles;
  r->o_lp = al(sizeof(int32_t) * (size_t)W * P.n);
  r->o_post = al(r->o_lp + sizeof(double) * W);
  r->o_st = al(r->o_post + sizeof(double) * (size_t)W * P.sum_card);
  r->io_tile = al(r->o_st + sizeof(int32_t) * W);
  const size_t need = al(arena_layout(P).bytes(tiles));
  auto fail = [&](jt_status st, const char *msg) {
    roll_release(*r);
    set_error(msg);
    return st;
  };
  // the ticks of a rolling plan are short launches: on a stream of the
  // highest priority their blocks are dispatched before those of the batch
  // slots' long passes, so a tick does not queue behind a whole layer of a
  // large plan
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  bool ok = cudaStreamCreateWithPriority(&r->stream, cudaStreamNonBlocking, greatest) == cudaSuccess;
  for (int i = 0; ok && i < kRollDepth; ++i)
    ok = cudaEventCreateWithFlags(&r->ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return fail(JT_ECUDA, "rolling plan: stream or events");
  }
  if (cudaMalloc(&r->d_io, r->io_tile * tiles) != cudaSuccess ||
      cudaHostAlloc(&r->h_io, r->io_tile * tiles, cudaHostAllocDefault) != cudaSuccess ||
      cudaMalloc((void **)&r->d_units, sizeof(int2) * 2 * kRollDepth * r->cap) != cudaSuccess ||
      cudaHostAlloc((void **)&r->h_units, sizeof(int2) * 2 * kRollDepth * r->cap, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return fail(JT_ENOMEM, "rolling plan: staging buffers");
  }
  std::lock_guard<std::mutex> lk(S->mu);
  size_t off = 0;
  if (!pool_alloc(S, need, &off)) return fail(JT_ENOMEM, "rolling plan: its tiles do not fit the server's free pool");
  if (arena_wrap(P, r->arena, S->pool + off, need, tiles) != JT_OK) {
    pool_free(S, off, need);
    return fail(JT_ENOMEM, "rolling plan: arena");
  }
  r->off = off;
  r->bytes = need;
  S->bytes_in_use += (int64_t)need;
  S->peak_bytes = std::max(S->peak_bytes, S->bytes_in_use);
  // the region may hold another plan's old data: the flag the finalize
  // kernels read starts cleared
  cudaMemsetAsync(r->arena.da.errflag, 0, sizeof(uint32_t), r->stream);
  PlanEntry pe;
  pe.plan = pl;
  pe.roll = std::move(r);
  S->plans.push_back(std::move(pe));
  *plan_id = (int32_t)S->plans.size() - 1;
  return JT_OK;
}

extern "C" jt_status jt_server_add_plan_rolling(jt_server *S, jt_plan *pl, int32_t tiles, int32_t *plan_id) {
  return guarded([&] { return jt_server_add_plan_rolling_impl(S, pl, tiles, plan_id); });
}

extern "C" jt_status jt_server_add_plan(jt_server *S, jt_plan *pl, int32_t *plan_id) {
  return guarded([&] { return jt_server_add_plan_impl(S, pl, plan_id); });
}

static jt_status jt_submit_impl(jt_server *S, int32_t plan_id, const int32_t *ev, const int32_t *query,
                               int32_t n_query, uint64_t *ticket) {
  if (!S || !ev || !ticket) { set_error("null argument"); return JT_EINVAL; }
  Request r;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (plan_id < 0 || plan_id >= (int32_t)S->plans.size()) { set_error("unknown plan id"); return JT_ENOTFOUND; }
    const Plan &P = S->plans[plan_id].plan->P;
    if (n_query < 0 || (n_query > 0 && !query)) { set_error("bad query"); return JT_EINVAL; }
    for (int i = 0; i < n_query; ++i)
      if (query[i] < 0 || query[i] >= P.n) { set_error("query variable out of range"); return JT_EINVAL; }
    r.ticket = S->next_ticket++;
    r.plan_id = plan_id;
    r.ev.assign(ev, ev + P.n);
    if (n_query > 0) r.query.assign(query, query + n_query);
    r.t_submit = Clock::now();
    *ticket = r.ticket;
    S->results[r.ticket] = Result{};
    S->plans[plan_id].pending.push_back(std::move(r));
    ++S->pending;
  }
  S->cv_work.notify_one();
  return JT_OK;
}

extern "C" jt_status jt_submit(jt_server *S, int32_t plan_id, const int32_t *ev, const int32_t *query,
                               int32_t n_query, uint64_t *ticket) {
  return guarded([&] { return jt_submit_impl(S, plan_id, ev, query, n_query, ticket); });
}

static jt_status jt_poll_impl(jt_server *S, uint64_t ticket, double *log_pe, double *post, int32_t *cst) {
  if (!S) { set_error("null server"); return JT_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->results.find(ticket);
  if (it == S->results.end()) { set_error("unknown ticket"); return JT_ENOTFOUND; }
  Result &r = it->second;
  if (!r.ready) return JT_EBUSY;
  if (r.status < 0) {
    S->results.erase(it);
    set_error("the batch of this request failed on the device");
    return JT_ECUDA;
  }
  const Plan &P = S->plans[r.plan_id].plan->P;
  if (log_pe) *log_pe = r.log_pe;
  if (cst) *cst = r.status;
  if (post) {
    if (r.query.empty()) {
      std::memcpy(post, r.post.data(), sizeof(double) * r.post.size());
    } else {
      size_t k = 0;
      for (int v : r.query)
        for (int j = 0; j < P.card[v]; ++j) post[k++] = r.post[P.post_off[v] + j];
    }
  }
  S->results.erase(it);
  return JT_OK;
}

extern "C" jt_status jt_poll(jt_server *S, uint64_t ticket, double *log_pe, double *post, int32_t *cst) {
  return guarded([&] { return jt_poll_impl(S, ticket, log_pe, post, cst); });
}

extern "C" jt_status jt_server_drain(jt_server *S) {
  if (!S) { set_error("null server"); return JT_EINVAL; }
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv_work.notify_one();
  S->cv_done.wait(lk, [&] { return S->pending == 0 && S->inflight == 0; });
  return JT_OK;
}

static jt_status jt_server_stats_impl(jt_server *S, int64_t *out) {
  if (!S || !out) { set_error("null argument"); return JT_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  out[0] = S->completed;
  out[1] = S->batches;
  out[2] = S->largest;
  out[3] = S->peak_bytes;
  out[4] = percentile(S->latencies, 0.50);
  out[5] = percentile(S->latencies, 0.99);
  out[6] = S->pending + S->inflight;
  out[7] = S->slot_creations;
  out[8] = S->slot_evictions;
  return JT_OK;
}

static jt_status jt_server_plan_stats_impl(jt_server *S, int32_t plan_id, int64_t *out) {
  if (!S || !out) { set_error("null argument"); return JT_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  if (plan_id < 0 || plan_id >= (int32_t)S->plans.size()) { set_error("unknown plan id"); return JT_ENOTFOUND; }
  const PlanEntry &pe = S->plans[plan_id];
  out[0] = pe.completed;
  out[1] = pe.batches;
  out[2] = percentile(pe.latencies, 0.50);
  out[3] = percentile(pe.latencies, 0.99);
  return JT_OK;
}

extern "C" jt_status jt_server_reset_latency(jt_server *S) {
  if (!S) { set_error("null argument"); return JT_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  S->latencies.clear();
  for (PlanEntry &pe : S->plans) pe.latencies.clear();
  return JT_OK;
}

extern "C" jt_status jt_server_set_priority(jt_server *S, int32_t plan_id, int32_t high) {
  if (!S) { set_error("null argument"); return JT_EINVAL; }
  std::lock_guard<std::mutex> lk(S->mu);
  if (plan_id < 0 || plan_id >= (int32_t)S->plans.size()) {
    set_error("unknown plan id");
    return JT_ENOTFOUND;
  }
  S->plans[plan_id].high = high ? 1 : 0;
  return JT_OK;
}

extern "C" jt_status jt_server_plan_stats(jt_server *S, int32_t plan_id, int64_t *out) {
  return guarded([&] { return jt_server_plan_stats_impl(S, plan_id, out); });
}

extern "C" jt_status jt_server_stats(jt_server *S, int64_t *out) {
  return guarded([&] { return jt_server_stats_impl(S, out); });
}

extern "C" void jt_server_destroy(jt_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (cudaStream_t st : S->streams)
    if (st) cudaStreamSynchronize(st);
  server_release(S);
  delete S;
}
