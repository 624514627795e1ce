// Serving loop: continuous batching of single-case requests over resident plans.
//
// One worker thread owns the device side.  Requests queue per plan; the
// worker repeatedly (1) retires finished batches -- copies their results to
// the request records and frees their arena bytes -- and (2) admits new
// batches: for a plan with pending requests it takes up to max_batch of them
// (FIFO), picks an idle slot of that plan or creates one if the arena budget
// allows, and enqueues H2D copy, the batched inference chunk and the D2H copy
// on the slot's own stream.  Batches of different plans, and several batches
// of the same plan, are therefore in flight at once and overlap on the GPU;
// requests that arrive meanwhile are admitted as soon as a slot and arena
// bytes free up.  A case's result does not depend on its batch: every case
// occupies one lane of a tile and its reductions run in a fixed order.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
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

struct Slot {
  int plan_id = -1;
  jt::Arena arena;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  void *d_io = nullptr, *h_io = nullptr;
  size_t o_lp = 0, o_post = 0, o_st = 0;
  size_t bytes = 0;            // arena + device io bytes counted against the budget
  bool busy = false;
  std::vector<Request> reqs;
};

struct PlanEntry {
  jt_plan *plan;
  std::deque<Request> pending;
};

}  // namespace

struct jt_server {
  int64_t budget = 0;
  int max_batch = 256;
  int max_inflight = 8;
  int device = 0;
  std::vector<PlanEntry> plans;
  std::vector<std::unique_ptr<Slot>> slots;
  std::unordered_map<uint64_t, Result> results;
  uint64_t next_ticket = 1;
  int64_t bytes_in_use = 0, peak_bytes = 0;
  int64_t completed = 0, batches = 0, largest = 0, pending = 0, inflight = 0;
  std::vector<int64_t> latencies;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread worker;
  size_t rr = 0;  // round-robin cursor over plans
};

namespace {

void slot_free(Slot &s) {
  arena_free(s.arena);
  if (s.d_io) cudaFree(s.d_io);
  if (s.h_io) cudaFreeHost(s.h_io);
  if (s.stream) cudaStreamDestroy(s.stream);
  if (s.done) cudaEventDestroy(s.done);
  s.d_io = s.h_io = nullptr;
  s.stream = nullptr;
  s.done = nullptr;
}

size_t slot_bytes(const jt_plan *pl, int max_batch, size_t *io_bytes) {
  const Plan &P = pl->P;
  const int tiles = (max_batch + P.tile - 1) / P.tile;
  const size_t io = sizeof(int32_t) * (size_t)max_batch * P.n + sizeof(double) * max_batch +
                    sizeof(double) * (size_t)max_batch * P.sum_card + sizeof(int32_t) * max_batch + 4 * 256;
  if (io_bytes) *io_bytes = io;
  return arena_layout(P).bytes(tiles) + io;
}

bool slot_create(jt_server *S, int plan_id, Slot &s) {
  jt_plan *pl = S->plans[plan_id].plan;
  const Plan &P = pl->P;
  const int tiles = (S->max_batch + P.tile - 1) / P.tile;
  size_t io = 0;
  s.bytes = slot_bytes(pl, S->max_batch, &io);
  if (arena_alloc(P, s.arena, tiles) != JT_OK) return false;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t o_ev = 0;
  s.o_lp = al(o_ev + sizeof(int32_t) * (size_t)S->max_batch * P.n);
  s.o_post = al(s.o_lp + sizeof(double) * S->max_batch);
  s.o_st = al(s.o_post + sizeof(double) * (size_t)S->max_batch * P.sum_card);
  const size_t total = al(s.o_st + sizeof(int32_t) * S->max_batch);
  if (cudaMalloc(&s.d_io, total) != cudaSuccess || cudaHostAlloc(&s.h_io, total, cudaHostAllocDefault) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    slot_free(s);
    return false;
  }
  s.plan_id = plan_id;
  return true;
}

// Launch one batch on a slot.  Called with S->mu held.
bool slot_launch(jt_server *S, Slot &s, std::vector<Request> &&reqs) {
  jt_plan *pl = S->plans[s.plan_id].plan;
  const Plan &P = pl->P;
  const int nb = (int)reqs.size();
  char *h = static_cast<char *>(s.h_io), *d = static_cast<char *>(s.d_io);
  int32_t *h_ev = reinterpret_cast<int32_t *>(h);
  for (int i = 0; i < nb; ++i) std::memcpy(h_ev + (size_t)i * P.n, reqs[i].ev.data(), sizeof(int32_t) * P.n);
  cudaMemcpyAsync(d, h, sizeof(int32_t) * (size_t)nb * P.n, cudaMemcpyHostToDevice, s.stream);
  // a batch that hit an expired device wait left the slot's flag set (its
  // cases reported JT_CASE_INCOMPLETE); the slot is idle, so clear it
  cudaMemsetAsync(s.arena.da.errflag, 0, sizeof(uint32_t), s.stream);
  jt_status st;
  {
    std::lock_guard<std::mutex> lk(pl->mu);
    st = run_chunk(pl, s.arena, reinterpret_cast<int32_t *>(d), nb, reinterpret_cast<double *>(d + s.o_lp),
                   reinterpret_cast<double *>(d + s.o_post), reinterpret_cast<int32_t *>(d + s.o_st), s.stream);
  }
  cudaMemcpyAsync(h + s.o_lp, d + s.o_lp, sizeof(double) * nb, cudaMemcpyDeviceToHost, s.stream);
  cudaMemcpyAsync(h + s.o_post, d + s.o_post, sizeof(double) * (size_t)nb * P.sum_card, cudaMemcpyDeviceToHost,
                  s.stream);
  cudaMemcpyAsync(h + s.o_st, d + s.o_st, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s.stream);
  cudaEventRecord(s.done, s.stream);
  s.reqs = std::move(reqs);
  s.busy = true;
  return st == JT_OK;
}

// Copy a finished slot's results to the request records.  S->mu held.
void slot_retire(jt_server *S, Slot &s, bool failed) {
  jt_plan *pl = S->plans[s.plan_id].plan;
  const Plan &P = pl->P;
  const char *h = static_cast<const char *>(s.h_io);
  const double *lp = reinterpret_cast<const double *>(h + s.o_lp);
  const double *po = reinterpret_cast<const double *>(h + s.o_post);
  const int32_t *st = reinterpret_cast<const int32_t *>(h + s.o_st);
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
    S->latencies.push_back(std::chrono::duration_cast<std::chrono::nanoseconds>(now - s.reqs[i].t_submit).count());
    ++S->completed;
  }
  S->inflight -= (int64_t)s.reqs.size();
  s.reqs.clear();
  s.busy = false;
}

void worker_main(jt_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    bool progress = false;
    // (1) retire finished batches
    for (auto &sp : S->slots) {
      Slot &s = *sp;
      if (!s.busy) continue;
      cudaError_t q = cudaEventQuery(s.done);
      if (q == cudaErrorNotReady) continue;
      slot_retire(S, s, q != cudaSuccess);
      if (q != cudaSuccess) cudaGetLastError();
      progress = true;
    }
    if (progress) S->cv_done.notify_all();
    // (2) admit new batches, round-robin over plans
    const size_t np = S->plans.size();
    int busy = 0;
    for (auto &sp : S->slots) busy += sp->busy;
    for (size_t k = 0; k < np && busy < S->max_inflight; ++k) {
      const int pid = (int)((S->rr + k) % np);
      PlanEntry &pe = S->plans[pid];
      if (pe.pending.empty()) continue;
      Slot *slot = nullptr;
      for (auto &sp : S->slots)
        if (!sp->busy && sp->plan_id == pid) { slot = sp.get(); break; }
      if (!slot) {
        const int64_t need = (int64_t)slot_bytes(pe.plan, S->max_batch, nullptr);
        if (S->bytes_in_use + need > S->budget) {
          // reclaim an idle slot of another plan if that makes room
          for (size_t j = 0; j < S->slots.size(); ++j) {
            Slot &o = *S->slots[j];
            if (!o.busy && o.plan_id != pid) {
              S->bytes_in_use -= (int64_t)o.bytes;
              slot_free(o);
              S->slots.erase(S->slots.begin() + j);
              break;
            }
          }
        }
        if (S->bytes_in_use + need > S->budget) continue;  // wait for memory
        auto ns = std::make_unique<Slot>();
        if (!slot_create(S, pid, *ns)) continue;
        S->bytes_in_use += (int64_t)ns->bytes;
        S->peak_bytes = std::max(S->peak_bytes, S->bytes_in_use);
        slot = ns.get();
        S->slots.push_back(std::move(ns));
      }
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
        cudaStreamSynchronize(slot->stream);
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
  try {
    S->worker = std::thread(worker_main, S);
  } catch (const std::exception &e) {
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
  std::lock_guard<std::mutex> lk(S->mu);
  if ((int64_t)slot_bytes(pl, S->max_batch, nullptr) > S->budget) {
    set_error("one batch of this plan does not fit the server's arena budget");
    return JT_ENOMEM;
  }
  S->plans.push_back(PlanEntry{pl, {}});
  *plan_id = (int32_t)S->plans.size() - 1;
  return JT_OK;
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
  std::vector<int64_t> l = S->latencies;
  if (l.empty()) {
    out[4] = out[5] = 0;
  } else {
    auto pct = [&](double q) {
      size_t k = (size_t)std::min<double>((double)l.size() - 1, std::floor(q * (double)(l.size() - 1) + 0.5));
      std::nth_element(l.begin(), l.begin() + k, l.end());
      return l[k];
    };
    out[4] = pct(0.50);
    out[5] = pct(0.99);
  }
  out[6] = S->pending + S->inflight;
  return JT_OK;
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
  for (auto &sp : S->slots) {
    if (sp->stream) cudaStreamSynchronize(sp->stream);
    slot_free(*sp);
  }
  delete S;
}
