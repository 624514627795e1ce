// Multi-core CPU comparator in the style of the paper's own design
// (Section 2): cases are processed one at a time; the junction tree is
// walked layer by layer, with cliques and separators as the nodes of the
// layering; at each layer every table entry of every node in the layer is a
// task of ONE parallel loop, split statically over the worker threads (the
// hybrid inter- and intra-clique parallelism obtained by flattening the
// nested loops); the table operations (reduction, extension,
// marginalisation) find each entry's index in the other table from the
// entry's mixed-radix digits.  Tables are FP64 and unscaled (FP64's range
// suffices for the workloads this comparator is timed on); a case whose P(e)
// underflows reports JT_CASE_ZERO_EVIDENCE.
//
// Long marginalisations are cut into chunks of at most kChunk source entries
// whose partial sums are added in chunk order in a second step, so results
// do not depend on the number of threads.
//
// This is a context measurement of the paper's design on the host cores; no
// other call of the library uses it.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

#include "jt_internal.h"

namespace jt {
namespace {

constexpr int64_t kChunk = 1024;

// ---------------------------------------------------------------------------
// a pool of threads that run phases: every thread takes a static slice of
// the phase's flat task range, then all meet at a barrier
// ---------------------------------------------------------------------------
class Barrier {
 public:
  explicit Barrier(int n) : n_(n) {}
  void wait() {
    const unsigned gen = gen_.load(std::memory_order_acquire);
    if (count_.fetch_add(1, std::memory_order_acq_rel) + 1 == n_) {
      count_.store(0, std::memory_order_relaxed);
      gen_.fetch_add(1, std::memory_order_acq_rel);
      return;
    }
    for (int spin = 0; gen_.load(std::memory_order_acquire) == gen; ++spin)
      if (spin > 256) std::this_thread::yield();
  }

 private:
  const int n_;
  std::atomic<int> count_{0};
  std::atomic<unsigned> gen_{0};
};

struct Phase {
  // task i of the phase is task i - pref[j] of job j (pref ascending)
  std::vector<int64_t> pref;
  virtual void run(int job, int64_t first, int64_t last) const = 0;
  virtual ~Phase() = default;
};

class Pool {
 public:
  explicit Pool(int threads) : t_(threads), bar_(threads) {
    for (int i = 1; i < t_; ++i) th_.emplace_back([this, i] { worker(i); });
  }
  ~Pool() {
    stop_ = true;
    bar_.wait();
    for (auto &t : th_) t.join();
  }
  void run(const Phase &ph) {
    cur_ = &ph;
    bar_.wait();   // start
    slice(0);
    bar_.wait();   // end
  }

 private:
  void worker(int i) {
    for (;;) {
      bar_.wait();
      if (stop_) return;
      slice(i);
      bar_.wait();
    }
  }
  // thread i: tasks [i*N/T, (i+1)*N/T) of the flat range, job by job
  void slice(int i) const {
    const Phase &ph = *cur_;
    const int64_t N = ph.pref.empty() ? 0 : ph.pref.back();
    int64_t a = N * i / t_, b = N * (i + 1) / t_;
    if (a >= b) return;
    int j = (int)(std::upper_bound(ph.pref.begin(), ph.pref.end(), a) - ph.pref.begin()) - 1;
    while (a < b) {
      const int64_t end = std::min(b, ph.pref[j + 1]);
      if (end > a) ph.run(j, a - ph.pref[j], end - ph.pref[j]);
      a = end;
      ++j;
    }
  }
  const int t_;
  Barrier bar_;
  std::vector<std::thread> th_;
  const Phase *cur_ = nullptr;
  bool stop_ = false;
};

// ---------------------------------------------------------------------------
// index mappings
// ---------------------------------------------------------------------------
// A walk over the entries of a table (vars with cards, last fastest) that
// keeps the entry's index in other tables: idx[k] = sum_i digit_i * w[k][i].
struct Walker {
  std::vector<int> card;
  std::vector<std::vector<int64_t>> w;  // per target, weight of each variable
  std::vector<int> digit;
  std::vector<int64_t> idx;
  void start(int64_t e) {
    digit.assign(card.size(), 0);
    idx.assign(w.size(), 0);
    for (int i = (int)card.size() - 1; i >= 0; --i) {
      digit[i] = (int)(e % card[i]);
      e /= card[i];
      for (size_t k = 0; k < w.size(); ++k) idx[k] += digit[i] * w[k][i];
    }
  }
  void next() {
    for (int i = (int)card.size() - 1; i >= 0; --i) {
      for (size_t k = 0; k < w.size(); ++k) idx[k] += w[k][i];
      if (++digit[i] < card[i]) return;
      for (size_t k = 0; k < w.size(); ++k) idx[k] -= (int64_t)card[i] * w[k][i];
      digit[i] = 0;
    }
  }
};

// weight of each of `vars` in a table laid out as `tvars` (last fastest);
// 0 for variables the table does not hold
std::vector<int64_t> weights_in(const std::vector<int> &vars, const std::vector<int> &tvars,
                                const std::vector<int> &card) {
  std::vector<int64_t> stride(tvars.size(), 1);
  for (int i = (int)tvars.size() - 2; i >= 0; --i) stride[i] = stride[i + 1] * card[tvars[i + 1]];
  std::vector<int64_t> w(vars.size(), 0);
  for (size_t i = 0; i < vars.size(); ++i) {
    auto it = std::find(tvars.begin(), tvars.end(), vars[i]);
    if (it != tvars.end()) w[i] = stride[it - tvars.begin()];
  }
  return w;
}

// A marginalisation target: entry t of a table of `tvars` sums the source
// entries whose digits of tvars equal t's (the remaining variables `uvars`
// run over all their states).  Cut into chunks of kChunk source entries.
struct Marg {
  int64_t src_off = 0;               // source table in the case's psi
  std::vector<int> tcard, ucard;
  std::vector<int64_t> tw, uw;       // weights in the source table
  int64_t T = 1, U = 1, nchunk = 1;
  int64_t part_off = 0;              // into the partials buffer
};

Marg make_marg(const Plan &P, int src_clique, int64_t src_off, const std::vector<int> &tvars) {
  const HostClique &C = P.cl[src_clique];
  Marg m;
  m.src_off = src_off;
  std::vector<int> uvars;
  for (int v : C.vars)
    if (std::find(tvars.begin(), tvars.end(), v) == tvars.end()) uvars.push_back(v);
  for (int v : tvars) { m.tcard.push_back(P.card[v]); m.T *= P.card[v]; }
  for (int v : uvars) { m.ucard.push_back(P.card[v]); m.U *= P.card[v]; }
  m.tw = weights_in(tvars, C.vars, P.card);
  m.uw = weights_in(uvars, C.vars, P.card);
  m.nchunk = (m.U + kChunk - 1) / kChunk;
  return m;
}

// ---------------------------------------------------------------------------
// the phases of one case
// ---------------------------------------------------------------------------
struct CaseState {
  std::vector<double> psi;      // all clique tables, clique c at psi_off[c]
  std::vector<double> phis;     // upward messages phi*, clique c at sep_off[c]
  std::vector<double> ratio;    // phi** / phi*
  std::vector<double> partial;  // chunk sums of the current marginalisation
  std::vector<double> marg;     // posterior marginals (sum card)
  const int32_t *ev = nullptr;  // this case's evidence [n]
};

// reduction + initialisation: psi_C = base_C x prod_{v in C observed} [x_v = e_v]
struct InitPhase : Phase {
  const Plan *P;
  CaseState *S;
  const std::vector<int64_t> *psi_off;
  std::vector<int> job_clique;
  void run(int job, int64_t first, int64_t last) const override {
    const int c = job_clique[job];
    const HostClique &C = P->cl[c];
    const double *b = P->base64.data() + P->p_base_off[c];
    double *psi = S->psi.data() + (*psi_off)[c];
    const int64_t e0 = first * kChunk, e1 = std::min(C.size, last * kChunk);
    std::vector<int> obs;  // positions of observed variables
    for (size_t i = 0; i < C.vars.size(); ++i)
      if (S->ev[C.vars[i]] >= 0) obs.push_back((int)i);
    Walker wk;
    wk.card = C.card;
    wk.start(e0);
    for (int64_t e = e0; e < e1; ++e, wk.next()) {
      bool keep = true;
      for (int i : obs) keep = keep && wk.digit[i] == S->ev[C.vars[i]];
      psi[e] = keep ? b[e] : 0.0;
    }
  }
};

// marginalisation, step 1: chunk sums
struct MargPhase : Phase {
  const std::vector<Marg> *jobs;
  CaseState *S;
  void run(int job, int64_t first, int64_t last) const override {
    const Marg &m = (*jobs)[job];
    const double *src = S->psi.data() + m.src_off;
    Walker wk;
    wk.card = m.ucard;
    wk.w = {m.uw};
    for (int64_t q = first; q < last; ++q) {
      const int64_t t = q / m.nchunk, k = q - t * m.nchunk;
      int64_t a = 0, r = t;
      for (int i = (int)m.tcard.size() - 1; i >= 0; --i) {
        a += (r % m.tcard[i]) * m.tw[i];
        r /= m.tcard[i];
      }
      const int64_t u0 = k * kChunk, u1 = std::min(m.U, u0 + kChunk);
      wk.start(u0);
      double s = 0.0;
      for (int64_t u = u0; u < u1; ++u, wk.next()) s += src[a + wk.idx[0]];
      S->partial[m.part_off + q] = s;
    }
  }
};

// marginalisation, step 2: chunk sums added in chunk order into `out`
// (divide = 1: out receives sum / phi* with 0/0 := 0, the separator division)
struct CombinePhase : Phase {
  const std::vector<Marg> *jobs;
  std::vector<double *> out;
  std::vector<const double *> divisor;  // nullptr: plain sum
  CaseState *S;
  void run(int job, int64_t first, int64_t last) const override {
    const Marg &m = (*jobs)[job];
    for (int64_t t = first; t < last; ++t) {
      double s = 0.0;
      for (int64_t k = 0; k < m.nchunk; ++k) s += S->partial[m.part_off + t * m.nchunk + k];
      if (divisor[job]) {
        const double d = divisor[job][t];
        s = d > 0.0 ? s / d : 0.0;
      }
      out[job][t] = s;
    }
  }
};

// extension: psi_C[e] *= prod_k msg_k[idx_k(e)] (collect: children's phi*;
// distribute: the clique's own ratio on its upward separator)
struct ExtendPhase : Phase {
  const Plan *P;
  CaseState *S;
  const std::vector<int64_t> *psi_off;
  std::vector<int> job_clique;
  std::vector<std::vector<const double *>> msg;  // per job, per factor: per-case message base
  std::vector<std::vector<std::vector<int64_t>>> w;  // per job, per factor: weights of the clique's vars
  void run(int job, int64_t first, int64_t last) const override {
    const HostClique &C = P->cl[job_clique[job]];
    double *psi = S->psi.data() + (*psi_off)[job_clique[job]];
    const int64_t e0 = first * kChunk, e1 = std::min(C.size, last * kChunk);
    Walker wk;
    wk.card = C.card;
    wk.w = w[job];
    wk.start(e0);
    const auto &M = msg[job];
    for (int64_t e = e0; e < e1; ++e, wk.next()) {
      double x = psi[e];
      for (size_t k = 0; k < M.size(); ++k) x *= M[k][wk.idx[k]];
      psi[e] = x;
    }
  }
};

int64_t chunks(int64_t n) { return (n + kChunk - 1) / kChunk; }

}  // namespace

jt_status cpu_layers_infer(const Plan &P, int32_t n_cases, const int32_t *ev, double *log_pe, double *post,
                           int32_t *status, int threads) {
  if (P.n_sliced > 0 || P.n_pruned > 0) {
    set_error("the CPU comparator runs unspecialised plans only");
    return JT_EINVAL;
  }
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
  const int m = (int)P.cl.size(), n = P.n;
  std::vector<int64_t> psi_off(m), sep_off(m);
  int64_t sum_psi = 0, sum_sep = 0;
  for (int c = 0; c < m; ++c) {
    psi_off[c] = sum_psi;
    sum_psi += P.cl[c].size;
    sep_off[c] = sum_sep;
    sum_sep += P.cl[c].nsep;
  }
  CaseState S;
  S.psi.assign(sum_psi, 0.0);
  S.phis.assign(sum_sep, 0.0);
  S.ratio.assign(sum_sep, 0.0);
  S.marg.assign(P.sum_card, 0.0);
  std::vector<std::vector<int>> at_depth(P.height + 1);
  for (int c = 0; c < m; ++c) at_depth[P.cl[c].depth].push_back(c);
  auto upsep = [&](int c) {
    const HostClique &C = P.cl[c];
    return std::vector<int>(C.vars.begin(), C.vars.begin() + C.n_up);
  };

  // ---- phases that do not depend on the evidence values: built once ----
  InitPhase init;
  init.P = &P;
  init.S = &S;
  init.psi_off = &psi_off;
  init.pref = {0};
  for (int c = 0; c < m; ++c) {
    init.job_clique.push_back(c);
    init.pref.push_back(init.pref.back() + chunks(P.cl[c].size));
  }
  int64_t max_part = 1;
  // collect, layer d: separators of the depth-d cliques, then their parents absorb
  struct Layer {
    std::vector<Marg> marg;
    MargPhase mp;
    CombinePhase cp;
    ExtendPhase xp;
  };
  auto finish_marg = [&](Layer &L) {
    L.mp.jobs = &L.marg;
    L.mp.S = &S;
    L.cp.jobs = &L.marg;
    L.cp.S = &S;
    L.mp.pref = {0};
    L.cp.pref = {0};
    int64_t part = 0;
    for (Marg &g : L.marg) {
      g.part_off = part;
      part += g.T * g.nchunk;
      L.mp.pref.push_back(L.mp.pref.back() + g.T * g.nchunk);
      L.cp.pref.push_back(L.cp.pref.back() + g.T);
    }
    max_part = std::max(max_part, part);
  };
  std::vector<Layer> up(P.height + 1), down(P.height + 1);
  for (int d = P.height; d >= 1; --d) {
    Layer &L = up[d];
    for (int c : at_depth[d]) {
      L.marg.push_back(make_marg(P, c, psi_off[c], upsep(c)));
      L.cp.out.push_back(S.phis.data() + sep_off[c]);
      L.cp.divisor.push_back(nullptr);
    }
    finish_marg(L);
    L.xp.P = &P;
    L.xp.S = &S;
    L.xp.psi_off = &psi_off;
    L.xp.pref = {0};
    for (int p : at_depth[d - 1]) {
      const HostClique &Cp = P.cl[p];
      if (Cp.children.empty()) continue;
      std::vector<const double *> msg;
      std::vector<std::vector<int64_t>> w;
      for (int k : Cp.children) {
        msg.push_back(S.phis.data() + sep_off[k]);
        w.push_back(weights_in(Cp.vars, upsep(k), P.card));
      }
      L.xp.job_clique.push_back(p);
      L.xp.msg.push_back(msg);
      L.xp.w.push_back(w);
      L.xp.pref.push_back(L.xp.pref.back() + chunks(Cp.size));
    }
  }
  // root total
  Layer rootL;
  rootL.marg.push_back(make_marg(P, P.root, psi_off[P.root], {}));
  double root_total = 0.0;
  rootL.cp.out.push_back(&root_total);
  rootL.cp.divisor.push_back(nullptr);
  finish_marg(rootL);
  // distribute, layer d: separators of the depth-(d+1) cliques from their
  // parents (division by phi* fused), then those cliques absorb
  for (int d = 0; d < P.height; ++d) {
    Layer &L = down[d];
    for (int c : at_depth[d + 1]) {
      L.marg.push_back(make_marg(P, P.cl[c].parent, psi_off[P.cl[c].parent], upsep(c)));
      L.cp.out.push_back(S.ratio.data() + sep_off[c]);
      L.cp.divisor.push_back(S.phis.data() + sep_off[c]);
    }
    finish_marg(L);
    L.xp.P = &P;
    L.xp.S = &S;
    L.xp.psi_off = &psi_off;
    L.xp.pref = {0};
    for (int c : at_depth[d + 1]) {
      const HostClique &C = P.cl[c];
      L.xp.job_clique.push_back(c);
      L.xp.msg.push_back({S.ratio.data() + sep_off[c]});
      L.xp.w.push_back({weights_in(C.vars, upsep(c), P.card)});
      L.xp.pref.push_back(L.xp.pref.back() + chunks(C.size));
    }
  }
  // posterior marginals: each variable from the smallest clique holding it
  Layer postL;
  for (int v = 0; v < n; ++v) {
    postL.marg.push_back(make_marg(P, P.post_src[v], psi_off[P.post_src[v]], {v}));
    postL.cp.out.push_back(S.marg.data() + P.post_off[v]);
    postL.cp.divisor.push_back(nullptr);
  }
  finish_marg(postL);
  S.partial.assign(max_part, 0.0);

  Pool pool(threads);
  for (int32_t i = 0; i < n_cases; ++i) {
    S.ev = ev + (int64_t)i * n;
    double *po = post + (int64_t)i * P.sum_card;
    bool bad = false;
    for (int v = 0; v < n; ++v) bad = bad || S.ev[v] < -1 || S.ev[v] >= P.card[v];
    if (bad) {
      log_pe[i] = NAN;
      status[i] = JT_CASE_BAD_EVIDENCE;
      for (int64_t j = 0; j < P.sum_card; ++j) po[j] = NAN;
      continue;
    }
    pool.run(init);
    for (int d = P.height; d >= 1; --d) {
      pool.run(up[d].mp);
      pool.run(up[d].cp);
      pool.run(up[d].xp);
    }
    pool.run(rootL.mp);
    pool.run(rootL.cp);
    if (!(root_total > 0.0)) {
      log_pe[i] = -INFINITY;
      status[i] = JT_CASE_ZERO_EVIDENCE;
      for (int64_t j = 0; j < P.sum_card; ++j) po[j] = NAN;
      continue;
    }
    for (int d = 0; d < P.height; ++d) {
      pool.run(down[d].mp);
      pool.run(down[d].cp);
      pool.run(down[d].xp);
    }
    pool.run(postL.mp);
    pool.run(postL.cp);
    log_pe[i] = std::log(root_total);
    status[i] = JT_CASE_OK;
    for (int v = 0; v < n; ++v) {
      const int64_t o = P.post_off[v];
      const int r = P.card[v];
      if (S.ev[v] >= 0) {
        for (int j = 0; j < r; ++j) po[o + j] = j == S.ev[v] ? 1.0 : 0.0;
        continue;
      }
      double s = 0.0;
      for (int j = 0; j < r; ++j) s += S.marg[o + j];
      for (int j = 0; j < r; ++j) po[o + j] = S.marg[o + j] / s;
    }
  }
  return JT_OK;
}

}  // namespace jt
