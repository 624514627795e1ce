// Host-side network compiler: BN -> junction tree -> device work description.
//
// Section 1 of the paper: a BN is converted into a secondary structure, the
// junction tree, whose nodes (cliques) and edges (separators) carry
// potential tables.  Section 2: the tree is traversed breadth-first and
// every clique is tagged with its layer; a root-selection strategy keeps
// the number of layers small; table operations are driven by index
// mappings between the original and the updated table.  This file builds
// all of that once per network:
//   moral graph -> min-fill elimination -> maximal cliques -> maximum-weight
//   spanning tree -> root -> BFS layers -> per-clique variable layout ->
//   index maps of every table operation -> per-layer thread-block lists.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <queue>
#include <tuple>

#include "jt_internal.h"

namespace jt {
namespace {

using Bits = std::vector<uint64_t>;

inline bool bit(const Bits &b, int i) { return (b[i >> 6] >> (i & 63)) & 1ull; }
inline void setbit(Bits &b, int i) { b[i >> 6] |= 1ull << (i & 63); }
inline void clearbit(Bits &b, int i) { b[i >> 6] &= ~(1ull << (i & 63)); }

int popcount_and(const Bits &a, const Bits &b) {
  int k = 0;
  for (size_t w = 0; w < a.size(); ++w) k += __builtin_popcountll(a[w] & b[w]);
  return k;
}

bool subset_of(const Bits &a, const Bits &b) {
  for (size_t w = 0; w < a.size(); ++w)
    if (a[w] & ~b[w]) return false;
  return true;
}

std::vector<int> members(const Bits &b, int n) {
  std::vector<int> out;
  for (int i = 0; i < n; ++i)
    if (bit(b, i)) out.push_back(i);
  return out;
}

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
jt_status validate(int32_t n, const int32_t *card, const int32_t *pptr, const int32_t *par,
                   const double *cpt, std::string &err) {
  if (n <= 0 || !card || !pptr || !cpt) { err = "empty network or null array"; return JT_EINVAL; }
  if (pptr[0] != 0) { err = "parent_ptr[0] must be 0"; return JT_EINVAL; }
  for (int v = 0; v < n; ++v) {
    if (card[v] < 2 || card[v] > (1 << 20)) { err = "card out of range at variable " + std::to_string(v); return JT_EINVAL; }
    if (pptr[v + 1] < pptr[v]) { err = "parent_ptr not monotone"; return JT_EINVAL; }
  }
  if (pptr[n] > 0 && !par) { err = "null parents"; return JT_EINVAL; }
  for (int v = 0; v < n; ++v) {
    for (int k = pptr[v]; k < pptr[v + 1]; ++k) {
      int p = par[k];
      if (p < 0 || p >= n || p == v) { err = "bad parent of variable " + std::to_string(v); return JT_EINVAL; }
      for (int q = pptr[v]; q < k; ++q)
        if (par[q] == p) { err = "duplicate parent of variable " + std::to_string(v); return JT_EINVAL; }
    }
  }
  // Kahn's algorithm: every node must be removable
  std::vector<int> indeg(n, 0);
  std::vector<std::vector<int>> kids(n);
  for (int v = 0; v < n; ++v)
    for (int k = pptr[v]; k < pptr[v + 1]; ++k) { kids[par[k]].push_back(v); ++indeg[v]; }
  std::vector<int> stack;
  for (int v = 0; v < n; ++v)
    if (!indeg[v]) stack.push_back(v);
  int seen = 0;
  while (!stack.empty()) {
    int v = stack.back();
    stack.pop_back();
    ++seen;
    for (int c : kids[v])
      if (--indeg[c] == 0) stack.push_back(c);
  }
  if (seen != n) { err = "parent graph has a directed cycle"; return JT_ECYCLE; }
  // CPT rows
  int64_t off = 0;
  for (int v = 0; v < n; ++v) {
    double rows = 1;
    for (int k = pptr[v]; k < pptr[v + 1]; ++k) rows *= card[par[k]];
    if (rows * card[v] > 2147483647.0) { err = "CPT of variable " + std::to_string(v) + " too large"; return JT_ETOOBIG; }
    for (int64_t r = 0; r < (int64_t)rows; ++r) {
      double s = 0;
      for (int x = 0; x < card[v]; ++x) {
        double p = cpt[off + r * card[v] + x];
        if (!(p >= 0.0) || !std::isfinite(p)) {
          err = "negative or non-finite CPT entry of variable " + std::to_string(v);
          return JT_EINVAL;
        }
        s += p;
      }
      if (std::fabs(s - 1.0) > 1e-6) {
        err = "CPT row of variable " + std::to_string(v) + " does not sum to 1";
        return JT_EINVAL;
      }
    }
    off += (int64_t)rows * card[v];
  }
  return JT_OK;
}

// ---------------------------------------------------------------------------
// triangulation and clique tree
// ---------------------------------------------------------------------------

// Min-fill elimination (fill = number of missing edges among the current
// neighbours; ties to the lowest variable id).  Returns the maximal
// elimination cliques in order of creation.
std::vector<Bits> eliminate_min_fill(int n, std::vector<Bits> adj) {
  const int W = (n + 63) / 64;
  Bits alive(W, 0);
  for (int v = 0; v < n; ++v) setbit(alive, v);
  std::vector<Bits> kept;
  std::vector<int64_t> fill(n, 0);
  std::vector<char> dirty(n, 1);
  auto compute_fill = [&](int v) {
    std::vector<int> nb = members(adj[v], n);
    int64_t present = 0;  // ordered pairs (a, b) of adjacent neighbours
    for (int a : nb) present += popcount_and(adj[a], adj[v]);
    int64_t d = (int64_t)nb.size();
    return d * (d - 1) / 2 - present / 2;
  };
  for (int step = 0; step < n; ++step) {
    int best = -1;
    for (int v = 0; v < n; ++v) {
      if (!bit(alive, v)) continue;
      if (dirty[v]) { fill[v] = compute_fill(v); dirty[v] = 0; }
      if (best < 0 || fill[v] < fill[best]) best = v;
    }
    const int v = best;
    std::vector<int> nb = members(adj[v], n);
    Bits clique = adj[v];
    setbit(clique, v);
    // connect the neighbours pairwise, then drop v
    for (int a : nb) {
      for (int b : nb)
        if (a != b) setbit(adj[a], b);
      clearbit(adj[a], v);
    }
    clearbit(alive, v);
    adj[v].assign(W, 0);
    // fill scores change only within distance two of v
    for (int a : nb) {
      dirty[a] = 1;
      for (int b = 0; b < n; ++b)
        if (bit(adj[a], b)) dirty[b] = 1;
    }
    bool maximal = true;
    for (const Bits &k : kept)
      if (subset_of(clique, k)) { maximal = false; break; }
    if (maximal) kept.push_back(clique);
  }
  return kept;
}

struct Tree {
  std::vector<std::vector<int>> nbr;
};

// Kruskal maximum-weight spanning tree over all clique pairs, weight = the
// number of shared variables (zero allowed: components join by empty
// separators); ties by (i, j).
Tree spanning_tree(const std::vector<Bits> &cl) {
  const int m = (int)cl.size();
  std::vector<std::tuple<int, int, int>> edges;  // (-w, i, j)
  edges.reserve((size_t)m * (m - 1) / 2);
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) edges.emplace_back(-popcount_and(cl[i], cl[j]), i, j);
  std::sort(edges.begin(), edges.end());
  std::vector<int> uf(m);
  std::iota(uf.begin(), uf.end(), 0);
  auto find = [&](int a) {
    while (uf[a] != a) { uf[a] = uf[uf[a]]; a = uf[a]; }
    return a;
  };
  Tree t;
  t.nbr.resize(m);
  int joined = 0;
  for (auto &e : edges) {
    if (joined == m - 1) break;
    int i = std::get<1>(e), j = std::get<2>(e);
    int a = find(i), b = find(j);
    if (a == b) continue;
    uf[a] = b;
    t.nbr[i].push_back(j);
    t.nbr[j].push_back(i);
    ++joined;
  }
  for (auto &v : t.nbr) std::sort(v.begin(), v.end());
  return t;
}

std::vector<int> bfs_dist(const Tree &t, int s) {
  std::vector<int> d(t.nbr.size(), -1);
  std::queue<int> q;
  q.push(s);
  d[s] = 0;
  while (!q.empty()) {
    int a = q.front();
    q.pop();
    for (int b : t.nbr[a])
      if (d[b] < 0) { d[b] = d[a] + 1; q.push(b); }
  }
  return d;
}

// ---------------------------------------------------------------------------
// layout helpers
// ---------------------------------------------------------------------------

// Table of weights over an ordered variable list (last fastest): for every
// entry of the mixed-radix space of `vars`, sum_i digit_i * weight[i].
void linear_table(const std::vector<int> &cards, const std::vector<int64_t> &weight,
                  std::vector<int32_t> &out) {
  int64_t size = 1;
  for (int c : cards) size *= c;
  out.assign(size, 0);
  const int k = (int)cards.size();
  std::vector<int> dig(k, 0);
  int64_t acc = 0;
  for (int64_t e = 0; e < size; ++e) {
    out[e] = (int32_t)acc;
    for (int i = k - 1; i >= 0; --i) {
      ++dig[i];
      acc += weight[i];
      if (dig[i] < cards[i]) break;
      acc -= weight[i] * cards[i];
      dig[i] = 0;
    }
  }
}

int64_t append_pool(std::vector<int32_t> &pool, const std::vector<int32_t> &t) {
  int64_t off = (int64_t)pool.size();
  pool.insert(pool.end(), t.begin(), t.end());
  return off;
}

}  // namespace

// Size bucket of a table of `rows` entries: floor(log2(rows)).
int size_bucket(int64_t rows) {
  int b = 0;
  while (b + 1 < JT_SIZE_BUCKETS && (rows >> (b + 1)) > 0) ++b;
  return b;
}

namespace {

bool all_zero(const std::vector<int64_t> &w) {
  for (auto x : w)
    if (x) return false;
  return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// work lists: per-layer warp work items of both passes, the dataflow
// schedule's flow layers and producer counts.  Depends only on the tree,
// the tasks and the work-shape options, so a compiled plan can be given a
// new work shape (jt_autotune's per-bucket tuning) without recompiling.
// ---------------------------------------------------------------------------
jt_status emit_work(Plan &P, const jt_compile_opts &opts, std::string &err) {
  const int m = (int)P.cl.size();
  // distribute tasks of each clique, in creation order
  std::vector<std::vector<int>> tasks_of(m);
  for (int t = 0; t < (int)P.dtask.size(); ++t) tasks_of[P.dtask[t].clique].push_back(t);
  const int NW = 8;  // warps per block
  // Rows per warp item: fixed by the option (rows per block / warps), else
  // chosen per layer so that a layer has about items_per_tile (default 192)
  // warp items per case tile, between a minimum (32 rows, one index batch,
  // for collect; 16 for distribute, whose rows carry less work) and 512: a
  // small layer is latency-bound and finishes sooner in short items, a big
  // one amortises each item's set-up over long ones.
  P.rows_per_cta = opts.rows_per_cta > 0 ? opts.rows_per_cta : 0;
  auto layer_rows = [&](int64_t total, bool distribute) -> int64_t {
    if (opts.rows_per_cta > 0) return std::max<int64_t>(1, opts.rows_per_cta / NW);
    int64_t items = opts.items_per_tile > 0 ? opts.items_per_tile : 192;
    if (distribute && opts.items_per_tile_distribute > 0) items = opts.items_per_tile_distribute;
    int64_t r = distribute ? 16 : 32;
    while (r < 512 && r * 2 * items <= total) r *= 2;
    return r;
  };
  P.citems.clear();
  P.ditems.clear();
  P.n_groups = 0;
  P.n_partials = 0;
  // one item per warp: whole segments when a segment fits the warp's rows,
  // else the segment is split into pieces combined in piece order
  auto emit = [&](std::vector<DItem> &out, int task, int64_t nseg, int64_t rows, int64_t ROWS) {
    if (rows <= ROWS) {
      int64_t per = std::max<int64_t>(1, ROWS / rows);
      for (int64_t t0 = 0; t0 < nseg; t0 += per) {
        DItem it{};
        it.t0 = t0;
        it.nt = std::min(per, nseg - t0);
        it.u0 = 0;
        it.nu = rows;
        it.task = task;
        it.split = 0;
        it.npieces = 1;
        it.piece = 0;
        it.group = -1;
        it.partial = -1;
        out.push_back(it);
      }
    } else {
      int64_t np = (rows + ROWS - 1) / ROWS;
      int64_t per = (rows + np - 1) / np;
      np = (rows + per - 1) / per;
      for (int64_t s = 0; s < nseg; ++s) {
        int32_t group = -1, first = -1;
        if (np > 1) {
          group = (int32_t)P.n_groups++;
          first = (int32_t)P.n_partials;
          P.n_partials += np;
        }
        for (int64_t p = 0; p < np; ++p) {
          DItem it{};
          it.t0 = s;
          it.nt = 1;
          it.u0 = p * per;
          it.nu = std::min(per, rows - p * per);
          it.task = task;
          it.split = 1;
          it.npieces = (int32_t)np;
          it.piece = (int32_t)p;
          it.group = group;
          it.partial = np > 1 ? first + (int32_t)p : -1;
          out.push_back(it);
        }
      }
    }
  };
  // Per size bucket (bucket b: 2^b <= rows < 2^(b+1)) the caller may fix
  // the rows of a work item; jt_autotune times these per bucket.  A value
  // is rounded down to a power of two in [16, 4096].
  auto bucket_rows = [&](const int32_t *table, int64_t rows, int64_t layer_value) -> int64_t {
    if (opts.rows_per_cta > 0) return layer_value;
    const int b = size_bucket(rows);
    if (table[b] <= 0) return layer_value;
    int64_t r = 16;
    while (r < 4096 && r * 2 <= table[b]) r *= 2;
    return r;
  };
  P.c_bucket_rows.fill(0);
  P.d_bucket_rows.fill(0);
  P.c_bucket_entries.fill(0);
  P.d_bucket_entries.fill(0);
  // A fused task's items hold whole primary targets inside one F-block, or
  // whole F-blocks; an F-block larger than an item, or whose secondary
  // targets would sum more than kFusedTerms rows, is cut into pieces that
  // write their secondary sums as partials, which the last piece to finish
  // adds in piece order.
  auto emit_fused = [&](int task, int64_t ROWS) {
    const DTask &T = P.dtask[task];
    const int64_t a = T.sec_a, b = T.sec_b, U = T.U, nF = T.T / a, Q = U / b;
    const int64_t R2 = ROWS;
    int64_t tp = std::max<int64_t>(1, std::min<int64_t>(R2 / U, kFusedTerms / Q));
    if (tp >= a) {
      const int64_t per = std::max<int64_t>(1, R2 / (a * U));
      for (int64_t f0 = 0; f0 < nF; f0 += per) {
        DItem it{};
        it.t0 = f0 * a;
        it.nt = std::min(per, nF - f0) * a;
        it.u0 = 0;
        it.nu = U;
        it.task = task;
        it.split = 0;
        it.npieces = 1;
        it.group = -1;
        it.partial = -1;
        it.fused = 1;
        P.ditems.push_back(it);
      }
      return;
    }
    int64_t np = (a + tp - 1) / tp;
    tp = (a + np - 1) / np;
    np = (a + tp - 1) / tp;
    for (int64_t f = 0; f < nF; ++f) {
      const int32_t group = (int32_t)P.n_groups++;
      const int32_t first = (int32_t)P.n_partials;
      P.n_partials += np * b;
      for (int64_t p = 0; p < np; ++p) {
        DItem it{};
        it.t0 = f * a + p * tp;
        it.nt = std::min(tp, a - p * tp);
        it.u0 = 0;
        it.nu = U;
        it.task = task;
        it.split = 0;
        it.npieces = (int32_t)np;
        it.piece = (int32_t)p;
        it.group = group;
        it.partial = first + (int32_t)(p * b);
        it.fused = 1;
        P.ditems.push_back(it);
      }
    }
  };
  P.levels.assign(P.height + 1, Level{});
  for (int L = 0; L <= P.height; ++L) {
    Level &lv = P.levels[L];
    lv.c_item_begin = (int64_t)P.citems.size();
    int64_t crows = 0, drows = 0;
    for (int c = 0; c < m; ++c) {
      if (P.cl[c].depth != L) continue;
      crows += P.cl[c].size;
      for (int t : tasks_of[c]) drows += P.dtask[t].T * P.dtask[t].U;
    }
    const int64_t cR = layer_rows(crows, false), dR = layer_rows(drows, true);
    for (int c = 0; c < m; ++c) {
      if (P.cl[c].depth != L) continue;
      const int64_t r = bucket_rows(opts.collect_rows_by_bucket, P.cl[c].size, cR);
      const int b = size_bucket(P.cl[c].size);
      P.c_bucket_rows[b] = std::max<int32_t>(P.c_bucket_rows[b], (int32_t)r);
      P.c_bucket_entries[b] += P.cl[c].size;
      emit(P.citems, c, P.cl[c].nsep, P.cl[c].R, r);
      lv.c_max_maps = std::max(lv.c_max_maps, P.dcl[c].sev_end - P.dcl[c].map_begin);
    }
    lv.c_item_end = (int64_t)P.citems.size();
    lv.d_item_begin = (int64_t)P.ditems.size();
    for (int c = 0; c < m; ++c) {
      if (P.cl[c].depth != L) continue;
      // a pair is fused where its items are long enough for the partial
      // sums of F-block pieces to cost little; elsewhere both tasks get
      // plain items
      for (int t : tasks_of[c]) {
        DTask &T = P.dtask[t];
        if (T.sec_b > 0) {
          const int64_t r = bucket_rows(opts.distribute_rows_by_bucket, T.T * T.U, dR);
          P.dtask[T.sec_task].absorbed = r >= kFusedMinRows ? 1 : 0;
        }
      }
      for (int t : tasks_of[c]) {
        if (P.dtask[t].absorbed) continue;  // computed by its fused partner's items
        const int64_t rows = P.dtask[t].T * P.dtask[t].U;
        const int64_t r = bucket_rows(opts.distribute_rows_by_bucket, rows, dR);
        const int b = size_bucket(rows);
        P.d_bucket_rows[b] = std::max<int32_t>(P.d_bucket_rows[b], (int32_t)r);
        P.d_bucket_entries[b] += rows;
        if (P.dtask[t].sec_b > 0 && P.dtask[P.dtask[t].sec_task].absorbed) emit_fused(t, r);
        else emit(P.ditems, t, P.dtask[t].T, P.dtask[t].U, r);
      }
    }
    lv.d_item_end = (int64_t)P.ditems.size();
  }
  // dataflow schedule: flow layers (collect deepest first, distribute from
  // the root) and each clique's producers on its tile
  P.c_flow_pref.assign(1, 0);
  P.d_flow_pref.assign(1, 0);
  P.c_flow_begin.clear();
  P.d_flow_begin.clear();
  for (int k = 0; k <= P.height; ++k) {
    const Level &lc = P.levels[P.height - k];
    P.c_flow_begin.push_back(lc.c_item_begin);
    P.c_flow_pref.push_back(P.c_flow_pref.back() + (lc.c_item_end - lc.c_item_begin));
    const Level &ld = P.levels[k];
    P.d_flow_begin.push_back(ld.d_item_begin);
    P.d_flow_pref.push_back(P.d_flow_pref.back() + (ld.d_item_end - ld.d_item_begin));
  }
  P.c_need.assign(m, 0);
  P.d_need.assign(m, 0);
  P.c_notify.assign(m, -1);
  for (const DItem &it : P.citems) {
    const HostClique &K = P.cl[it.task];
    if (K.parent >= 0 && K.n_up > 0) {
      P.c_notify[it.task] = K.parent;
      ++P.c_need[K.parent];
    }
  }
  for (const DItem &it : P.ditems) {
    const DTask &T = P.dtask[it.task];
    if (T.kind == TASK_CHILD) ++P.d_need[T.dst];
    if (it.fused && T.sec_kind == TASK_CHILD) ++P.d_need[T.sec_dst];
  }
  if (opts.stall_clique > 0) {
    if (opts.stall_clique > m) {
      err = "stall_clique out of range";
      return JT_EINVAL;
    }
    ++P.c_need[opts.stall_clique - 1];  // a producer that never comes
  }

  return JT_OK;
}

// ---------------------------------------------------------------------------
// build_plan
// ---------------------------------------------------------------------------
jt_status build_plan(int32_t n, const int32_t *card, const int32_t *pptr, const int32_t *par,
                     const double *cpt, const jt_compile_opts &opts, Plan &P, std::string &err) {
  jt_status st = validate(n, card, pptr, par, cpt, err);
  if (st != JT_OK) return st;
  P.opts = opts;
  P.n = n;
  P.card.assign(card, card + n);
  P.pptr.assign(pptr, pptr + n + 1);
  P.par.assign(par, par + pptr[n]);
  P.cpt_off.assign(n + 1, 0);
  for (int v = 0; v < n; ++v) {
    int64_t rows = 1;
    for (int k = pptr[v]; k < pptr[v + 1]; ++k) rows *= card[par[k]];
    P.cpt_off[v + 1] = P.cpt_off[v] + rows * card[v];
  }
  P.cpt.assign(cpt, cpt + P.cpt_off[n]);
  P.post_off.assign(n, 0);
  P.sum_card = 0;
  for (int v = 0; v < n; ++v) { P.post_off[v] = P.sum_card; P.sum_card += card[v]; }
  // rows of evidence and posteriors (build_plan_pruned widens them to the
  // full network after building a pruned plan)
  P.io_n = n;
  P.io_sum_card = P.sum_card;
  P.n_pruned = 0;
  P.io_var.clear();
  P.io_dropped.clear();
  P.io_post_col.clear();
  P.io_nan_cols.clear();
  // observed set of a specialised plan
  P.slice_var.assign(n, 0);
  P.n_sliced = 0;
  if (opts.n_observed_set < 0 || (opts.n_observed_set > 0 && opts.observed_set == nullptr)) {
    err = "bad observed set";
    return JT_EINVAL;
  }
  for (int i = 0; i < opts.n_observed_set; ++i) {
    const int v = opts.observed_set[i];
    if (v < 0 || v >= n || P.slice_var[v]) {
      err = "observed set: variable out of range or listed twice";
      return JT_EINVAL;
    }
    P.slice_var[v] = 1;
    ++P.n_sliced;
  }
  P.opts.observed_set = nullptr;  // the caller's array is read during compilation only
  auto sliced = [&](int v) { return P.slice_var[v] != 0; };

  // moral graph
  const int W = (n + 63) / 64;
  std::vector<Bits> adj(n, Bits(W, 0));
  for (int v = 0; v < n; ++v) {
    for (int k = pptr[v]; k < pptr[v + 1]; ++k) {
      int p = par[k];
      setbit(adj[v], p);
      setbit(adj[p], v);
      for (int q = k + 1; q < pptr[v + 1]; ++q) {
        setbit(adj[p], par[q]);
        setbit(adj[par[q]], p);
      }
    }
  }
  std::vector<Bits> cbits = eliminate_min_fill(n, adj);
  const int m = (int)cbits.size();
  const int64_t max_entries = opts.max_clique_entries > 0 ? opts.max_clique_entries : 2147483647LL;
  P.cl.assign(m, HostClique());
  std::vector<double> csize(m, 1.0);
  for (int c = 0; c < m; ++c) {
    for (int v : members(cbits[c], n)) csize[c] *= card[v];
    if (csize[c] > (double)max_entries) {
      err = "clique " + std::to_string(c) + " has " + std::to_string(csize[c]) + " entries";
      return JT_ETOOBIG;
    }
  }
  Tree tree = spanning_tree(cbits);

  // root
  int root = 0;
  if (opts.root_rule == JT_ROOT_LARGEST) {
    for (int c = 1; c < m; ++c)
      if (csize[c] > csize[root]) root = c;
  } else {
    int best = -1;
    for (int s = 0; s < m; ++s) {
      std::vector<int> d = bfs_dist(tree, s);
      int ecc = *std::max_element(d.begin(), d.end());
      if (best < 0 || ecc < best || (ecc == best && csize[s] > csize[root])) {
        best = ecc;
        root = s;
      }
    }
  }
  P.root = root;

  // orient: BFS from the root, neighbours ascending
  std::vector<int> parent(m, -2), depth(m, 0);
  P.bfs.clear();
  P.bfs.push_back(root);
  parent[root] = -1;
  for (size_t h = 0; h < P.bfs.size(); ++h) {
    int a = P.bfs[h];
    for (int b : tree.nbr[a])
      if (parent[b] == -2) {
        parent[b] = a;
        depth[b] = depth[a] + 1;
        P.bfs.push_back(b);
      }
  }
  P.height = 0;
  for (int c = 0; c < m; ++c) P.height = std::max(P.height, depth[c]);

  // variable layout: upward separator first (in the parent's order), then
  // the remaining variables in ascending id
  for (int c : P.bfs) {
    HostClique &C = P.cl[c];
    C.parent = parent[c];
    C.depth = depth[c];
    C.vars.clear();
    if (C.parent >= 0)
      for (int v : P.cl[C.parent].vars)
        if (bit(cbits[c], v)) C.vars.push_back(v);
    C.n_up = (int)C.vars.size();
    for (int v = 0; v < n; ++v)
      if (bit(cbits[c], v) && std::find(C.vars.begin(), C.vars.begin() + C.n_up, v) == C.vars.begin() + C.n_up)
        C.vars.push_back(v);
    const int k = (int)C.vars.size();
    C.card.resize(k);
    C.stride.resize(k);
    int64_t s = 1;
    for (int i = k - 1; i >= 0; --i) {
      C.card[i] = card[C.vars[i]];
      C.stride[i] = s;
      s *= C.card[i];
    }
    C.size = s;
    C.nsep = 1;
    for (int i = 0; i < C.n_up; ++i) C.nsep *= C.card[i];
    C.R = C.size / C.nsep;
    if (C.parent >= 0) P.cl[C.parent].children.push_back(c);
  }
  for (auto &C : P.cl) std::sort(C.children.begin(), C.children.end());
  // Full layout (base tables) and, in a specialised plan, the sliced layout
  // of every other table: the observed set's variables left out, the order
  // kept (so each child's upward separator stays a prefix in its parent's
  // order).
  for (auto &C : P.cl) {
    C.fvars = C.vars;
    C.fstride = C.stride;
    C.fsize = C.size;
    if (P.n_sliced == 0) continue;
    std::vector<int> v2;
    int up2 = 0;
    for (int i = 0; i < (int)C.vars.size(); ++i) {
      if (sliced(C.vars[i])) continue;
      v2.push_back(C.vars[i]);
      if (i < C.n_up) ++up2;
    }
    C.vars = v2;
    C.n_up = up2;
    const int k = (int)C.vars.size();
    C.card.assign(k, 0);
    C.stride.assign(k, 0);
    int64_t s2 = 1;
    for (int i = k - 1; i >= 0; --i) {
      C.card[i] = card[C.vars[i]];
      C.stride[i] = s2;
      s2 *= C.card[i];
    }
    C.size = s2;
    C.nsep = 1;
    for (int i = 0; i < C.n_up; ++i) C.nsep *= C.card[i];
    C.R = C.size / C.nsep;
  }

  // CPT assignment (smallest clique containing the family, lowest id on
  // ties); posterior owner (smallest clique containing the variable)
  P.assign.assign(n, -1);
  P.post_src.assign(n, -1);
  for (int v = 0; v < n; ++v) {
    Bits fam(W, 0);
    setbit(fam, v);
    for (int k = pptr[v]; k < pptr[v + 1]; ++k) setbit(fam, par[k]);
    for (int c = 0; c < m; ++c) {
      if (bit(cbits[c], v) && (P.post_src[v] < 0 || csize[c] < csize[P.post_src[v]])) P.post_src[v] = c;
      if (subset_of(fam, cbits[c]) && (P.assign[v] < 0 || csize[c] < csize[P.assign[v]])) P.assign[v] = c;
    }
    if (P.assign[v] < 0) { err = "internal: no clique covers a family"; return JT_EINVAL; }
    P.cl[P.assign[v]].homed.push_back(v);
  }
  // Posterior source of each variable in the batched path: the smallest
  // table holding it -- a separator (its calibrated marginal is phi* x rho)
  // when one is no larger than the smallest clique, else that clique.
  for (int v = 0; v < n; ++v) {
    if (sliced(v)) continue;  // always observed: a point mass, no table needed
    int best_sep = -1;
    double best_sep_size = 0;
    for (int c = 0; c < m; ++c) {
      const HostClique &C = P.cl[c];
      if (C.parent < 0 || C.n_up == 0) continue;
      if (std::find(C.vars.begin(), C.vars.begin() + C.n_up, v) == C.vars.begin() + C.n_up) continue;
      double sz = 1;
      for (int i = 0; i < C.n_up; ++i) sz *= C.card[i];
      if (best_sep < 0 || sz < best_sep_size) { best_sep = c; best_sep_size = sz; }
    }
    if (best_sep >= 0 && best_sep_size <= (double)P.cl[P.post_src[v]].size)
      P.cl[best_sep].owned_sep.push_back(v);
    else
      P.cl[P.post_src[v]].owned.push_back(v);
  }

  // Evidence placement of the batched path.  Hugin enters an observed
  // variable's 0/1 indicator into one table holding the variable; entering
  // it into a child's upward message before the parent absorbs it gives the
  // parent the same product, and the later division by that message stays
  // exact (the indicator is 0 or 1, the calibrated separator is 0 wherever
  // it is 0, and 0/0 := 0).  Each variable goes to the smallest such table:
  // an upward separator (one indicator per message entry, applied when the
  // entry is written) or a clique (one indicator per clique entry), ties to
  // the separator and then to the lowest clique id.
  for (int v = 0; v < n; ++v) {
    if (sliced(v)) continue;  // sliced out: each case reads its own slice
    int best = -1;
    bool best_sep = false;
    int64_t best_cost = 0;
    for (int c = 0; c < m; ++c) {
      const HostClique &C = P.cl[c];
      if (!bit(cbits[c], v)) continue;
      const bool in_up = C.parent >= 0 && C.n_up > 0 &&
                         std::find(C.vars.begin(), C.vars.begin() + C.n_up, v) != C.vars.begin() + C.n_up;
      if (in_up && (best < 0 || C.nsep < best_cost || (C.nsep == best_cost && !best_sep))) {
        best = c;
        best_sep = true;
        best_cost = C.nsep;
      }
      if (best < 0 || C.size < best_cost) {
        best = c;
        best_sep = false;
        best_cost = C.size;
      }
    }
    (best_sep ? P.cl[best].ev_sep : P.cl[best].ev_clique).push_back(v);
  }

  P.sum_cl = P.max_cl = P.sum_sep = P.sum_base = 0;
  for (int c = 0; c < m; ++c) {
    P.sum_cl += P.cl[c].size;
    P.sum_base += P.cl[c].fsize;
    P.max_cl = std::max(P.max_cl, P.cl[c].size);
    if (c != root) P.sum_sep += P.cl[c].nsep;
  }

  // base tables: product of the assigned CPTs, in each clique's full layout
  P.base64.assign(P.sum_base, 1.0);
  P.base32.assign(P.sum_base, 1.0f);
  P.p_base_off.assign(m, 0);
  std::vector<int64_t> psi_row(m, 0);
  {
    int64_t off = 0, prow = 0;
    for (int c = 0; c < m; ++c) {
      P.p_base_off[c] = off;
      off += P.cl[c].fsize;
      psi_row[c] = prow;
      prow += P.cl[c].size;
    }
  }
  for (int v = 0; v < n; ++v) {
    const HostClique &C = P.cl[P.assign[v]];
    // weight of each clique variable inside v's CPT (parents listed order, child fastest)
    std::vector<int64_t> w(C.fvars.size(), 0);
    int64_t s = 1;
    auto pos_of = [&](int x) { return (int)(std::find(C.fvars.begin(), C.fvars.end(), x) - C.fvars.begin()); };
    w[pos_of(v)] = s;
    s *= card[v];
    for (int k = pptr[v + 1] - 1; k >= pptr[v]; --k) {
      w[pos_of(par[k])] = s;
      s *= card[par[k]];
    }
    std::vector<int> fcard;
    for (int x : C.fvars) fcard.push_back(card[x]);
    std::vector<int32_t> idx;
    linear_table(fcard, w, idx);
    double *b = P.base64.data() + P.p_base_off[P.assign[v]];
    const double *t = P.cpt.data() + P.cpt_off[v];
    for (int64_t e = 0; e < C.fsize; ++e) b[e] *= t[idx[e]];
  }
  // FP32 copy, each clique scaled by a power of two so that its maximum is
  // in [1, 2); the exponents are a per-plan constant added to log P(e)
  std::vector<int> base_exp(m, 0);
  for (int c = 0; c < m; ++c) {
    const double *b = P.base64.data() + P.p_base_off[c];
    double mx = 0;
    for (int64_t e = 0; e < P.cl[c].fsize; ++e) mx = std::max(mx, b[e]);
    int ex = 0;
    if (mx > 0) { std::frexp(mx, &ex); ex -= 1; }
    base_exp[c] = ex;
    for (int64_t e = 0; e < P.cl[c].fsize; ++e)
      P.base32[P.p_base_off[c] + e] = (float)std::ldexp(b[e], -ex);
  }

  // ---------------------------------------------------------------------
  // device descriptors
  // ---------------------------------------------------------------------
  P.ipool.clear();
  P.dcl.assign(m, DClique{});
  P.dmap.clear();
  P.dtask.clear();
  int64_t zero_len = 1;
  for (int c = 0; c < m; ++c) zero_len = std::max({zero_len, P.cl[c].nsep, P.cl[c].R, P.cl[c].size});
  // one shared all-zero table serves every map part that no variable feeds
  const int64_t zero_off = 0;
  P.ipool.assign(zero_len, 0);

  std::vector<int64_t> sep_row(m, 0);
  {
    int64_t r = 0;
    for (int c = 0; c < m; ++c) { sep_row[c] = r; r += P.cl[c].nsep; }
    P.sep_rows = r;
  }

  auto table_or_zero = [&](const std::vector<int> &cards, const std::vector<int64_t> &w) -> int64_t {
    if (all_zero(w)) return zero_off;
    std::vector<int32_t> t;
    linear_table(cards, w, t);
    return append_pool(P.ipool, t);
  };

  for (int c = 0; c < m; ++c) {
    HostClique &C = P.cl[c];
    DClique &D = P.dcl[c];
    D.psi_row = psi_row[c];
    D.nsep = C.nsep;
    D.R = C.R;
    D.base_off = P.p_base_off[c];
    D.sep_row = sep_row[c];
    D.parent = C.parent;
    // Empty separators (disconnected parts of the network) split the tree
    // into independent component trees: such a child sends no message to
    // its parent, its own total enters log P(e) directly.
    D.is_root = (c == root) || (C.n_up == 0);
    D.map_begin = (int32_t)P.dmap.size();
    std::vector<int> up_card(C.card.begin(), C.card.begin() + C.n_up);
    std::vector<int> res_card(C.card.begin() + C.n_up, C.card.end());
    // child messages
    for (int ch : C.children) {
      const HostClique &K = P.cl[ch];
      if (K.n_up == 0) continue;
      // stride of each separator variable in the child's message (K's up block)
      std::vector<int64_t> wa(C.n_up, 0), wb(C.vars.size() - C.n_up, 0);
      for (int i = 0; i < K.n_up; ++i) {
        int v = K.vars[i];
        int64_t sstride = K.stride[i] / K.R;
        int pos = (int)(std::find(C.vars.begin(), C.vars.end(), v) - C.vars.begin());
        if (pos < C.n_up) wa[pos] = sstride; else wb[pos - C.n_up] = sstride;
      }
      DMap mp{};
      mp.kind = MAP_CHILD;
      mp.src = ch;
      mp.src_row = sep_row[ch];
      mp.A_off = table_or_zero(up_card, wa);
      mp.B_off = table_or_zero(res_card, wb);
      P.dmap.push_back(mp);
    }
    // evidence digits of the variables whose indicator this clique gathers
    for (int v : C.ev_clique) {
      std::vector<int64_t> wa(C.n_up, 0), wb(C.vars.size() - C.n_up, 0);
      int pos = (int)(std::find(C.vars.begin(), C.vars.end(), v) - C.vars.begin());
      if (pos < C.n_up) wa[pos] = 1; else wb[pos - C.n_up] = 1;
      DMap mp{};
      mp.kind = MAP_EVIDENCE;
      mp.src = v;
      mp.src_row = P.post_off[v];  // first row of v's indicator table
      mp.A_off = table_or_zero(up_card, wa);
      mp.B_off = table_or_zero(res_card, wb);
      P.dmap.push_back(mp);
    }
    D.map_end = (int32_t)P.dmap.size();
    // evidence applied to the upward message: state of v per message entry
    D.sev_begin = D.map_end;
    for (int v : C.ev_sep) {
      std::vector<int64_t> wa(C.n_up, 0);
      const int pos = (int)(std::find(C.vars.begin(), C.vars.begin() + C.n_up, v) - C.vars.begin());
      wa[pos] = 1;
      DMap mp{};
      mp.kind = MAP_SEP_EVIDENCE;
      mp.src = v;
      mp.src_row = P.post_off[v];
      mp.A_off = table_or_zero(up_card, wa);
      mp.B_off = 0;
      P.dmap.push_back(mp);
    }
    D.sev_end = (int32_t)P.dmap.size();
    // sliced plan: the clique's observed-set variables (stride in the full
    // base table) and the base entry of each table entry
    D.slice_begin = D.sev_end;
    D.bmap_A = D.bmap_B = zero_off;
    if (P.n_sliced > 0) {
      for (size_t i = 0; i < C.fvars.size(); ++i) {
        if (!sliced(C.fvars[i])) continue;
        DMap mp{};
        mp.kind = MAP_SLICE;
        mp.src = C.fvars[i];
        mp.A_off = C.fstride[i];
        P.dmap.push_back(mp);
      }
      auto fstride_of = [&](int v) {
        return C.fstride[std::find(C.fvars.begin(), C.fvars.end(), v) - C.fvars.begin()];
      };
      std::vector<int64_t> wa(C.n_up, 0), wb(C.vars.size() - C.n_up, 0);
      for (int i = 0; i < (int)C.vars.size(); ++i)
        (i < C.n_up ? wa[i] : wb[i - C.n_up]) = fstride_of(C.vars[i]);
      D.bmap_A = table_or_zero(up_card, wa);
      D.bmap_B = table_or_zero(res_card, wb);
    }
    D.slice_end = (int32_t)P.dmap.size();
  }
  P.cpt_per_thread = opts.cases_per_thread > 0 ? opts.cases_per_thread : 4;
  if (P.cpt_per_thread != 1 && P.cpt_per_thread != 2 && P.cpt_per_thread != 4 && P.cpt_per_thread != 8) {
    err = "cases_per_thread must be 1, 2, 4 or 8";
    return JT_EINVAL;
  }
  if (opts.schedule != JT_SCHEDULE_DATAFLOW && opts.schedule != JT_SCHEDULE_LAYERS) {
    err = "schedule must be JT_SCHEDULE_DATAFLOW or JT_SCHEDULE_LAYERS";
    return JT_EINVAL;
  }
  if (opts.rescale != 0 && opts.rescale != 1) {
    err = "rescale must be 0 or 1";
    return JT_EINVAL;
  }
  P.tile = 32 * P.cpt_per_thread;
  if (opts.recompute_psi != 0 && opts.recompute_psi != 1) {
    err = "recompute_psi must be 0 or 1";
    return JT_EINVAL;
  }
  // recomputed clique tables: standard plans (a sliced plan's base-table
  // gather stays in the collect pass)
  P.recompute = (opts.recompute_psi && P.n_sliced == 0) ? 1 : 0;
  // distribute tasks: children first (ascending), then owned posteriors
  std::vector<std::vector<int>> tasks_of(m);
  std::vector<std::vector<int>> task_vars;  // target variables of each task
  for (int c = 0; c < m; ++c) {
    const HostClique &C = P.cl[c];
    auto make_task = [&](const std::vector<int> &target, int kind, int dst, int64_t dst_row, bool from_sep = false) {
      // target variables in the source table's layout order (the clique, or
      // its upward separator = the first n_up variables)
      const int nv = from_sep ? C.n_up : (int)C.vars.size();
      std::vector<int> tpos, upos;
      for (int i = 0; i < nv; ++i) {
        bool in = std::find(target.begin(), target.end(), C.vars[i]) != target.end();
        (in ? tpos : upos).push_back(i);
      }
      std::vector<int> tcard, ucard;
      std::vector<int64_t> wa, wsa, wb, wsb;
      // stride inside the source table / inside the upward separator
      auto xs = [&](int i) { return from_sep ? C.stride[i] / C.R : C.stride[i]; };
      for (int i : tpos) {
        tcard.push_back(C.card[i]);
        wa.push_back(xs(i));
        wsa.push_back(i < C.n_up ? C.stride[i] / C.R : 0);
      }
      for (int i : upos) {
        ucard.push_back(C.card[i]);
        wb.push_back(xs(i));
        wsb.push_back(i < C.n_up ? C.stride[i] / C.R : 0);
      }
      DTask t{};
      t.T = 1;
      for (int x : tcard) t.T *= x;
      t.U = 1;
      for (int x : ucard) t.U *= x;
      t.A_off = table_or_zero(tcard, wa);
      t.sA_off = table_or_zero(tcard, wsa);
      t.B_off = table_or_zero(ucard, wb);
      t.sB_off = table_or_zero(ucard, wsb);
      t.clique = c;
      t.kind = kind;
      t.dst = dst;
      t.dst_row = dst_row;
      t.src_sep = from_sep ? 1 : 0;
      t.op_off = -1;
      t.sec_task = -1;
      tasks_of[c].push_back((int)P.dtask.size());
      P.dtask.push_back(t);
      task_vars.push_back(target);
    };
    for (int ch : C.children) {
      const HostClique &K = P.cl[ch];
      if (K.n_up == 0) continue;
      std::vector<int> sv(K.vars.begin(), K.vars.begin() + K.n_up);
      make_task(sv, TASK_CHILD, ch, sep_row[ch]);
    }
    for (int v : C.owned) make_task(std::vector<int>{v}, TASK_POSTERIOR, v, P.post_off[v]);
    for (int v : C.owned_sep) make_task(std::vector<int>{v}, TASK_POSTERIOR, v, P.post_off[v], true);
  }

  // Fused pairs: two tasks reading the same clique table share one pass
  // over it (see DTask).  The secondary's per-F-block sums live in shared
  // memory, kFusedRowBytes per warp at most, so its targets per F-block
  // are bounded by that over the tile's row bytes.
  P.sec_rows = 0;
  if (opts.fuse_distribute && !P.recompute) {
    const int64_t bmax = kFusedRowBytes / (4 * (int64_t)P.tile);
    for (int c = 0; c < m; ++c) {
      const HostClique &C = P.cl[c];
      std::vector<int> cand;
      for (int t : tasks_of[c])
        if (!P.dtask[t].src_sep) cand.push_back(t);
      auto in = [](const std::vector<int> &vs, int v) { return std::find(vs.begin(), vs.end(), v) != vs.end(); };
      auto card_of = [&](const std::vector<int> &vs) {
        int64_t r = 1;
        for (int v : vs) r *= card[v];
        return r;
      };
      while (cand.size() >= 2) {
        // the pair whose secondary needs the fewest shared-memory rows
        int bi = -1, bj = -1;
        int64_t best_b = 0;
        for (int i : cand)
          for (int j : cand) {
            if (i == j) continue;
            const std::vector<int> &Ti = task_vars[i], &Tj = task_vars[j];
            std::vector<int> only_j;
            for (int v : Tj)
              if (!in(Ti, v)) only_j.push_back(v);
            const int64_t b = card_of(only_j);
            if (b > bmax || P.dtask[i].U > kFusedMaxRows) continue;
            if (bi < 0 || b < best_b) { bi = i; bj = j; best_b = b; }
          }
        if (bi < 0) break;
        const std::vector<int> &Ti = task_vars[bi], &Tj = task_vars[bj];
        // layout-ordered variable lists: F, T1 \ F, (T2 \ T1), the rest
        std::vector<int> fpos, tpos, kpos, rpos;
        for (int i = 0; i < (int)C.vars.size(); ++i) {
          const int v = C.vars[i];
          const bool a1 = in(Ti, v), a2 = in(Tj, v);
          (a1 && a2 ? fpos : a1 ? tpos : a2 ? kpos : rpos).push_back(i);
        }
        auto cards_at = [&](const std::vector<int> &pos) {
          std::vector<int> r;
          for (int i : pos) r.push_back(C.card[i]);
          return r;
        };
        // row-major stride of clique position i inside the enumeration of a
        // target's variables taken in layout order
        auto target_stride = [&](const std::vector<int> &tv, int i) -> int64_t {
          int64_t s2 = 1;
          for (int q = (int)C.vars.size() - 1; q >= 0; --q) {
            if (!in(tv, C.vars[q])) continue;
            if (q == i) return s2;
            s2 *= C.card[q];
          }
          return 0;
        };
        std::vector<int> tord = fpos;  // primary targets: F outermost
        tord.insert(tord.end(), tpos.begin(), tpos.end());
        std::vector<int> uord = kpos;  // rows: the secondary's own variables outermost
        uord.insert(uord.end(), rpos.begin(), rpos.end());
        std::vector<int64_t> wa, wsa, wop, wb, wsb, wku;
        for (int i : tord) {
          wa.push_back(C.stride[i]);
          wsa.push_back(i < C.n_up ? C.stride[i] / C.R : 0);
          wop.push_back(target_stride(Ti, i));
        }
        int64_t ks = 1;
        std::vector<int64_t> kstride(kpos.size());
        for (int q = (int)kpos.size() - 1; q >= 0; --q) { kstride[q] = ks; ks *= C.card[kpos[q]]; }
        for (size_t q = 0; q < uord.size(); ++q) {
          const int i = uord[q];
          wb.push_back(C.stride[i]);
          wsb.push_back(i < C.n_up ? C.stride[i] / C.R : 0);
          wku.push_back(q < kpos.size() ? kstride[q] : 0);
        }
        std::vector<int64_t> wosf, wosk;
        for (int i : fpos) wosf.push_back(target_stride(Tj, i));
        for (int i : kpos) wosk.push_back(target_stride(Tj, i));
        DTask &T = P.dtask[bi];
        const DTask &S = P.dtask[bj];
        T.fA_off = table_or_zero(cards_at(tord), wa);
        T.fsA_off = table_or_zero(cards_at(tord), wsa);
        T.op_off = table_or_zero(cards_at(tord), wop);
        T.fB_off = table_or_zero(cards_at(uord), wb);
        T.fsB_off = table_or_zero(cards_at(uord), wsb);
        T.ku_off = table_or_zero(cards_at(uord), wku);
        T.osf_off = table_or_zero(cards_at(fpos), wosf);
        T.osk_off = table_or_zero(cards_at(kpos), wosk);
        T.sec_a = (int32_t)card_of([&] { std::vector<int> r; for (int i : tpos) r.push_back(C.vars[i]); return r; }());
        T.sec_b = (int32_t)best_b;
        T.sec_kind = S.kind;
        T.sec_dst = S.dst;
        T.sec_dst_row = S.dst_row;
        T.sec_task = bj;
        P.dtask[bj].absorbed = 1;
        P.sec_rows = std::max<int>(P.sec_rows, (int)best_b);
        cand.erase(std::find(cand.begin(), cand.end(), bi));
        cand.erase(std::find(cand.begin(), cand.end(), bj));
      }
    }
  }

  st = emit_work(P, opts, err);
  if (st != JT_OK) return st;

  P.base_exp_sum = 0;
  for (int c = 0; c < m; ++c) P.base_exp_sum += base_exp[c];

  // variable groups of the posterior kernel (a block per tile and group)
  P.pgroup_ptr.assign(1, 0);
  {
    int cols = 0;
    for (int v = 0; v < n; ++v) {
      if (cols > 0 && cols + card[v] > 16) { P.pgroup_ptr.push_back(v); cols = 0; }
      cols += card[v];
    }
    P.pgroup_ptr.push_back(n);
  }

  // component trees: every variable belongs to exactly one (an empty
  // separator shares no variable), listed under the component's root
  {
    std::vector<int> comp_root(m, -1);
    for (int c : P.bfs) comp_root[c] = (c == root || P.cl[c].n_up == 0) ? c : comp_root[P.cl[c].parent];
    std::vector<std::vector<int32_t>> members_of(m);
    // every variable of the component's tables; an observed-set variable
    // (sliced out of the tables, but read through the base tables) is listed
    // in every component whose cliques hold it
    std::vector<std::vector<char>> seen_in(m);
    for (int c : P.bfs) {
      std::vector<char> &seen = seen_in[comp_root[c]];
      if (seen.empty()) seen.assign(n, 0);
      for (int v : P.cl[c].fvars)
        if (!seen[v]) { seen[v] = 1; members_of[comp_root[c]].push_back(v); }
    }
    P.comp_ptr.assign(m + 1, 0);
    P.comp_vars.clear();
    for (int c = 0; c < m; ++c) {
      P.comp_vars.insert(P.comp_vars.end(), members_of[c].begin(), members_of[c].end());
      P.comp_ptr[c + 1] = (int32_t)P.comp_vars.size();
    }
    std::vector<std::vector<int32_t>> cliques_of(m);
    for (int c = 0; c < m; ++c) {
      P.dcl[comp_root[c]].comp_base_exp += base_exp[c];
      if (comp_root[c] != c) cliques_of[comp_root[c]].push_back(c);
    }
    P.comp_cliques.clear();
    P.comp_roots.clear();
    for (int c = 0; c < m; ++c)
      if (comp_root[c] == c) P.comp_roots.push_back(c);
    for (int c = 0; c < m; ++c) {
      P.dcl[c].comp_begin = (int32_t)P.comp_cliques.size();
      P.comp_cliques.insert(P.comp_cliques.end(), cliques_of[c].begin(), cliques_of[c].end());
      P.dcl[c].comp_end = (int32_t)P.comp_cliques.size();
    }
    // component (index into comp_roots) of each comp_cliques entry
    P.comp_owner.assign(P.comp_cliques.size(), 0);
    for (size_t q = 0; q < P.comp_roots.size(); ++q) {
      const DClique &D = P.dcl[P.comp_roots[q]];
      for (int k = D.comp_begin; k < D.comp_end; ++k) P.comp_owner[k] = (int32_t)q;
    }
    // component of each comp_vars entry (only component roots list variables)
    P.comp_var_owner.assign(P.comp_vars.size(), 0);
    for (size_t q = 0; q < P.comp_roots.size(); ++q) {
      const int cl = P.comp_roots[q];
      for (int k = P.comp_ptr[cl]; k < P.comp_ptr[cl + 1]; ++k) P.comp_var_owner[k] = (int32_t)q;
    }
  }

  // ---------------------------------------------------------------------
  // plain FP64 path maps: (var, card, src stride, dst stride) quadruples
  // (the comparator runs unspecialised plans only)
  // ---------------------------------------------------------------------
  P.pmap.clear();
  P.ppool.clear();
  if (P.n_sliced > 0) return JT_OK;
  auto plain_map = [&](const HostClique &X, const std::vector<int> &dst_vars) -> int {
    // dst is row-major over dst_vars (last fastest)
    DPlainMap pm{};
    pm.size = X.size;
    pm.nv = (int32_t)X.vars.size();
    pm.var_off = (int64_t)P.ppool.size();
    for (int i = 0; i < (int)X.vars.size(); ++i) {
      int64_t ds = 0, s = 1;
      for (int j = (int)dst_vars.size() - 1; j >= 0; --j) {
        if (dst_vars[j] == X.vars[i]) ds = s;
        s *= card[dst_vars[j]];
      }
      P.ppool.push_back(X.vars[i]);
      P.ppool.push_back(X.card[i]);
      P.ppool.push_back(X.stride[i]);
      P.ppool.push_back(ds);
    }
    P.pmap.push_back(pm);
    return (int)P.pmap.size() - 1;
  };
  P.p_child_map.assign(m, -1);
  P.p_parent_map.assign(m, -1);
  P.p_init_map.assign(m, -1);
  P.p_post_map.assign(n, -1);
  P.p_sep_off.assign(m, 0);
  {
    int64_t off = 0;
    for (int c = 0; c < m; ++c) { P.p_sep_off[c] = off; off += P.cl[c].nsep; }
  }
  for (int c = 0; c < m; ++c) {
    const HostClique &C = P.cl[c];
    P.p_init_map[c] = plain_map(C, std::vector<int>{});
    if (c == root) continue;
    std::vector<int> sv(C.vars.begin(), C.vars.begin() + C.n_up);
    P.p_child_map[c] = plain_map(C, sv);
    P.p_parent_map[c] = plain_map(P.cl[C.parent], sv);
  }
  P.p_root_map.assign(1, plain_map(P.cl[root], std::vector<int>{}));
  for (int v = 0; v < n; ++v) P.p_post_map[v] = plain_map(P.cl[P.post_src[v]], std::vector<int>{v});
  return JT_OK;
}

// ---------------------------------------------------------------------------
// query-set pruning: the plan keeps the query set, the observed set and all
// their ancestors.  The rest is barren: no kept variable has a removed
// parent, so the removed variables sum out of the joint one CPT at a time
// (children first), each sum being exactly 1, and the joint of the kept
// variables is the product of their own CPTs (the marginalisation of
// Section 2 applied to whole variables).
// ---------------------------------------------------------------------------
jt_status build_plan_pruned(int32_t n, const int32_t *card, const int32_t *pptr, const int32_t *par,
                            const double *cpt, const jt_compile_opts &opts, Plan &P, std::string &err) {
  if (opts.n_query_set == 0) return build_plan(n, card, pptr, par, cpt, opts, P, err);
  if (opts.n_query_set < 0 || opts.query_set == nullptr) {
    err = "bad query set";
    return JT_EINVAL;
  }
  jt_status st = validate(n, card, pptr, par, cpt, err);
  if (st != JT_OK) return st;
  if (opts.n_observed_set < 0 || (opts.n_observed_set > 0 && opts.observed_set == nullptr)) {
    err = "bad observed set";
    return JT_EINVAL;
  }
  std::vector<char> keep(n, 0), listed(n, 0);
  std::vector<int> stack;
  for (int i = 0; i < opts.n_query_set; ++i) {
    const int v = opts.query_set[i];
    if (v < 0 || v >= n || listed[v]) {
      err = "query set: variable out of range or listed twice";
      return JT_EINVAL;
    }
    listed[v] = 1;
    stack.push_back(v);
  }
  for (int i = 0; i < opts.n_observed_set; ++i) {
    const int v = opts.observed_set[i];
    if (v < 0 || v >= n) {
      err = "observed set: variable out of range or listed twice";
      return JT_EINVAL;
    }
    stack.push_back(v);
  }
  while (!stack.empty()) {  // ancestral closure
    const int v = stack.back();
    stack.pop_back();
    if (keep[v]) continue;
    keep[v] = 1;
    for (int k = pptr[v]; k < pptr[v + 1]; ++k) stack.push_back(par[k]);
  }
  std::vector<int32_t> sub_of(n, -1), orig;
  for (int v = 0; v < n; ++v)
    if (keep[v]) {
      sub_of[v] = (int32_t)orig.size();
      orig.push_back(v);
    }
  jt_compile_opts so = opts;
  so.n_query_set = 0;
  so.query_set = nullptr;
  if ((int)orig.size() == n) return build_plan(n, card, pptr, par, cpt, so, P, err);  // nothing barren
  // the kept network, variables renumbered in their original order
  const int k = (int)orig.size();
  std::vector<int32_t> kcard(k), kpptr(k + 1, 0), kpar;
  std::vector<double> kcpt;
  std::vector<int64_t> off(n + 1, 0);
  for (int v = 0; v < n; ++v) {
    int64_t rows = 1;
    for (int q = pptr[v]; q < pptr[v + 1]; ++q) rows *= card[par[q]];
    off[v + 1] = off[v] + rows * card[v];
  }
  for (int i = 0; i < k; ++i) {
    const int v = orig[i];
    kcard[i] = card[v];
    for (int q = pptr[v]; q < pptr[v + 1]; ++q) kpar.push_back(sub_of[par[q]]);  // kept: ancestors are kept
    kpptr[i + 1] = (int32_t)kpar.size();
    kcpt.insert(kcpt.end(), cpt + off[v], cpt + off[v + 1]);
  }
  if (kpar.empty()) kpar.push_back(0);
  std::vector<int32_t> kobs;
  for (int i = 0; i < opts.n_observed_set; ++i) kobs.push_back(sub_of[opts.observed_set[i]]);
  so.observed_set = kobs.empty() ? nullptr : kobs.data();
  st = build_plan(k, kcard.data(), kpptr.data(), kpar.data(), kcpt.data(), so, P, err);
  if (st != JT_OK) return st;
  // rows of evidence and posteriors keep the full network's layout
  std::vector<int64_t> full_off(n, 0);
  int64_t sc = 0;
  for (int v = 0; v < n; ++v) { full_off[v] = sc; sc += card[v]; }
  P.io_n = n;
  P.io_sum_card = sc;
  P.n_pruned = n - k;
  P.io_var.assign(orig.begin(), orig.end());
  P.io_dropped.clear();
  P.io_nan_cols.clear();
  for (int v = 0; v < n; ++v)
    if (!keep[v]) {
      P.io_dropped.push_back(v);
      for (int j = 0; j < card[v]; ++j) P.io_nan_cols.push_back((int32_t)(full_off[v] + j));
    }
  P.io_post_col.assign(P.sum_card, 0);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < kcard[i]; ++j) P.io_post_col[P.post_off[i] + j] = (int32_t)(full_off[orig[i]] + j);
  P.opts.n_query_set = 0;
  P.opts.query_set = nullptr;
  return JT_OK;
}

}  // namespace jt
