// Test of the library's host compiler: every index map of a compiled plan
// against a direct mixed-radix restatement (digits decoded by division).
//
// Input: a network file (int64 n, number of parent entries, number of CPT
// entries; int32 card[n]; int32 parent_ptr[n+1]; int32 parents[]; double
// cpt[]), then optional "obs=v1,v2,..." and "query=v1,..." arguments.
// Checks, for every clique C of the plan:
//   * its strides are the row-major strides of its variable order and the
//     upward separator is the outermost block (entry e = s*R + u);
//   * child maps: A[s] + B[u] is the index, in the child's message, of the
//     child-separator digits of entry e (the extension step);
//   * evidence maps: A[s] + B[u] is the digit of the variable at e;
//   * upward-message evidence maps: A[s] is the digit of the variable at s;
//   * base maps of an observed-set plan: A[s] + B[u] is the entry of the
//     full base table with e's digits (observed-set digits 0);
// and for every distribute task: over t < T, u < U the entries
// A[t] + B[u] visit each entry of the source table exactly once, the
// target digits of that entry encode t (through the output map OP of a
// fused pair; the marginalisation), and sA[t] + sB[u] is its entry of the
// clique's upward separator; for a fused pair also that the secondary
// index Ku[u] is in range and OSf[t / a] + OSk[Ku[u]] encodes the entry's
// digits of the secondary target, one target per (F-block, index), every
// secondary target written; and that fused work items hold whole F-blocks
// or pieces of one, with partial slots in range.  Options fuse=0|1,
// cpt=N (cases per thread) and rows=N (distribute rows per item in every
// size bucket) vary the compiled shape.
// Prints the number of failed checks and exits non-zero if any failed.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>

#include "../../paper_2212_04241_gb300/csrc/jt_internal.h"

namespace jt {
void set_error(const std::string &) {}
}
using namespace jt;

static long long g_fail = 0, g_checks = 0;
static void expect(bool ok, const char *what, int c, long long e) {
  ++g_checks;
  if (!ok && g_fail++ < 20) std::printf("FAIL %s: clique %d entry %lld\n", what, c, e);
}

static std::vector<int> parse_list(const char *s) {
  std::vector<int> out;
  while (*s) {
    out.push_back(std::atoi(s));
    const char *comma = std::strchr(s, ',');
    if (!comma) break;
    s = comma + 1;
  }
  return out;
}

int main(int argc, char **argv) {
  if (argc < 2) return 2;
  FILE *f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t hdr[3];
  if (std::fread(hdr, 8, 3, f) != 3) return 2;
  const int n = (int)hdr[0];
  std::vector<int32_t> card(n), pptr(n + 1), par(std::max<int64_t>(1, hdr[1]));
  std::vector<double> cpt(hdr[2]);
  size_t got = std::fread(card.data(), 4, n, f) + std::fread(pptr.data(), 4, n + 1, f);
  if (hdr[1] > 0) got += std::fread(par.data(), 4, hdr[1], f);
  got += std::fread(cpt.data(), 8, hdr[2], f);
  std::fclose(f);
  if (got != (size_t)(n + n + 1 + hdr[1] + hdr[2])) return 2;
  std::vector<int> obs, query;
  int fuse = 1, cpt_opt = 0, rows = 0;
  for (int i = 2; i < argc; ++i) {
    if (!std::strncmp(argv[i], "obs=", 4)) obs = parse_list(argv[i] + 4);
    if (!std::strncmp(argv[i], "query=", 6)) query = parse_list(argv[i] + 6);
    if (!std::strncmp(argv[i], "fuse=", 5)) fuse = std::atoi(argv[i] + 5);
    if (!std::strncmp(argv[i], "cpt=", 4)) cpt_opt = std::atoi(argv[i] + 4);
    if (!std::strncmp(argv[i], "rows=", 5)) rows = std::atoi(argv[i] + 5);
  }
  jt_compile_opts o;
  std::memset(&o, 0, sizeof(o));
  o.root_rule = JT_ROOT_MIN_HEIGHT;
  o.host_only = 1;
  o.use_graphs = 1;
  o.rescale = 1;
  o.fuse_distribute = fuse;
  o.cases_per_thread = cpt_opt;
  for (int b = 0; b < JT_SIZE_BUCKETS; ++b) o.distribute_rows_by_bucket[b] = rows;
  o.n_observed_set = (int32_t)obs.size();
  o.observed_set = obs.empty() ? nullptr : obs.data();
  o.n_query_set = (int32_t)query.size();
  o.query_set = query.empty() ? nullptr : query.data();
  Plan P;
  std::string err;
  if (build_plan_pruned(n, card.data(), pptr.data(), par.data(), cpt.data(), o, P, err) != JT_OK) {
    std::printf("compile failed: %s\n", err.c_str());
    return 1;
  }
  const int m = (int)P.cl.size();
  const int32_t *pool = P.ipool.data();
  for (int c = 0; c < m; ++c) {
    const HostClique &C = P.cl[c];
    const DClique &D = P.dcl[c];
    const int nv = (int)C.vars.size();
    // row-major strides, separator outermost
    int64_t s_expect = 1;
    for (int i = nv - 1; i >= 0; --i) {
      expect(C.stride[i] == s_expect, "row-major stride", c, i);
      s_expect *= C.card[i];
    }
    expect(s_expect == C.size, "table size", c, -1);
    int64_t nsep = 1;
    for (int i = 0; i < C.n_up; ++i) nsep *= C.card[i];
    expect(nsep == C.nsep && C.nsep * C.R == C.size, "separator block", c, -1);
    if (C.parent >= 0) {
      const HostClique &Pa = P.cl[C.parent];
      std::vector<int> sep;
      for (int v : Pa.vars)
        if (std::find(C.vars.begin(), C.vars.end(), v) != C.vars.end()) sep.push_back(v);
      expect((int)sep.size() == C.n_up && std::equal(sep.begin(), sep.end(), C.vars.begin()),
             "upward separator outermost, parent's order", c, -1);
    }
    auto digit = [&](int64_t e, int v) -> int {
      const int i = (int)(std::find(C.vars.begin(), C.vars.end(), v) - C.vars.begin());
      return i < nv ? (int)((e / C.stride[i]) % C.card[i]) : -1;
    };
    // collect maps
    for (int k = D.map_begin; k < D.map_end; ++k) {
      const DMap &mp = P.dmap[k];
      for (int64_t e = 0; e < C.size; ++e) {
        const int64_t s = e / C.R, u = e % C.R;
        const int64_t got_idx = (int64_t)pool[mp.A_off + s] + pool[mp.B_off + u];
        if (mp.kind == MAP_CHILD) {
          const HostClique &K = P.cl[mp.src];
          int64_t want = 0;
          for (int i = 0; i < K.n_up; ++i) {
            int64_t w = 1;  // row-major stride of K.vars[i] inside K's separator block
            for (int j = i + 1; j < K.n_up; ++j) w *= K.card[j];
            want += (int64_t)digit(e, K.vars[i]) * w;
          }
          expect(got_idx == want, "child message index", c, e);
        } else if (mp.kind == MAP_EVIDENCE) {
          expect(got_idx == digit(e, mp.src), "evidence digit", c, e);
        }
      }
    }
    for (int k = D.sev_begin; k < D.sev_end; ++k) {
      const DMap &mp = P.dmap[k];
      for (int64_t s = 0; s < C.nsep; ++s) expect(pool[mp.A_off + s] == digit(s * C.R, mp.src), "message evidence digit", c, s);
    }
    if (D.slice_end > D.slice_begin || P.n_sliced > 0) {
      for (int64_t e = 0; e < C.size; ++e) {
        int64_t want = 0;
        for (int i = 0; i < nv; ++i) {
          int64_t fw = 1;  // row-major stride of vars[i] in the full layout
          const int fi = (int)(std::find(C.fvars.begin(), C.fvars.end(), C.vars[i]) - C.fvars.begin());
          for (size_t j = fi + 1; j < C.fvars.size(); ++j) fw *= P.card[C.fvars[j]];
          want += (int64_t)digit(e, C.vars[i]) * fw;
        }
        const int64_t got_idx = (int64_t)pool[D.bmap_A + e / C.R] + pool[D.bmap_B + e % C.R];
        expect(got_idx == want, "base-table slice map", c, e);
      }
    }
  }
  // distribute tasks
  for (size_t ti = 0; ti < P.dtask.size(); ++ti) {
    const DTask &T = P.dtask[ti];
    const HostClique &C = P.cl[T.clique];
    const int64_t xsize = T.src_sep ? C.nsep : C.size;
    std::vector<int> target;
    if (T.kind == TASK_CHILD) {
      const HostClique &K = P.cl[T.dst];
      target.assign(K.vars.begin(), K.vars.begin() + K.n_up);
    } else {
      target.push_back(T.dst);
    }
    // a target's code: its variables' digits at entry e, in layout order
    auto code_of = [&](const std::vector<int> &tv, int64_t e) {
      std::vector<int> ordered;
      for (int v : C.vars)
        if (std::find(tv.begin(), tv.end(), v) != tv.end()) ordered.push_back(v);
      int64_t code = 0;
      for (int v : ordered) {
        const int i = (int)(std::find(C.vars.begin(), C.vars.end(), v) - C.vars.begin());
        code = code * C.card[i] + (int64_t)((e / C.stride[i]) % C.card[i]);
      }
      return code;
    };
    // the task's plain enumeration: every source entry once, target t
    auto check_enumeration = [&](int64_t A_off, int64_t B_off, int64_t sA_off, int64_t sB_off, bool fused) {
      std::vector<char> seen(xsize, 0);
      bool once = T.T * T.U == xsize;
      std::vector<int> target2;
      int64_t size2 = 1;
      std::vector<char> seen2;
      std::vector<int64_t> fcode;
      if (fused) {
        const DTask &S = P.dtask[T.sec_task];
        expect(S.clique == T.clique && S.kind == T.sec_kind && S.dst == T.sec_dst && S.dst_row == T.sec_dst_row &&
                   !S.src_sep && !T.src_sep && S.sec_b == 0,
               "fused pair descriptor", T.clique, (long long)ti);
        if (S.kind == TASK_CHILD) {
          const HostClique &K = P.cl[S.dst];
          target2.assign(K.vars.begin(), K.vars.begin() + K.n_up);
        } else {
          target2.push_back(S.dst);
        }
        for (int v : target2) size2 *= P.card[v];
        expect(T.sec_a > 0 && T.T % T.sec_a == 0 && T.U % T.sec_b == 0 && T.sec_b <= P.sec_rows, "fused pair sizes",
               T.clique, (long long)ti);
        seen2.assign(size2, 0);
        fcode.assign((T.T / T.sec_a) * T.sec_b, -1);
      }
      for (int64_t t = 0; t < T.T; ++t)
        for (int64_t u = 0; u < T.U; ++u) {
          const int64_t x = (int64_t)pool[A_off + t] + pool[B_off + u];
          if (x < 0 || x >= xsize || seen[x]) { once = false; continue; }
          seen[x] = 1;
          const int64_t e = T.src_sep ? x * C.R : x;  // an entry of C with the same separator digits
          const int64_t tcode = code_of(target, e);
          const int64_t tout = fused ? (int64_t)pool[T.op_off + t] : t;
          expect(tout >= 0 && tout < T.T && tcode == tout, "task target digits", T.clique, x);
          const int64_t y = (int64_t)pool[sA_off + t] + pool[sB_off + u];
          const bool root_like = !T.src_sep && P.dcl[T.clique].is_root;  // scaled by 2^-k, no ratio
          expect(root_like || y == e / C.R, "task ratio entry", T.clique, x);
          if (fused) {
            const int64_t k = pool[T.ku_off + u];
            const int64_t f = t / T.sec_a;
            expect(k >= 0 && k < T.sec_b, "fused secondary index in range", T.clique, x);
            if (k < 0 || k >= T.sec_b) continue;
            const int64_t got = (int64_t)pool[T.osf_off + f] + pool[T.osk_off + k];
            expect(got >= 0 && got < size2 && got == code_of(target2, e), "fused secondary target digits", T.clique, x);
            // (F-block, k) names one secondary target, the same for every row
            int64_t &fc = fcode[f * T.sec_b + k];
            expect(fc < 0 || fc == got, "fused secondary target fixed per F-block", T.clique, x);
            fc = got;
            if (got >= 0 && got < size2) seen2[got] = 1;
          }
        }
      expect(once, "task visits every source entry once", T.clique, (long long)ti);
      if (fused) {
        bool all = true;
        for (char c2 : seen2) all = all && c2;
        expect(all, "fused pair writes every secondary target", T.clique, (long long)ti);
      }
    };
    check_enumeration(T.A_off, T.B_off, T.sA_off, T.sB_off, false);
    if (T.sec_b > 0) check_enumeration(T.fA_off, T.fB_off, T.fsA_off, T.fsB_off, true);
  }
  // work items of fused tasks: whole primary targets inside one F-block (or
  // whole F-blocks), partial slots and split groups in range
  for (const DItem &it : P.ditems) {
    const DTask &T = P.dtask[it.task];
    expect(!T.absorbed, "no items for an absorbed task", T.clique, it.task);
    // a pair either has fused items (partner absorbed) or both tasks plain items
    expect(!it.fused || (T.sec_b > 0 && P.dtask[T.sec_task].absorbed), "fused item of a fused pair", T.clique,
           it.task);
    expect(it.fused || T.sec_b <= 0 || !P.dtask[T.sec_task].absorbed, "plain item of an unfused pair", T.clique,
           it.task);
    if (!it.fused) continue;
    const int64_t a = T.sec_a;
    expect(it.split == 0 && it.u0 == 0 && it.nu == T.U && it.t0 >= 0 && it.t0 + it.nt <= T.T, "fused item range",
           T.clique, it.t0);
    if (it.npieces == 1) {
      expect(it.t0 % a == 0 && it.nt % a == 0, "fused item holds whole F-blocks", T.clique, it.t0);
    } else {
      expect(it.t0 / a == (it.t0 + it.nt - 1) / a, "fused piece inside one F-block", T.clique, it.t0);
      expect(it.group >= 0 && it.group < P.n_groups && it.partial >= 0 &&
                 it.partial + (int64_t)it.npieces * T.sec_b - (int64_t)it.piece * T.sec_b <= P.n_partials &&
                 it.partial - (int64_t)it.piece * T.sec_b >= 0,
             "fused piece partial slots", T.clique, it.t0);
    }
  }
  long long fused = 0, pieces = 0;
  for (const DTask &T : P.dtask) fused += T.sec_b > 0;
  long long fused_items = 0;
  for (const DItem &it : P.ditems) {
    pieces += it.fused && it.npieces > 1;
    fused_items += it.fused;
  }
  std::printf("fused pairs %lld, fused items %lld, of them pieces %lld\n", fused, fused_items, pieces);
  std::printf("%lld checks, %lld failed\n", g_checks, g_fail);
  return g_fail ? 1 : 0;
}
