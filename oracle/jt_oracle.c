/*
 * jt_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 junction-tree (Hugin) inference
 * engine used as the correctness oracle for the GPU library.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the GPU library: it has
 * its own network compiler, its own table layout and its own message
 * passing, written for readability rather than speed.
 *
 * What it computes (Section 1 of the paper, the problem statement): for
 * evidence e, P(e) and the posterior marginal P(X_v | e) of every
 * unobserved variable v.  The route is the junction-tree algorithm the
 * paper describes (Section 1: cliques as tree nodes, separators as edges,
 * potential tables, messages passed along the tree): moralise the DAG,
 * triangulate, build the clique tree, then collect (leaves -> root) and
 * distribute (root -> leaves) messages.  The table operations are the
 * three the paper names in Section 2 -- marginalisation, extension and
 * reduction -- plus the Hugin separator division.  Details the poster does
 * not state are filled with standard readings:
 *   - triangulation: min-fill elimination, ties to the lowest variable id
 *     (min-degree available for invariance tests);
 *   - cliques: maximal elimination cliques, numbered in creation order;
 *   - tree: Kruskal maximum-weight spanning tree over all clique pairs,
 *     weight = number of shared variables (zero-weight pairs included, so
 *     disconnected networks become one tree), ties by (clique i, clique j);
 *   - root: largest table (ties to the lowest id), or the clique of least
 *     eccentricity (fewest layers, Section 2's root selection), or a given id;
 *   - CPT v goes to the smallest clique containing {v} u parents(v);
 *   - evidence ("reduction", Section 2): every clique containing an
 *     observed variable has the contradicting entries set to zero;
 *   - separator division 0/0 := 0;
 *   - optional power-of-two rescaling of every message by its maximum,
 *     with the integer exponents summed into log P(e); exact in FP64.
 *
 * Table layout (the oracle's own): a table over an ordered variable list
 * is a dense row-major array, the LAST listed variable varying fastest.
 * Clique and separator variable lists are ascending variable ids.
 *
 * Parity status of every exported function is listed in the test suite;
 * all of them are pinned by brute-force enumeration of the joint, a
 * hand-derived closed form, or an independent variable-elimination solver.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0 /* >0 only in the mutation tests (planted mistakes) */
#endif

#define MAXV 64 /* variables per table; 2^64 entries is far beyond memory */

typedef struct {
  int nv;
  int vars[MAXV];
  int card[MAXV];
  long size;
} scope_t;

typedef struct {
  int n;
  int *card;
  int *pptr, *par;
  double *cpt;
  long *cpt_off;
  int ncl;
  scope_t *cl;      /* cliques, ascending vars */
  scope_t *sep;     /* sep[c] = clique c intersect its parent (c != root) */
  int root;
  int *parent;      /* parent clique, -1 for the root */
  int *bfs;         /* BFS order from the root */
  int *depth;
  int *assign;      /* CPT of variable v multiplied into clique assign[v] */
  int *post_src;    /* posterior of v read from clique post_src[v] */
  long *post_off;   /* offset of v's marginal in the posterior output */
  long sum_card;
  long sum_cl, sum_sep, max_cl;
} orc_t;

/* ------------------------------------------------------------------ */
/* table index mapping                                                 */
/* ------------------------------------------------------------------ */

/* For every variable of x, its stride inside y (0 when y lacks it).  y is a
 * row-major table over its own variable list, last variable fastest. */
static void map_strides(const scope_t *x, const scope_t *y, long *ystride) {
  for (int i = 0; i < x->nv; ++i) ystride[i] = 0;
  long s = 1;
  for (int j = y->nv - 1; j >= 0; --j) {
    for (int i = 0; i < x->nv; ++i)
      if (x->vars[i] == y->vars[j]) ystride[i] = s;
    s *= y->card[j];
  }
}

/* Advance the mixed-radix digits of x by one entry and keep idx, the
 * matching index into y, in step. */
static void odometer_step(const scope_t *x, int *dig, const long *ystride, long *idx) {
  for (int i = x->nv - 1; i >= 0; --i) {
    dig[i]++;
    *idx += ystride[i];
    if (dig[i] < x->card[i]) return;
    *idx -= ystride[i] * x->card[i];
    dig[i] = 0;
  }
}

/* Marginalisation (Section 2): ty = sum over the variables of x not in y. */
static void marginalize(const scope_t *x, const double *tx, const scope_t *y, double *ty) {
  long ys[MAXV];
  int dig[MAXV];
  memset(ty, 0, sizeof(double) * y->size);
  memset(dig, 0, sizeof(dig));
  map_strides(x, y, ys);
  long idx = 0;
  long n = x->size;
#if ORACLE_MUTANT == 5
  n -= 1; /* planted: a dropped term */
#endif
  for (long e = 0; e < n; ++e) {
    ty[idx] += tx[e];
    odometer_step(x, dig, ys, &idx);
  }
}

/* Extension (Section 2): tx[e] *= ty[entry of y that e maps to]. */
static void extend_multiply(const scope_t *x, double *tx, const scope_t *y, const double *ty) {
  long ys[MAXV];
  int dig[MAXV];
  memset(dig, 0, sizeof(dig));
  map_strides(x, y, ys);
  long idx = 0;
  for (long e = 0; e < x->size; ++e) {
    tx[e] *= ty[idx];
    odometer_step(x, dig, ys, &idx);
  }
}

/* Reduction (Section 2): zero the entries of x whose state of v is not s. */
static void reduce_evidence(const scope_t *x, double *tx, int v, int s) {
  int pos = -1;
  for (int i = 0; i < x->nv; ++i)
    if (x->vars[i] == v) pos = i;
  if (pos < 0) return;
  long stride = 1;
  for (int i = x->nv - 1; i > pos; --i) stride *= x->card[i];
  for (long e = 0; e < x->size; ++e) {
    int d = (int)((e / stride) % x->card[pos]);
#if ORACLE_MUTANT == 2
    if (d == s) tx[e] = 0.0; /* planted: inverted test */
#else
    if (d != s) tx[e] = 0.0;
#endif
  }
}

static int scope_contains(const scope_t *x, int v) {
  for (int i = 0; i < x->nv; ++i)
    if (x->vars[i] == v) return 1;
  return 0;
}

static void scope_finish(scope_t *x, const int *card) {
  x->size = 1;
  for (int i = 0; i < x->nv; ++i) {
    x->card[i] = card[x->vars[i]];
    x->size *= x->card[i];
  }
}

/* Exponent k with m * 2^-k in [1, 2) (m > 0). */
static int pow2_exponent(double m) {
  int ex;
  frexp(m, &ex);
  return ex - 1;
}

/* ------------------------------------------------------------------ */
/* compiler: moralise, triangulate, clique tree                         */
/* ------------------------------------------------------------------ */

typedef struct { int w, i, j; } edge_t;

static int edge_cmp(const void *a, const void *b) {
  const edge_t *x = a, *y = b;
#if ORACLE_MUTANT == 8
  if (x->w != y->w) return x->w < y->w ? -1 : 1; /* planted: minimum tree */
#else
  if (x->w != y->w) return x->w > y->w ? -1 : 1;
#endif
  if (x->i != y->i) return x->i < y->i ? -1 : 1;
  if (x->j != y->j) return x->j < y->j ? -1 : 1;
  return 0;
}

static int uf_find(int *p, int a) {
  while (p[a] != a) a = p[a] = p[p[a]];
  return a;
}

static int is_subset(const scope_t *a, const scope_t *b) {
  for (int i = 0; i < a->nv; ++i)
    if (!scope_contains(b, a->vars[i])) return 0;
  return 1;
}

static int shared_count(const scope_t *a, const scope_t *b) {
  int k = 0;
  for (int i = 0; i < a->nv; ++i) k += scope_contains(b, a->vars[i]);
  return k;
}

void orc_free(void *h);

/* elim_rule: 0 = min-fill, 1 = min-degree.  root_rule: 0 = largest table,
 * 1 = least eccentricity, r >= 2 = clique r-2. */
int orc_compile(int n, const int *card, const int *pptr, const int *par, const double *cpt,
                int elim_rule, int root_rule, void **out) {
  *out = NULL;
  if (n <= 0) return -1;
  orc_t *o = calloc(1, sizeof(orc_t));
  o->n = n;
  o->card = malloc(sizeof(int) * n);
  memcpy(o->card, card, sizeof(int) * n);
  o->pptr = malloc(sizeof(int) * (n + 1));
  memcpy(o->pptr, pptr, sizeof(int) * (n + 1));
  o->par = malloc(sizeof(int) * (pptr[n] > 0 ? pptr[n] : 1));
  memcpy(o->par, par, sizeof(int) * pptr[n]);
  o->cpt_off = malloc(sizeof(long) * (n + 1));
  o->cpt_off[0] = 0;
  for (int v = 0; v < n; ++v) {
    long rows = 1;
    for (int k = pptr[v]; k < pptr[v + 1]; ++k) rows *= card[par[k]];
    o->cpt_off[v + 1] = o->cpt_off[v] + rows * card[v];
  }
  o->cpt = malloc(sizeof(double) * o->cpt_off[n]);
  memcpy(o->cpt, cpt, sizeof(double) * o->cpt_off[n]);

  /* moral graph */
  char *adj = calloc((size_t)n * n, 1);
  for (int v = 0; v < n; ++v) {
    for (int a = pptr[v]; a < pptr[v + 1]; ++a) {
      int p = par[a];
      adj[(size_t)v * n + p] = adj[(size_t)p * n + v] = 1;
#if ORACLE_MUTANT != 9 /* planted (9): parents are not married */
      for (int b = a + 1; b < pptr[v + 1]; ++b) {
        int q = par[b];
        adj[(size_t)p * n + q] = adj[(size_t)q * n + p] = 1;
      }
#endif
    }
  }

  /* elimination */
  char *alive = malloc(n);
  memset(alive, 1, n);
  int *nb = malloc(sizeof(int) * n);
  scope_t *ecl = malloc(sizeof(scope_t) * n);
  int necl = 0;
  int ret = 0;
  for (int step = 0; step < n; ++step) {
    int best = -1;
    long best_score = 0;
    for (int v = 0; v < n; ++v) {
      if (!alive[v]) continue;
      int k = 0;
      for (int u = 0; u < n; ++u)
        if (u != v && alive[u] && adj[(size_t)v * n + u]) nb[k++] = u;
      long score;
      if (elim_rule == 1) {
        score = k;
      } else {
        score = 0;
        for (int a = 0; a < k; ++a)
          for (int b = a + 1; b < k; ++b)
            if (!adj[(size_t)nb[a] * n + nb[b]]) ++score;
      }
      if (best < 0 || score < best_score) {
        best = v;
        best_score = score;
      }
    }
    int v = best;
    int k = 0;
    for (int u = 0; u < n; ++u)
      if (u != v && alive[u] && adj[(size_t)v * n + u]) nb[k++] = u;
    if (k + 1 > MAXV) { ret = -3; break; }
    scope_t c;
    c.nv = 0;
    /* ascending variable ids */
    int placed = 0;
    for (int a = 0; a < k; ++a) {
      if (!placed && nb[a] > v) { c.vars[c.nv++] = v; placed = 1; }
      c.vars[c.nv++] = nb[a];
    }
    if (!placed) c.vars[c.nv++] = v;
    scope_finish(&c, card);
    for (int a = 0; a < k; ++a)
      for (int b = a + 1; b < k; ++b)
        adj[(size_t)nb[a] * n + nb[b]] = adj[(size_t)nb[b] * n + nb[a]] = 1;
    alive[v] = 0;
    int maximal = 1;
    for (int q = 0; q < necl; ++q)
      if (is_subset(&c, &ecl[q])) { maximal = 0; break; }
    if (maximal) ecl[necl++] = c;
  }
  free(adj);
  free(alive);
  free(nb);
  if (ret) { free(ecl); orc_free(o); return ret; }

  o->ncl = necl;
  o->cl = ecl;
  o->sum_cl = 0;
  o->max_cl = 0;
  for (int c = 0; c < necl; ++c) {
    o->sum_cl += ecl[c].size;
    if (ecl[c].size > o->max_cl) o->max_cl = ecl[c].size;
  }

  /* Kruskal maximum-weight spanning tree over all clique pairs */
  long npairs = (long)necl * (necl - 1) / 2;
  edge_t *ed = malloc(sizeof(edge_t) * (npairs > 0 ? npairs : 1));
  long m = 0;
  for (int i = 0; i < necl; ++i)
    for (int j = i + 1; j < necl; ++j) {
      ed[m].w = shared_count(&ecl[i], &ecl[j]);
      ed[m].i = i;
      ed[m].j = j;
      ++m;
    }
  qsort(ed, m, sizeof(edge_t), edge_cmp);
  int *uf = malloc(sizeof(int) * necl);
  for (int i = 0; i < necl; ++i) uf[i] = i;
  int *tadj = calloc((size_t)necl * necl, sizeof(int)); /* tree adjacency matrix */
  int taken = 0;
  for (long e = 0; e < m && taken < necl - 1; ++e) {
    int a = uf_find(uf, ed[e].i), b = uf_find(uf, ed[e].j);
    if (a == b) continue;
    uf[a] = b;
    tadj[(size_t)ed[e].i * necl + ed[e].j] = tadj[(size_t)ed[e].j * necl + ed[e].i] = 1;
    ++taken;
  }
  free(ed);
  free(uf);

  /* root */
  int *dist = malloc(sizeof(int) * necl);
  int *queue = malloc(sizeof(int) * necl);
  int root = 0;
  if (root_rule == 0) {
    for (int c = 1; c < necl; ++c)
      if (ecl[c].size > ecl[root].size) root = c;
  } else if (root_rule == 1) {
    int best_ecc = -1;
    for (int s = 0; s < necl; ++s) {
      for (int c = 0; c < necl; ++c) dist[c] = -1;
      int qh = 0, qt = 0;
      queue[qt++] = s;
      dist[s] = 0;
      int ecc = 0;
      while (qh < qt) {
        int a = queue[qh++];
        if (dist[a] > ecc) ecc = dist[a];
        for (int b = 0; b < necl; ++b)
          if (tadj[(size_t)a * necl + b] && dist[b] < 0) { dist[b] = dist[a] + 1; queue[qt++] = b; }
      }
      if (best_ecc < 0 || ecc < best_ecc ||
          (ecc == best_ecc && ecl[s].size > ecl[root].size)) {
        best_ecc = ecc;
        root = s;
      }
    }
  } else {
    root = root_rule - 2;
    if (root < 0 || root >= necl) root = 0;
  }
  o->root = root;

  /* orient the tree: BFS from the root, neighbours in ascending id order */
  o->parent = malloc(sizeof(int) * necl);
  o->bfs = malloc(sizeof(int) * necl);
  o->depth = malloc(sizeof(int) * necl);
  for (int c = 0; c < necl; ++c) o->parent[c] = -2;
  int qh = 0, qt = 0;
  o->bfs[qt++] = root;
  o->parent[root] = -1;
  o->depth[root] = 0;
  while (qh < qt) {
    int a = o->bfs[qh++];
    for (int b = 0; b < necl; ++b)
      if (tadj[(size_t)a * necl + b] && o->parent[b] == -2) {
        o->parent[b] = a;
        o->depth[b] = o->depth[a] + 1;
        o->bfs[qt++] = b;
      }
  }
  free(tadj);
  free(dist);
  free(queue);

  o->sep = calloc(necl, sizeof(scope_t));
  o->sum_sep = 0;
  for (int c = 0; c < necl; ++c) {
    if (c == root) continue;
    const scope_t *a = &ecl[c], *b = &ecl[o->parent[c]];
    o->sep[c].nv = 0;
    for (int i = 0; i < a->nv; ++i)
      if (scope_contains(b, a->vars[i])) o->sep[c].vars[o->sep[c].nv++] = a->vars[i];
    scope_finish(&o->sep[c], card);
    o->sum_sep += o->sep[c].size;
  }

  /* CPT assignment and posterior sources */
  o->assign = malloc(sizeof(int) * n);
  o->post_src = malloc(sizeof(int) * n);
  o->post_off = malloc(sizeof(long) * n);
  o->sum_card = 0;
  for (int v = 0; v < n; ++v) {
    o->post_off[v] = o->sum_card;
    o->sum_card += card[v];
    int best = -1, bestp = -1;
    for (int c = 0; c < necl; ++c) {
      if (!scope_contains(&ecl[c], v)) continue;
      if (bestp < 0 || ecl[c].size < ecl[bestp].size) bestp = c;
      int ok = 1;
      for (int k = pptr[v]; k < pptr[v + 1]; ++k)
        if (!scope_contains(&ecl[c], par[k])) ok = 0;
      if (ok && (best < 0 || ecl[c].size < ecl[best].size)) best = c;
    }
    if (best < 0) { orc_free(o); return -4; } /* no clique covers the family */
    o->assign[v] = best;
    o->post_src[v] = bestp;
  }
  *out = o;
  return 0;
}

void orc_free(void *h) {
  orc_t *o = h;
  if (!o) return;
  free(o->card); free(o->pptr); free(o->par); free(o->cpt); free(o->cpt_off);
  free(o->cl); free(o->sep); free(o->parent); free(o->bfs); free(o->depth);
  free(o->assign); free(o->post_src); free(o->post_off);
  free(o);
}

/* ------------------------------------------------------------------ */
/* inference                                                           */
/* ------------------------------------------------------------------ */

typedef struct {
  double **psi;   /* clique tables */
  double **phi;   /* separator tables (message from collect) */
  double *tmp;    /* scratch separator table */
  long *sc;       /* true psi_c = psi_c * 2^sc[c] */
  long *ksep;     /* true phi_c = phi_c * 2^ksep[c] */
} work_t;

static work_t *work_alloc(const orc_t *o) {
  work_t *w = calloc(1, sizeof(work_t));
  w->psi = calloc(o->ncl, sizeof(double *));
  w->phi = calloc(o->ncl, sizeof(double *));
  long maxsep = 1;
  for (int c = 0; c < o->ncl; ++c) {
    w->psi[c] = malloc(sizeof(double) * o->cl[c].size);
    long s = (c == o->root) ? 1 : o->sep[c].size;
    w->phi[c] = malloc(sizeof(double) * s);
    if (s > maxsep) maxsep = s;
  }
  w->tmp = malloc(sizeof(double) * maxsep);
  w->sc = calloc(o->ncl, sizeof(long));
  w->ksep = calloc(o->ncl, sizeof(long));
  return w;
}

static void work_free(const orc_t *o, work_t *w) {
  for (int c = 0; c < o->ncl; ++c) { free(w->psi[c]); free(w->phi[c]); }
  free(w->psi); free(w->phi); free(w->tmp); free(w->sc); free(w->ksep);
  free(w);
}

/* Scale t (size n) by 2^-k where k is the exponent of its maximum; returns k
 * (0 for an all-zero table).  Exact in FP64. */
static long rescale_table(double *t, long n) {
  double m = 0.0;
  for (long i = 0; i < n; ++i)
    if (t[i] > m) m = t[i];
  if (m <= 0.0) return 0;
  int k = pow2_exponent(m);
  for (long i = 0; i < n; ++i) t[i] = ldexp(t[i], -k);
  return k;
}

/* One evidence case.  Returns 0, or 1 when P(e) = 0. */
static int infer_one(const orc_t *o, work_t *w, const int *ev, int rescale,
                     double *log_pe, double *post) {
  const int n = o->n, ncl = o->ncl;
  /* initial potentials: product of the assigned CPTs */
  for (int c = 0; c < ncl; ++c) {
    for (long e = 0; e < o->cl[c].size; ++e) w->psi[c][e] = 1.0;
    w->sc[c] = 0;
  }
  for (int v = 0; v < n; ++v) {
    scope_t f;
    f.nv = 0;
#if ORACLE_MUTANT == 3
    f.vars[f.nv++] = v; /* planted: child state taken as the slowest digit */
    for (int k = o->pptr[v]; k < o->pptr[v + 1]; ++k) f.vars[f.nv++] = o->par[k];
#else
    for (int k = o->pptr[v]; k < o->pptr[v + 1]; ++k) f.vars[f.nv++] = o->par[k];
    f.vars[f.nv++] = v;
#endif
    scope_finish(&f, o->card);
    extend_multiply(&o->cl[o->assign[v]], w->psi[o->assign[v]], &f, o->cpt + o->cpt_off[v]);
  }
  /* evidence */
  for (int v = 0; v < n; ++v) {
    if (ev[v] < 0) continue;
    for (int c = 0; c < ncl; ++c) reduce_evidence(&o->cl[c], w->psi[c], v, ev[v]);
  }
  /* collect: children before parents (reverse BFS order) */
  for (int q = ncl - 1; q >= 1; --q) {
#if ORACLE_MUTANT == 6
    int c = o->bfs[ncl - q]; /* planted: parents before children */
#else
    int c = o->bfs[q];
#endif
    int p = o->parent[c];
    marginalize(&o->cl[c], w->psi[c], &o->sep[c], w->phi[c]);
    long k = rescale ? rescale_table(w->phi[c], o->sep[c].size) : 0;
    w->ksep[c] = k + w->sc[c];
    extend_multiply(&o->cl[p], w->psi[p], &o->sep[c], w->phi[c]);
#if ORACLE_MUTANT == 4
    (void)0; /* planted: the exponent is dropped */
#else
    w->sc[p] += w->ksep[c];
#endif
  }
  /* P(e) from the root */
  double z = 0.0;
  for (long e = 0; e < o->cl[o->root].size; ++e) z += w->psi[o->root][e];
  if (!(z > 0.0)) {
    *log_pe = -INFINITY;
    for (long i = 0; i < o->sum_card; ++i) post[i] = NAN;
    return 1;
  }
  *log_pe = log(z) + (double)w->sc[o->root] * log(2.0);
  /* distribute: parents before children (BFS order) */
  for (int q = 1; q < ncl; ++q) {
    int c = o->bfs[q];
    int p = o->parent[c];
    const scope_t *s = &o->sep[c];
    marginalize(&o->cl[p], w->psi[p], s, w->tmp);
    long k = rescale ? rescale_table(w->tmp, s->size) : 0;
    for (long i = 0; i < s->size; ++i) {
      double num = w->tmp[i], den = w->phi[c][i];
#if ORACLE_MUTANT == 1
      w->tmp[i] = num; /* planted: no division by the old separator */
      (void)den;
#else
      w->tmp[i] = (den != 0.0) ? num / den : 0.0; /* 0/0 := 0 */
#endif
    }
    extend_multiply(&o->cl[c], w->psi[c], s, w->tmp);
    w->sc[c] = w->sc[c] + k + w->sc[p] - w->ksep[c];
  }
  /* posteriors */
  for (int v = 0; v < n; ++v) {
    double *pv = post + o->post_off[v];
    int r = o->card[v];
    if (ev[v] >= 0) {
      for (int s = 0; s < r; ++s) pv[s] = (s == ev[v]) ? 1.0 : 0.0;
      continue;
    }
    scope_t one;
    one.nv = 1;
    one.vars[0] = v;
    scope_finish(&one, o->card);
    marginalize(&o->cl[o->post_src[v]], w->psi[o->post_src[v]], &one, pv);
    double t = 0.0;
    for (int s = 0; s < r; ++s) t += pv[s];
    for (int s = 0; s < r; ++s) pv[s] /= t;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* exported API                                                        */
/* ------------------------------------------------------------------ */

int orc_info(void *h, long *out) {
  /* out: ncl, root, height, sum_cl, max_cl, sum_sep, sum_card */
  orc_t *o = h;
  int height = 0;
  for (int c = 0; c < o->ncl; ++c)
    if (o->depth[c] > height) height = o->depth[c];
  out[0] = o->ncl;
  out[1] = o->root;
  out[2] = height;
  out[3] = o->sum_cl;
  out[4] = o->max_cl;
  out[5] = o->sum_sep;
  out[6] = o->sum_card;
  return 0;
}

/* Variables of clique c (ascending) and its parent clique (-1 for root). */
int orc_clique(void *h, int c, int *vars, int *parent) {
  orc_t *o = h;
  if (c < 0 || c >= o->ncl) return -1;
  memcpy(vars, o->cl[c].vars, sizeof(int) * o->cl[c].nv);
  *parent = o->parent[c];
  return o->cl[c].nv;
}

int orc_infer(void *h, const int *ev, int rescale, double *log_pe, double *post) {
  orc_t *o = h;
  work_t *w = work_alloc(o);
  int st = infer_one(o, w, ev, rescale, log_pe, post);
  work_free(o, w);
  return st;
}

/* After a full inference, copy out the calibrated table of clique c (oracle
 * layout: ascending variables, last fastest) and its power-of-two exponent:
 * the calibrated potential is table * 2^exponent. */
int orc_calibrated(void *h, const int *ev, int rescale, int c, double *table, long *exponent) {
  orc_t *o = h;
  if (c < 0 || c >= o->ncl) return -1;
  work_t *w = work_alloc(o);
  double lp;
  double *post = malloc(sizeof(double) * o->sum_card);
  int st = infer_one(o, w, ev, rescale, &lp, post);
  memcpy(table, w->psi[c], sizeof(double) * o->cl[c].size);
  *exponent = w->sc[c];
  free(post);
  work_free(o, w);
  return st;
}

typedef struct {
  const orc_t *o;
  int ncases, tid, nthreads, rescale;
  const int *ev;
  double *log_pe, *post;
  int *status;
} job_t;

static void *batch_worker(void *arg) {
  job_t *j = arg;
  work_t *w = work_alloc(j->o);
  for (int i = j->tid; i < j->ncases; i += j->nthreads)
    j->status[i] = infer_one(j->o, w, j->ev + (size_t)i * j->o->n, j->rescale,
                             j->log_pe + i, j->post + (size_t)i * j->o->sum_card);
  work_free(j->o, w);
  return NULL;
}

/* Independent cases on nthreads threads, one case per thread at a time. */
int orc_infer_batch(void *h, int ncases, const int *ev, int rescale, double *log_pe,
                    double *post, int *status, int nthreads) {
  orc_t *o = h;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > ncases) nthreads = ncases > 0 ? ncases : 1;
  pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
  job_t *jobs = malloc(sizeof(job_t) * nthreads);
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = (job_t){o, ncases, t, nthreads, rescale, ev, log_pe, post, status};
    if (nthreads == 1) batch_worker(&jobs[t]);
    else pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
  }
  if (nthreads > 1)
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(th);
  free(jobs);
  return 0;
}
