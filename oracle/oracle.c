/*
 * CPU oracle for the particle-in-tree (PIT) / particle-in-dual-tree (PIDT)
 * particle step of Weinzierl, Verleye, Henri, Roose, "Two Particle-in-Grid
 * Realisations on Spacetrees" (arXiv:1508.02435).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant generator with the CUDA path; it is plain, serial,
 * double precision C (plus an FP32 mirror of the split-precision arithmetic)
 * written for readability, not speed.  Compile with -ffp-contract=off and
 * without -ffast-math: every floating point operation below is one IEEE
 * operation in program order.
 *
 * What it computes, with the passage each part follows:
 *   - k = 3 spacetree from level-order refinement flags (Section 4, cells,
 *     levels, leaves; children split 3 times per axis).
 *   - PIT owner: the leaf covering a particle position -- the end state of the
 *     lifts and drops of Algorithm 1 (Theorem 1).
 *   - PIDT owner: the vertex whose dual cell covers the position, on the level
 *     of the leaf covering it -- the end state of Algorithms 2-3 (Theorem 2,
 *     Section 4.2 "vertex holds the particles closer to it than to any other").
 *   - Charge deposit rho = sum_i R(x_i) with d-linear R on the 2^d vertices of
 *     the covering leaf (Section 3, item 1), hanging vertices constrained.
 *   - L(V) = rho with L the (negative) Laplacian in d-linear finite elements,
 *     a fixed number of damped Jacobi sweeps (Section 3, item 2).
 *   - E = -grad V at the vertices and the gather E_i = R^T(x_i) E (item 3).
 *   - Leapfrog push d_t v = (q/m) E, d_t x = v (item 4), periodic wrap.
 *   - Re-binning into buckets: stable by (new key, old storage index).
 *   - Re-refinement by the particles-per-cell criterion (Section 6 setup).
 *
 * Readings where the paper is silent are listed in the repository design
 * notes; the ones that change results are repeated next to the code.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

/* Positions are quantised once onto 2*3^18 integer steps per axis: every cell
 * face and every dual-cell face of levels 0..18 is then an exact integer, so
 * all containment decisions are integer comparisons (reading: faces belong to
 * the upper cell, cells and dual cells are half-open [lo, hi)). */
#define OR_QSCALE 774840978.0
#define OR_QSTEPS 774840978LL
#define OR_MAXLEV 18

static int64_t p3(int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= 3;
  return r;
}

/* ------------------------------------------------------------------------ */
/* Tree                                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t n;
  int64_t cap;
  int32_t *vid;
  double *w;
} explist;

typedef struct ortree {
  int d, nch, ncorner, depth;
  int64_t n_nodes, n_leaves;
  int32_t *level;   /* per node */
  int64_t *coords;  /* per node, 3 entries (unused axes 0) */
  int32_t *child0;  /* first child node or -1 */
  int32_t *leaf_id; /* dense leaf id in depth-first order or -1 */
  int32_t *leaf_node;

  /* finite element grid, built on demand */
  int grid_ready;
  int64_t M;          /* 3^depth grid points per axis at the finest level */
  int64_t n_vert;     /* non-hanging grid points */
  int64_t *vert_key;  /* sorted row-major keys (x fastest) at level depth */
  int64_t *cexp_ptr;  /* per leaf corner (leaf*ncorner + a): expansion range */
  int32_t *cexp_vid;
  double *cexp_w;
  double *ion_load;   /* integral of each vertex hat function */
  double *diag;       /* diagonal of the constrained stiffness matrix */
  int64_t *direct_cnt;/* leaves that have the vertex as an unconstrained corner */

  /* PIDT vertices: (level, j) of every leaf corner, sorted by (level, row-major j) */
  int pidt_ready;
  int64_t n_pv;
  int32_t *pv_level;
  int64_t *pv_j;      /* 3 entries per vertex */
  int32_t *corner_pv; /* per leaf corner: PIDT vertex id */
} ortree;

static void tree_free_grid(ortree *t) {
  free(t->vert_key); free(t->cexp_ptr); free(t->cexp_vid); free(t->cexp_w);
  free(t->ion_load); free(t->diag); free(t->direct_cnt);
  t->vert_key = NULL; t->cexp_ptr = NULL; t->cexp_vid = NULL; t->cexp_w = NULL;
  t->ion_load = NULL; t->diag = NULL; t->direct_cnt = NULL;
  free(t->pv_level); free(t->pv_j); free(t->corner_pv);
  t->pv_level = NULL; t->pv_j = NULL; t->corner_pv = NULL;
  t->grid_ready = 0; t->pidt_ready = 0;
}

OR_API void or_tree_free(ortree *t) {
  if (!t) return;
  tree_free_grid(t);
  free(t->level); free(t->coords); free(t->child0); free(t->leaf_id); free(t->leaf_node);
  free(t);
}

/* Depth-first pre-order numbering of the leaves, children in digit order. */
static void number_leaves(ortree *t) {
  int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * (size_t)(t->n_nodes + 1));
  int64_t sp = 0, next = 0;
  stack[sp++] = 0;
  while (sp > 0) {
    int32_t nd = stack[--sp];
    if (t->child0[nd] < 0) {
      t->leaf_id[nd] = (int32_t)next;
      t->leaf_node[next] = nd;
      ++next;
    } else {
      for (int c = t->nch - 1; c >= 0; --c) stack[sp++] = t->child0[nd] + c;
    }
  }
  free(stack);
}

/* Returns NULL and sets *err when the flags do not describe a k=3 tree:
 * -1 wrong d, -2 flag count does not match the implied node count,
 * -3 deeper than level 18, -4 allocation failure. */
OR_API ortree *or_tree_new(int d, int64_t n_flags, const uint8_t *flags, int *err) {
  *err = 0;
  if (d != 2 && d != 3) { *err = -1; return NULL; }
  if (n_flags < 1) { *err = -2; return NULL; }
  ortree *t = (ortree *)calloc(1, sizeof(ortree));
  t->d = d; t->nch = (int)p3(d); t->ncorner = 1 << d;
  t->n_nodes = n_flags;
  t->level = (int32_t *)malloc(sizeof(int32_t) * n_flags);
  t->coords = (int64_t *)calloc((size_t)n_flags * 3, sizeof(int64_t));
  t->child0 = (int32_t *)malloc(sizeof(int32_t) * n_flags);
  t->leaf_id = (int32_t *)malloc(sizeof(int32_t) * n_flags);
  t->leaf_node = (int32_t *)malloc(sizeof(int32_t) * n_flags);
  if (!t->level || !t->coords || !t->child0 || !t->leaf_id || !t->leaf_node) {
    or_tree_free(t); *err = -4; return NULL;
  }
  t->level[0] = 0;
  int64_t next = 1, leaves = 0;
  int depth = 0;
  for (int64_t i = 0; i < n_flags; ++i) {
    if (i >= next) { or_tree_free(t); *err = -2; return NULL; }
    t->leaf_id[i] = -1;
    if (flags[i]) {
      if (t->level[i] + 1 > OR_MAXLEV) { or_tree_free(t); *err = -3; return NULL; }
      if (next + t->nch > n_flags) { or_tree_free(t); *err = -2; return NULL; }
      t->child0[i] = (int32_t)next;
      for (int c = 0; c < t->nch; ++c) {
        int64_t k = next + c;
        t->level[k] = t->level[i] + 1;
        for (int a = 0; a < d; ++a)
          t->coords[k * 3 + a] = 3 * t->coords[i * 3 + a] + (c / p3(a)) % 3;
        if (t->level[k] > depth) depth = t->level[k];
      }
      next += t->nch;
    } else {
      t->child0[i] = -1;
      ++leaves;
    }
  }
  if (next != n_flags) { or_tree_free(t); *err = -2; return NULL; }
  t->n_leaves = leaves;
  t->depth = depth;
  number_leaves(t);
  return t;
}

OR_API int64_t or_n_leaves(const ortree *t) { return t->n_leaves; }
OR_API int or_depth(const ortree *t) { return t->depth; }

/* Leaf table in leaf order: level and integer coordinates (d per leaf). */
OR_API void or_leaf_info(const ortree *t, int32_t *level, int64_t *coords) {
  for (int64_t l = 0; l < t->n_leaves; ++l) {
    int32_t nd = t->leaf_node[l];
    level[l] = t->level[nd];
    for (int a = 0; a < t->d; ++a) coords[l * t->d + a] = t->coords[nd * 3 + a];
  }
}

/* ------------------------------------------------------------------------ */
/* Owners (keys)                                                             */
/* ------------------------------------------------------------------------ */

/* Wrap into [0,1) (periodic domain) and quantise: Q = floor(RN(x * 2*3^18)). */
static double wrap01(double x) {
  double y = x - floor(x);
  if (y >= 1.0) y = 0.0;
  return y;
}

static int64_t quantise(double x) {
  double y = wrap01(x);
  double s = y * OR_QSCALE;
  int64_t q = (int64_t)floor(s);
  if (q < 0) q = 0;
  if (q > OR_QSTEPS - 1) q = OR_QSTEPS - 1;
  return q;
}

/* Descend from the root, at each refined cell choosing the child whose
 * closure-open box contains Q: the chain of drops of Algorithm 1.  Returns the
 * covering leaf's node. */
static int32_t descend_q(const ortree *t, const int64_t Q[3]) {
  int32_t nd = 0;
  while (t->child0[nd] >= 0) {
    int m = t->level[nd] + 1;
    int64_t step = 2 * p3(OR_MAXLEV - m);
    int digit = 0;
    for (int a = 0; a < t->d; ++a) digit += (int)(((Q[a] / step) % 3) * p3(a));
    nd = t->child0[nd] + digit;
  }
  return nd;
}

/* a1: PIT owner leaf (leaf order id) for every particle; x is [d][n]. */
OR_API void or_pit_owner(const ortree *t, int64_t n, const double *x, int32_t *leaf) {
  for (int64_t p = 0; p < n; ++p) {
    int64_t Q[3] = {0, 0, 0};
    for (int a = 0; a < t->d; ++a) Q[a] = quantise(x[a * n + p]);
    leaf[p] = t->leaf_id[descend_q(t, Q)];
  }
}

/* Corner of the covering leaf whose dual cell holds Q: per axis 1 iff Q lies
 * in the upper half of the leaf (the dual-cell face through the leaf centre
 * belongs to the upper vertex). */
static int pidt_corner(const ortree *t, int32_t nd, const int64_t Q[3]) {
  int lev = t->level[nd];
  int64_t half = p3(OR_MAXLEV - lev);
  int a_idx = 0;
  for (int a = 0; a < t->d; ++a) {
    int64_t rel = Q[a] - t->coords[nd * 3 + a] * 2 * half;
    if (rel >= half) a_idx |= 1 << a;
  }
  return a_idx;
}

/* a2: PIDT owner vertex (level, j) for every particle; j is [d][n].
 * Reading of Algorithms 2-3: drops happen in enterCell of every refined cell
 * that contains the particle, into the child-level vertex whose dual cell
 * holds it; the move happens in the leaf.  So the owner sits on the level of
 * the covering leaf, at the leaf corner nearest to the particle. */
OR_API void or_pidt_owner(const ortree *t, int64_t n, const double *x, int32_t *vlevel,
                          int64_t *vj) {
  for (int64_t p = 0; p < n; ++p) {
    int64_t Q[3] = {0, 0, 0};
    for (int a = 0; a < t->d; ++a) Q[a] = quantise(x[a * n + p]);
    int32_t nd = descend_q(t, Q);
    int lev = t->level[nd];
    int64_t half = p3(OR_MAXLEV - lev), per = p3(lev);
    vlevel[p] = lev;
    for (int a = 0; a < t->d; ++a) vj[a * n + p] = ((Q[a] + half) / (2 * half)) % per;
  }
}

/* ------------------------------------------------------------------------ */
/* Finite element grid with hanging-vertex constraints                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t cap, n;
  int64_t *key;
  int32_t *val;
} hmap;

static void hm_init(hmap *h, int64_t expect) {
  int64_t cap = 1024;
  while (cap < 2 * expect + 16) cap <<= 1;
  h->cap = cap; h->n = 0;
  h->key = (int64_t *)malloc(sizeof(int64_t) * cap);
  h->val = (int32_t *)malloc(sizeof(int32_t) * cap);
  for (int64_t i = 0; i < cap; ++i) h->key[i] = -1;
}
static void hm_free(hmap *h) { free(h->key); free(h->val); }
static uint64_t hm_hash(int64_t k) {
  uint64_t x = (uint64_t)k;
  x ^= x >> 33; x *= 0xff51afd7ed558ccdULL; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL; x ^= x >> 33;
  return x;
}
/* returns slot; *found tells whether the key was present */
static int64_t hm_slot(const hmap *h, int64_t k, int *found) {
  uint64_t i = hm_hash(k) & (uint64_t)(h->cap - 1);
  while (h->key[i] != -1 && h->key[i] != k) i = (i + 1) & (uint64_t)(h->cap - 1);
  *found = h->key[i] == k;
  return (int64_t)i;
}
static void hm_grow(hmap *h) {
  hmap g;
  hm_init(&g, h->cap);
  for (int64_t i = 0; i < h->cap; ++i)
    if (h->key[i] != -1) {
      int f;
      int64_t s = hm_slot(&g, h->key[i], &f);
      g.key[s] = h->key[i]; g.val[s] = h->val[i]; g.n++;
    }
  hm_free(h);
  *h = g;
}

typedef struct {
  int state;        /* 0 unknown, 1 in progress, 2 done */
  int hanging;
  explist ex;       /* expansion onto point keys (vid holds point index) */
} ptinfo;

typedef struct {
  ortree *t;
  hmap map;
  int64_t n_pts, cap_pts;
  int64_t *pkey;
  ptinfo *info;
} gridbuild;

static int64_t point_key(const ortree *t, const int64_t p[3]) {
  int64_t k = 0, m = 1;
  for (int a = 0; a < t->d; ++a) { k += p[a] * m; m *= t->M; }
  return k;
}

static int64_t gb_point(gridbuild *g, const int64_t p[3]) {
  int64_t k = point_key(g->t, p);
  int f;
  if (2 * (g->map.n + 1) > g->map.cap) hm_grow(&g->map);
  int64_t s = hm_slot(&g->map, k, &f);
  if (f) return g->map.val[s];
  if (g->n_pts == g->cap_pts) {
    g->cap_pts = g->cap_pts ? 2 * g->cap_pts : 1024;
    g->pkey = (int64_t *)realloc(g->pkey, sizeof(int64_t) * g->cap_pts);
    g->info = (ptinfo *)realloc(g->info, sizeof(ptinfo) * g->cap_pts);
  }
  int64_t id = g->n_pts++;
  g->pkey[id] = k;
  memset(&g->info[id], 0, sizeof(ptinfo));
  g->map.key[s] = k; g->map.val[s] = (int32_t)id; g->map.n++;
  return id;
}

static void ex_add(explist *e, int32_t vid, double w) {
  for (int64_t i = 0; i < e->n; ++i)
    if (e->vid[i] == vid) { e->w[i] += w; return; }
  if (e->n == e->cap) {
    e->cap = e->cap ? 2 * e->cap : 4;
    e->vid = (int32_t *)realloc(e->vid, sizeof(int32_t) * e->cap);
    e->w = (double *)realloc(e->w, sizeof(double) * e->cap);
  }
  e->vid[e->n] = vid; e->w[e->n] = w; e->n++;
}

/* Classify grid point id and build its expansion onto non-hanging points.
 * A grid point is non-hanging iff it is a corner of the coarsest leaf whose
 * closure contains it; otherwise its value is the d-linear interpolant of
 * that leaf's corners (continuity across the coarse face), recursively. */
static void gb_resolve(gridbuild *g, int64_t id) {
  if (g->info[id].state == 2) return;
  ortree *t = g->t;
  int d = t->d;
  int64_t key = g->pkey[id], p[3] = {0, 0, 0};
  for (int a = 0; a < d; ++a) { p[a] = key % t->M; key /= t->M; }
  int64_t qs = 2 * p3(OR_MAXLEV - t->depth);
  int32_t best = -1;
  for (int e = 0; e < (1 << d); ++e) {
    int64_t Q[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      int64_t q = p[a] * qs - (((e >> a) & 1) ? 0 : 1);
      if (q < 0) q += OR_QSTEPS;
      Q[a] = q;
    }
    int32_t nd = descend_q(t, Q);
    if (best < 0 || t->level[nd] < t->level[best]) best = nd;
  }
  int lev = t->level[best];
  int64_t s = p3(t->depth - lev);
  int64_t r[3] = {0, 0, 0};
  int is_corner = 1;
  for (int a = 0; a < d; ++a) {
    int64_t rr = p[a] - t->coords[best * 3 + a] * s;
    if (rr < 0) rr += t->M;
    r[a] = rr;
    if (rr != 0 && rr != s) is_corner = 0;
  }
  g->info[id].state = 1;
  if (is_corner) {
    g->info[id].hanging = 0;
    ex_add(&g->info[id].ex, (int32_t)id, 1.0);
  } else {
    g->info[id].hanging = 1;
    for (int e = 0; e < (1 << d); ++e) {
      double w = 1.0;
      int64_t q[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) {
        int ea = (e >> a) & 1;
        double f = ea ? (double)r[a] / (double)s : (double)(s - r[a]) / (double)s;
        w = w * f;
        q[a] = ((t->coords[best * 3 + a] + ea) * s) % t->M;
      }
      if (w == 0.0) continue;
      int64_t cid = gb_point(g, q);
      gb_resolve(g, cid);
      ptinfo *ci = &g->info[cid];
      for (int64_t i = 0; i < ci->ex.n; ++i) ex_add(&g->info[id].ex, ci->ex.vid[i], w * ci->ex.w[i]);
    }
  }
  g->info[id].state = 2;
}

static int cmp_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x > y) - (x < y);
}

static int64_t find_sorted(const int64_t *arr, int64_t n, int64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (arr[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < n && arr[lo] == key) ? lo : -1;
}

/* Reference element stiffness of -Laplace for d-linear elements on the unit
 * cell, by the number of axes in which corners e and f differ. */
static double kref(int d, int e, int f) {
  int diff = __builtin_popcount((unsigned)(e ^ f));
  if (d == 2) {
    static const double k2[3] = {4.0 / 6.0, -1.0 / 6.0, -2.0 / 6.0};
    return k2[diff];
  }
  static const double k3[4] = {4.0 / 12.0, 0.0, -1.0 / 12.0, -1.0 / 12.0};
  return k3[diff];
}

static double leaf_h(const ortree *t, int64_t l) { return 1.0 / (double)p3(t->level[t->leaf_node[l]]); }

OR_API int or_grid_build(ortree *t) {
  if (t->grid_ready) return 0;
  if (t->depth > 12) return -1;
  int d = t->d, nc = t->ncorner;
  t->M = p3(t->depth);
  gridbuild g;
  memset(&g, 0, sizeof(g));
  g.t = t;
  hm_init(&g.map, t->n_leaves * 2);
  int64_t nlc = t->n_leaves * nc;
  int64_t *corner_pt = (int64_t *)malloc(sizeof(int64_t) * nlc);
  for (int64_t l = 0; l < t->n_leaves; ++l) {
    int32_t nd = t->leaf_node[l];
    int64_t s = p3(t->depth - t->level[nd]);
    for (int e = 0; e < nc; ++e) {
      int64_t q[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) q[a] = ((t->coords[nd * 3 + a] + ((e >> a) & 1)) * s) % t->M;
      corner_pt[l * nc + e] = gb_point(&g, q);
    }
  }
  for (int64_t l = 0; l < nlc; ++l) gb_resolve(&g, corner_pt[l]);
  /* number the non-hanging points by row-major key */
  int64_t nv = 0;
  for (int64_t i = 0; i < g.n_pts; ++i) nv += !g.info[i].hanging;
  t->n_vert = nv;
  t->vert_key = (int64_t *)malloc(sizeof(int64_t) * (nv ? nv : 1));
  nv = 0;
  for (int64_t i = 0; i < g.n_pts; ++i) if (!g.info[i].hanging) t->vert_key[nv++] = g.pkey[i];
  qsort(t->vert_key, (size_t)nv, sizeof(int64_t), cmp_i64);
  /* leaf corner expansions onto vertex ids, sorted by vertex id */
  t->cexp_ptr = (int64_t *)malloc(sizeof(int64_t) * (nlc + 1));
  int64_t tot = 0;
  for (int64_t i = 0; i < nlc; ++i) tot += g.info[corner_pt[i]].ex.n;
  t->cexp_vid = (int32_t *)malloc(sizeof(int32_t) * (tot ? tot : 1));
  t->cexp_w = (double *)malloc(sizeof(double) * (tot ? tot : 1));
  int64_t k = 0;
  for (int64_t i = 0; i < nlc; ++i) {
    t->cexp_ptr[i] = k;
    explist *ex = &g.info[corner_pt[i]].ex;
    int64_t k0 = k;
    for (int64_t j = 0; j < ex->n; ++j) {
      int32_t v = (int32_t)find_sorted(t->vert_key, t->n_vert, g.pkey[ex->vid[j]]);
      double w = ex->w[j];
      /* insertion by vertex id */
      int64_t pos = k;
      while (pos > k0 && t->cexp_vid[pos - 1] > v) {
        t->cexp_vid[pos] = t->cexp_vid[pos - 1]; t->cexp_w[pos] = t->cexp_w[pos - 1]; --pos;
      }
      t->cexp_vid[pos] = v; t->cexp_w[pos] = w;
      ++k;
    }
  }
  t->cexp_ptr[nlc] = k;
  /* integral of each hat function, direct-corner counts, stiffness diagonal:
   * all accumulated in leaf order, corner order, expansion order */
  t->ion_load = (double *)calloc((size_t)(t->n_vert ? t->n_vert : 1), sizeof(double));
  t->diag = (double *)calloc((size_t)(t->n_vert ? t->n_vert : 1), sizeof(double));
  t->direct_cnt = (int64_t *)calloc((size_t)(t->n_vert ? t->n_vert : 1), sizeof(int64_t));
  for (int64_t l = 0; l < t->n_leaves; ++l) {
    double h = leaf_h(t, l);
    double vol = 1.0;
    for (int a = 0; a < d; ++a) vol = vol * h;
    double cint = vol / (double)nc;
    double hs = d == 2 ? 1.0 : h;
    for (int e = 0; e < nc; ++e) {
      int64_t i = l * nc + e;
      for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j)
        t->ion_load[t->cexp_vid[j]] += t->cexp_w[j] * cint;
      if (t->cexp_ptr[i + 1] - t->cexp_ptr[i] == 1 && !g.info[corner_pt[i]].hanging)
        t->direct_cnt[t->cexp_vid[t->cexp_ptr[i]]] += 1;
      for (int f = 0; f < nc; ++f) {
        int64_t jf = l * nc + f;
        double kef = kref(d, e, f) * hs;
        for (int64_t a1 = t->cexp_ptr[i]; a1 < t->cexp_ptr[i + 1]; ++a1)
          for (int64_t a2 = t->cexp_ptr[jf]; a2 < t->cexp_ptr[jf + 1]; ++a2)
            if (t->cexp_vid[a1] == t->cexp_vid[a2])
              t->diag[t->cexp_vid[a1]] += kef * t->cexp_w[a1] * t->cexp_w[a2];
      }
    }
  }
  for (int64_t i = 0; i < g.n_pts; ++i) { free(g.info[i].ex.vid); free(g.info[i].ex.w); }
  free(g.info); free(g.pkey); hm_free(&g.map); free(corner_pt);
  t->grid_ready = 1;
  return 0;
}

OR_API int64_t or_n_vertices(ortree *t) {
  if (or_grid_build(t)) return -1;
  return t->n_vert;
}

/* Vertex positions in units of 3^-depth, [d][n_vert]. */
OR_API void or_vertex_pos(ortree *t, int64_t *pos) {
  or_grid_build(t);
  for (int64_t v = 0; v < t->n_vert; ++v) {
    int64_t k = t->vert_key[v];
    for (int a = 0; a < t->d; ++a) { pos[a * t->n_vert + v] = k % t->M; k /= t->M; }
  }
}

OR_API void or_vertex_aux(ortree *t, double *ion_load, double *diag) {
  or_grid_build(t);
  memcpy(ion_load, t->ion_load, sizeof(double) * t->n_vert);
  memcpy(diag, t->diag, sizeof(double) * t->n_vert);
}

/* Number of expansion entries and the expansion table itself (for tests). */
OR_API int64_t or_corner_expansion(ortree *t, int64_t *ptr, int32_t *vid, double *w) {
  or_grid_build(t);
  int64_t nlc = t->n_leaves * t->ncorner;
  if (ptr) {
    memcpy(ptr, t->cexp_ptr, sizeof(int64_t) * (nlc + 1));
    memcpy(vid, t->cexp_vid, sizeof(int32_t) * t->cexp_ptr[nlc]);
    memcpy(w, t->cexp_w, sizeof(double) * t->cexp_ptr[nlc]);
  }
  return t->cexp_ptr[nlc];
}

/* ------------------------------------------------------------------------ */
/* PIDT vertex table                                                          */
/* ------------------------------------------------------------------------ */

typedef struct { int64_t lev, rm, l; int a; } pvrec;
static int cmp_pv(const void *x, const void *y) {
  const pvrec *a = (const pvrec *)x, *b = (const pvrec *)y;
  if (a->lev != b->lev) return (a->lev > b->lev) - (a->lev < b->lev);
  if (a->rm != b->rm) return (a->rm > b->rm) - (a->rm < b->rm);
  if (a->l != b->l) return (a->l > b->l) - (a->l < b->l);
  return (a->a > b->a) - (a->a < b->a);
}

/* Owner vertices of PIDT are (level, j) pairs of leaf corners on the leaf's
 * level; they are ordered by (level, row-major j).  Hanging corners own
 * particles too: the drop of Algorithm 2 reaches them. */
OR_API int or_pidt_build(ortree *t) {
  if (t->pidt_ready) return 0;
  int d = t->d, nc = t->ncorner;
  int64_t nlc = t->n_leaves * nc;
  pvrec *r = (pvrec *)malloc(sizeof(pvrec) * (nlc ? nlc : 1));
  for (int64_t l = 0; l < t->n_leaves; ++l) {
    int32_t nd = t->leaf_node[l];
    int lev = t->level[nd];
    int64_t per = p3(lev);
    for (int e = 0; e < nc; ++e) {
      int64_t rm = 0, m = 1;
      for (int a = 0; a < d; ++a) {
        int64_t j = (t->coords[nd * 3 + a] + ((e >> a) & 1)) % per;
        rm += j * m; m *= per;
      }
      pvrec *q = &r[l * nc + e];
      q->lev = lev; q->rm = rm; q->l = l; q->a = e;
    }
  }
  qsort(r, (size_t)nlc, sizeof(pvrec), cmp_pv);
  t->corner_pv = (int32_t *)malloc(sizeof(int32_t) * (nlc ? nlc : 1));
  t->pv_level = (int32_t *)malloc(sizeof(int32_t) * (nlc ? nlc : 1));
  t->pv_j = (int64_t *)malloc(sizeof(int64_t) * 3 * (nlc ? nlc : 1));
  int64_t nv = 0;
  for (int64_t i = 0; i < nlc; ++i) {
    if (i == 0 || r[i].lev != r[i - 1].lev || r[i].rm != r[i - 1].rm) {
      int64_t per = p3((int)r[i].lev), rm = r[i].rm;
      t->pv_level[nv] = (int32_t)r[i].lev;
      for (int a = 0; a < 3; ++a) { t->pv_j[nv * 3 + a] = a < d ? rm % per : 0; if (a < d) rm /= per; }
      ++nv;
    }
    t->corner_pv[r[i].l * nc + r[i].a] = (int32_t)(nv - 1);
  }
  t->n_pv = nv;
  free(r);
  t->pidt_ready = 1;
  return 0;
}

OR_API int64_t or_n_pidt_vertices(ortree *t) { or_pidt_build(t); return t->n_pv; }

OR_API void or_pidt_vertex_info(ortree *t, int32_t *level, int64_t *j) {
  or_pidt_build(t);
  for (int64_t v = 0; v < t->n_pv; ++v) {
    level[v] = t->pv_level[v];
    for (int a = 0; a < t->d; ++a) j[v * t->d + a] = t->pv_j[v * 3 + a];
  }
}

/* ------------------------------------------------------------------------ */
/* FP64 particle step                                                        */
/* ------------------------------------------------------------------------ */

enum { OR_PIT = 0, OR_PIDT = 1 };

/* Per particle: covering leaf, local coordinates t in [0,1]^d, PIDT corner. */
static void locate64(const ortree *t, const double *x, int64_t n, int64_t p, int32_t *leaf,
                     double tl[3], int *corner) {
  int64_t Q[3] = {0, 0, 0};
  for (int a = 0; a < t->d; ++a) Q[a] = quantise(x[a * n + p]);
  int32_t nd = descend_q(t, Q);
  *leaf = t->leaf_id[nd];
  double s = (double)p3(t->level[nd]);
  for (int a = 0; a < t->d; ++a) {
    double y = wrap01(x[a * n + p]);
    double u = y * s - (double)t->coords[nd * 3 + a];
    if (u < 0.0) u = 0.0;
    if (u > 1.0) u = 1.0;
    tl[a] = u;
  }
  *corner = pidt_corner(t, nd, Q);
}

/* d-linear shape function of corner e at local coordinates tl. */
static double shape64(int d, int e, const double tl[3]) {
  double w = 1.0;
  for (int a = 0; a < d; ++a) {
    double f = ((e >> a) & 1) ? tl[a] : 1.0 - tl[a];
    w = w * f;
  }
  return w;
}

/* Bucket key of a particle: PIT = leaf id; PIDT = owner vertex id * 2^d + the
 * quadrant of the covering leaf seen from that vertex (complement of corner). */
static int64_t key_of(const ortree *t, int scheme, int32_t leaf, int corner) {
  if (scheme == OR_PIT) return leaf;
  int nc = t->ncorner;
  return (int64_t)t->corner_pv[(int64_t)leaf * nc + corner] * nc + (nc - 1 - corner);
}

OR_API int64_t or_n_keys(ortree *t, int scheme) {
  if (scheme == OR_PIT) return t->n_leaves;
  or_pidt_build(t);
  return t->n_pv * t->ncorner;
}

OR_API void or_keys64(ortree *t, int scheme, int64_t n, const double *x, int64_t *key) {
  if (scheme == OR_PIDT) or_pidt_build(t);
  for (int64_t p = 0; p < n; ++p) {
    int32_t leaf; double tl[3]; int c;
    locate64(t, x, n, p, &leaf, tl, &c);
    key[p] = key_of(t, scheme, leaf, c);
  }
}

/* Stable counting sort: perm[i] = storage index of the i-th particle in the
 * new order, start = bucket offsets (n_keys + 1). */
OR_API void or_stable_bucket(int64_t n, const int64_t *key, int64_t n_keys, int64_t *start,
                             int64_t *perm) {
  memset(start, 0, sizeof(int64_t) * (n_keys + 1));
  for (int64_t p = 0; p < n; ++p) start[key[p] + 1]++;
  for (int64_t k = 0; k < n_keys; ++k) start[k + 1] += start[k];
  int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (n_keys ? n_keys : 1));
  memcpy(cur, start, sizeof(int64_t) * n_keys);
  for (int64_t p = 0; p < n; ++p) perm[cur[key[p]]++] = p;
  free(cur);
}

/* a7: deposit.  For every leaf, corner partial sums of the shape functions in
 * storage order (PIDT: the leaf's particles grouped by owning corner, corner
 * order, storage order within); every vertex then adds w * partial over the
 * leaf corners that expand onto it, in leaf, corner, expansion order.
 * Q_v = q * S_v + ion * integral(phi_v).  Returns the FP64 sum of all Q_v. */
OR_API double or_deposit64(ortree *t, int scheme, int64_t n, const double *x, double q,
                           double ion, double *Qv) {
  or_grid_build(t);
  int d = t->d, nc = t->ncorner;
  int64_t nlc = t->n_leaves * nc;
  int32_t *leaf = (int32_t *)malloc(sizeof(int32_t) * (n ? n : 1));
  int *corner = (int *)malloc(sizeof(int) * (n ? n : 1));
  double *tl = (double *)malloc(sizeof(double) * 3 * (n ? n : 1));
  for (int64_t p = 0; p < n; ++p) locate64(t, x, n, p, &leaf[p], &tl[3 * p], &corner[p]);
  /* group particles by (leaf, sub-bucket corner), stable in storage order */
  int64_t *gk = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
  for (int64_t p = 0; p < n; ++p) gk[p] = (int64_t)leaf[p] * nc + (scheme == OR_PIDT ? corner[p] : 0);
  int64_t *gs = (int64_t *)malloc(sizeof(int64_t) * (nlc + 1));
  int64_t *gp = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
  or_stable_bucket(n, gk, nlc, gs, gp);
  double *part = (double *)calloc((size_t)(nlc ? nlc : 1), sizeof(double));
  for (int64_t i = 0; i < n; ++i) {
    int64_t p = gp[i];
    for (int e = 0; e < nc; ++e) part[(int64_t)leaf[p] * nc + e] += shape64(d, e, &tl[3 * p]);
  }
  double *S = (double *)calloc((size_t)t->n_vert, sizeof(double));
  for (int64_t i = 0; i < nlc; ++i)
    for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j)
      S[t->cexp_vid[j]] += t->cexp_w[j] * part[i];
  double tot = 0.0;
  for (int64_t v = 0; v < t->n_vert; ++v) {
    Qv[v] = q * S[v] + ion * t->ion_load[v];
    tot += Qv[v];
  }
  free(S); free(part); free(gp); free(gs); free(gk); free(tl); free(corner); free(leaf);
  return tot;
}

/* y = A V with A the constrained d-linear stiffness matrix of -Laplace,
 * assembled leaf by leaf. */
static void apply64(const ortree *t, const double *V, double *y) {
  int d = t->d, nc = t->ncorner;
  memset(y, 0, sizeof(double) * t->n_vert);
  double vc[8], yc[8];
  for (int64_t l = 0; l < t->n_leaves; ++l) {
    double hs = d == 2 ? 1.0 : leaf_h(t, l);
    for (int e = 0; e < nc; ++e) {
      int64_t i = l * nc + e;
      double s = 0.0;
      for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j) s += t->cexp_w[j] * V[t->cexp_vid[j]];
      vc[e] = s;
    }
    for (int e = 0; e < nc; ++e) {
      double s = 0.0;
      for (int f = 0; f < nc; ++f) s += (kref(d, e, f) * hs) * vc[f];
      yc[e] = s;
    }
    for (int e = 0; e < nc; ++e) {
      int64_t i = l * nc + e;
      for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j) y[t->cexp_vid[j]] += t->cexp_w[j] * yc[e];
    }
  }
}

OR_API void or_apply64(ortree *t, const double *V, double *y) { or_grid_build(t); apply64(t, V, y); }

/* a8 (auxiliary): right-hand side b = Q - (sum Q) * integral(phi) (periodic
 * compatibility), then `sweeps` damped Jacobi sweeps
 * V <- V + omega (b - A V) / diag(A), warm-started from V.  Returns the
 * Euclidean norm of b - A V after the sweeps. */
OR_API double or_solve64(ortree *t, const double *Q, double *V, int sweeps, double omega) {
  or_grid_build(t);
  int64_t nv = t->n_vert;
  double tot = 0.0;
  for (int64_t v = 0; v < nv; ++v) tot += Q[v];
  double *b = (double *)malloc(sizeof(double) * nv);
  double *y = (double *)malloc(sizeof(double) * nv);
  for (int64_t v = 0; v < nv; ++v) b[v] = Q[v] - tot * t->ion_load[v];
  for (int it = 0; it < sweeps; ++it) {
    apply64(t, V, y);
    for (int64_t v = 0; v < nv; ++v) V[v] = V[v] + omega * (b[v] - y[v]) / t->diag[v];
  }
  apply64(t, V, y);
  double r2 = 0.0;
  for (int64_t v = 0; v < nv; ++v) { double r = b[v] - y[v]; r2 += r * r; }
  free(b); free(y);
  return sqrt(r2);
}

/* E = -grad V at the vertices: minus the mean, over the leaves that have the
 * vertex as an unconstrained corner, of the gradient of the leaf's d-linear
 * interpolant at that corner (on uniform grids: central differences).
 * Ev is [d][n_vert]. */
OR_API void or_efield64(ortree *t, const double *V, double *Ev) {
  or_grid_build(t);
  int d = t->d, nc = t->ncorner;
  int64_t nv = t->n_vert;
  memset(Ev, 0, sizeof(double) * d * nv);
  double vc[8];
  for (int64_t l = 0; l < t->n_leaves; ++l) {
    double h = leaf_h(t, l);
    for (int e = 0; e < nc; ++e) {
      int64_t i = l * nc + e;
      double s = 0.0;
      for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j) s += t->cexp_w[j] * V[t->cexp_vid[j]];
      vc[e] = s;
    }
    for (int e = 0; e < nc; ++e) {
      int64_t i = l * nc + e;
      if (t->cexp_ptr[i + 1] - t->cexp_ptr[i] != 1 || t->cexp_w[t->cexp_ptr[i]] != 1.0) continue;
      int32_t v = t->cexp_vid[t->cexp_ptr[i]];
      for (int a = 0; a < d; ++a) {
        double g = (vc[e | (1 << a)] - vc[e & ~(1 << a)]) / h;
        Ev[a * nv + v] += g;
      }
    }
  }
  for (int64_t v = 0; v < nv; ++v) {
    double c = (double)t->direct_cnt[v];
    for (int a = 0; a < d; ++a) Ev[a * nv + v] = -(Ev[a * nv + v] / c);
  }
}

/* a3 + a4: gather E_i = sum_e phi_e(x_i) E(corner e) with hanging corners
 * interpolated, then the leapfrog kick and drift
 *   v <- v + (q/m dt) E_i,  x <- wrap(x + v dt)   (one rounding per operation). */
OR_API void or_push64(ortree *t, int64_t n, double *x, double *v, const double *Ev, double qm,
                      double dt) {
  or_grid_build(t);
  int d = t->d, nc = t->ncorner;
  int64_t nv = t->n_vert;
  double qmdt = qm * dt;
  for (int64_t p = 0; p < n; ++p) {
    int32_t leaf; double tl[3]; int c;
    locate64(t, x, n, p, &leaf, tl, &c);
    double E[3] = {0.0, 0.0, 0.0};
    for (int e = 0; e < nc; ++e) {
      int64_t i = (int64_t)leaf * nc + e;
      double w = shape64(d, e, tl);
      for (int a = 0; a < d; ++a) {
        double ec = 0.0;
        for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j) ec += t->cexp_w[j] * Ev[a * nv + t->cexp_vid[j]];
        E[a] += w * ec;
      }
    }
    for (int a = 0; a < d; ++a) {
      double vn = v[a * n + p] + qmdt * E[a];
      v[a * n + p] = vn;
      x[a * n + p] = wrap01(x[a * n + p] + vn * dt);
    }
  }
}

/* The particle-handling step of the paper's experiments (Section 6): no PDE
 * and no particle-grid interplay, every particle moves with its own velocity,
 * x <- x + RN(v dt), and either wraps (periodic, reflect = 0) or is reflected
 * at the walls of the unit box without any other change of its velocity
 * (reflect = 1).  Reading of the reflection for any number of wall hits:
 * y = x + v dt is folded into [0, 2) (y - 2 floor(y / 2), exact), and
 * y >= 1 becomes 2 - y (exact) with the velocity component negated (an odd
 * number of reflections); a particle that lands exactly on the far wall
 * (y == 1) is placed at the largest double below 1. */
static const double OR_ONE_MINUS64 = 0x1.fffffffffffffp-1;

static double fold64(double y, int *flip) {
  double m = y - 2.0 * floor(y * 0.5);
  *flip = 0;
  if (m >= 1.0) {
    m = 2.0 - m;
    *flip = 1;
    if (m >= 1.0) m = OR_ONE_MINUS64;
  }
  return m;
}

OR_API void or_move64(ortree *t, int64_t n, double *x, double *v, double dt, int reflect) {
  int d = t->d;
  for (int64_t p = 0; p < n; ++p)
    for (int a = 0; a < d; ++a) {
      double y = x[a * n + p] + v[a * n + p] * dt;
      if (reflect) {
        int flip;
        x[a * n + p] = fold64(y, &flip);
        if (flip) v[a * n + p] = -v[a * n + p];
      } else {
        x[a * n + p] = wrap01(y);
      }
    }
}

/* Only the gather (for tests): E at the particles, [d][n]. */
OR_API void or_gather64(ortree *t, int64_t n, const double *x, const double *Ev, double *Ep) {
  or_grid_build(t);
  int d = t->d, nc = t->ncorner;
  int64_t nv = t->n_vert;
  for (int64_t p = 0; p < n; ++p) {
    int32_t leaf; double tl[3]; int c;
    locate64(t, x, n, p, &leaf, tl, &c);
    double E[3] = {0.0, 0.0, 0.0};
    for (int e = 0; e < nc; ++e) {
      int64_t i = (int64_t)leaf * nc + e;
      double w = shape64(d, e, tl);
      for (int a = 0; a < d; ++a) {
        double ec = 0.0;
        for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j) ec += t->cexp_w[j] * Ev[a * nv + t->cexp_vid[j]];
        E[a] += w * ec;
      }
    }
    for (int a = 0; a < d; ++a) Ep[a * n + p] = E[a];
  }
}

/* ------------------------------------------------------------------------ */
/* FP32 split-precision mirror                                                */
/* ------------------------------------------------------------------------ */
/* State per particle: covering leaf + FP32 offset o in [0,1)^d in leaf-cell
 * units + FP32 velocity in domain units.  The leaf after a move is resolved
 * with integer arithmetic only:
 *   s_l = RN32(dt 3^l);  t = RN32(o + RN32(v s_l));  n = floor(t);  f = t - n;
 *   target integer cell c + n (mod 3^l) on the particle's level, then
 *   lift to level m: c' = I div 3^(l-m), o' = RN32(RN32(r + f) / 3^(l-m)),
 *   drop one level: u = RN32(3 f), digit = min(floor u, 2), f = u - digit;
 * an offset that rounds to 1 becomes the largest float below 1. */

static const float OR_ONE_MINUS = 0x1.fffffep-1f;

static float clamp_off(float f) {
  if (f < 0.0f) return 0.0f;
  if (f > OR_ONE_MINUS) return OR_ONE_MINUS;
  return f;
}

/* Resolve the leaf covering the integer cell I (level lev, already periodic)
 * plus fraction f.  Writes the new leaf node and offsets. */
static int32_t resolve32(const ortree *t, int lev, const int64_t I[3], const float f_in[3],
                         float o_out[3]) {
  int d = t->d;
  int32_t nd = 0;
  /* descend with the integer digits of I while the cell is refined and above lev */
  while (t->child0[nd] >= 0 && t->level[nd] < lev) {
    int m = t->level[nd] + 1;
    int64_t sh = p3(lev - m);
    int digit = 0;
    for (int a = 0; a < d; ++a) digit += (int)(((I[a] / sh) % 3) * p3(a));
    nd = t->child0[nd] + digit;
  }
  float f[3] = {f_in[0], f_in[1], f_in[2]};
  if (t->level[nd] < lev) {
    /* lift: the covering leaf is coarser than lev */
    int m = t->level[nd];
    int64_t sh = p3(lev - m);
    for (int a = 0; a < d; ++a) {
      int64_t r = I[a] % sh;
      float num = (float)r + f[a];
      o_out[a] = clamp_off(num / (float)sh);
    }
    return nd;
  }
  /* drops below lev, digits from the fraction */
  while (t->child0[nd] >= 0) {
    int digit = 0;
    for (int a = 0; a < d; ++a) {
      float u = 3.0f * f[a];
      int dg = (int)floorf(u);
      if (dg > 2) dg = 2;
      f[a] = clamp_off(u - (float)dg);
      digit += dg * (int)p3(a);
    }
    nd = t->child0[nd] + digit;
  }
  for (int a = 0; a < d; ++a) o_out[a] = clamp_off(f[a]);
  return nd;
}

/* Conversion of FP64 positions into the split state: leaf by the FP64 PIT
 * owner, o = RN32(clamp(RN64(x 3^l) - c)), v = RN32(v). */
OR_API void or_split_from64(ortree *t, int64_t n, const double *x, const double *v,
                            int32_t *leaf, float *o, float *vf) {
  int d = t->d;
  for (int64_t p = 0; p < n; ++p) {
    int64_t Q[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) Q[a] = quantise(x[a * n + p]);
    int32_t nd = descend_q(t, Q);
    leaf[p] = t->leaf_id[nd];
    double s = (double)p3(t->level[nd]);
    for (int a = 0; a < d; ++a) {
      double u = wrap01(x[a * n + p]) * s - (double)t->coords[nd * 3 + a];
      if (u < 0.0) u = 0.0;
      o[a * n + p] = clamp_off((float)u);
      vf[a * n + p] = (float)v[a * n + p];
    }
  }
}

/* Absolute positions (c + o) / 3^l in FP64. */
OR_API void or_split_to64(ortree *t, int64_t n, const int32_t *leaf, const float *o, double *x) {
  for (int64_t p = 0; p < n; ++p) {
    int32_t nd = t->leaf_node[leaf[p]];
    double s = (double)p3(t->level[nd]);
    for (int a = 0; a < t->d; ++a)
      x[a * n + p] = ((double)t->coords[nd * 3 + a] + (double)o[a * n + p]) / s;
  }
}

static float shape32(int d, int e, const float *o, int64_t n, int64_t p) {
  float w = 1.0f;
  for (int a = 0; a < d; ++a) {
    float oa = o[a * n + p];
    float f = ((e >> a) & 1) ? oa : 1.0f - oa;
    w = w * f;
  }
  return w;
}

static int corner32(int d, const float *o, int64_t n, int64_t p) {
  int c = 0;
  for (int a = 0; a < d; ++a) if (o[a * n + p] >= 0.5f) c |= 1 << a;
  return c;
}

OR_API void or_keys32(ortree *t, int scheme, int64_t n, const int32_t *leaf, const float *o,
                      int64_t *key) {
  if (scheme == OR_PIDT) or_pidt_build(t);
  for (int64_t p = 0; p < n; ++p) key[p] = key_of(t, scheme, leaf[p], corner32(t->d, o, n, p));
}

/* FP32 deposit with the same grouping and order as the FP64 one; the vertex
 * charges are FP32, the returned total is an FP64 sum of them. */
OR_API double or_deposit32(ortree *t, int scheme, int64_t n, const int32_t *leaf, const float *o,
                           float q, float ion, float *Qv) {
  or_grid_build(t);
  int d = t->d, nc = t->ncorner;
  int64_t nlc = t->n_leaves * nc;
  int64_t *gk = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
  for (int64_t p = 0; p < n; ++p) gk[p] = (int64_t)leaf[p] * nc + (scheme == OR_PIDT ? corner32(d, o, n, p) : 0);
  int64_t *gs = (int64_t *)malloc(sizeof(int64_t) * (nlc + 1));
  int64_t *gp = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
  or_stable_bucket(n, gk, nlc, gs, gp);
  float *part = (float *)calloc((size_t)(nlc ? nlc : 1), sizeof(float));
  for (int64_t i = 0; i < n; ++i) {
    int64_t p = gp[i];
    for (int e = 0; e < nc; ++e) part[(int64_t)leaf[p] * nc + e] += shape32(d, e, o, n, p);
  }
  float *S = (float *)calloc((size_t)t->n_vert, sizeof(float));
  for (int64_t i = 0; i < nlc; ++i)
    for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j)
      S[t->cexp_vid[j]] += (float)t->cexp_w[j] * part[i];
  double tot = 0.0;
  for (int64_t v = 0; v < t->n_vert; ++v) {
    Qv[v] = q * S[v] + ion * (float)t->ion_load[v];
    tot += (double)Qv[v];
  }
  free(S); free(part); free(gp); free(gs); free(gk);
  return tot;
}

static void apply32(const ortree *t, const float *V, float *y) {
  int d = t->d, nc = t->ncorner;
  memset(y, 0, sizeof(float) * t->n_vert);
  float vc[8], yc[8];
  for (int64_t l = 0; l < t->n_leaves; ++l) {
    float hs = d == 2 ? 1.0f : (float)leaf_h(t, l);
    for (int e = 0; e < nc; ++e) {
      int64_t i = l * nc + e;
      float s = 0.0f;
      for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j) s += (float)t->cexp_w[j] * V[t->cexp_vid[j]];
      vc[e] = s;
    }
    for (int e = 0; e < nc; ++e) {
      float s = 0.0f;
      for (int f = 0; f < nc; ++f) s += ((float)kref(d, e, f) * hs) * vc[f];
      yc[e] = s;
    }
    for (int e = 0; e < nc; ++e) {
      int64_t i = l * nc + e;
      for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j) y[t->cexp_vid[j]] += (float)t->cexp_w[j] * yc[e];
    }
  }
}

/* FP32 Jacobi; the compatibility sum and the residual norm in FP64. */
OR_API double or_solve32(ortree *t, const float *Q, float *V, int sweeps, float omega) {
  or_grid_build(t);
  int64_t nv = t->n_vert;
  double tot = 0.0;
  for (int64_t v = 0; v < nv; ++v) tot += (double)Q[v];
  float ftot = (float)tot;
  float *b = (float *)malloc(sizeof(float) * nv);
  float *y = (float *)malloc(sizeof(float) * nv);
  for (int64_t v = 0; v < nv; ++v) b[v] = Q[v] - ftot * (float)t->ion_load[v];
  for (int it = 0; it < sweeps; ++it) {
    apply32(t, V, y);
    for (int64_t v = 0; v < nv; ++v) V[v] = V[v] + omega * (b[v] - y[v]) / (float)t->diag[v];
  }
  apply32(t, V, y);
  double r2 = 0.0;
  for (int64_t v = 0; v < nv; ++v) { double r = (double)b[v] - (double)y[v]; r2 += r * r; }
  free(b); free(y);
  return sqrt(r2);
}

OR_API void or_efield32(ortree *t, const float *V, float *Ev) {
  or_grid_build(t);
  int d = t->d, nc = t->ncorner;
  int64_t nv = t->n_vert;
  memset(Ev, 0, sizeof(float) * d * nv);
  float vc[8];
  for (int64_t l = 0; l < t->n_leaves; ++l) {
    float h = (float)leaf_h(t, l);
    for (int e = 0; e < nc; ++e) {
      int64_t i = l * nc + e;
      float s = 0.0f;
      for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j) s += (float)t->cexp_w[j] * V[t->cexp_vid[j]];
      vc[e] = s;
    }
    for (int e = 0; e < nc; ++e) {
      int64_t i = l * nc + e;
      if (t->cexp_ptr[i + 1] - t->cexp_ptr[i] != 1 || t->cexp_w[t->cexp_ptr[i]] != 1.0) continue;
      int32_t v = t->cexp_vid[t->cexp_ptr[i]];
      for (int a = 0; a < d; ++a) Ev[a * nv + v] += (vc[e | (1 << a)] - vc[e & ~(1 << a)]) / h;
    }
  }
  for (int64_t v = 0; v < nv; ++v) {
    float c = (float)t->direct_cnt[v];
    for (int a = 0; a < d; ++a) Ev[a * nv + v] = -(Ev[a * nv + v] / c);
  }
}

/* FP32 corner fields (hanging corners interpolated) in leaf, corner, axis order. */
static void corner_field32(const ortree *t, const float *Ev, float *Ec) {
  int d = t->d, nc = t->ncorner;
  int64_t nv = t->n_vert;
  for (int64_t i = 0; i < t->n_leaves * nc; ++i)
    for (int a = 0; a < d; ++a) {
      float s = 0.0f;
      for (int64_t j = t->cexp_ptr[i]; j < t->cexp_ptr[i + 1]; ++j) s += (float)t->cexp_w[j] * Ev[a * nv + t->cexp_vid[j]];
      Ec[i * d + a] = s;
    }
}

/* Split push (a3 + a4 + a1 in the split representation): gather in FP32,
 * kick, drift in leaf-cell units, integer re-location.  Updates leaf, o, v in
 * place (storage order unchanged). */
OR_API void or_push32(ortree *t, int64_t n, int32_t *leaf, float *o, float *v, const float *Ev,
                      double qm, double dt) {
  or_grid_build(t);
  int d = t->d, nc = t->ncorner;
  float *Ec = (float *)malloc(sizeof(float) * t->n_leaves * nc * d);
  corner_field32(t, Ev, Ec);
  float qmdt = (float)(qm * dt);
  for (int64_t p = 0; p < n; ++p) {
    int32_t nd = t->leaf_node[leaf[p]];
    int lev = t->level[nd];
    int64_t per = p3(lev);
    float sl = (float)(dt * (double)per);
    float E[3] = {0.0f, 0.0f, 0.0f};
    for (int e = 0; e < nc; ++e) {
      float w = shape32(d, e, o, n, p);
      for (int a = 0; a < d; ++a) E[a] += w * Ec[((int64_t)leaf[p] * nc + e) * d + a];
    }
    int64_t I[3] = {0, 0, 0};
    float f[3] = {0.0f, 0.0f, 0.0f};
    for (int a = 0; a < d; ++a) {
      float vn = v[a * n + p] + qmdt * E[a];
      v[a * n + p] = vn;
      float tt = o[a * n + p] + vn * sl;
      float fl = floorf(tt);
      f[a] = tt - fl;
      int64_t c = t->coords[nd * 3 + a] + (int64_t)fl;
      c %= per;
      if (c < 0) c += per;
      I[a] = c;
    }
    float on[3];
    int32_t nn = resolve32(t, lev, I, f, on);
    leaf[p] = t->leaf_id[nn];
    for (int a = 0; a < d; ++a) o[a * n + p] = on[a];
  }
  free(Ec);
}

/* The particle-handling step (or_move64) in the split representation: t =
 * RN32(o + RN32(v s_l)), n = floor t, f = t - n, target cell I = c + n on the
 * leaf's level (per = 3^l cells).  Periodic: I mod per.  Reflecting: with
 * Im = I mod 2 per, Im < per keeps (Im, f); otherwise the point is mirrored,
 * (2 per - 1 - Im, RN32(1 - f)) for f > 0 and (2 per - Im, 0) for f = 0, and
 * the velocity component negated; a point on the far wall goes to the last
 * cell with the largest offset below 1.  Then the integer lift/drop
 * re-location of or_push32. */
OR_API void or_move32(ortree *t, int64_t n, int32_t *leaf, float *o, float *v, double dt, int reflect) {
  int d = t->d;
  for (int64_t p = 0; p < n; ++p) {
    int32_t nd = t->leaf_node[leaf[p]];
    int lev = t->level[nd];
    int64_t per = p3(lev);
    float sl = (float)(dt * (double)per);
    int64_t I[3] = {0, 0, 0};
    float f[3] = {0.0f, 0.0f, 0.0f};
    for (int a = 0; a < d; ++a) {
      float vn = v[a * n + p];
      float tt = o[a * n + p] + vn * sl;
      float fl = floorf(tt);
      float fr = tt - fl;
      int64_t c = t->coords[nd * 3 + a] + (int64_t)fl;
      if (!reflect) {
        c %= per;
        if (c < 0) c += per;
      } else {
        int64_t p2 = 2 * per, im = c % p2;
        if (im < 0) im += p2;
        if (im < per) {
          c = im;
        } else {
          v[a * n + p] = -vn;
          if (fr > 0.0f) {
            c = p2 - 1 - im;
            fr = clamp_off(1.0f - fr);
          } else {
            c = p2 - im;
            if (c >= per) {
              c = per - 1;
              fr = OR_ONE_MINUS;
            }
          }
        }
      }
      I[a] = c;
      f[a] = fr;
    }
    float on[3];
    int32_t nn = resolve32(t, lev, I, f, on);
    leaf[p] = t->leaf_id[nn];
    for (int a = 0; a < d; ++a) o[a * n + p] = on[a];
  }
}

OR_API void or_gather32(ortree *t, int64_t n, const int32_t *leaf, const float *o, const float *Ev,
                        float *Ep) {
  or_grid_build(t);
  int d = t->d, nc = t->ncorner;
  float *Ec = (float *)malloc(sizeof(float) * t->n_leaves * nc * d);
  corner_field32(t, Ev, Ec);
  for (int64_t p = 0; p < n; ++p) {
    float E[3] = {0.0f, 0.0f, 0.0f};
    for (int e = 0; e < nc; ++e) {
      float w = shape32(d, e, o, n, p);
      for (int a = 0; a < d; ++a) E[a] += w * Ec[((int64_t)leaf[p] * nc + e) * d + a];
    }
    for (int a = 0; a < d; ++a) Ep[a * n + p] = E[a];
  }
  free(Ec);
}

/* ------------------------------------------------------------------------ */
/* Re-refinement by the particles-per-cell criterion                          */
/* ------------------------------------------------------------------------ */
/* Reading of the Section 6 setup (refine a cell whose particle count exceeds
 * ppc, coarsen children whose union does not): cell C on level m is refined
 * iff m < dmin, or m < dmax and count(C) > ppc.  The result depends only on
 * the positions.  Positions are integer cells on level dmax, computed from Q
 * (FP64) or from leaf + offset digits (split, same drop rule as the push). */

static int64_t cellkey(int d, const int64_t *I, int64_t per) {
  int64_t k = 0, m = 1;
  for (int a = 0; a < d; ++a) { k += I[a] * m; m *= per; }
  return k;
}

static int64_t count_range(const int64_t *sorted, int64_t n, int64_t lo, int64_t hi) {
  int64_t a = 0, b = n;
  while (a < b) { int64_t m = (a + b) / 2; if (sorted[m] < lo) a = m + 1; else b = m; }
  int64_t s = a;
  a = s; b = n;
  while (a < b) { int64_t m = (a + b) / 2; if (sorted[m] < hi) a = m + 1; else b = m; }
  return a - s;
}

/* fine: integer cell coords on level dmax, [n][d]; returns malloc'd flags. */
static uint8_t *retree_from_cells(int d, int64_t n, const int64_t *fine, int64_t ppc, int dmin,
                                  int dmax, int64_t *n_flags) {
  int nch = (int)p3(d);
  /* per level sorted cell keys of all particles */
  int64_t **keys = (int64_t **)malloc(sizeof(int64_t *) * (dmax + 1));
  for (int m = 0; m <= dmax; ++m) {
    keys[m] = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
    int64_t sh = p3(dmax - m), per = p3(m);
    for (int64_t p = 0; p < n; ++p) {
      int64_t I[3] = {0, 0, 0};
      for (int a = 0; a < d; ++a) I[a] = fine[p * d + a] / sh;
      keys[m][p] = cellkey(d, I, per);
    }
    qsort(keys[m], (size_t)n, sizeof(int64_t), cmp_i64);
  }
  int64_t cap = 1024, nf = 0;
  uint8_t *flags = (uint8_t *)malloc(cap);
  int64_t ncur = 1;
  int64_t *cur = (int64_t *)calloc(3, sizeof(int64_t));
  for (int m = 0; m <= dmax && ncur > 0; ++m) {
    int64_t per = p3(m);
    int64_t *nxt = (int64_t *)malloc(sizeof(int64_t) * 3 * ncur * nch);
    int64_t nn = 0;
    for (int64_t i = 0; i < ncur; ++i) {
      int64_t *c = &cur[i * 3];
      int refine = 0;
      if (m < dmin) refine = 1;
      else if (m < dmax) {
        int64_t k = cellkey(d, c, per);
        refine = count_range(keys[m], n, k, k + 1) > ppc;
      }
      if (nf == cap) { cap *= 2; flags = (uint8_t *)realloc(flags, cap); }
      flags[nf++] = (uint8_t)refine;
      if (refine)
        for (int ch = 0; ch < nch; ++ch) {
          for (int a = 0; a < 3; ++a) nxt[nn * 3 + a] = a < d ? 3 * c[a] + (ch / p3(a)) % 3 : 0;
          ++nn;
        }
    }
    free(cur);
    cur = nxt;
    ncur = nn;
  }
  free(cur);
  for (int m = 0; m <= dmax; ++m) free(keys[m]);
  free(keys);
  *n_flags = nf;
  return flags;
}

static uint8_t *g_last_flags = NULL;
static int64_t g_last_nflags = 0;

/* Builds the new flags; returns their count; fetch them with or_retree_fetch. */
OR_API int64_t or_retree64(int d, int64_t n, const double *x, int64_t ppc, int dmin, int dmax) {
  int64_t *fine = (int64_t *)malloc(sizeof(int64_t) * d * (n ? n : 1));
  int64_t step = 2 * p3(OR_MAXLEV - dmax);
  for (int64_t p = 0; p < n; ++p)
    for (int a = 0; a < d; ++a) fine[p * d + a] = quantise(x[a * n + p]) / step;
  free(g_last_flags);
  g_last_flags = retree_from_cells(d, n, fine, ppc, dmin, dmax, &g_last_nflags);
  free(fine);
  return g_last_nflags;
}

OR_API int64_t or_retree32(ortree *t, int64_t n, const int32_t *leaf, const float *o, int64_t ppc,
                           int dmin, int dmax) {
  int d = t->d;
  int64_t *fine = (int64_t *)malloc(sizeof(int64_t) * d * (n ? n : 1));
  for (int64_t p = 0; p < n; ++p) {
    int32_t nd = t->leaf_node[leaf[p]];
    int lev = t->level[nd];
    for (int a = 0; a < d; ++a) {
      int64_t I = t->coords[nd * 3 + a];
      if (lev >= dmax) {
        I /= p3(lev - dmax);
      } else {
        float f = o[a * n + p];
        for (int m = lev; m < dmax; ++m) {
          float u = 3.0f * f;
          int dg = (int)floorf(u);
          if (dg > 2) dg = 2;
          f = clamp_off(u - (float)dg);
          I = 3 * I + dg;
        }
      }
      fine[p * d + a] = I;
    }
  }
  free(g_last_flags);
  g_last_flags = retree_from_cells(d, n, fine, ppc, dmin, dmax, &g_last_nflags);
  free(fine);
  return g_last_nflags;
}

OR_API void or_retree_fetch(uint8_t *out) { memcpy(out, g_last_flags, (size_t)g_last_nflags); }

/* Re-bin split particles of tree `from` into tree `to` (same positions):
 * the resolve rule of the push with zero displacement. */
OR_API void or_rebin32(const ortree *from, const ortree *to, int64_t n, int32_t *leaf, float *o) {
  int d = from->d;
  for (int64_t p = 0; p < n; ++p) {
    int32_t nd = from->leaf_node[leaf[p]];
    int lev = from->level[nd];
    int64_t I[3] = {0, 0, 0};
    float f[3] = {0.0f, 0.0f, 0.0f};
    for (int a = 0; a < d; ++a) { I[a] = from->coords[nd * 3 + a]; f[a] = o[a * n + p]; }
    float on[3];
    int32_t nn = resolve32(to, lev, I, f, on);
    leaf[p] = to->leaf_id[nn];
    for (int a = 0; a < d; ++a) o[a * n + p] = on[a];
  }
}
