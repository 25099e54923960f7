/*
 * mm_oracle.c -- plain, slow, FP64 CPU oracle for the MulMent hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; every function below is written from the
 * paper (Meyerhenke, Noellenburg, Schulz, "Drawing Large Graphs by Multilevel
 * Maxent-Stress Optimization", arXiv 1506.04383) and cites the passage it
 * follows.  Arithmetic is double precision throughout.
 *
 * Conventions (where the paper leaves a choice, the function comment states
 * the reading taken):
 *   positions      x[2*v+0], x[2*v+1]
 *   CSR            rp[n+1] (int64), col[nnz] (int32), symmetric, no loops
 *   coincident pair (|x_u - x_v| == 0): unit vector and r-value are 0,
 *                  ln|x_u - x_v| contributes 0.
 *
 * Parity status per function (see the module docstring of oracle/__init__.py
 * for the pins that check each one):
 *   orc_philox4x32_10      pinned (published known-answer vectors)
 *   orc_build_S            pinned (cycle / path closed forms, brute force)
 *   orc_repulsion_exact    pinned (cycle closed form)
 *   orc_repulsion_bh       pinned (theta=0 equals exact; 2-D multipole bound)
 *   orc_sweep              pinned (regular-polygon closed form, K2 map,
 *                                  equivariance)
 *   orc_objective          pinned (K2 and cycle closed forms)
 *   orc_sclap              pinned by invariants and order-free cases
 *   orc_contract           pinned (hand-worked example, invariants)
 *   orc_prolong            pinned (radius bound, distribution moments)
 *   orc_repulsion_h        pinned (identity map and single cluster equal the
 *                                  exact sum; far-field error order; scaling)
 *   orc_full_stress        pinned (path on a line, K2 and scaled closed forms;
 *                                  distances equal a library BFS)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Ten rounds of the */
/* 4x32 Philox bijection; the key is bumped by the Weyl constants between    */
/* rounds.  The paper (Sec. 3.2, prolongation) draws a uniform angle and a   */
/* uniform radius; the generator is unspecified there, this one is chosen.   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24 high bits of a 32-bit draw mapped to [0, 1). */
static double u01(uint32_t z) { return (double)(z >> 8) * (1.0 / 16777216.0); }

static void draw4(uint64_t seed, uint32_t a, uint32_t b, uint32_t c,
                  uint32_t d, uint32_t out[4]) {
  uint32_t ctr[4] = {a, b, c, d};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Edge length on a level (Sec. 3.2, "Local Improvement"): on a coarse level */
/* the target distance of adjacent u, v is sqrt(c(u)) + sqrt(c(v)); on the   */
/* input level it is the input length d (default 1, Sec. 2.1).               */
/* ------------------------------------------------------------------------ */
static double edge_len(int coarse, const double* c, const double* elen,
                       int64_t e, int32_t u, int32_t v) {
  if (coarse) return sqrt(c[u]) + sqrt(c[v]);
  return elen ? elen[e] : 1.0;
}

/* ------------------------------------------------------------------------ */
/* k-hop pair set S (Sec. 2.3 footnote: the general model with S a superset  */
/* of E).  For each u, S_u = every v != u reachable by a path of at most k   */
/* edges; d_uv = the shortest such path length (hop count on the input      */
/* level with unit lengths); w_uv = d_uv^-2 (Sec. 2.3); rho_u = sum_S w_uv   */
/* (Eq. 2).  Computed by k rounds of hop-limited Bellman-Ford per source.    */
/* Entries of each row are in ascending v.                                   */
/*                                                                            */
/* Call once with scol == NULL to obtain the row pointer sp and the total;   */
/* then again with buffers of that size.  Returns nnz(S) or -1 on error.     */
/* ------------------------------------------------------------------------ */
int64_t orc_build_S(int32_t n, const int64_t* rp, const int32_t* col,
                    const double* elen, const double* c, int coarse, int k,
                    int64_t* sp, int32_t* scol, double* sd, double* rho) {
  if (n < 0 || k < 1) return -1;
  double* cur = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* nxt = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  char* seen = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!cur || !nxt || !touched || !seen) return -1;
  for (int32_t i = 0; i < n; ++i) cur[i] = nxt[i] = INFINITY;
  int64_t total = 0;
  sp[0] = 0;
  for (int32_t u = 0; u < n; ++u) {
    int32_t nt = 0;
    cur[u] = 0.0; nxt[u] = 0.0;
    touched[nt++] = u; seen[u] = 1;
    for (int hop = 0; hop < k; ++hop) {
      /* relax every edge out of every vertex reached within `hop` hops */
      int32_t nt_before = nt;
      for (int32_t t = 0; t < nt_before; ++t) {
        int32_t a = touched[t];
        if (!(cur[a] < INFINITY)) continue;
        for (int64_t e = rp[a]; e < rp[a + 1]; ++e) {
          int32_t b = col[e];
          double nd = cur[a] + edge_len(coarse, c, elen, e, a, b);
          if (!seen[b]) { seen[b] = 1; touched[nt++] = b; }
          if (nd < nxt[b]) nxt[b] = nd;
        }
      }
      for (int32_t t = 0; t < nt; ++t) cur[touched[t]] = nxt[touched[t]];
    }
    /* collect S_u in ascending vertex id */
    int32_t cnt = 0;
    for (int32_t t = 0; t < nt; ++t) if (touched[t] != u) ++cnt;
    if (scol) {
      /* simple insertion into sorted order (rows are small) */
      int64_t base = sp[u];
      int32_t m = 0;
      for (int32_t t = 0; t < nt; ++t) {
        int32_t v = touched[t];
        if (v == u) continue;
        int32_t pos = m++;
        while (pos > 0 && scol[base + pos - 1] > v) {
          scol[base + pos] = scol[base + pos - 1];
          sd[base + pos] = sd[base + pos - 1];
          --pos;
        }
        scol[base + pos] = v;
        sd[base + pos] = cur[v];
      }
      double r = 0.0;
      for (int32_t j = 0; j < cnt; ++j) r += 1.0 / (sd[base + j] * sd[base + j]);
      rho[u] = r;
    }
    total += cnt;
    sp[u + 1] = total;
    for (int32_t t = 0; t < nt; ++t) {
      cur[touched[t]] = nxt[touched[t]] = INFINITY;
      seen[touched[t]] = 0;
    }
  }
  free(cur); free(nxt); free(touched); free(seen);
  return total;
}

/* r-value r(u,v) = (x_u - x_v) / |x_u - x_v|^2 (Sec. 2.3, after Eq. 2). */
static void rvalue(const double* x, int32_t u, int32_t v, double* rx, double* ry) {
  double dx = x[2 * u] - x[2 * v], dy = x[2 * u + 1] - x[2 * v + 1];
  double q = dx * dx + dy * dy;
  if (q > 0.0) { *rx = dx / q; *ry = dy / q; } else { *rx = 0.0; *ry = 0.0; }
}

/* Exact long-range sum F_u = sum_{v != u} r(u,v) over all vertices. */
void orc_repulsion_exact(int32_t n, const double* x, double* F) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int32_t u = 0; u < n; ++u) {
    double fx = 0.0, fy = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      if (v == u) continue;
      double rx, ry;
      rvalue(x, u, v, &rx, &ry);
      fx += rx; fy += ry;
    }
    F[2 * u] = fx; F[2 * u + 1] = fy;
  }
}

/* ------------------------------------------------------------------------ */
/* The hierarchy approximation of the entropy sum, Eq. 3 (Sec. 3.2, "Faster  */
/* Local Improvement"), without its last term (the sum over E, subtracted by */
/* the caller exactly as for the other modes):                               */
/*   F_u = sum_{v != u, M(v) = M(u)} r(u,v)                                   */
/*       + sum_{v' != M(u)} nu(v') (x_u - x'_{v'}) / |x_u - x'_{v'}|^2        */
/* M maps the n current-level vertices to the nc vertices of the level used  */
/* for the approximation (h levels down, or the coarsest), nu(v') counts the */
/* current-level vertices mapped to v', and x'_{v'} is their midpoint, each  */
/* current-level vertex weighted by what it stands for on the current level, */
/* i.e. once: x'_{v'} = (1/nu(v')) sum_{M(v) = v'} x_v.                       */
/* ------------------------------------------------------------------------ */
void orc_repulsion_h(int32_t n, const double* x, const int32_t* cmap, int32_t nc,
                     double* F) {
  double* xc = (double*)calloc(2 * (size_t)(nc > 0 ? nc : 1), sizeof(double));
  double* nu = (double*)calloc((size_t)(nc > 0 ? nc : 1), sizeof(double));
  for (int32_t v = 0; v < n; ++v) {
    nu[cmap[v]] += 1.0;
    xc[2 * cmap[v]] += x[2 * v];
    xc[2 * cmap[v] + 1] += x[2 * v + 1];
  }
  for (int32_t c = 0; c < nc; ++c) {
    if (nu[c] > 0.0) { xc[2 * c] /= nu[c]; xc[2 * c + 1] /= nu[c]; }
  }
  /* the vertices of every representative, in ascending order */
  int64_t* off = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
  int32_t* mem = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t v = 0; v < n; ++v) off[cmap[v] + 1] += 1;
  for (int32_t c = 0; c < nc; ++c) off[c + 1] += off[c];
  {
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nc + 1));
    memcpy(fill, off, sizeof(int64_t) * ((size_t)nc + 1));
    for (int32_t v = 0; v < n; ++v) mem[fill[cmap[v]]++] = v;
    free(fill);
  }
#pragma omp parallel for schedule(dynamic, 64)
  for (int32_t u = 0; u < n; ++u) {
    double fx = 0.0, fy = 0.0;
    /* close vertices: the same coarse representative, exact r-values */
    for (int64_t j = off[cmap[u]]; j < off[cmap[u] + 1]; ++j) {
      int32_t v = mem[j];
      if (v == u) continue;
      double rx, ry;
      rvalue(x, u, v, &rx, &ry);
      fx += rx; fy += ry;
    }
    /* far vertices: one r-value per other coarse vertex, scaled by nu */
    for (int32_t c = 0; c < nc; ++c) {
      if (c == cmap[u] || nu[c] == 0.0) continue;
      double dx = x[2 * u] - xc[2 * c], dy = x[2 * u + 1] - xc[2 * c + 1];
      double q = dx * dx + dy * dy;
      if (q > 0.0) { fx += nu[c] * dx / q; fy += nu[c] * dy / q; }
    }
    F[2 * u] = fx; F[2 * u + 1] = fy;
  }
  free(xc); free(nu); free(off); free(mem);
}

/* ------------------------------------------------------------------------ */
/* Barnes-Hut quadtree (Barnes and Hut 1986; cited in Sec. 2.2 and as the    */
/* approximation used by the maxent-stress solver of Gansner et al., Sec.    */
/* 2.3).  A classic recursive pointer quadtree over the bounding square of   */
/* the layout: root corner = (min x, min y), side = max extent.  A cell is   */
/* split at its midpoint; a point goes to the upper half when its coordinate */
/* is >= the midpoint.  Splitting stops at a single point or at depth        */
/* max_depth (a bucket).  Mass of a cell = number of vertices in it.         */
/* ------------------------------------------------------------------------ */
typedef struct {
  double x0, y0, w;      /* lower-left corner and side of the cell */
  double cx, cy;         /* centroid of the points inside */
  int32_t count, depth;
  int32_t child[4];      /* -1 if empty */
  int32_t pbeg, pend;    /* leaf: range in the point permutation */
} orc_qnode;

typedef struct {
  orc_qnode* nodes;
  int32_t nn, cap;
  int32_t* perm;         /* point ids grouped by leaf */
  const double* x;
  int max_depth;
} orc_qtree;

static int32_t qt_new(orc_qtree* t) {
  if (t->nn == t->cap) {
    t->cap = t->cap ? 2 * t->cap : 1024;
    t->nodes = (orc_qnode*)realloc(t->nodes, sizeof(orc_qnode) * (size_t)t->cap);
  }
  return t->nn++;
}

static int quadrant(const double* p, double mx, double my) {
  return (p[0] >= mx ? 1 : 0) + (p[1] >= my ? 2 : 0);
}

/* builds the subtree for perm[beg, end) inside cell (x0, y0, w) */
static int32_t qt_build(orc_qtree* t, int32_t beg, int32_t end, double x0,
                        double y0, double w, int depth, int32_t* scratch) {
  int32_t id = qt_new(t);
  orc_qnode nd;
  nd.x0 = x0; nd.y0 = y0; nd.w = w; nd.depth = depth;
  nd.count = end - beg;
  nd.child[0] = nd.child[1] = nd.child[2] = nd.child[3] = -1;
  nd.pbeg = beg; nd.pend = end;
  double sx = 0.0, sy = 0.0;
  for (int32_t i = beg; i < end; ++i) {
    sx += t->x[2 * t->perm[i]];
    sy += t->x[2 * t->perm[i] + 1];
  }
  nd.cx = sx / nd.count; nd.cy = sy / nd.count;
  t->nodes[id] = nd;
  if (nd.count <= 1 || depth >= t->max_depth) return id;   /* leaf */
  double h = 0.5 * w, mx = x0 + h, my = y0 + h;
  int32_t cnt[4] = {0, 0, 0, 0};
  for (int32_t i = beg; i < end; ++i) ++cnt[quadrant(&t->x[2 * t->perm[i]], mx, my)];
  int32_t off[4];
  off[0] = beg; off[1] = off[0] + cnt[0]; off[2] = off[1] + cnt[1]; off[3] = off[2] + cnt[2];
  int32_t fill[4] = {off[0], off[1], off[2], off[3]};
  for (int32_t i = beg; i < end; ++i) {
    int32_t p = t->perm[i];
    scratch[fill[quadrant(&t->x[2 * p], mx, my)]++] = p;
  }
  memcpy(t->perm + beg, scratch + beg, sizeof(int32_t) * (size_t)(end - beg));
  for (int q = 0; q < 4; ++q) {
    if (!cnt[q]) continue;
    double cx0 = (q & 1) ? mx : x0, cy0 = (q & 2) ? my : y0;
    int32_t ch = qt_build(t, off[q], off[q] + cnt[q], cx0, cy0, h, depth + 1, scratch);
    t->nodes[id].child[q] = ch;
  }
  t->nodes[id].pbeg = t->nodes[id].pend = 0;   /* internal: no point list */
  return id;
}

static void qt_visit(const orc_qtree* t, int32_t id, int32_t u, int u_inside,
                     double theta, double* fx, double* fy, int64_t* nacc) {
  const orc_qnode* nd = &t->nodes[id];
  const double* xu = &t->x[2 * u];
  if (!u_inside) {
    double dx = xu[0] - nd->cx, dy = xu[1] - nd->cy;
    double q = dx * dx + dy * dy;
    /* acceptance: side / distance < theta, u not in the cell */
    if (theta > 0.0 && nd->w * nd->w < theta * theta * q) {
      *fx += nd->count * dx / q;
      *fy += nd->count * dy / q;
      if (nacc) ++*nacc;
      return;
    }
  }
  int leaf = nd->child[0] < 0 && nd->child[1] < 0 && nd->child[2] < 0 && nd->child[3] < 0;
  if (leaf) {
    for (int32_t i = nd->pbeg; i < nd->pend; ++i) {
      int32_t v = t->perm[i];
      if (v == u) continue;
      double rx, ry;
      rvalue(t->x, u, v, &rx, &ry);
      *fx += rx; *fy += ry;
      if (nacc) ++*nacc;
    }
    return;
  }
  double h = 0.5 * nd->w, mx = nd->x0 + h, my = nd->y0 + h;
  int uq = u_inside ? quadrant(xu, mx, my) : -1;
  for (int q = 0; q < 4; ++q)
    if (nd->child[q] >= 0)
      qt_visit(t, nd->child[q], u, u_inside && uq == q, theta, fx, fy, nacc);
}

/* F_u ~ sum_{v != u} r(u,v) by Barnes-Hut with opening parameter theta.
 * theta == 0 opens every cell, giving the exact sum.  nacc (nullable)
 * receives per-vertex interaction counts. */
void orc_repulsion_bh(int32_t n, const double* x, double theta, int max_depth,
                      double* F, int64_t* nacc) {
  if (n <= 0) return;
  orc_qtree t;
  memset(&t, 0, sizeof(t));
  t.x = x; t.max_depth = max_depth;
  t.perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* scratch = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  double lox = x[0], hix = x[0], loy = x[1], hiy = x[1];
  for (int32_t i = 0; i < n; ++i) {
    t.perm[i] = i;
    if (x[2 * i] < lox) lox = x[2 * i];
    if (x[2 * i] > hix) hix = x[2 * i];
    if (x[2 * i + 1] < loy) loy = x[2 * i + 1];
    if (x[2 * i + 1] > hiy) hiy = x[2 * i + 1];
  }
  double side = (hix - lox) > (hiy - loy) ? (hix - lox) : (hiy - loy);
  qt_build(&t, 0, n, lox, loy, side, 0, scratch);
#pragma omp parallel for schedule(dynamic, 64)
  for (int32_t u = 0; u < n; ++u) {
    double fx = 0.0, fy = 0.0;
    int64_t cnt = 0;
    qt_visit(&t, 0, u, 1, theta, &fx, &fy, nacc ? &cnt : NULL);
    F[2 * u] = fx; F[2 * u + 1] = fy;
    if (nacc) nacc[u] = cnt;
  }
  free(t.nodes); free(t.perm); free(scratch);
}

/* ------------------------------------------------------------------------ */
/* One Jacobi iteration of Eq. 2 (Sec. 2.3), general model over S:           */
/*   x'_u = (1/rho_u) sum_{v in S_u} w_uv (x_v + d_uv (x_u-x_v)/|x_u-x_v|)   */
/*        + (alpha/rho_u) sum_{v not in S_u, v != u} r(u,v).                 */
/* The iteration reads only the previous coordinates (Sec. 3.2).             */
/* rep_mode 0: the entropy sum is taken literally, pair by pair.             */
/* rep_mode 1: the entropy sum is the Barnes-Hut total minus the exact       */
/*             r-values over S (the subtraction of Eq. 3).                   */
/* rep_mode 2: the entropy sum is Eq. 3: orc_repulsion_h with the map cmap   */
/*             to nc coarse vertices, minus the exact r-values over S.       */
/* stats[0] = sum |x'-x|^2, stats[1] = sum |x|^2 (relative change,           */
/* Sec. 3.2), stats[2] = stress of x over the unordered pairs of S (Eq. 1).  */
/* ------------------------------------------------------------------------ */
void orc_sweep(int32_t n, const double* x, const int64_t* sp,
               const int32_t* scol, const double* sd, const double* rho,
               double alpha, int rep_mode, double theta, int max_depth,
               const int32_t* cmap, int32_t nc, double* xout, double* stats) {
  double* F = NULL;
  if (rep_mode == 1 || rep_mode == 2) {
    F = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
    if (rep_mode == 1)
      orc_repulsion_bh(n, x, theta, max_depth, F, NULL);
    else
      orc_repulsion_h(n, x, cmap, nc, F);
  }
  double s_dx = 0.0, s_x = 0.0, s_stress = 0.0;
#pragma omp parallel
  {
    char* inS = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
#pragma omp for schedule(dynamic, 64) reduction(+ : s_dx, s_x, s_stress)
    for (int32_t u = 0; u < n; ++u) {
      double gx = 0.0, gy = 0.0;      /* stress part of Eq. 2 */
      double sx = 0.0, sy = 0.0;      /* r-values over S */
      for (int64_t e = sp[u]; e < sp[u + 1]; ++e) {
        int32_t v = scol[e];
        double d = sd[e], w = 1.0 / (d * d);
        double dx = x[2 * u] - x[2 * v], dy = x[2 * u + 1] - x[2 * v + 1];
        double dist = sqrt(dx * dx + dy * dy);
        double ux = 0.0, uy = 0.0;
        if (dist > 0.0) { ux = dx / dist; uy = dy / dist; }
        gx += w * (x[2 * v] + d * ux);
        gy += w * (x[2 * v + 1] + d * uy);
        double rx, ry;
        rvalue(x, u, v, &rx, &ry);
        sx += rx; sy += ry;
        s_stress += 0.5 * w * (dist - d) * (dist - d);
      }
      double ex = 0.0, ey = 0.0;      /* sum over v not in S_u */
      if (rep_mode == 1 || rep_mode == 2) {
        ex = F[2 * u] - sx; ey = F[2 * u + 1] - sy;
      } else {
        for (int64_t e = sp[u]; e < sp[u + 1]; ++e) inS[scol[e]] = 1;
        for (int32_t v = 0; v < n; ++v) {
          if (v == u || inS[v]) continue;
          double rx, ry;
          rvalue(x, u, v, &rx, &ry);
          ex += rx; ey += ry;
        }
        for (int64_t e = sp[u]; e < sp[u + 1]; ++e) inS[scol[e]] = 0;
      }
      double nx = (gx + alpha * ex) / rho[u];
      double ny = (gy + alpha * ey) / rho[u];
      xout[2 * u] = nx; xout[2 * u + 1] = ny;
      s_dx += (nx - x[2 * u]) * (nx - x[2 * u]) + (ny - x[2 * u + 1]) * (ny - x[2 * u + 1]);
      s_x += x[2 * u] * x[2 * u] + x[2 * u + 1] * x[2 * u + 1];
    }
    free(inS);
  }
  if (stats) { stats[0] = s_dx; stats[1] = s_x; stats[2] = s_stress; }
  free(F);
}

/* ------------------------------------------------------------------------ */
/* Maxent-stress objective, Eq. 1, general model over S:                     */
/*   M(x) = sum_{{u,v} in S} w (|x_u-x_v| - d)^2                             */
/*        - alpha * sum_{{u,v} not in S} ln |x_u - x_v|                      */
/* over unordered pairs.  out[0] = stress, out[1] = the ln-sum over pairs    */
/* not in S, out[2] = M.                                                     */
/* ------------------------------------------------------------------------ */
void orc_objective(int32_t n, const double* x, const int64_t* sp,
                   const int32_t* scol, const double* sd, double alpha,
                   double* out) {
  double stress = 0.0, lns = 0.0;
#pragma omp parallel
  {
    char* inS = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
#pragma omp for schedule(dynamic, 64) reduction(+ : stress, lns)
    for (int32_t u = 0; u < n; ++u) {
      for (int64_t e = sp[u]; e < sp[u + 1]; ++e) {
        int32_t v = scol[e];
        inS[v] = 1;
        if (v <= u) continue;
        double d = sd[e], w = 1.0 / (d * d);
        double dx = x[2 * u] - x[2 * v], dy = x[2 * u + 1] - x[2 * v + 1];
        double dist = sqrt(dx * dx + dy * dy);
        stress += w * (dist - d) * (dist - d);
      }
      for (int32_t v = u + 1; v < n; ++v) {
        if (inS[v]) continue;
        double dx = x[2 * u] - x[2 * v], dy = x[2 * u + 1] - x[2 * v + 1];
        double q = dx * dx + dy * dy;
        if (q > 0.0) lns += 0.5 * log(q);
      }
      for (int64_t e = sp[u]; e < sp[u + 1]; ++e) inS[scol[e]] = 0;
    }
    free(inS);
  }
  out[0] = stress; out[1] = lns; out[2] = stress - alpha * lns;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1 for graphs too large for the O(n^2) ln-sum: the stress over S is    */
/* summed exactly, the ln-sum over the unordered pairs not in S is estimated */
/* from `samples` uniformly drawn ordered pairs u != v (an unordered pair is */
/* then uniform too): pairs in S are rejected, the rest give ln |x_u - x_v|  */
/* (0 for coincident points).  With N = n(n-1)/2 - |S|/2 pairs outside S,   */
/* the estimate is N * mean and its standard error N * sd / sqrt(kept).     */
/* Draw i uses Philox counter (i, 0, 0, 5), key = seed; u and v are 64-bit   */
/* draws reduced mod n.  S rows must be sorted ascending (binary search).    */
/* out[0] = stress, out[1] = ln-sum estimate, out[2] = M estimate,           */
/* out[3] = standard error of out[1], out[4] = samples kept.                 */
/* ------------------------------------------------------------------------ */
static int in_row(const int32_t* scol, int64_t a, int64_t b, int32_t v) {
  while (a < b) {
    int64_t m = a + (b - a) / 2;
    if (scol[m] == v) return 1;
    if (scol[m] < v) a = m + 1; else b = m;
  }
  return 0;
}

void orc_objective_sampled(int32_t n, const double* x, const int64_t* sp,
                           const int32_t* scol, const double* sd, double alpha,
                           int64_t samples, uint64_t seed, double* out) {
  /* fixed chunks, each summed in order, then the chunks in order: the     */
  /* result does not depend on the thread count or schedule                */
  enum { CH = 256 };
  double cs[CH], c1[CH], c2[CH], ck[CH];
#pragma omp parallel for schedule(dynamic, 1)
  for (int c = 0; c < CH; ++c) {
    double st = 0.0, s1 = 0.0, s2 = 0.0, kk = 0.0;
    int32_t u0 = (int32_t)((int64_t)n * c / CH), u1 = (int32_t)((int64_t)n * (c + 1) / CH);
    for (int32_t u = u0; u < u1; ++u)
      for (int64_t e = sp[u]; e < sp[u + 1]; ++e) {
        int32_t v = scol[e];
        if (v <= u) continue;
        double d = sd[e], w = 1.0 / (d * d);
        double dx = x[2 * u] - x[2 * v], dy = x[2 * u + 1] - x[2 * v + 1];
        double dist = sqrt(dx * dx + dy * dy);
        st += w * (dist - d) * (dist - d);
      }
    int64_t i0 = samples * c / CH, i1 = samples * (c + 1) / CH;
    for (int64_t i = i0; i < i1; ++i) {
      uint32_t z[4];
      draw4(seed, (uint32_t)i, (uint32_t)(i >> 32), 0u, 5u, z);
      int32_t u = (int32_t)((((uint64_t)z[0] << 32) | z[1]) % (uint64_t)n);
      int32_t v = (int32_t)((((uint64_t)z[2] << 32) | z[3]) % (uint64_t)n);
      if (u == v || in_row(scol, sp[u], sp[u + 1], v)) continue;
      double dx = x[2 * u] - x[2 * v], dy = x[2 * u + 1] - x[2 * v + 1];
      double q = dx * dx + dy * dy;
      double l = q > 0.0 ? 0.5 * log(q) : 0.0;
      s1 += l;
      s2 += l * l;
      kk += 1.0;
    }
    cs[c] = st; c1[c] = s1; c2[c] = s2; ck[c] = kk;
  }
  double stress = 0.0, sum = 0.0, sum2 = 0.0, kept = 0.0;
  for (int c = 0; c < CH; ++c) { stress += cs[c]; sum += c1[c]; sum2 += c2[c]; kept += ck[c]; }
  double N = 0.5 * (double)n * (double)(n - 1) - 0.5 * (double)sp[n];
  double mean = kept > 0.0 ? sum / kept : 0.0;
  double var = kept > 1.0 ? (sum2 - kept * mean * mean) / (kept - 1.0) : 0.0;
  if (var < 0.0) var = 0.0;
  out[0] = stress;
  out[1] = N * mean;
  out[2] = stress - alpha * N * mean;
  out[3] = kept > 0.0 ? N * sqrt(var / kept) : 0.0;
  out[4] = kept;
}

/* ------------------------------------------------------------------------ */
/* Size-constrained label propagation, SCLaP (Sec. 3.1).  Start from         */
/* singletons; each round visits the vertices in a random order and moves a  */
/* vertex to the neighbouring cluster of strongest connection (sum of edge   */
/* weights omega) that is not overloaded after the move (cluster weight +    */
/* c(v) <= U).  Ties keep the current cluster if it is among the best, else  */
/* take the smallest cluster id.  At most `rounds` rounds; stops early when  */
/* a round moves nothing.  The random order is a Fisher-Yates shuffle drawn  */
/* from Philox with counter (i, round, level, 3); a caller may pass the      */
/* orders instead (order_in: rounds x n, row r = the visiting order of round */
/* r; NULL = the Philox shuffle), the way a test fixes the random draws.     */
/* ------------------------------------------------------------------------ */
void orc_sclap(int32_t n, const int64_t* rp, const int32_t* col,
               const double* ew, const double* c, double U, int rounds,
               uint64_t seed, int32_t level, const int32_t* order_in,
               int32_t* labels) {
  double* wt = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* conn = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  char* mark = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int32_t v = 0; v < n; ++v) { labels[v] = v; wt[v] = c[v]; }
  for (int r = 0; r < rounds; ++r) {
    if (order_in) {
      for (int32_t i = 0; i < n; ++i) order[i] = order_in[(size_t)r * n + i];
    } else {
      for (int32_t i = 0; i < n; ++i) order[i] = i;
      for (int32_t i = n - 1; i > 0; --i) {
        uint32_t z[4];
        draw4(seed, (uint32_t)i, (uint32_t)r, (uint32_t)level, 3u, z);
        uint64_t big = ((uint64_t)z[0] << 32) | z[1];
        int32_t j = (int32_t)(big % (uint64_t)(i + 1));
        int32_t tmp = order[i]; order[i] = order[j]; order[j] = tmp;
      }
    }
    int64_t moved = 0;
    for (int32_t i = 0; i < n; ++i) {
      int32_t v = order[i];
      int32_t own = labels[v];
      int32_t nc = 0;
      for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
        int32_t L = labels[col[e]];
        if (!mark[L]) { mark[L] = 1; cand[nc++] = L; conn[L] = 0.0; }
        conn[L] += ew ? ew[e] : 1.0;
      }
      double own_conn = mark[own] ? conn[own] : 0.0;
      double best = own_conn;
      for (int32_t j = 0; j < nc; ++j) {
        int32_t L = cand[j];
        if (L == own || wt[L] + c[v] > U) continue;
        if (conn[L] > best) best = conn[L];
      }
      int32_t target = own;
      if (best > own_conn) {
        target = -1;
        for (int32_t j = 0; j < nc; ++j) {
          int32_t L = cand[j];
          if (L == own || wt[L] + c[v] > U) continue;
          if (conn[L] == best && (target < 0 || L < target)) target = L;
        }
      }
      for (int32_t j = 0; j < nc; ++j) mark[cand[j]] = 0;
      if (target != own) {
        wt[own] -= c[v]; wt[target] += c[v];
        labels[v] = target;
        ++moved;
      }
    }
    if (!moved) break;
  }
  free(wt); free(conn); free(order); free(cand); free(mark);
}

/* ------------------------------------------------------------------------ */
/* Cluster contraction (Sec. 3.1): each block becomes one node whose weight  */
/* is the sum of its members' weights; two coarse nodes are adjacent iff     */
/* their blocks are joined by at least one edge, with weight the sum of the  */
/* weights of the joining edges.  Coarse ids: the rank of the label among    */
/* the distinct labels (ascending).  Coarse rows are in ascending column     */
/* order; each coarse edge weight is summed in fine-entry order.             */
/* Outputs must have room for n nodes and nnz entries.  Returns n'.          */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t a, b; int64_t idx; } orc_trip;
static int trip_cmp(const void* p, const void* q) {
  const orc_trip* s = (const orc_trip*)p; const orc_trip* t = (const orc_trip*)q;
  if (s->a != t->a) return s->a < t->a ? -1 : 1;
  if (s->b != t->b) return s->b < t->b ? -1 : 1;
  return s->idx < t->idx ? -1 : (s->idx > t->idx ? 1 : 0);
}

int32_t orc_contract(int32_t n, const int64_t* rp, const int32_t* col,
                     const double* ew, const double* c, const int32_t* labels,
                     int32_t* map, double* cc, int64_t* crp, int32_t* ccol,
                     double* cew, int64_t* cnnz_out) {
  int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) rank[i] = 0;
  for (int32_t v = 0; v < n; ++v) rank[labels[v]] = 1;
  int32_t nc = 0;
  for (int32_t i = 0; i < n; ++i) { int32_t used = rank[i]; rank[i] = nc; nc += used; }
  for (int32_t v = 0; v < n; ++v) map[v] = rank[labels[v]];
  for (int32_t i = 0; i < nc; ++i) cc[i] = 0.0;
  for (int32_t v = 0; v < n; ++v) cc[map[v]] += c[v];
  int64_t nnz = rp[n];
  orc_trip* tr = (orc_trip*)malloc(sizeof(orc_trip) * (size_t)(nnz > 0 ? nnz : 1));
  int64_t m = 0;
  for (int32_t u = 0; u < n; ++u)
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
      int32_t a = map[u], b = map[col[e]];
      if (a == b) continue;
      tr[m].a = a; tr[m].b = b; tr[m].idx = e; ++m;
    }
  qsort(tr, (size_t)m, sizeof(orc_trip), trip_cmp);
  for (int32_t i = 0; i <= nc; ++i) crp[i] = 0;
  int64_t k = 0;
  for (int64_t i = 0; i < m; ++i) {
    if (i > 0 && tr[i].a == tr[i - 1].a && tr[i].b == tr[i - 1].b) {
      cew[k - 1] += ew ? ew[tr[i].idx] : 1.0;
      continue;
    }
    ccol[k] = tr[i].b;
    cew[k] = ew ? ew[tr[i].idx] : 1.0;
    crp[tr[i].a + 1]++;
    ++k;
  }
  for (int32_t i = 0; i < nc; ++i) crp[i + 1] += crp[i];
  *cnnz_out = k;
  free(rank); free(tr);
  return nc;
}

/* ------------------------------------------------------------------------ */
/* Prolongation (Sec. 3.2, "Uncoarsening"): a fine vertex v represented by  */
/* the coarse vertex v' at P is placed at polar coordinates around P with    */
/* angle uniform in [0, 2 pi) and radius uniform in [0, sqrt(c(v'))).  The   */
/* two draws come from Philox with counter (v, level, 0, 0), key = seed.     */
/* ------------------------------------------------------------------------ */
void orc_prolong(int32_t n_fine, const int32_t* map, const double* xc,
                 const double* cc, uint64_t seed, int32_t level, double* xf) {
  for (int32_t v = 0; v < n_fine; ++v) {
    uint32_t z[4];
    draw4(seed, (uint32_t)v, (uint32_t)level, 0u, 0u, z);
    int32_t p = map[v];
    double phi = 2.0 * ORC_PI * u01(z[0]);
    double rad = sqrt(cc[p]) * u01(z[1]);
    xf[2 * v] = xc[2 * p] + rad * cos(phi);
    xf[2 * v + 1] = xc[2 * p + 1] + rad * sin(phi);
  }
}

/* Initial layout of a coarsest level with more than two vertices: the same
 * polar placement around the origin, with radius sqrt(sum c) (a virtual
 * parent holding every vertex); Philox counter (v, level, 1, 0). */
void orc_place_coarsest(int32_t n, const double* c, uint64_t seed,
                        int32_t level, double* x) {
  double tot = 0.0;
  for (int32_t v = 0; v < n; ++v) tot += c[v];
  double R = sqrt(tot);
  for (int32_t v = 0; v < n; ++v) {
    uint32_t z[4];
    draw4(seed, (uint32_t)v, (uint32_t)level, 1u, 0u, z);
    double phi = 2.0 * ORC_PI * u01(z[0]);
    double rad = R * u01(z[1]);
    x[2 * v] = rad * cos(phi);
    x[2 * v + 1] = rad * sin(phi);
  }
}

/* ------------------------------------------------------------------------ */
/* Full stress and its optimal scale (Sec. 4, methodology):                  */
/*   F(x) = sum over unordered pairs {u,v} of w_uv (|x_u - x_v| - d_uv)^2    */
/* with d_uv the shortest-path (hop) distance and w_uv = d_uv^-2, and the    */
/* scalar s minimising sum w (s |x_u - x_v| - d)^2:                          */
/*   s = sum w d |x_u - x_v| / sum w |x_u - x_v|^2,                          */
/*   F(s x) = sum w d^2 - (sum w d |dx|)^2 / sum w |dx|^2.                   */
/* One breadth-first search per source (plain queue).  out[0] = F(x),        */
/* out[1] = s, out[2] = F(s x), out[3] = number of connected pairs.          */
/* ------------------------------------------------------------------------ */
void orc_full_stress(int32_t n, const int64_t* rp, const int32_t* col, const double* x,
                     double* out) {
  double F = 0.0, A = 0.0, B = 0.0, C = 0.0, pairs = 0.0;
#pragma omp parallel reduction(+ : F, A, B, C, pairs)
  {
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
    for (int32_t s = 0; s < n; ++s) {
      for (int32_t v = 0; v < n; ++v) dist[v] = -1;
      int32_t head = 0, tail = 0;
      dist[s] = 0;
      queue[tail++] = s;
      while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
          int32_t v = col[e];
          if (dist[v] < 0) { dist[v] = dist[u] + 1; queue[tail++] = v; }
        }
      }
      for (int32_t v = s + 1; v < n; ++v) {       /* unordered pairs */
        if (dist[v] <= 0) continue;
        double d = (double)dist[v], w = 1.0 / (d * d);
        double dx = x[2 * s] - x[2 * v], dy = x[2 * s + 1] - x[2 * v + 1];
        double len = sqrt(dx * dx + dy * dy);
        F += w * (len - d) * (len - d);
        A += w * d * len;
        B += w * len * len;
        C += w * d * d;
        pairs += 1.0;
      }
    }
    free(dist); free(queue);
  }
  out[0] = F;
  out[1] = B > 0.0 ? A / B : 0.0;
  out[2] = B > 0.0 ? C - A * A / B : C;
  out[3] = pairs;
}
