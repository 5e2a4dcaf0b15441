/*
 * Plain sequential CPU oracle of the terminal-edge-region polygonal mesher of
 * Salinas, Ojeda, Hitschfeld and Ortiz-Bernardin, "GPU parallel algorithm for the
 * generation of polygonal meshes based on terminal-edge regions" (IMR 2022).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this file's library.  It shares no code, header or
 * helper with the CUDA library; both read the same generated meshes.
 *
 * Mesh layout (the paper's Section 2 arrays, with an explicit twin instead of the
 * Neighbor array): xy[2v], xy[2v+1] are the lattice coordinates of vertex v;
 * tri[3t+k] is the k-th vertex of the ccw triangle t; half-edge h = 3t+k runs from
 * tri[h] to tri[3t+(k+1)%3]; twin[h] is the opposite half-edge, or -1 on the border.
 *
 * Readings of the paper that this file fixes (the paper is silent or ambiguous):
 *  - Edge length is the exact int64 squared length; among equal lengths the edge
 *    with the lower undirected id min(h, twin(h)) counts as longer (Section 3.2.1
 *    gives no tie rule).  This is a strict total order on edges.
 *  - A border edge is always a frontier edge; a border longest edge is also a
 *    (border) terminal edge (Algorithm 2, LabelSeed / LabelFrontier).
 *  - A polygon is emitted starting at its frontier half-edge with the smallest
 *    (origin vertex, half-edge id), one origin per frontier half-edge, ccw.
 *  - Reparation: in a polygon with several barrier-edge tips the tip with the
 *    smallest vertex id is split first; the "middle internal edge" is e_ceil(k/2)
 *    among the k internal edges at the tip, counted ccw starting after the barrier
 *    edge; the two new polygons replace the old one in place, the one containing
 *    the half-edge tip->x first.
 *
 * Every routine below is a direct restatement; nothing is blocked, fused or
 * reordered beyond the paper's own steps.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "polylla_oracle.h"

/* ---------------------------------------------------------------- half-edge basics */
static int64_t he_next(int64_t h) { return 3 * (h / 3) + (h % 3 + 1) % 3; }
static int64_t he_prev(int64_t h) { return 3 * (h / 3) + (h % 3 + 2) % 3; }
static int64_t he_origin(const int32_t* tri, int64_t h) { return tri[h]; }
static int64_t he_dest(const int32_t* tri, int64_t h) { return tri[he_next(h)]; }

/* squared length of the edge of half-edge h, exact */
static int64_t edge_len2(const int64_t* xy, const int32_t* tri, int64_t h) {
  int64_t a = he_origin(tri, h), b = he_dest(tri, h);
  int64_t dx = xy[2 * b] - xy[2 * a];
  int64_t dy = xy[2 * b + 1] - xy[2 * a + 1];
  return dx * dx + dy * dy;
}

/* undirected edge id: the lower of the two half-edge ids */
static int64_t edge_id(const int32_t* twin, int64_t h) {
  int64_t g = twin[h];
  return (g >= 0 && g < h) ? g : h;
}

/* 1 if the edge of h is longer than the edge of g (length, then lower edge id) */
static int edge_longer(const int64_t* xy, const int32_t* tri, const int32_t* twin, int64_t h,
                       int64_t g) {
  int64_t lh = edge_len2(xy, tri, h), lg = edge_len2(xy, tri, g);
  if (lh != lg) return lh > lg;
  return edge_id(twin, h) < edge_id(twin, g);
}

/* ---------------------------------------------------------------- Algorithm 2 */
/* LabelMax: for every triangle, the local index of its longest edge (Max array). */
int oracle_label_max(const int64_t* xy, const int32_t* tri, const int32_t* twin, int64_t m,
                     uint8_t* max_edge) {
  if (m < 0 || (m > 0 && (!xy || !tri || !twin || !max_edge))) return ORACLE_ERR_ARG;
  for (int64_t t = 0; t < m; ++t) {
    int best = 0;
    for (int k = 1; k < 3; ++k)
      if (edge_longer(xy, tri, twin, 3 * t + k, 3 * t + best)) best = k;
    max_edge[t] = (uint8_t)best;
  }
  return ORACLE_OK;
}

static int is_longest(const uint8_t* max_edge, int64_t h) { return max_edge[h / 3] == h % 3; }

/* LabelSeed: per edge.  A border edge that is the longest edge of its triangle is
 * a border terminal edge and that triangle is a seed.  An interior edge that is
 * the longest edge of both triangles t_a, t_b is a terminal edge and the triangle
 * with the lower index is a seed.  terminal[h] marks both half-edges. */
int oracle_label_seed(const int32_t* twin, int64_t m, const uint8_t* max_edge, uint8_t* seed,
                      uint8_t* terminal) {
  if (m < 0) return ORACLE_ERR_ARG;
  memset(seed, 0, (size_t)m);
  memset(terminal, 0, (size_t)(3 * m));
  for (int64_t h = 0; h < 3 * m; ++h) {
    int64_t g = twin[h];
    if (g >= 0 && g < h) continue; /* each undirected edge once */
    if (g < 0) {
      if (is_longest(max_edge, h)) {
        terminal[h] = 1;
        seed[h / 3] = 1;
      }
      continue;
    }
    if (is_longest(max_edge, h) && is_longest(max_edge, g)) {
      int64_t ta = h / 3, tb = g / 3;
      terminal[h] = terminal[g] = 1;
      seed[ta < tb ? ta : tb] = 1;
    }
  }
  return ORACLE_OK;
}

/* LabelFrontier: per edge.  Frontier iff it is a border edge, or it is the longest
 * edge of neither of its two triangles. */
int oracle_label_frontier(const int32_t* twin, int64_t m, const uint8_t* max_edge,
                          uint8_t* frontier) {
  if (m < 0) return ORACLE_ERR_ARG;
  memset(frontier, 0, (size_t)(3 * m));
  for (int64_t h = 0; h < 3 * m; ++h) {
    int64_t g = twin[h];
    if (g >= 0 && g < h) continue;
    if (g < 0) {
      frontier[h] = 1;
    } else if (!is_longest(max_edge, h) && !is_longest(max_edge, g)) {
      frontier[h] = frontier[g] = 1;
    }
  }
  return ORACLE_OK;
}

/* The seed triangles in ascending order (the Seed array read front to back). */
/*
 * Longest-edge propagation paths (the Lepp that defines terminal-edge regions,
 * Section 2; Lepp kernels are the paper's future work, Section 5).  From triangle t,
 * follow the neighbour across the longest edge until that edge is the longest
 * edge of both its triangles, or a border edge -- a terminal edge.  region[t] is
 * the seed of the terminal edge reached (its lower triangle, or the border
 * triangle itself); depth[t] is the number of links followed.  Returns the largest
 * depth, or ORACLE_ERR_NOT_DISK if a path runs longer than m links.
 */
int64_t oracle_lepp(const int32_t* twin, int64_t m, const uint8_t* max_edge, int32_t* region,
                    int32_t* depth) {
  if (!twin || !max_edge || !region || !depth || m < 1) return ORACLE_ERR_ARG;
  int64_t deepest = 0;
  for (int64_t t = 0; t < m; ++t) {
    int64_t u = t, d = 0;
    for (;;) {
      const int64_t h = 3 * u + max_edge[u];
      const int64_t g = twin[h];
      if (g < 0) {  /* border terminal edge */
        region[t] = (int32_t)u;
        break;
      }
      if (is_longest(max_edge, g)) {  /* longest of both triangles */
        region[t] = (int32_t)(u < g / 3 ? u : g / 3);
        break;
      }
      u = g / 3;
      if (++d > m) return ORACLE_ERR_NOT_DISK;
    }
    depth[t] = (int32_t)d;
    if (d > deepest) deepest = d;
  }
  return deepest;
}

int64_t oracle_seed_list(const uint8_t* seed, int64_t m, int32_t* seeds) {
  int64_t ns = 0;
  for (int64_t t = 0; t < m; ++t)
    if (seed[t]) seeds[ns++] = (int32_t)t;
  return ns;
}

/* ---------------------------------------------------------------- polygon of a region */
typedef struct {
  int64_t m;
  const int32_t* tri;
  const int32_t* twin;
  const uint8_t* frontier;
  int32_t* stamp; /* per triangle: id of the last region search that reached it */
  int32_t cur;
  int32_t* queue; /* m entries */
  int64_t* fh;    /* frontier half-edges of the current region (3m entries) */
} region_ctx;

static int ctx_init(region_ctx* c, int64_t m, const int32_t* tri, const int32_t* twin,
                    const uint8_t* frontier) {
  c->m = m;
  c->tri = tri;
  c->twin = twin;
  c->frontier = frontier;
  c->cur = 0;
  c->stamp = (int32_t*)calloc((size_t)(m > 0 ? m : 1), sizeof(int32_t));
  c->queue = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  c->fh = (int64_t*)malloc((size_t)(3 * (m > 0 ? m : 1)) * sizeof(int64_t));
  if (!c->stamp || !c->queue || !c->fh) return ORACLE_ERR_OOM;
  return ORACLE_OK;
}

static void ctx_free(region_ctx* c) {
  free(c->stamp);
  free(c->queue);
  free(c->fh);
}

/*
 * PolyConstruction (Algorithm 4), restated.  The terminal-edge region of triangle t
 * is the set of triangles reachable from t without crossing a frontier edge; its
 * polygon is the cycle of its frontier half-edges, walked ccw with the region on
 * the left: from a frontier half-edge h the next one is found by turning around
 * the endpoint of h through internal edges,
 *     g = next(h);  while (g is not frontier) g = next(twin(g)),
 * and each visited frontier half-edge contributes its origin vertex.  The walk
 * starts at the region's frontier half-edge with the smallest (origin, id).
 * Appends the polygon's origins (and half-edges, if `hout` is given) and returns
 * its length, or ORACLE_ERR_NOT_DISK if the walk does not visit every frontier
 * half-edge of the region exactly once (the region boundary is not one cycle).
 */
static int64_t region_polygon(region_ctx* c, int64_t t, int32_t* vout, int64_t* hout) {
  const int32_t* tri = c->tri;
  const int32_t* twin = c->twin;
  const uint8_t* fr = c->frontier;
  c->cur += 1;
  const int32_t id = c->cur;
  int64_t qh = 0, qt = 0, nfh = 0;
  c->queue[qt++] = (int32_t)t;
  c->stamp[t] = id;
  while (qh < qt) {
    int64_t u = c->queue[qh++];
    for (int k = 0; k < 3; ++k) {
      int64_t h = 3 * u + k;
      if (fr[h]) {
        c->fh[nfh++] = h;
        continue;
      }
      int64_t g = twin[h];
      if (g < 0) return ORACLE_ERR_NOT_DISK; /* a border edge must be frontier */
      int64_t w = g / 3;
      if (c->stamp[w] != id) {
        c->stamp[w] = id;
        c->queue[qt++] = (int32_t)w;
      }
    }
  }
  if (nfh == 0) return ORACLE_ERR_NOT_DISK;
  int64_t start = c->fh[0];
  for (int64_t i = 1; i < nfh; ++i) {
    int64_t h = c->fh[i];
    if (tri[h] < tri[start] || (tri[h] == tri[start] && h < start)) start = h;
  }
  int64_t len = 0, h = start, limit = 3 * c->m + 3;
  do {
    if (len >= nfh) return ORACLE_ERR_NOT_DISK;
    vout[len] = tri[h];
    if (hout) hout[len] = h;
    ++len;
    int64_t g = he_next(h);
    int64_t steps = 0;
    while (!fr[g]) {
      if (twin[g] < 0 || ++steps > limit) return ORACLE_ERR_NOT_DISK;
      g = he_next(twin[g]);
    }
    h = g;
  } while (h != start);
  if (len != nfh) return ORACLE_ERR_NOT_DISK;
  return len;
}

/* ---------------------------------------------------------------- Algorithm 3 */
/* TraversalTriangulation: one polygon per seed, in ascending seed order; the Mesh
 * and Position arrays are written as CSR (off[i]..off[i+1] holds polygon i).
 * Returns the total number of polygon vertices or a negative error. */
int64_t oracle_traverse(const int32_t* tri, const int32_t* twin, int64_t m, const uint8_t* frontier,
                        const int32_t* seeds, int64_t ns, int64_t* off, int32_t* vtx,
                        int64_t cap_vtx) {
  region_ctx c;
  int rc = ctx_init(&c, m, tri, twin, frontier);
  if (rc) {
    ctx_free(&c);
    return rc;
  }
  int32_t* buf = (int32_t*)malloc((size_t)(3 * (m > 0 ? m : 1)) * sizeof(int32_t));
  if (!buf) {
    ctx_free(&c);
    return ORACLE_ERR_OOM;
  }
  int64_t total = 0;
  off[0] = 0;
  for (int64_t i = 0; i < ns; ++i) {
    int64_t len = region_polygon(&c, seeds[i], buf, NULL);
    if (len < 0) {
      total = len;
      break;
    }
    if (total + len > cap_vtx) {
      total = ORACLE_ERR_CAPACITY;
      break;
    }
    memcpy(vtx + total, buf, (size_t)len * sizeof(int32_t));
    total += len;
    off[i + 1] = total;
  }
  free(buf);
  ctx_free(&c);
  return total;
}

/* ---------------------------------------------------------------- Algorithm 5 */
/* Trivertex array: one half-edge leaving each vertex (Section 2). */
static void build_trivertex(const int32_t* tri, int64_t m, int64_t n, int64_t* tv) {
  for (int64_t v = 0; v < n; ++v) tv[v] = -1;
  for (int64_t h = 0; h < 3 * m; ++h)
    if (tv[tri[h]] < 0) tv[tri[h]] = h;
}

/* The Trivertex array as a public routine (Section 2): tv[v] = the smallest
 * half-edge leaving v, or -1 for a vertex no triangle uses.  Returns 0. */
int oracle_trivertex(const int32_t* tri, int64_t m, int64_t n, int64_t* tv) {
  if (!tri || !tv || m < 0 || n < 0) return ORACLE_ERR_ARG;
  for (int64_t h = 0; h < 3 * m; ++h)
    if (tri[h] < 0 || tri[h] >= n) return ORACLE_ERR_ARG;
  build_trivertex(tri, m, n, tv);
  return ORACLE_OK;
}

/* ccw successor of an out-half-edge o around its origin: twin(prev(o)) */
static int64_t rot_ccw(const int32_t* twin, int64_t o) { return twin[he_prev(o)]; }

/*
 * Split one polygon at its barrier-edge tip (Section 3.2.3).  `v` holds the
 * polygon's vertices.  Returns 0 if it has no tip, 1 if it was split (the two new
 * polygons are appended to `dst` in order), or a negative error.
 */
typedef struct {
  int64_t* off;
  int32_t* vtx;
  int64_t np, nv, cap_poly, cap_vtx;
} csr_out;

static int emit(csr_out* o, const int32_t* v, int64_t len) {
  if (o->np + 1 > o->cap_poly || o->nv + len > o->cap_vtx) return ORACLE_ERR_CAPACITY;
  memcpy(o->vtx + o->nv, v, (size_t)len * sizeof(int32_t));
  o->nv += len;
  o->np += 1;
  o->off[o->np] = o->nv;
  return ORACLE_OK;
}

static int split_polygon(region_ctx* c, uint8_t* frontier, const int64_t* tv, const int32_t* v,
                         int64_t len, csr_out* dst, int32_t* buf) {
  const int32_t* tri = c->tri;
  const int32_t* twin = c->twin;
  /* barrier-edge tips: consecutive v_a, v_b, v_c with v_a == v_c (cyclic) */
  int64_t tip = -1, tip_a = -1;
  for (int64_t i = 0; i < len; ++i) {
    int32_t va = v[i], vb = v[(i + 1) % len], vc = v[(i + 2) % len];
    if (va == vc && (tip < 0 || vb < tip)) {
      tip = vb;
      tip_a = va;
    }
  }
  if (tip < 0) return 0;
  /* the out-half-edge tip -> a, found through the Trivertex array */
  int64_t o = tv[tip];
  if (o < 0) return ORACLE_ERR_NOT_DISK;
  int64_t guard = 0;
  while (he_dest(tri, o) != tip_a) {
    int64_t r = rot_ccw(twin, o);
    if (r < 0 || ++guard > 3 * c->m) return ORACLE_ERR_NOT_DISK; /* a tip is interior */
    o = r;
  }
  const int64_t o0 = o;
  /* internal edges e_1..e_k at the tip, ccw after the barrier edge */
  int64_t k = 0;
  for (int64_t r = rot_ccw(twin, o0); r != o0; r = rot_ccw(twin, r)) {
    if (r < 0 || frontier[r]) return ORACLE_ERR_NOT_DISK; /* not a barrier-edge tip */
    ++k;
  }
  if (k < 2) return ORACLE_ERR_NOT_DISK;
  const int64_t j = (k + 1) / 2; /* ceil(k/2), 1-based */
  int64_t oj = o0;
  for (int64_t s = 0; s < j; ++s) oj = rot_ccw(twin, oj);
  /* label e_j as a frontier edge and rebuild the two polygons on its sides */
  frontier[oj] = 1;
  frontier[twin[oj]] = 1;
  int64_t la = region_polygon(c, oj / 3, buf, NULL);
  if (la < 0) return (int)la;
  int rc = emit(dst, buf, la);
  if (rc) return rc;
  int64_t lb = region_polygon(c, twin[oj] / 3, buf, NULL);
  if (lb < 0) return (int)lb;
  rc = emit(dst, buf, lb);
  if (rc) return rc;
  return 1;
}

/*
 * PolygonReparation (Algorithm 5) with the outer loop of Algorithm 1: every round
 * splits each polygon of M_in that has a barrier-edge tip once, writing the two
 * halves in its place in M_out (other polygons are copied), and counts the split
 * polygons in Total bet; rounds repeat until Total bet is 0.  `frontier` is
 * updated in place with the new frontier edges.  stats[0] = rounds that split
 * something, stats[1] = total splits.  Returns the final vertex count (and the
 * final polygon count in *np_out) or a negative error.
 */
int64_t oracle_repair(int64_t n, const int32_t* tri, const int32_t* twin, int64_t m,
                      uint8_t* frontier, const int64_t* off_in, const int32_t* vtx_in,
                      int64_t np_in, int64_t* off_out, int32_t* vtx_out, int64_t cap_poly,
                      int64_t cap_vtx, int64_t* np_out, int64_t* stats) {
  region_ctx c;
  int rc = ctx_init(&c, m, tri, twin, frontier);
  int64_t* tv = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int32_t* buf = (int32_t*)malloc((size_t)(3 * (m > 0 ? m : 1)) * sizeof(int32_t));
  /* ping-pong Mesh / Position arrays (the paper's auxiliary mesh) */
  csr_out a = {(int64_t*)malloc((size_t)(cap_poly + 1) * sizeof(int64_t)),
               (int32_t*)malloc((size_t)(cap_vtx > 0 ? cap_vtx : 1) * sizeof(int32_t)), 0, 0,
               cap_poly, cap_vtx};
  csr_out b = {(int64_t*)malloc((size_t)(cap_poly + 1) * sizeof(int64_t)),
               (int32_t*)malloc((size_t)(cap_vtx > 0 ? cap_vtx : 1) * sizeof(int32_t)), 0, 0,
               cap_poly, cap_vtx};
  int64_t result = 0;
  if (rc || !tv || !buf || !a.off || !a.vtx || !b.off || !b.vtx) {
    result = ORACLE_ERR_OOM;
    goto done;
  }
  build_trivertex(tri, m, n, tv);
  if (stats) stats[0] = stats[1] = 0;
  a.off[0] = 0;
  for (int64_t i = 0; i < np_in; ++i) {
    rc = emit(&a, vtx_in + off_in[i], off_in[i + 1] - off_in[i]);
    if (rc) {
      result = rc;
      goto done;
    }
  }
  csr_out* in = &a;
  csr_out* out = &b;
  for (;;) {
    int64_t total_bet = 0;
    out->np = 0;
    out->nv = 0;
    out->off[0] = 0;
    for (int64_t i = 0; i < in->np; ++i) {
      const int32_t* v = in->vtx + in->off[i];
      int64_t len = in->off[i + 1] - in->off[i];
      int s = split_polygon(&c, frontier, tv, v, len, out, buf);
      if (s < 0) {
        result = s;
        goto done;
      }
      if (s == 0) {
        rc = emit(out, v, len);
        if (rc) {
          result = rc;
          goto done;
        }
      }
      total_bet += s;
    }
    csr_out* tmp = in;
    in = out;
    out = tmp;
    if (total_bet == 0) break;
    if (stats) {
      stats[0] += 1;
      stats[1] += total_bet;
    }
  }
  memcpy(off_out, in->off, (size_t)(in->np + 1) * sizeof(int64_t));
  memcpy(vtx_out, in->vtx, (size_t)in->nv * sizeof(int32_t));
  *np_out = in->np;
  result = in->nv;
done:
  ctx_free(&c);
  free(tv);
  free(buf);
  free(a.off);
  free(a.vtx);
  free(b.off);
  free(b.vtx);
  return result;
}

/* ---------------------------------------------------------------- Algorithm 1 */
/* The whole mesher: label, seeds, traversal, reparation.  Outputs the final
 * polygons (CSR) and the per-triangle max / per-half-edge frontier labels after
 * reparation.  Returns the vertex count or a negative error. */
int64_t oracle_run(const int64_t* xy, int64_t n, const int32_t* tri, const int32_t* twin,
                   int64_t m, uint8_t* max_edge, uint8_t* frontier, int64_t* off, int32_t* vtx,
                   int64_t* np_out, int64_t* stats) {
  uint8_t* seed = (uint8_t*)malloc((size_t)(m > 0 ? m : 1));
  uint8_t* terminal = (uint8_t*)malloc((size_t)(3 * (m > 0 ? m : 1)));
  int32_t* seeds = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int64_t* off0 = (int64_t*)malloc((size_t)(m + 1) * sizeof(int64_t));
  int32_t* vtx0 = (int32_t*)malloc((size_t)(3 * (m > 0 ? m : 1)) * sizeof(int32_t));
  int64_t r = ORACLE_ERR_OOM;
  if (seed && terminal && seeds && off0 && vtx0) {
    r = oracle_label_max(xy, tri, twin, m, max_edge);
    if (!r) r = oracle_label_seed(twin, m, max_edge, seed, terminal);
    if (!r) r = oracle_label_frontier(twin, m, max_edge, frontier);
    if (!r) {
      int64_t ns = oracle_seed_list(seed, m, seeds);
      r = oracle_traverse(tri, twin, m, frontier, seeds, ns, off0, vtx0, 3 * m);
      if (r >= 0)
        r = oracle_repair(n, tri, twin, m, frontier, off0, vtx0, ns, off, vtx, m, 3 * m, np_out,
                          stats);
    }
  }
  free(seed);
  free(terminal);
  free(seeds);
  free(off0);
  free(vtx0);
  return r;
}
