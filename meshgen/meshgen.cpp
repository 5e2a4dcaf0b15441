// Seeded synthetic input generator: integer-lattice point sets and their exact
// Delaunay triangulation, as ccw triangles plus a half-edge twin array.
//
// This module produces INPUTS only.  It holds none of the mesher's arithmetic
// (no longest edges, labels, regions or polygons); both the CUDA library and the
// CPU oracle consume what it writes.
//
// Points.  SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) drives everything.  Gaussian draws use the Marsaglia
// polar method with a logarithm computed here from +,-,*,/ only, and the file is
// compiled with -ffp-contract=off, so x86_64 and aarch64 hosts draw bit-identical
// point sets.  Points are snapped to the lattice, deduplicated and Hilbert-sorted,
// so vertex ids are spatially coherent.
//
// Triangulation.  Incremental Bowyer-Watson insertion in Hilbert order with a
// visibility walk for point location and "ghost" triangles (one symbolic vertex at
// infinity) for the convex hull.  Predicates are exact: orient2d in int64 and
// incircle in __int128, valid for coordinates in [0, 2^28).  Co-circular lattice
// points are legal (incircle == 0 is not a conflict), so the result is a valid
// Delaunay triangulation; ties are resolved by insertion order, deterministically.
//
// Output layout.  tri[3t+k] is the k-th vertex of triangle t (ccw); half-edge
// h = 3t+k runs from tri[h] to tri[3t+(k+1)%3]; twin[h] is the opposite half-edge or
// -1 on the hull.  Triangles are ordered by their smallest vertex id and rotated so
// that the smallest vertex comes first.

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------- random numbers
struct SplitMix64 {
  uint64_t s;
  explicit SplitMix64(uint64_t seed) : s(seed) {}
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  // uniform integer in [0, bound) by rejection (exact, no modulo bias)
  uint64_t below(uint64_t bound) {
    uint64_t lim = UINT64_MAX - (UINT64_MAX % bound);
    for (;;) {
      uint64_t r = next();
      if (r < lim) return r % bound;
    }
  }
  // uniform double in [0, 1) with 53 random bits
  double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// Natural logarithm from basic IEEE operations only: s = f * 2^e with f in
// [0.5, 1); ln f = 2 atanh(z), z = (f-1)/(f+1) in [-1/3, 0), summed as the odd
// power series until the terms vanish.  Deterministic on every IEEE-754 host.
double det_log(double s) {
  int e = 0;
  double f = s;
  while (f >= 1.0) { f *= 0.5; ++e; }
  while (f < 0.5) { f *= 2.0; --e; }
  const double z = (f - 1.0) / (f + 1.0);
  const double z2 = z * z;
  double term = z, sum = 0.0;
  for (int k = 1; k < 80; k += 2) {
    double add = term / (double)k;
    if (add == 0.0) break;
    sum += add;
    term *= z2;
  }
  const double kLn2 = 0.69314718055994530942;
  return 2.0 * sum + (double)e * kLn2;
}

// One pair of independent standard normal draws (Marsaglia polar method).
void gauss2(SplitMix64& r, double* g0, double* g1) {
  for (;;) {
    double u = 2.0 * r.unit() - 1.0, v = 2.0 * r.unit() - 1.0;
    double s = u * u + v * v;
    if (s >= 1.0 || s == 0.0) continue;
    double f = __builtin_sqrt(-2.0 * det_log(s) / s);
    *g0 = u * f;
    *g1 = v * f;
    return;
  }
}

// ---------------------------------------------------------------- Hilbert order
uint64_t hilbert_key(uint32_t x, uint32_t y, int order) {
  uint64_t d = 0;
  for (uint32_t s = 1u << (order - 1); s > 0; s >>= 1) {
    uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
    d += (uint64_t)s * (uint64_t)s * (uint64_t)((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) { x = ~x; y = ~y; }
      uint32_t t = x; x = y; y = t;
    }
  }
  return d;
}

int order_for_side(int64_t side) {
  int o = 1;
  while (o < 31 && ((int64_t)1 << o) < side) ++o;
  return o;
}

struct Draw {
  uint64_t key;
  int64_t idx;  // draw index: first draw of a duplicated lattice point wins
  int64_t x, y;
};

// Deduplicate, keep exactly n points (smallest draw indices), emit Hilbert-sorted.
template <class Gen>
int64_t make_points(int64_t n, int64_t side, Gen gen, int64_t* xy) {
  const int ord = order_for_side(side);
  std::vector<Draw> pts;
  pts.reserve((size_t)n + n / 16 + 64);
  int64_t drawn = 0;
  int64_t want = n;
  for (int iter = 0; iter < 64; ++iter) {
    for (int64_t i = 0; i < want; ++i) {
      int64_t x, y;
      gen(&x, &y);
      pts.push_back(Draw{hilbert_key((uint32_t)x, (uint32_t)y, ord), drawn++, x, y});
    }
    std::sort(pts.begin(), pts.end(), [](const Draw& a, const Draw& b) {
      return a.key != b.key ? a.key < b.key : a.idx < b.idx;
    });
    size_t w = 0;
    for (size_t i = 0; i < pts.size(); ++i)
      if (w == 0 || pts[i].key != pts[w - 1].key) pts[w++] = pts[i];
    pts.resize(w);
    if ((int64_t)w >= n) break;
    want = (n - (int64_t)w) + (n - (int64_t)w) / 8 + 16;
  }
  if ((int64_t)pts.size() < n) return -1;
  if ((int64_t)pts.size() > n) {
    std::nth_element(pts.begin(), pts.begin() + n, pts.end(),
                     [](const Draw& a, const Draw& b) { return a.idx < b.idx; });
    pts.resize((size_t)n);
    std::sort(pts.begin(), pts.end(), [](const Draw& a, const Draw& b) { return a.key < b.key; });
  }
  for (int64_t i = 0; i < n; ++i) {
    xy[2 * i] = pts[(size_t)i].x;
    xy[2 * i + 1] = pts[(size_t)i].y;
  }
  return n;
}

// ---------------------------------------------------------------- exact predicates
inline int64_t orient(const int64_t* a, const int64_t* b, const int64_t* c) {
  return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]);
}

// > 0 iff d lies strictly inside the circle through the ccw triangle (a, b, c).
inline int incircle_sign(const int64_t* a, const int64_t* b, const int64_t* c, const int64_t* d) {
  const __int128 adx = a[0] - d[0], ady = a[1] - d[1];
  const __int128 bdx = b[0] - d[0], bdy = b[1] - d[1];
  const __int128 cdx = c[0] - d[0], cdy = c[1] - d[1];
  const __int128 al = adx * adx + ady * ady;
  const __int128 bl = bdx * bdx + bdy * bdy;
  const __int128 cl = cdx * cdx + cdy * cdy;
  const __int128 det = al * (bdx * cdy - cdx * bdy) + bl * (cdx * ady - adx * cdy) +
                       cl * (adx * bdy - bdx * ady);
  return det > 0 ? 1 : (det < 0 ? -1 : 0);
}

// p strictly between a and b, given a, b, p collinear.
inline bool strictly_between(const int64_t* a, const int64_t* b, const int64_t* p) {
  if (a[0] != b[0]) {
    int64_t lo = std::min(a[0], b[0]), hi = std::max(a[0], b[0]);
    return p[0] > lo && p[0] < hi;
  }
  int64_t lo = std::min(a[1], b[1]), hi = std::max(a[1], b[1]);
  return p[1] > lo && p[1] < hi;
}

// ---------------------------------------------------------------- Bowyer-Watson
constexpr int32_t INF = -1;

struct Delaunay {
  const int64_t* xy;
  int64_t n;
  std::vector<int32_t> V;  // 3 per triangle slot; INF marks the ghost vertex
  std::vector<int32_t> T;  // twin half-edge per half-edge slot
  std::vector<uint8_t> dead;
  std::vector<int32_t> freelist;
  std::vector<uint32_t> stamp;
  uint32_t cur_stamp = 0;
  std::vector<int32_t> stack, cavity, bnd_t, bnd_k;
  std::vector<int32_t> newtri_of;  // per vertex (+1 slot for INF): new triangle id
  std::vector<int32_t> outer, ea, eb, made;
  int32_t last = 0;
  uint64_t rot = 0;

  const int64_t* P(int32_t v) const { return xy + 2 * (int64_t)v; }

  int32_t alloc_tri() {
    int32_t t;
    if (!freelist.empty()) {
      t = freelist.back();
      freelist.pop_back();
      dead[(size_t)t] = 0;
    } else {
      t = (int32_t)(V.size() / 3);
      V.resize(V.size() + 3);
      T.resize(T.size() + 3);
      dead.push_back(0);
      stamp.push_back(0);
    }
    return t;
  }

  bool is_ghost(int32_t t) const {
    return V[3 * (size_t)t] == INF || V[3 * (size_t)t + 1] == INF || V[3 * (size_t)t + 2] == INF;
  }

  bool conflict(int32_t t, const int64_t* p) const {
    const int32_t* v = &V[3 * (size_t)t];
    for (int k = 0; k < 3; ++k) {
      if (v[k] == INF) {
        const int64_t* a = P(v[(k + 1) % 3]);
        const int64_t* b = P(v[(k + 2) % 3]);
        int64_t o = orient(a, b, p);
        if (o > 0) return true;
        return o == 0 && strictly_between(a, b, p);
      }
    }
    return incircle_sign(P(v[0]), P(v[1]), P(v[2]), p) > 0;
  }

  // Visibility walk from `last`; returns a triangle in conflict with p.
  int32_t locate(const int64_t* p) {
    int32_t t = last;
    if (dead[(size_t)t]) {
      t = 0;
      while (dead[(size_t)t]) ++t;
    }
    for (int64_t steps = 0;; ++steps) {
      if (is_ghost(t)) return t;
      const int32_t* v = &V[3 * (size_t)t];
      int off = (int)(rot++ % 3);
      bool moved = false;
      for (int i = 0; i < 3; ++i) {
        int k = (i + off) % 3;
        if (orient(P(v[k]), P(v[(k + 1) % 3]), p) < 0) {
          t = T[3 * (size_t)t + k] / 3;
          moved = true;
          break;
        }
      }
      if (!moved) return t;
    }
  }

  int insert(int32_t pv) {
    const int64_t* p = P(pv);
    int32_t t0 = locate(p);
    if (!conflict(t0, p)) return -2;  // duplicate point or broken state
    ++cur_stamp;
    stack.clear();
    cavity.clear();
    bnd_t.clear();
    bnd_k.clear();
    stack.push_back(t0);
    stamp[(size_t)t0] = cur_stamp;
    while (!stack.empty()) {
      int32_t t = stack.back();
      stack.pop_back();
      cavity.push_back(t);
      for (int k = 0; k < 3; ++k) {
        int32_t nb = T[3 * (size_t)t + k] / 3;
        if (stamp[(size_t)nb] == cur_stamp) continue;  // already in the cavity
        if (conflict(nb, p)) {
          stamp[(size_t)nb] = cur_stamp;
          stack.push_back(nb);
        } else {
          bnd_t.push_back(t);
          bnd_k.push_back(k);
        }
      }
    }
    // Boundary edges record the outside twin before cavity slots are recycled.
    const size_t nb_edges = bnd_t.size();
    outer.resize(nb_edges);
    ea.resize(nb_edges);
    eb.resize(nb_edges);
    made.resize(nb_edges);
    for (size_t i = 0; i < nb_edges; ++i) {
      int32_t t = bnd_t[i], k = bnd_k[i];
      ea[i] = V[3 * (size_t)t + k];
      eb[i] = V[3 * (size_t)t + (k + 1) % 3];
      outer[i] = T[3 * (size_t)t + k];
    }
    for (int32_t t : cavity) {
      dead[(size_t)t] = 1;
      freelist.push_back(t);
    }
    for (size_t i = 0; i < nb_edges; ++i) {
      int32_t nt = alloc_tri();
      made[i] = nt;
      V[3 * (size_t)nt] = ea[i];
      V[3 * (size_t)nt + 1] = eb[i];
      V[3 * (size_t)nt + 2] = pv;
      T[3 * (size_t)nt] = outer[i];
      T[(size_t)outer[i]] = 3 * nt;
      newtri_of[(size_t)(ea[i] + 1)] = nt;
    }
    for (size_t i = 0; i < nb_edges; ++i) {
      int32_t nt = made[i];
      int32_t other = newtri_of[(size_t)(eb[i] + 1)];  // triangle whose edge starts at eb
      T[3 * (size_t)nt + 1] = 3 * other + 2;
      T[3 * (size_t)other + 2] = 3 * nt + 1;
    }
    for (size_t i = 0; i < nb_edges; ++i)
      if (!is_ghost(made[i])) last = made[i];
    return 0;
  }

  // Returns 0 on success.
  int build() {
    if (n < 3) return -1;
    newtri_of.assign((size_t)n + 1, -1);
    // first non-collinear triple (0, 1, k)
    int64_t k = 2;
    while (k < n && orient(P(0), P(1), P((int32_t)k)) == 0) ++k;
    if (k >= n) return -1;
    int32_t a = 0, b = 1, c = (int32_t)k;
    if (orient(P(a), P(b), P(c)) < 0) std::swap(b, c);
    int32_t t = alloc_tri(), g0 = alloc_tri(), g1 = alloc_tri(), g2 = alloc_tri();
    int32_t vs[3] = {a, b, c};
    int32_t gs[3] = {g0, g1, g2};
    for (int i = 0; i < 3; ++i) V[3 * (size_t)t + i] = vs[i];
    for (int i = 0; i < 3; ++i) {
      // ghost across edge vs[i] -> vs[i+1]: (vs[i+1], vs[i], INF)
      int32_t g = gs[i];
      V[3 * (size_t)g] = vs[(i + 1) % 3];
      V[3 * (size_t)g + 1] = vs[i];
      V[3 * (size_t)g + 2] = INF;
      T[3 * (size_t)t + i] = 3 * g;
      T[3 * (size_t)g] = 3 * t + i;
    }
    for (int i = 0; i < 3; ++i) {
      // ghost gs[i] edge 1 (vs[i] -> INF) twins ghost gs[i-1] edge 2 (INF -> vs[i])
      int32_t g = gs[i], gp = gs[(i + 2) % 3];
      T[3 * (size_t)g + 1] = 3 * gp + 2;
      T[3 * (size_t)gp + 2] = 3 * g + 1;
    }
    last = t;
    for (int64_t i = 2; i < n; ++i) {
      if (i == k) continue;
      if (insert((int32_t)i) != 0) return -2;
    }
    return 0;
  }
};

}  // namespace

extern "C" {

// n unique points uniform on [0, side)^2, Hilbert-sorted.  Returns n, or -1.
int64_t mg_points_uniform(uint64_t seed, int64_t n, int64_t side, int64_t* xy) {
  if (n <= 0 || side <= 1 || side > ((int64_t)1 << 28)) return -1;
  if ((double)n > 0.5 * (double)side * (double)side) return -1;
  SplitMix64 r(seed);
  auto gen = [&](int64_t* x, int64_t* y) {
    *x = (int64_t)r.below((uint64_t)side);
    *y = (int64_t)r.below((uint64_t)side);
  };
  return make_points(n, side, gen, xy);
}

// n unique points from an ncomp-component equal-weight isotropic Gaussian mixture
// snapped to the lattice [0, side)^2 (draws outside the square are rejected).
// Means are uniform in the square; sigma_c is uniform in [smin, smax] * side.
int64_t mg_points_gmm(uint64_t seed, int64_t n, int32_t ncomp, int64_t side, double smin,
                      double smax, int64_t* xy) {
  if (n <= 0 || ncomp <= 0 || side <= 1 || side > ((int64_t)1 << 28)) return -1;
  SplitMix64 r(seed);
  std::vector<double> mx((size_t)ncomp), my((size_t)ncomp), sg((size_t)ncomp);
  for (int c = 0; c < ncomp; ++c) {
    mx[(size_t)c] = r.unit() * (double)side;
    my[(size_t)c] = r.unit() * (double)side;
    sg[(size_t)c] = (smin + (smax - smin) * r.unit()) * (double)side;
  }
  auto gen = [&](int64_t* x, int64_t* y) {
    for (;;) {
      int c = (int)r.below((uint64_t)ncomp);
      double g0, g1;
      gauss2(r, &g0, &g1);
      double fx = mx[(size_t)c] + sg[(size_t)c] * g0;
      double fy = my[(size_t)c] + sg[(size_t)c] * g1;
      if (!(fx >= 0.0 && fy >= 0.0)) continue;
      int64_t ix = (int64_t)(fx + 0.5), iy = (int64_t)(fy + 0.5);
      if (ix >= side || iy >= side) continue;
      *x = ix;
      *y = iy;
      return;
    }
  };
  return make_points(n, side, gen, xy);
}

// Delaunay triangulation of n distinct points with coordinates in [0, 2^28).
// tri/twin need room for 3*(2n) int32 each.  Returns m (number of triangles) or a
// negative error: -1 bad input / all collinear, -2 internal failure, -3 capacity.
int64_t mg_delaunay(const int64_t* xy, int64_t n, int32_t* tri, int32_t* twin, int64_t cap_tri) {
  if (n < 3 || n > (int64_t)1 << 30) return -1;
  for (int64_t i = 0; i < 2 * n; ++i)
    if (xy[i] < 0 || xy[i] >= ((int64_t)1 << 28)) return -1;
  Delaunay D;
  D.xy = xy;
  D.n = n;
  D.V.reserve((size_t)(6 * n + 64));
  D.T.reserve((size_t)(6 * n + 64));
  int rc = D.build();
  if (rc != 0) return rc;
  const int64_t slots = (int64_t)D.dead.size();
  // renumber real triangles: counting sort by smallest vertex, stable in slot order
  std::vector<int64_t> start((size_t)n + 1, 0);
  std::vector<int32_t> minv((size_t)slots, -1);
  int64_t m = 0;
  for (int64_t t = 0; t < slots; ++t) {
    if (D.dead[(size_t)t] || D.is_ghost((int32_t)t)) continue;
    const int32_t* v = &D.V[3 * (size_t)t];
    int32_t mv = std::min(v[0], std::min(v[1], v[2]));
    minv[(size_t)t] = mv;
    start[(size_t)mv + 1]++;
    ++m;
  }
  if (m > cap_tri) return -3;
  for (int64_t i = 0; i < n; ++i) start[(size_t)i + 1] += start[(size_t)i];
  std::vector<int32_t> newid((size_t)slots, -1);
  std::vector<int8_t> rot((size_t)slots, 0);
  for (int64_t t = 0; t < slots; ++t) {
    if (minv[(size_t)t] < 0) continue;
    int32_t id = (int32_t)start[(size_t)minv[(size_t)t]]++;
    newid[(size_t)t] = id;
    const int32_t* v = &D.V[3 * (size_t)t];
    int r = (v[0] == minv[(size_t)t]) ? 0 : (v[1] == minv[(size_t)t] ? 1 : 2);
    rot[(size_t)t] = (int8_t)r;
    for (int k = 0; k < 3; ++k) tri[3 * (int64_t)id + k] = v[(k + r) % 3];
  }
  for (int64_t t = 0; t < slots; ++t) {
    int32_t id = newid[(size_t)t];
    if (id < 0) continue;
    int r = rot[(size_t)t];
    for (int k = 0; k < 3; ++k) {
      int32_t ok = (k + r) % 3;  // old local edge index of new edge k
      int32_t oh = D.T[3 * (size_t)t + ok];
      int32_t ot = oh / 3, okk = oh % 3;
      int32_t nid = newid[(size_t)ot];
      int32_t tw = -1;
      if (nid >= 0) tw = 3 * nid + (okk - rot[(size_t)ot] + 3) % 3;
      twin[3 * (int64_t)id + k] = tw;
    }
  }
  return m;
}

// Many meshes at once on `threads` host threads.  Mesh i has n[i] points drawn
// with seed[i] (kind[i]: 0 uniform, 1 Gaussian mixture with 16 components and
// sigma in [0.5%, 5%] of the side) on a lattice of side[i].  Outputs are
// concatenated: points at xy + 2*vtx_off[i]; triangles and twins of mesh i start
// at 3 * (2 * (n[0] + ... + n[i-1])) in tri/twin (a capacity of 2*n[i] triangles
// per mesh), with vertex and half-edge ids local to the mesh.  tri_count[i]
// receives the number of triangles of mesh i.  Returns the total or a negative
// error.
int64_t mg_batch(int64_t count, const int64_t* n, const uint64_t* seed, const int32_t* kind,
                 const int64_t* side, const int64_t* vtx_off, int64_t* xy, int32_t* tri,
                 int32_t* twin, int64_t* tri_count, int32_t threads) {
  if (threads < 1) threads = 1;
  std::vector<int64_t> res((size_t)count, 0);
  std::vector<std::thread> pool;
  std::vector<int64_t> cap_off((size_t)count + 1, 0);
  for (int64_t i = 0; i < count; ++i) cap_off[(size_t)i + 1] = cap_off[(size_t)i] + 2 * n[i];
  std::vector<int64_t> order((size_t)count);
  for (int64_t i = 0; i < count; ++i) order[(size_t)i] = i;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return n[a] > n[b]; });
  std::atomic<int64_t> cursor(0);
  auto worker = [&]() {
    for (;;) {
      int64_t j = cursor.fetch_add(1);
      if (j >= count) return;
      int64_t i = order[(size_t)j];
      int64_t* pxy = xy + 2 * vtx_off[i];
      int64_t got = kind[i] == 0 ? mg_points_uniform(seed[i], n[i], side[i], pxy)
                                 : mg_points_gmm(seed[i], n[i], 16, side[i], 0.005, 0.05, pxy);
      if (got != n[i]) { res[(size_t)i] = -1; continue; }
      res[(size_t)i] = mg_delaunay(pxy, n[i], tri + 3 * cap_off[(size_t)i],
                                   twin + 3 * cap_off[(size_t)i], 2 * n[i]);
    }
  };
  for (int i = 0; i < threads; ++i) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  int64_t total = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (res[(size_t)i] < 0) return res[(size_t)i];
    tri_count[i] = res[(size_t)i];
    total += res[(size_t)i];
  }
  return total;
}

}  // extern "C"
