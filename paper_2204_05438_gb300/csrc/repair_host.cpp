// Sequential reparation on the host: the paper's "mixed" variant (Section 3.2,
// Section 4: GPU labelling and traversal, then the reparation phase on the CPU,
// which the paper found faster than its GPU reparation for the few polygons that
// need it).
//
// Input: the mesh (tri, twin), the frontier bits of the label bytes and the
// traversal polygons as vertex lists (CSR).  Section 3.2.3: a polygon with a
// barrier-edge tip (consecutive vertices v_a, v_b, v_a) is split at the middle
// internal edge of the tip's fan, found through the Trivertex array; here one
// thread repairs the polygons one after another:
//   * the polygon's first half-edge v0 -> v1 is found among the half-edges leaving
//     v0 (the Trivertex array gives one, the rest by rotating around v0);
//   * its pieces are kept in order by their start half-edges; the first piece with
//     a tip is re-walked (turning around each vertex through internal edges, as in
//     Algorithm 4), split at its smallest tip b along e_ceil(k/2) -- the k
//     internal edges at b counted ccw after the barrier edge -- which becomes a
//     frontier edge, and replaced by the piece containing the new half-edge b -> x
//     followed by the other one;
//   * finished pieces are written from their canonical start (smallest (origin,
//     half-edge)).
// This gives exactly the polygons of the device reparation (the same readings of
// the paper: smallest tip first, the middle internal edge, halves in place).
#include <cstdint>
#include <cstring>
#include <vector>

namespace polylla {

namespace {

inline int64_t nxt(int64_t h) { return (h % 3 == 2) ? h - 2 : h + 1; }
inline int64_t prv(int64_t h) { return (h % 3 == 0) ? h + 2 : h - 1; }

struct HostMesh {
  const int32_t* tri;
  const int32_t* twin;
  uint8_t* lab;  // label bytes; frontier bits 2-4 updated by the splits
  int64_t m;
  bool fr(int64_t h) const { return (lab[h / 3] >> (2 + h % 3)) & 1; }
  void set_fr(int64_t h) { lab[h / 3] |= (uint8_t)(1u << (2 + h % 3)); }
  int64_t dest(int64_t h) const { return tri[nxt(h)]; }
  // next frontier half-edge of the region boundary after frontier half-edge h
  int64_t turn(int64_t h) const {
    int64_t g = nxt(h);
    for (int64_t steps = 0; !fr(g); ++steps) {
      const int64_t t = twin[g];
      if (t < 0 || steps > 3 * m) return -1;
      g = nxt(t);
    }
    return g;
  }
};

// One piece: its walk from start half-edge h0, with length, canonical start and
// the barrier half-edge a -> b of its smallest tip b (or -1).
struct Walk {
  int64_t len = 0, start = -1, tip = -1;
  bool ok = false;
};

Walk walk_piece(const HostMesh& M, int64_t h0) {
  Walk w;
  int64_t h = h0;
  int64_t best_o = INT64_MAX, best_h = INT64_MAX, tipv = INT64_MAX;
  do {
    const int64_t o = M.tri[h];
    if (o < best_o || (o == best_o && h < best_h)) {
      best_o = o;
      best_h = h;
    }
    const int64_t g = M.turn(h);
    if (g < 0) return w;
    if (g == M.twin[h]) {  // the boundary turns back along h: dest(h) is a tip
      const int64_t b = M.dest(h);
      if (b < tipv) {
        tipv = b;
        w.tip = h;
      }
    }
    ++w.len;
    if (w.len > 3 * M.m) return w;
    h = g;
  } while (h != h0);
  w.start = best_h;
  w.ok = true;
  return w;
}

// The split edge at the tip b of barrier half-edge p = a -> b: o0 = b -> a, then the
// internal edges o_s = twin(prev(o_{s-1})) ccw around b; returns o_ceil(k/2), or -1.
int64_t middle_internal_edge(const HostMesh& M, int64_t p) {
  const int64_t o0 = M.twin[p];
  if (o0 < 0) return -1;
  std::vector<int64_t> fan;
  for (int64_t o = M.twin[prv(o0)]; o != o0; o = M.twin[prv(o)]) {
    if (o < 0 || M.fr(o) || (int64_t)fan.size() > 3 * M.m) return -1;
    fan.push_back(o);
  }
  const int64_t k = (int64_t)fan.size();
  if (k < 2) return -1;
  return fan[(size_t)((k + 1) / 2 - 1)];
}

}  // namespace

// Returns the number of splits, or -1 if a polygon could not be repaired (its
// first half-edge not found, a walk or a fan out of bounds).  out_off needs
// n_poly_in + splits + 1 entries (at most m + 1), out_vtx the final length (at most
// 3m).
int64_t host_repair(int64_t n, int64_t m, const int32_t* tri, const int32_t* twin, uint8_t* lab,
                    const int64_t* off, const int32_t* vtx, int64_t n_poly, int64_t* out_off,
                    int32_t* out_vtx, int64_t* out_np, int64_t* out_nv) {
  HostMesh M{tri, twin, lab, m};
  // Trivertex: the smallest half-edge leaving each vertex
  std::vector<int64_t> tv((size_t)n, -1);
  for (int64_t h = 0; h < 3 * m; ++h)
    if (tv[(size_t)tri[h]] < 0) tv[(size_t)tri[h]] = h;
  int64_t np = 0, nv = 0, splits = 0;
  out_off[0] = 0;
  std::vector<int64_t> pieces;
  for (int64_t i = 0; i < n_poly; ++i) {
    const int32_t* v = vtx + off[i];
    const int64_t L = off[i + 1] - off[i];
    bool tips = false;
    for (int64_t k = 0; k < L && !tips; ++k) tips = v[k] == v[(k + 2) % L];
    if (!tips || L < 3) {  // unchanged
      std::memcpy(out_vtx + nv, v, sizeof(int32_t) * (size_t)L);
      nv += L;
      out_off[++np] = nv;
      continue;
    }
    // the half-edge v0 -> v1 among those leaving v0: ccw from the Trivertex entry,
    // then cw (v0 may lie on the border)
    int64_t h0 = -1;
    const int64_t first = tv[(size_t)v[0]];
    for (int64_t o = first, s = 0; o >= 0 && s <= 3 * m; ++s) {
      if (M.dest(o) == v[1] && M.fr(o)) {
        h0 = o;
        break;
      }
      o = twin[prv(o)];
      if (o == first) break;
    }
    for (int64_t o = first, s = 0; h0 < 0 && o >= 0 && s <= 3 * m; ++s) {
      if (M.dest(o) == v[1] && M.fr(o)) h0 = o;
      const int64_t t = twin[o];
      o = t < 0 ? -1 : nxt(t);
      if (o == first) break;
    }
    if (h0 < 0) return -1;
    pieces.assign(1, h0);
    for (size_t j = 0; j < pieces.size();) {
      const Walk w = walk_piece(M, pieces[j]);
      if (!w.ok) return -1;
      if (w.tip < 0) {  // finished: from its canonical start
        int64_t h = w.start;
        for (int64_t k = 0; k < w.len; ++k) {
          out_vtx[nv++] = tri[h];
          h = M.turn(h);
          if (h < 0) return -1;
        }
        out_off[++np] = nv;
        ++j;
        continue;
      }
      const int64_t oj = middle_internal_edge(M, w.tip);
      if (oj < 0 || twin[oj] < 0) return -1;
      M.set_fr(oj);
      M.set_fr(twin[oj]);
      ++splits;
      pieces[j] = oj;  // the piece containing tip -> x first
      pieces.insert(pieces.begin() + (int64_t)j + 1, (int64_t)twin[oj]);
    }
  }
  *out_np = np;
  *out_nv = nv;
  return splits;
}

}  // namespace polylla
