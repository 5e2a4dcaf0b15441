// Region-boundary walks and the sequential reparation of one polygon
// (Algorithms 4 and 5, restated on half-edges).
//
// From a frontier half-edge h of a terminal-edge region, the next frontier
// half-edge of the region's boundary is found by turning around the endpoint of
// h through internal edges:
//     g = next(h);  while (g is not frontier) g = next(twin(g));
// The walk stays inside the region (it never crosses a frontier edge), visits the
// boundary ccw with the region on its left, and each frontier half-edge
// contributes its origin vertex.  A turn reads one tf word per step: tf[g] < 0
// iff g is frontier, and its low 31 bits are twin(g).
//
// The turn of every frontier half-edge is also precomputed into succ[h] (k_succ)
// for the first walk; bit 31 of succ[h] flags a barrier-edge tip: succ(h) ==
// twin(h), i.e. consecutive polygon vertices v_a, v_b, v_a with v_b = dest(h)
// (Section 3.2.3).  Every loop is bounded and every index range-checked, so a
// corrupt mesh ends in an error code, not a hang or a stray access.
#pragma once

#include "polylla_internal.cuh"

namespace polylla {

constexpr int kTipFlag = 1 << 31;
constexpr int kSuccMask = 0x7fffffff;

__device__ __forceinline__ int tf_twin(int x) { return x & 0x7fffffff; }

// Canonical key of a frontier half-edge: (origin vertex, half-edge id).
__device__ __forceinline__ unsigned long long he_key(const int* __restrict__ tri, int h) {
  return ((unsigned long long)(unsigned)tri[h] << 32) | (unsigned)h;
}

// A frontier half-edge of the region of triangle t: a frontier edge of t if it
// has one, else the first frontier half-edge met turning around tri[3t] (the
// shortest edge at every vertex is a frontier edge, so this ends).
__device__ __forceinline__ int region_entry_tf(const int* tf, int t, int H, long long limit) {
  for (int k = 0; k < 3; ++k)
    if (tf[3 * t + k] < 0) return 3 * t + k;
  int g = 3 * t;
  long long steps = 0;
  for (;;) {
    const int x = tf[g];
    if (x < 0) return g;
    if (x >= H || ++steps > limit) return -1;
    g = he_next(x);
  }
}

// Next frontier half-edge after h (the turn), or -1 on a bound violation.
__device__ __forceinline__ int turn_tf(const int* tf, int h, int H, long long& steps,
                                      long long limit) {
  int g = he_next(h);
  int x = tf[g];
  while (x >= 0) {
    if (x >= H || ++steps > limit) return -1;
    g = he_next(x);
    x = tf[g];
  }
  return g;
}

struct Cyc {
  int start;  // canonical start: the frontier half-edge with the smallest (origin, id)
  int len;
  int tip_h;  // barrier half-edge a->b ending at the smallest tip vertex b, or -1
  int ntips;
  bool ok;
};

// Walk the cycle through h0 with on-the-fly turns (current labels).
__device__ __forceinline__ Cyc cycle_tf(const int* __restrict__ tri, const int* tf, int h0, int H,
                                        long long limit) {
  Cyc c{h0, 0, -1, 0, false};
  unsigned long long best = ~0ull;
  int tipv = 0x7fffffff;
  long long steps = 0;
  int h = h0;
  do {
    const unsigned long long key = he_key(tri, h);
    if (key < best) best = key;
    const int g = turn_tf(tf, h, H, steps, limit);
    if (g < 0) return c;
    if (g == tf_twin(tf[h])) {  // the boundary turns back along h: dest(h) is a tip
      ++c.ntips;
      const int b = tri[g];
      if (b < tipv) {
        tipv = b;
        c.tip_h = h;
      }
    }
    ++c.len;
    h = g;
    if (++steps > limit) return c;
  } while (h != h0);
  c.start = (int)(best & 0xffffffffu);
  c.ok = true;
  return c;
}

// Write the origins of `len` consecutive frontier half-edges from h.
__device__ __forceinline__ bool write_tf(const int* __restrict__ tri, const int* tf, int h, int len,
                                         int H, long long limit, int* __restrict__ out) {
  long long steps = 0;
  for (int j = 0; j < len; ++j) {
    out[j] = tri[h];
    if (j + 1 < len) {
      h = turn_tf(tf, h, H, steps, limit);
      if (h < 0) return false;
    }
  }
  return true;
}

// Mark half-edge h frontier in tf and in its triangle's label byte.  Several
// split edges may touch one triangle, so both are atomic ORs.
__device__ __forceinline__ void set_frontier(uint8_t* lab, int* tf, int h) {
  atomicOr(tf + h, (int)0x80000000u);
  const int t = h / 3;
  const unsigned bit = 1u << (2 + (h - 3 * t));
  unsigned* word = reinterpret_cast<unsigned*>(lab + (t & ~3));
  atomicOr(word, bit << (8 * (t & 3)));
}

// The split edge of a barrier-edge tip (Section 3.2.3): with o_0 = b->a the
// barrier half-edge leaving the tip b and o_j = twin(prev(o_{j-1})) the k internal
// edges that follow ccw, the middle internal edge e_ceil(k/2) = o_ceil(k/2).
// barrier = a->b.  Returns o_ceil(k/2), or -1 if b is not a tip of an interior fan
// (a border or another frontier edge at b, or k < 2).
//
// The fan is walked from both ends at once -- forward o_1, o_2, ... and backward
// o_k = next(a->b), o_{k-1} = next(twin(o_k)), ... -- until the two meet, so k
// need not be known first and the chain of dependent loads is about k/2 long.
__device__ __forceinline__ int split_edge(const int* tf, int barrier, int H) {
  const int o0 = tf_twin(tf[barrier]);
  if (o0 >= H) return -1;
  int fwd = tf_twin(tf[he_prev(o0)]);  // o_s
  int bwd = he_next(barrier);          // o_{k+1-s}
  for (int s = 1; s <= H; ++s) {
    if (fwd >= H || fwd == o0) return -1;
    const int tfw = tf[fwd];
    const int tbw = tf[bwd];
    const int pf = tf[he_prev(fwd)];
    if (tfw < 0 || tbw < 0) return -1;  // o_s or o_{k+1-s} is frontier
    if (fwd == bwd) return s >= 2 ? fwd : -1;  // k = 2s - 1
    const int nf = tf_twin(pf);
    if (nf == bwd) return fwd;  // k = 2s
    fwd = nf;
    bwd = he_next(tf_twin(tbw));
  }
  return -1;
}

// Reparation of one polygon by one thread (Algorithm 5 with Algorithm 1's loop,
// per polygon).  The polygon is kept as an ordered list of pieces (their start
// half-edges in ps[]); the first piece with a tip is split at its smallest tip
// along split_edge(), which becomes frontier, and is replaced in place by the
// piece left of tip->x followed by the other one.  A split removes its tip (and x,
// if x is a tip) and creates none, so at most ntips + 1 pieces arise.  Finished
// pieces are written from their canonical start into out[], in order; piece j gets
// (pool position pos[j], length len[j]).  `first` is the walk of the whole
// polygon.  out[] holds out_cap entries (the polygon's length plus two per tip
// suffices for a valid mesh; a corrupt one may walk longer pieces, which end the
// split with an error instead of writing past it).  Returns the number of
// pieces, or -1 on an error.
__device__ __forceinline__ int repair_seq(const int* __restrict__ tri, int* tf, uint8_t* lab,
                                          Cyc first, int cap, int H, long long limit, int* ps,
                                          long long* pos, int* plen, int* out, long long out0,
                                          long long out_cap) {
  int count = 1;
  ps[0] = first.start;
  Cyc cur = first;
  bool known = true;
  long long acc = 0;
  int j = 0;
  while (j < count) {
    if (!known) {
      cur = cycle_tf(tri, tf, ps[j], H, limit);
      if (!cur.ok) return -1;
    }
    known = false;
    if (cur.tip_h < 0) {
      if (acc + cur.len > out_cap) return -1;
      if (!write_tf(tri, tf, cur.start, cur.len, H, limit, out + acc)) return -1;
      pos[j] = out0 + acc;
      plen[j] = cur.len;
      acc += cur.len;
      ++j;
      continue;
    }
    if (count + 1 > cap) return -1;
    const int oj = split_edge(tf, cur.tip_h, H);
    if (oj < 0) return -1;
    const int tw = tf_twin(tf[oj]);
    if (tw >= H) return -1;
    set_frontier(lab, tf, oj);
    set_frontier(lab, tf, tw);
    for (int q = count; q > j + 1; --q) ps[q] = ps[q - 1];
    ps[j] = oj;
    ps[j + 1] = tw;
    ++count;
  }
  return count;
}

}  // namespace polylla
