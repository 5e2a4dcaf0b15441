// The region walk shared by traversal and reparation (Algorithm 4,
// PolyConstruction, restated on half-edges).
//
// From a frontier half-edge h of a terminal-edge region, the next frontier
// half-edge of the region's boundary is found by turning around the endpoint of
// h through internal edges:
//     g = next(h);  while (g is not frontier) g = next(twin(g));
// The walk stays inside the region (it never crosses a frontier edge), visits
// the boundary ccw with the region on its left, and each frontier half-edge
// contributes its origin vertex.  Every step is bounded (3m + 3 in total) and
// every twin is range-checked, so a corrupt mesh ends in an error, not a hang.
#pragma once

#include "polylla_internal.cuh"

namespace polylla {

struct WalkInfo {
  int start;  // frontier half-edge with the smallest (origin, id): the canonical start
  int len;    // number of frontier half-edges = polygon length
  int tip_h;  // barrier half-edge a->b ending at the smallest tip vertex b, or -1
  int ntips;  // barrier-edge tips (v_a == v_c on consecutive vertices)
  bool ok;
};

// Next frontier half-edge after h; returns -1 on a bound violation.
__device__ __forceinline__ int walk_step(const int* __restrict__ tri, const int* __restrict__ twin,
                                         const uint8_t* lab, int h, int H, long long& steps,
                                         long long limit) {
  (void)tri;
  int g = he_next(h);
  while (!lab_frontier(lab, g)) {
    const int tw = twin[g];
    if ((unsigned)tw >= (unsigned)H || ++steps > limit) return -1;
    g = he_next(tw);
  }
  if (++steps > limit) return -1;
  return g;
}

// A frontier half-edge of the region of triangle t: a frontier edge of t if it
// has one, else the first frontier half-edge met turning around tri[3t] (the
// shortest edge at every vertex is a frontier edge, so this ends).
__device__ __forceinline__ int region_entry(const int* __restrict__ twin, const uint8_t* lab, int t,
                                            int H, long long limit) {
  const unsigned fr = (lab[t] >> 2) & 7u;
  if (fr) return 3 * t + (__ffs(fr) - 1);
  int g = 3 * t;
  long long steps = 0;
  while (!lab_frontier(lab, g)) {
    const int tw = twin[g];
    if ((unsigned)tw >= (unsigned)H || ++steps > limit) return -1;
    g = he_next(tw);
  }
  return g;
}

// Walk the whole boundary cycle through h0: length, canonical start and tips.
__device__ __forceinline__ WalkInfo walk_cycle(const int* __restrict__ tri,
                                               const int* __restrict__ twin, const uint8_t* lab,
                                               int h0, int H, long long limit) {
  WalkInfo w;
  w.start = h0;
  w.len = 0;
  w.tip_h = -1;
  w.ntips = 0;
  w.ok = false;
  long long steps = 0;
  int best_o = 0x7fffffff, best_h = 0x7fffffff;
  int v0 = -1, v1 = -1;
  int pp_o = -1, p_o = -1, pp_h = -1, p_h = -1;
  int tip_v = 0x7fffffff;
  int h = h0;
  int len = 0;
  do {
    const int o = tri[h];
    if (o < best_o || (o == best_o && h < best_h)) {
      best_o = o;
      best_h = h;
    }
    if (len >= 2 && pp_o == o) {  // consecutive v_a, v_b, v_c with v_a == v_c
      ++w.ntips;
      if (p_o < tip_v) {
        tip_v = p_o;
        w.tip_h = pp_h;
      }
    }
    if (len == 0) v0 = o;
    if (len == 1) v1 = o;
    pp_o = p_o;
    pp_h = p_h;
    p_o = o;
    p_h = h;
    ++len;
    h = walk_step(tri, twin, lab, h, H, steps, limit);
    if (h < 0) return w;
  } while (h != h0);
  if (len >= 3) {  // the two cyclic triples that wrap around the start
    if (pp_o == v0) {
      ++w.ntips;
      if (p_o < tip_v) {
        tip_v = p_o;
        w.tip_h = pp_h;
      }
    }
    if (p_o == v1) {
      ++w.ntips;
      if (v0 < tip_v) {
        tip_v = v0;
        w.tip_h = p_h;
      }
    }
  }
  w.start = best_h;
  w.len = len;
  w.ok = true;
  return w;
}

// Write the origins of `len` consecutive frontier half-edges starting at h.
__device__ __forceinline__ bool walk_write(const int* __restrict__ tri, const int* __restrict__ twin,
                                           const uint8_t* lab, int h, int len, int H,
                                           long long limit, int* __restrict__ out) {
  long long steps = 0;
  for (int j = 0; j < len; ++j) {
    out[j] = tri[h];
    if (j + 1 < len) {
      h = walk_step(tri, twin, lab, h, H, steps, limit);
      if (h < 0) return false;
    }
  }
  return true;
}

}  // namespace polylla
