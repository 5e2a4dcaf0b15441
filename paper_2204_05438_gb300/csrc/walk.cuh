// Region-boundary walks shared by traversal and reparation (Algorithm 4,
// PolyConstruction, restated on half-edges).
//
// From a frontier half-edge h of a terminal-edge region, the next frontier
// half-edge of the region's boundary is found by turning around the endpoint of
// h through internal edges:
//     g = next(h);  while (g is not frontier) g = next(twin(g));
// The walk stays inside the region (it never crosses a frontier edge), visits the
// boundary ccw with the region on its left, and each frontier half-edge
// contributes its origin vertex.
//
// The turn is precomputed once per frontier half-edge into succ[h] (k_succ), so a
// polygon walk is a chase of one dependent load per vertex.  Bit 31 of succ[h]
// flags a barrier-edge tip: succ(h) == twin(h), i.e. consecutive polygon vertices
// v_a, v_b, v_a with v_b = dest(h) (Section 3.2.3).  Every loop is bounded and every
// index range-checked, so a corrupt mesh ends in an error, not a hang.
#pragma once

#include "polylla_internal.cuh"

namespace polylla {

constexpr int kTipFlag = 1 << 31;
constexpr int kSuccMask = 0x7fffffff;
constexpr int kWalkCap = 64;  // longer polygons go to one thread block each (long.cu)

// Next frontier half-edge after h by turning through internal edges, or -1.
__device__ __forceinline__ int turn_to_frontier(const int* __restrict__ twin, const uint8_t* lab,
                                                int h, int H, long long limit) {
  int g = he_next(h);
  long long steps = 0;
  while (!lab_frontier(lab, g)) {
    const int tw = twin[g];
    if ((unsigned)tw >= (unsigned)H || ++steps > limit) return -1;
    g = he_next(tw);
  }
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

// region_entry on tf words (sign = frontier, low bits = twin).
__device__ __forceinline__ int region_entry_tf(const int* __restrict__ tf, int t, int H,
                                               long long limit) {
  int g = 3 * t;
  for (int k = 0; k < 3; ++k)
    if (tf[3 * t + k] < 0) return 3 * t + k;
  long long steps = 0;
  for (;;) {
    const int x = tf[g];
    if (x < 0) return g;
    if (x >= H || ++steps > limit) return -1;
    g = he_next(x);
  }
}

// Canonical key of a frontier half-edge: (origin vertex, half-edge id).
__device__ __forceinline__ unsigned long long he_key(const int* __restrict__ tri, int h) {
  return ((unsigned long long)(unsigned)tri[h] << 32) | (unsigned)h;
}

struct CycleInfo {
  int start;  // half-edge with the smallest (origin, id): the canonical start
  int len;    // number of frontier half-edges = polygon length
  int ntips;  // barrier-edge tips on the cycle
  bool ok;
};

// Walk the succ cycle through h0 (length, canonical start, tip count).  When
// tip_out is given, the barrier half-edge of every tip is appended to it.
__device__ __forceinline__ CycleInfo succ_cycle(const int* __restrict__ tri, const int* succ,
                                                int h0, int H, long long limit, int* tip_out,
                                                int tip_cap) {
  CycleInfo c;
  c.start = h0;
  c.len = 0;
  c.ntips = 0;
  c.ok = false;
  unsigned long long best = ~0ull;
  int h = h0;
  long long steps = 0;
  do {
    const unsigned long long k = he_key(tri, h);
    if (k < best) best = k;
    const int s = succ[h];
    if (s & kTipFlag) {
      if (tip_out && c.ntips < tip_cap) tip_out[c.ntips] = h;
      ++c.ntips;
    }
    ++c.len;
    h = s & kSuccMask;
    if ((unsigned)h >= (unsigned)H || ++steps > limit) return c;
  } while (h != h0);
  c.start = (int)(best & 0xffffffffu);
  c.ok = true;
  return c;
}

// Write the origins of the `len` half-edges of the succ cycle starting at h.
__device__ __forceinline__ bool succ_write(const int* __restrict__ tri, const int* succ, int h,
                                           int len, int H, int* __restrict__ out) {
  for (int j = 0; j < len; ++j) {
    if ((unsigned)h >= (unsigned)H) return false;
    out[j] = tri[h];
    h = succ[h] & kSuccMask;
  }
  return true;
}

}  // namespace polylla
