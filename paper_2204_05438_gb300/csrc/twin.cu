// The twin array from the triangles alone (the step before the paper's input: its
// Neighbor array, Section 2, comes from the triangulator).  Half-edge h = 3t + k
// runs from tri[h] to tri[3t + (k+1) % 3]; its twin is the half-edge running the
// other way, or -1.
//
//   k_twin_count   outgoing half-edges per vertex (atomics), and the per-tile sums
//                  of those counts for the tile scan;
//   k_twin_start   each vertex's first slot: its tile's offset + an in-tile scan;
//   k_twin_fill    every half-edge, with its destination, into its origin's slots;
//   k_twin_match   h = u->v finds v->u among v's outgoing half-edges (about six
//                  on a Delaunay mesh, one or two cache lines of (half-edge,
//                  destination) pairs).  A directed edge used twice, or an edge
//                  with more than two triangles, sets POLYLLA_ERR_TOPOLOGY: an
//                  edge with more than two triangles repeats a directed edge,
//                  and a repeated u->v is two hits for the thread of a v->u, or,
//                  with no v->u, two entries in u's list.
#include "polylla_internal.cuh"

namespace polylla {

constexpr int kTwinTile = kTriTile;  // vertices per tile of the count scan

// Lanes of a warp holding the same vertex add to its count with one atomic (the
// half-edges of neighbouring triangles share vertices).  The loop bound is
// rounded up to whole warps so that every lane takes part in the match.
__global__ void __launch_bounds__(kBlock) k_twin_count(const int* __restrict__ tri, long long m,
                                                       long long n, int* __restrict__ cnt,
                                                       Counters* C) {
  const long long H = 3 * m;
  const long long Hw = (H + 31) / 32 * 32;
  const int lane = threadIdx.x & 31;
  for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < Hw;
       h += (long long)gridDim.x * blockDim.x) {
    int v = h < H ? __ldg(tri + h) : -1;
    if (h < H && (v < 0 || v >= n)) {
      set_error(C, POLYLLA_ERR_RANGE, 140);
      v = -1;
    }
    const unsigned same = __match_any_sync(0xffffffffu, v);
    if (v >= 0 && lane == __ffs(same) - 1) atomicAdd(cnt + v, __popc(same));
  }
}

__global__ void __launch_bounds__(kBlock) k_twin_tiles(const int* __restrict__ cnt, long long n,
                                                       long long* __restrict__ tile_sum) {
  __shared__ long long sh[kBlock / 32];
  const long long ntiles = (n + kTwinTile - 1) / kTwinTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    long long s = 0;
    for (int j = threadIdx.x; j < kTwinTile; j += kBlock) {
      const long long v = tile * kTwinTile + j;
      if (v < n) s += cnt[v];
    }
    const long long tot = block_sum(s, sh);
    if (threadIdx.x == 0) {
      tile_sum[2 * tile] = tot;
      tile_sum[2 * tile + 1] = 0;
    }
  }
}

// start[v] = first slot of v; start[n] = 3m.  cnt is cleared for the fill.
__global__ void __launch_bounds__(kBlock) k_twin_start(int* __restrict__ cnt, long long n,
                                                       const long long* __restrict__ tile_off,
                                                       int* __restrict__ start, long long m) {
  __shared__ long long sh[kBlock / 32];
  constexpr int kPer = kTwinTile / kBlock;
  const long long ntiles = (n + kTwinTile - 1) / kTwinTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long v0 = tile * kTwinTile + (long long)threadIdx.x * kPer;
    int c[kPer];
    long long s = 0;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      c[j] = (v0 + j < n) ? cnt[v0 + j] : 0;
      s += c[j];
    }
    long long tot;
    long long p = tile_off[2 * tile] + block_exclusive_scan(s, &tot, sh);
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      if (v0 + j < n) {
        start[v0 + j] = (int)p;
        cnt[v0 + j] = 0;
      }
      p += c[j];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) start[n] = (int)(3 * m);
}

// Each origin's slots: the half-edges' destinations in adj_dst, the half-edges
// themselves at the same positions in adj_he.  Lanes with the same origin take
// consecutive slots from one atomic.
__global__ void __launch_bounds__(kBlock) k_twin_fill(const int* __restrict__ tri, long long m,
                                                      long long n, const int* __restrict__ start,
                                                      int* __restrict__ cnt,
                                                      int* __restrict__ adj_dst,
                                                      int* __restrict__ adj_he) {
  const long long H = 3 * m;
  const long long Hw = (H + 31) / 32 * 32;
  const int lane = threadIdx.x & 31;
  for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < Hw;
       h += (long long)gridDim.x * blockDim.x) {
    int v = h < H ? __ldg(tri + h) : -1;
    if (v >= n) v = -1;
    const unsigned same = __match_any_sync(0xffffffffu, v);
    const int leader = __ffs(same) - 1;
    int base = 0;
    if (v >= 0 && lane == leader) base = atomicAdd(cnt + v, __popc(same));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (v < 0) continue;
    const int q = start[v] + base + __popc(same & ((1u << lane) - 1u));
    adj_dst[q] = __ldg(tri + he_next((int)h));
    adj_he[q] = (int)h;
  }
}

__global__ void __launch_bounds__(kBlock) k_twin_match(const int* __restrict__ tri, long long m,
                                                       long long n, const int* __restrict__ start,
                                                       const int* __restrict__ adj_dst,
                                                       const int* __restrict__ adj_he,
                                                       int* __restrict__ twin, Counters* C) {
  const long long H = 3 * m;
  for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < H;
       h += (long long)gridDim.x * blockDim.x) {
    const int u = __ldg(tri + h);
    const int v = __ldg(tri + he_next((int)h));
    if (u < 0 || u >= n || v < 0 || v >= n) {
      twin[h] = -1;
      continue;
    }
    // the twin: v -> u among v's outgoing half-edges.  A second v -> u is a
    // non-manifold edge.  A second u -> v shows up as two hits in the scan of
    // u's list made for a v -> u, when there is one; so u's own list is scanned
    // only when h has no twin
    int g = -1, hits = 0;
    const int b0 = start[v], b1 = start[v + 1];
    for (int q = b0; q < b1; ++q) {
      if (__ldg(adj_dst + q) == u) {
        g = q;
        ++hits;
      }
    }
    if (hits) g = __ldg(adj_he + g);
    int same = 1;
    if (hits == 0) {
      same = 0;
      const int a0 = start[u], a1 = start[u + 1];
      for (int q = a0; q < a1; ++q) same += __ldg(adj_dst + q) == v;
    }
    if (hits > 1 || same != 1) set_error(C, POLYLLA_ERR_TOPOLOGY, 141);
    twin[h] = g;
  }
}

cudaError_t launch_build_twin(const int* tri, long long m, long long n, int* twin, int* cnt,
                              int* start, int2* adj, long long* tile_sum, long long* tile_off,
                              Counters* C, int sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n, s);
  if (e != cudaSuccess) return e;
  static std::atomic<int> c1{0}, c2{0}, c3{0}, c4{0}, c5{0};
  const long long H = 3 * m;
  const long long ntiles = (n + kTwinTile - 1) / kTwinTile;
  int g = resident_grid(reinterpret_cast<const void*>(k_twin_count), kBlock, 0,
                        (H + kBlock - 1) / kBlock, &c1);
  k_twin_count<<<g, kBlock, 0, s>>>(tri, m, n, cnt, C);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  g = resident_grid(reinterpret_cast<const void*>(k_twin_tiles), kBlock, 0, ntiles, &c2);
  k_twin_tiles<<<g, kBlock, 0, s>>>(cnt, n, tile_sum);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_scan_tiles(tile_sum, tile_off, n, nullptr, n, kTwinTile, &C->scratch0,
                             &C->scratch1, nullptr, 0, 0, C, s)) != cudaSuccess)
    return e;
  g = resident_grid(reinterpret_cast<const void*>(k_twin_start), kBlock, 0, ntiles, &c3);
  k_twin_start<<<g, kBlock, 0, s>>>(cnt, n, tile_off, start, m);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the pair buffer (3m int2) as two int arrays of 3m
  int* adj_dst = reinterpret_cast<int*>(adj);
  int* adj_he = adj_dst + H;
  g = resident_grid(reinterpret_cast<const void*>(k_twin_fill), kBlock, 0,
                    (H + kBlock - 1) / kBlock, &c4);
  k_twin_fill<<<g, kBlock, 0, s>>>(tri, m, n, start, cnt, adj_dst, adj_he);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  g = resident_grid(reinterpret_cast<const void*>(k_twin_match), kBlock, 0,
                    (H + kBlock - 1) / kBlock, &c5);
  (void)sms;
  k_twin_match<<<g, kBlock, 0, s>>>(tri, m, n, start, adj_dst, adj_he, twin, C);
  return cudaGetLastError();
}

}  // namespace polylla

namespace polylla {

// ------------------------------------------------------------------ Neighbor array
// The twin array from the triangulator's Neighbor array (Section 2): nb[3t + j] is
// the triangle across edge j of t, or -1 on the border.  Edge j is the one
// opposite vertex j (convention 0, the layout of Triangle's .neigh files) or the
// one from vertex j to vertex j+1 (convention 1).  The twin of h = 3t + k (from
// u = tri[h] to v = tri[3t + (k+1) % 3]) is the half-edge v -> u of that
// neighbour; a neighbour id outside [-1, m) is POLYLLA_ERR_RANGE, a neighbour
// without the reversed edge POLYLLA_ERR_TOPOLOGY (the twin is then -1).
__global__ void __launch_bounds__(kBlock) k_twin_from_neighbor(const int* __restrict__ tri,
                                                               const int* __restrict__ nb,
                                                               long long m, int convention,
                                                               int* __restrict__ twin,
                                                               Counters* C) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x) {
    const int a[3] = {__ldg(tri + 3 * t), __ldg(tri + 3 * t + 1), __ldg(tri + 3 * t + 2)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int j = convention ? k : (k + 2) % 3;  // the edge u -> v is opposite vertex k+2
      const int u = __ldg(nb + 3 * t + j);
      int g = -1;
      if (u >= 0 && u < m) {
        const int from = a[(k + 1) % 3], to = a[k];  // the twin runs v -> u
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (__ldg(tri + 3LL * u + q) == from && __ldg(tri + 3LL * u + (q + 1) % 3) == to)
            g = 3 * u + q;
        if (g < 0) set_error(C, POLYLLA_ERR_TOPOLOGY, 150);
      } else if (u < -1 || u >= m) {
        set_error(C, POLYLLA_ERR_RANGE, 151);
      }
      twin[3 * t + k] = g;
    }
  }
}

cudaError_t launch_twin_from_neighbor(const int* tri, const int* nb, long long m, int convention,
                                      int* twin, Counters* C, int grid, cudaStream_t s) {
  static std::atomic<int> cap{0};
  grid = resident_grid(reinterpret_cast<const void*>(k_twin_from_neighbor), kBlock, 0, grid, &cap);
  k_twin_from_neighbor<<<grid, kBlock, 0, s>>>(tri, nb, m, convention, twin, C);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Trivertex
// The Trivertex array (Section 2: one element incident to each vertex; the
// paper's reparation reaches a tip's fan through it): for every vertex, the
// smallest half-edge leaving it, or -1 for a vertex no triangle uses.  tv starts
// as all ones (0xffffffff = -1); each half-edge lowers its origin's word.
__global__ void __launch_bounds__(kBlock) k_trivertex(const int* __restrict__ tri, long long m,
                                                      long long n, unsigned* __restrict__ tv,
                                                      Counters* C) {
  const long long H = 3 * m;
  for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < H;
       h += (long long)gridDim.x * blockDim.x) {
    const int v = __ldg(tri + h);
    if (v < 0 || v >= n) {
      set_error(C, POLYLLA_ERR_RANGE, 152);
      continue;
    }
    atomicMin(tv + v, (unsigned)h);
  }
}

cudaError_t launch_trivertex(const int* tri, long long m, long long n, int* tv, Counters* C,
                             int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(tv, 0xff, sizeof(int) * (size_t)n, s);
  if (e != cudaSuccess) return e;
  static std::atomic<int> cap{0};
  grid = resident_grid(reinterpret_cast<const void*>(k_trivertex), kBlock, 0, grid, &cap);
  k_trivertex<<<grid, kBlock, 0, s>>>(tri, m, n, reinterpret_cast<unsigned*>(tv), C);
  return cudaGetLastError();
}

}  // namespace polylla
