// Traversal phase (Section 3.2.2, Algorithms 3 and 4).
//
//   k_succ        one thread per triangle: for each frontier half-edge, the next
//                 frontier half-edge of its region's boundary (the turn of
//                 PolyConstruction), with the barrier-edge tip flag.
//   k_trav_count  one seed per thread (grid-stride, no block barriers): enter the
//                 region, chase succ around the cycle, record the canonical start,
//                 the length, and every barrier-edge tip (appended to the tip list
//                 with its polygon and its vertex -> tip map entry).  A cycle
//                 longer than kWalkCap goes to k_long_trav (long.cu).
//   k_len_tiles / k_offsets  per-tile length sums, then (after the tile scan) each
//                 polygon's CSR offset -- the paper's AtomicAdd on i_Gmesh / i_Gpos
//                 becomes this deterministic scan.
//   k_trav_write  one polygon per thread: chase succ from the canonical start
//                 writing origins.
#include "walk.cuh"

namespace polylla {

// The three turns of a triangle advance together (independent loads in flight);
// each step reads one tf word: its sign says frontier, its low bits the twin.
__global__ void __launch_bounds__(kBlock) k_succ(DevMesh M, const int* __restrict__ tf,
                                                 int* __restrict__ succ, Counters* C) {
  const long long m = M.m;
  const int H = (int)(3 * m);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x) {
    int x[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = __ldg(tf + 3 * t + k);
    int cur[3], y[3];
    unsigned active = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (x[k] >= 0) continue;  // not frontier: no successor
      const int kn = (k == 2) ? 0 : k + 1;
      cur[k] = (int)(3 * t + kn);
      y[k] = x[kn];
      active |= 1u << k;
    }
    for (long long step = 0; active && step <= 3 * m; ++step) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        if (!((active >> k) & 1u)) continue;
        if (y[k] < 0) {  // reached a frontier half-edge
          const int h = (int)(3 * t + k);
          const int g = cur[k];
          succ[h] = (g == (x[k] & 0x7fffffff)) ? (g | kTipFlag) : g;
          active &= ~(1u << k);
          continue;
        }
        const int tw = y[k];
        if (tw >= H) {
          set_error(C, POLYLLA_ERR_LIMIT, 50);
          succ[3 * t + k] = (int)(3 * t + k);
          active &= ~(1u << k);
          continue;
        }
        cur[k] = he_next(tw);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if ((active >> k) & 1u) y[k] = tf[cur[k]];
    }
    if (active) set_error(C, POLYLLA_ERR_LIMIT, 50);
  }
}

cudaError_t launch_succ(const DevMesh& M, const int* tf, int* succ, Counters* C, int grid,
                        cudaStream_t s) {
  k_succ<<<grid, kBlock, 0, s>>>(M, tf, succ, C);
  return cudaGetLastError();
}

constexpr int kLocalTips = 8;

// Walks stop after kWalkCap half-edges: a longer polygon is handed to one block of
// k_long_trav (mode 1), so that no single thread walks a thousand-vertex cycle.
__global__ void __launch_bounds__(kBlock) k_trav_count(DevMesh M, const uint8_t* __restrict__ lab,
                                                       const int* __restrict__ seeds,
                                                       const int* __restrict__ succ,
                                                       PolyArrays P, TipArrays T, LongList Lg,
                                                       int epoch, Counters* C) {
  const long long n = C->n_seeds;
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  long long my_len = 0, my_tips = 0, my_tip_polys = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = seeds[i];
    const int e = region_entry(M.twin, lab, s, H, limit);
    int tips[kLocalTips];
    CycleInfo c;
    c.ok = false;
    if (e >= 0) c = succ_cycle(M.tri, succ, e, H, kWalkCap, tips, kLocalTips);
    if (e >= 0 && !c.ok && c.len >= kWalkCap) {
      // long polygon: one block of k_long_trav takes it over
      P.mode[i] = 1;
      P.len[i] = 0;
      P.ntip[i] = 0;
      const long long j = (long long)atomicAdd(
          reinterpret_cast<unsigned long long*>(&C->n_long), 1ull);
      if (j < Lg.cap) Lg.poly[j] = (int)i;
      continue;
    }
    P.mode[i] = 0;
    if (!c.ok) {
      set_error(C, POLYLLA_ERR_LIMIT, 51);
      c.start = 3 * s;
      c.len = 0;
      c.ntips = 0;
    }
    P.start[i] = c.start;
    P.len[i] = c.len;
    P.ntip[i] = c.ntips;
    my_len += c.len;
    if (c.ntips > 0) {
      my_tips += c.ntips;
      my_tip_polys += 1;
      const long long base = (long long)atomicAdd(
          reinterpret_cast<unsigned long long*>(&C->n_tips), (unsigned long long)c.ntips);
      P.tipbase[i] = (int)base;
      if (base + c.ntips > T.cap) {
        set_error(C, POLYLLA_ERR_LIMIT, 52);
        P.ntip[i] = 0;
        continue;
      }
      if (c.ntips > kLocalTips) {  // rare: record every tip with a second walk
        succ_cycle(M.tri, succ, e, H, limit, T.h + base, c.ntips);
      } else {
        for (int q = 0; q < c.ntips; ++q) T.h[base + q] = tips[q];
      }
      for (int q = 0; q < c.ntips; ++q) {
        const int g = T.h[base + q];
        T.poly[base + q] = (int)i;
        const int b = M.tri[he_next(g)];  // the tip vertex: dest of the barrier half-edge
        T.vtip[b] = ((long long)epoch << 32) | (unsigned)(base + q);
      }
    }
  }
  // warp-aggregated statistics
  my_len = __reduce_add_sync(0xffffffffu, (unsigned)my_len);
  my_tip_polys = __reduce_add_sync(0xffffffffu, (unsigned)my_tip_polys);
  if ((threadIdx.x & 31) == 0) {
    if (my_len)
      atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_vtx_trav), (unsigned long long)my_len);
    if (my_tip_polys)
      atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tip_polys),
                (unsigned long long)my_tip_polys);
  }
  (void)my_tips;
}

cudaError_t launch_trav_count(const DevMesh& M, const uint8_t* lab, const int* seeds,
                              const int* succ, const PolyArrays& P, const TipArrays& T,
                              const LongList& Lg, int epoch, Counters* C, int grid,
                              cudaStream_t s) {
  k_trav_count<<<grid, kBlock, 0, s>>>(M, lab, seeds, succ, P, T, Lg, epoch, C);
  return cudaGetLastError();
}

// Per-tile sums of the traversal polygon lengths.
__global__ void __launch_bounds__(kBlock) k_len_tiles(const int* __restrict__ len,
                                                      long long* __restrict__ tile_sum,
                                                      Counters* C) {
  __shared__ long long sh[kBlock / 32];
  const long long n = C->n_seeds;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    const long long v = (i < n) ? len[i] : 0;
    const long long tot = block_sum(v, sh);
    if (threadIdx.x == 0) {
      tile_sum[2 * tile] = tot;
      tile_sum[2 * tile + 1] = 0;
    }
  }
}

cudaError_t launch_len_tiles(const int* len, long long* tile_sum, Counters* C, int grid,
                             cudaStream_t s) {
  k_len_tiles<<<grid, kBlock, 0, s>>>(len, tile_sum, C);
  return cudaGetLastError();
}

// off[i] = tile offset + block-exclusive scan of the lengths.
__global__ void __launch_bounds__(kBlock) k_offsets(const int* __restrict__ len,
                                                    const long long* __restrict__ tile_off,
                                                    long long* __restrict__ off, Counters* C) {
  __shared__ long long sh[kBlock / 32];
  const long long n = C->n_seeds;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    const long long v = (i < n) ? len[i] : 0;
    long long tot;
    const long long pos = tile_off[2 * tile] + block_exclusive_scan(v, &tot, sh);
    if (i < n) off[i] = pos;
  }
}

cudaError_t launch_offsets(const int* len, const long long* tile_off, long long* off, Counters* C,
                           int grid, cudaStream_t s) {
  k_offsets<<<grid, kBlock, 0, s>>>(len, tile_off, off, C);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock) k_trav_write(DevMesh M, const int* __restrict__ succ,
                                                       const int* __restrict__ start,
                                                       const int* __restrict__ len,
                                                       const int* __restrict__ mode,
                                                       const long long* __restrict__ off,
                                                       int* __restrict__ vtx, Counters* C) {
  const long long n = C->n_seeds;
  const int H = (int)(3 * M.m);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (mode[i] == 1) continue;  // long polygons are written from their ranks
    const long long pos = off[i];
    const int L = len[i];
    if (pos + L > (long long)H) {
      set_error(C, POLYLLA_ERR_LIMIT, 53);  // only possible on an inconsistent mesh
      continue;
    }
    if (L > 0 && !succ_write(M.tri, succ, start[i], L, H, vtx + pos))
      set_error(C, POLYLLA_ERR_LIMIT, 54);
  }
}

cudaError_t launch_trav_write(const DevMesh& M, const int* succ, const int* start, const int* len,
                              const int* mode, const long long* off, int* vtx, Counters* C,
                              int grid, cudaStream_t s) {
  k_trav_write<<<grid, kBlock, 0, s>>>(M, succ, start, len, mode, off, vtx, C);
  return cudaGetLastError();
}

}  // namespace polylla
