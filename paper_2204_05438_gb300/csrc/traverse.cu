// Traversal phase (Section 3.2.2, Algorithms 3 and 4).
//
//   k_succ        one thread per triangle: for each frontier half-edge, the next
//                 frontier half-edge of its region's boundary (the turn of
//                 PolyConstruction), with the barrier-edge tip flag.
//   k_trav_count  one seed per thread (grid-stride, no block barriers, so a long
//                 walk holds up only its own thread): enter the region, chase succ
//                 around the cycle, record the canonical start, the length, and
//                 every barrier-edge tip (appended to the tip list with its
//                 polygon and its vertex -> tip map entry).
//   k_len_tiles / k_offsets  per-tile length sums, then (after the tile scan) each
//                 polygon's CSR offset -- the paper's AtomicAdd on i_Gmesh / i_Gpos
//                 becomes this deterministic scan.
//   k_trav_write  one polygon per thread: chase succ from the canonical start
//                 writing origins.
#include "walk.cuh"

namespace polylla {

__global__ void __launch_bounds__(kBlock) k_succ(DevMesh M, const uint8_t* __restrict__ lab,
                                                 int* __restrict__ succ, Counters* C) {
  const long long m = M.m;
  const int H = (int)(3 * m);
  const long long limit = 3 * m + 3;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x) {
    const unsigned fr = (__ldg(lab + t) >> 2) & 7u;
    if (!fr) continue;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (!((fr >> k) & 1u)) continue;
      const int h = (int)(3 * t + k);
      const int g = turn_to_frontier(M.twin, lab, h, H, limit);
      if (g < 0) {
        set_error(C, POLYLLA_ERR_LIMIT, 50);
        succ[h] = h;  // a one-element cycle keeps later walks bounded
        continue;
      }
      succ[h] = (g == __ldg(M.twin + h)) ? (g | kTipFlag) : g;
    }
  }
}

cudaError_t launch_succ(const DevMesh& M, const uint8_t* lab, int* succ, Counters* C, int grid,
                        cudaStream_t s) {
  k_succ<<<grid, kBlock, 0, s>>>(M, lab, succ, C);
  return cudaGetLastError();
}

constexpr int kLocalTips = 8;

__global__ void __launch_bounds__(kBlock) k_trav_count(DevMesh M, const uint8_t* __restrict__ lab,
                                                       const int* __restrict__ seeds,
                                                       const int* __restrict__ succ,
                                                       PolyArrays P, TipArrays T, int epoch,
                                                       Counters* C) {
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
    if (e >= 0) c = succ_cycle(M.tri, succ, e, H, limit, tips, kLocalTips);
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
                              const int* succ, const PolyArrays& P, const TipArrays& T, int epoch,
                              Counters* C, int grid, cudaStream_t s) {
  k_trav_count<<<grid, kBlock, 0, s>>>(M, lab, seeds, succ, P, T, epoch, C);
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
                                                       const long long* __restrict__ off,
                                                       int* __restrict__ vtx, Counters* C) {
  const long long n = C->n_seeds;
  const int H = (int)(3 * M.m);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
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
                              const long long* off, int* vtx, Counters* C, int grid,
                              cudaStream_t s) {
  k_trav_write<<<grid, kBlock, 0, s>>>(M, succ, start, len, off, vtx, C);
  return cudaGetLastError();
}

}  // namespace polylla
