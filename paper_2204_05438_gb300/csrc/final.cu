// Output CSR (the paper's Mesh and Position arrays, Section 2).  Every output
// polygon already sits in the vertex pool in its final vertex order (written by
// the thread or block that walked it); the order of the polygons is fixed here:
// traversal polygons in seed order, each split polygon replaced in place by its
// pieces.  One scan over the polygons' (piece count, vertex count) replaces the
// paper's AtomicAdd on i_Gmesh / i_Gpos, then each polygon's pieces are copied to
// their offsets.
#include "polylla_internal.cuh"

namespace polylla {

__device__ __forceinline__ void out_counts(const PolyArrays& P, long long i, long long* c,
                                           long long* l) {
  const int pc = P.pcnt[i];
  *c = pc == 0 ? 1 : pc;
  *l = P.flen[i];
}

__global__ void __launch_bounds__(kBlock) k_final_tiles(PolyArrays P, long long* __restrict__ tile_sum,
                                                        Counters* C) {
  __shared__ long long sh[kBlock / 32];
  const long long n = C->n_seeds;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    long long c = 0, l = 0;
    if (i < n) out_counts(P, i, &c, &l);
    const long long s0 = block_sum(c, sh);
    const long long s1 = block_sum(l, sh);
    if (threadIdx.x == 0) {
      tile_sum[2 * tile] = s0;
      tile_sum[2 * tile + 1] = s1;
    }
  }
}

cudaError_t launch_final_tiles(const PolyArrays& P, long long* tile_sum, Counters* C, int grid,
                               cudaStream_t s) {
  k_final_tiles<<<grid, kBlock, 0, s>>>(P, tile_sum, C);
  return cudaGetLastError();
}

// Every polygon's output -- its pieces in order, for a split one -- lies in one
// contiguous stretch of the pool, and the untouched polygons that one walk warp
// pooled (32 consecutive seeds) lie back to back.  So a warp's 32 polygons form a
// few runs that are contiguous both in the pool and in the output, broken where
// a polygon was split or walked elsewhere; each run is copied by the whole warp,
// coalesced.  Piece offsets are written by the polygon's own thread.
__global__ void __launch_bounds__(kBlock) k_final_write(PolyArrays P, FinalPieces F, Pool pool,
                                                        const long long* __restrict__ tile_off,
                                                        long long* __restrict__ off,
                                                        int* __restrict__ vtx, long long m,
                                                        Counters* C) {
  __shared__ long long sh[kBlock / 32];
  __shared__ unsigned long long shu[kBlock / 32];
  const long long n = C->n_seeds;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  const int lane = threadIdx.x & 31;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    long long c = 0, l = 0;
    if (i < n) out_counts(P, i, &c, &l);
    // one scan of (count << 40) + length, exact while every polygon of the tile has
    // fewer than 2^16 pieces (then the tile has fewer than 2^24; it always has
    // fewer than 2^40 vertices); otherwise two scans
    long long pb, vb;
    if (!__syncthreads_or(c >= (1ll << 16))) {
      unsigned long long t0;
      const unsigned long long x = block_exclusive_scan(
          ((unsigned long long)c << 40) + (unsigned long long)l, &t0, shu);
      pb = tile_off[2 * tile] + (long long)(x >> 40);
      vb = tile_off[2 * tile + 1] + (long long)(x & ((1ull << 40) - 1));
    } else {
      long long t0, t1;
      pb = tile_off[2 * tile] + block_exclusive_scan(c, &t0, sh);
      vb = tile_off[2 * tile + 1] + block_exclusive_scan(l, &t1, sh);
    }
    bool ok = i < n;
    if (ok && (pb + c > m || vb + l > 3 * m)) {
      set_error(C, POLYLLA_ERR_LIMIT, 80);
      ok = false;
    }
    long long src = -1;
    if (ok) {
      const int pc = P.pcnt[i];
      if (pc == 0) {
        src = P.pos[i];
        off[pb] = vb;
      } else {
        const long long fb = P.pbase[i];
        src = F.pos[fb];
        long long acc = 0;
        for (int r = 0; r < pc; ++r) {
          off[pb + r] = vb + acc;
          acc += F.len[fb + r];
        }
      }
      if (src < 0 || src + l > pool.cap) {
        set_error(C, POLYLLA_ERR_LIMIT, 81);
        src = -1;
      }
    }
    const unsigned um = __ballot_sync(0xffffffffu, src >= 0);
    const long long prev_end = __shfl_up_sync(0xffffffffu, src + l, 1);
    const bool first = src >= 0 && (lane == 0 || !((um >> (lane - 1)) & 1u) || prev_end != src);
    unsigned starts = __ballot_sync(0xffffffffu, first);
    const unsigned breaks = starts | ~um;
    while (starts) {
      const int a = __ffs(starts) - 1;
      starts &= starts - 1;
      const unsigned above = breaks & ~((2u << a) - 1u);
      const int e = above ? __ffs(above) - 1 : 32;
      const long long s0 = __shfl_sync(0xffffffffu, src, a);
      const long long d0 = __shfl_sync(0xffffffffu, vb, a);
      const long long s1 = __shfl_sync(0xffffffffu, src + l, e - 1);
      const long long run = s1 - s0;
      const int* from = pool.v + s0;
      int* to = vtx + d0;
      for (long long k = lane; k < run; k += 32) to[k] = from[k];
    }
  }
}

cudaError_t launch_final_write(const PolyArrays& P, const FinalPieces& F, const Pool& pool,
                               const long long* tile_off, long long* off, int* vtx, long long m,
                               Counters* C, int grid, cudaStream_t s) {
  k_final_write<<<grid, kBlock, 0, s>>>(P, F, pool, tile_off, off, vtx, m, C);
  return cudaGetLastError();
}

}  // namespace polylla
