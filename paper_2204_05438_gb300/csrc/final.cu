// Output CSR (the paper's Mesh and Position arrays, Section 2).  Every output
// polygon already sits in the vertex pool in its final vertex order (written by
// the thread or block that walked it); the order of the polygons is fixed here:
// traversal polygons in seed order, each split polygon replaced in place by its
// pieces.  One single-pass scan over the polygons' (piece count, vertex count)
// replaces the paper's AtomicAdd on i_Gmesh / i_Gpos, and each polygon's pieces
// are copied to their offsets in the same pass.
#include "polylla_internal.cuh"

namespace polylla {

__device__ __forceinline__ void out_counts(const PolyArrays& P, long long i, long long* c,
                                           long long* l) {
  const int pc = P.pcnt[i];
  *c = pc == 0 ? 1 : pc;
  *l = P.flen[i];
}

// Every polygon's output -- its pieces in order, for a split one -- lies in one
// contiguous stretch of the pool, and the untouched polygons that one walk warp
// pooled (32 consecutive seeds) lie back to back.  So a warp's 32 polygons form a
// few runs that are contiguous both in the pool and in the output, broken where
// a polygon was split or walked elsewhere; each run is copied by the whole warp,
// coalesced.  Piece offsets are written by the polygon's own thread.
//
// The tile offsets come from a look-back over `status` in the same pass (tiles in
// ticket order; one word per tile packs the piece count << 33 | vertex count,
// exact within the mesh size limits), and the last tile writes the totals and the
// CSR end marker.
__global__ void __launch_bounds__(kBlock) k_final_write(PolyArrays P, FinalPieces F, Pool pool,
                                                        unsigned long long* status,
                                                        long long* __restrict__ off,
                                                        int* __restrict__ vtx,
                                                        long long* __restrict__ obase, long long m,
                                                        Counters* C) {
  __shared__ long long sh[kBlock / 32];
  __shared__ unsigned long long shu[kBlock / 32];
  __shared__ long long s_tile, s_p, s_v;
  const long long n = C->n_seeds;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  const int lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0)
      s_tile = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&C->ticket), 1ull);
    __syncthreads();
    const long long tile = s_tile;
    __syncthreads();
    if (tile >= ntiles) break;
    const long long i = tile * kPolyTile + threadIdx.x;
    long long c = 0, l = 0;
    if (i < n) out_counts(P, i, &c, &l);
    // one scan of (count << 40) + length, exact while every polygon of the tile has
    // fewer than 2^16 pieces (then the tile has fewer than 2^24; it always has
    // fewer than 2^40 vertices); otherwise two scans
    long long pl, vl, tc, tl;  // in-tile exclusive offsets and tile totals
    if (!__syncthreads_or(c >= (1ll << 16))) {
      unsigned long long t0;
      const unsigned long long x = block_exclusive_scan(
          ((unsigned long long)c << 40) + (unsigned long long)l, &t0, shu);
      pl = (long long)(x >> 40);
      vl = (long long)(x & ((1ull << 40) - 1));
      tc = (long long)(t0 >> 40);
      tl = (long long)(t0 & ((1ull << 40) - 1));
    } else {
      pl = block_exclusive_scan(c, &tc, sh);
      vl = block_exclusive_scan(l, &tl, sh);
    }
    long long pb, vb;
    {
      if (threadIdx.x < 32) {
        const long long ex = lookback_warp(status, tile, (tc << 33) | tl, C);
        if (threadIdx.x == 0) {
          s_p = ex >> 33;
          s_v = ex & ((1ll << 33) - 1);
          if (tile == ntiles - 1) {
            const long long np = s_p + tc, nv = s_v + tl;
            C->n_poly = np;
            C->n_vtx = nv;
            if (np <= m) off[np] = nv;
            else set_error(C, POLYLLA_ERR_LIMIT, 82);
          }
        }
      }
      __syncthreads();
      pb = s_p + pl;
      vb = s_v + vl;
    }
    bool ok = i < n;
    if (ok && (pb + c > m || vb + l > 3 * m)) {
      set_error(C, POLYLLA_ERR_LIMIT, 80);
      ok = false;
    }
    long long src = -1;
    if (ok) {
      if (obase) obase[i] = pb;
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
      const int* __restrict__ from = pool.v + s0;
      int* __restrict__ to = vtx + d0;
      // up to four loads in flight per lane before their stores
      for (long long k = lane; k < run; k += 128) {
        int v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (k + 32 * u < run) v[u] = from[k + 32 * u];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (k + 32 * u < run) to[k + 32 * u] = v[u];
      }
    }
  }
}

cudaError_t launch_final_write(const PolyArrays& P, const FinalPieces& F, const Pool& pool,
                               unsigned long long* status, long long* off, int* vtx,
                               long long* obase, long long m, Counters* C, int grid,
                               cudaStream_t s) {
  static int cap = 0;
  grid = resident_grid(reinterpret_cast<const void*>(k_final_write), kBlock, 0, grid, &cap);
  k_final_write<<<grid, kBlock, 0, s>>>(P, F, pool, status, off, vtx, obase, m, C);
  return cudaGetLastError();
}

}  // namespace polylla
