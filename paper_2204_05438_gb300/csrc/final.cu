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
// A block takes kSub consecutive 256-polygon sub-tiles per ticket (one look-back
// tile), so one block scan and one look-back serve 1024 polygons.  The tile
// offsets come from a look-back over `status` in the same pass (tiles in ticket
// order; one word per tile packs the piece count << 33 | vertex count, exact
// within the mesh size limits), and the last tile writes the totals and the CSR
// end marker.  The status words clean themselves: the block that completes the
// last look-back (C->out_done counts them) clears them and the count.
constexpr int kSub = 4;
constexpr int kOutTile = kSub * kPolyTile;

__global__ void __launch_bounds__(kBlock, 5) k_final_write(PolyArrays P, FinalPieces F, Pool pool,
                                                        unsigned long long* status,
                                                        long long* __restrict__ off,
                                                        int* __restrict__ vtx,
                                                        long long* __restrict__ obase, long long m,
                                                        Counters* C) {
  __shared__ long long s_src[kSub][kBlock];  // pool position of each polygon (or -1)
  __shared__ int s_len[kSub][kBlock], s_pc[kSub][kBlock];
  __shared__ long long s_xc[kSub][kBlock], s_xl[kSub][kBlock];  // in-warp exclusive sums
  __shared__ long long s_wc[kBlock / 32][kSub], s_wl[kBlock / 32][kSub];  // warp sums
  __shared__ long long s_tile, s_p, s_v;
  __shared__ int s_clear;
  const long long n = C->n_seeds;
  const long long ntiles = (n + kOutTile - 1) / kOutTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0)
      s_tile = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&C->ticket), 1ull);
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= ntiles) break;
    // this thread's polygon in each sub-tile; every load issued before any use
    int pcj[kSub], lj[kSub];
#pragma unroll
    for (int j = 0; j < kSub; ++j) {
      const long long i = tile * kOutTile + (long long)j * kPolyTile + threadIdx.x;
      pcj[j] = i < n ? P.pcnt[i] : 0;
      lj[j] = i < n ? P.flen[i] : 0;
    }
#pragma unroll
    for (int j = 0; j < kSub; ++j) {
      const long long i = tile * kOutTile + (long long)j * kPolyTile + threadIdx.x;
      const long long src = i < n ? (pcj[j] == 0 ? P.pos[i] : F.pos[P.pbase[i]]) : -1;
      s_src[j][threadIdx.x] = src;
      // the polygon's first vertex (and its line) to L2 while the tile waits for
      // its look-back
      if (src >= 0 && src < pool.cap) asm volatile("prefetch.global.L2 [%0];" ::"l"(pool.v + src));
      s_len[j][threadIdx.x] = lj[j];
      s_pc[j][threadIdx.x] = pcj[j];
      long long xc = i < n ? (pcj[j] == 0 ? 1 : pcj[j]) : 0, xl = lj[j];
      const long long c0 = xc, l0 = xl;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const long long yc = __shfl_up_sync(0xffffffffu, xc, d);
        const long long yl = __shfl_up_sync(0xffffffffu, xl, d);
        if (lane >= d) {
          xc += yc;
          xl += yl;
        }
      }
      s_xc[j][threadIdx.x] = xc - c0;
      s_xl[j][threadIdx.x] = xl - l0;
      if (lane == 31) {
        s_wc[warp][j] = xc;
        s_wl[warp][j] = xl;
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      long long ac = 0, al = 0;
      for (int j = 0; j < kSub; ++j)
        for (int w = 0; w < kBlock / 32; ++w) {
          ac += s_wc[w][j];
          al += s_wl[w][j];
        }
      const long long ex = lookback_warp(status, tile, (ac << 33) | al, C);
      if (threadIdx.x == 0) {
        s_p = ex >> 33;
        s_v = ex & ((1ll << 33) - 1);
        // the last look-back to complete clears the status words for the next pass
        const unsigned long long done =
            atomicAdd(reinterpret_cast<unsigned long long*>(&C->out_done), 1ull);
        s_clear = done == (unsigned long long)(ntiles - 1);
        if (tile == ntiles - 1) {
          const long long np = s_p + ac, nv = s_v + al;
          C->n_poly = np;
          C->n_vtx = nv;
          if (np <= m) off[np] = nv;
          else set_error(C, POLYLLA_ERR_LIMIT, 82);
        }
      }
    }
    __syncthreads();
    long long bp = s_p, bv = s_v;  // offsets of sub-tile j's first polygon
    for (int j = 0; j < kSub; ++j) {
      long long wp = 0, wv = 0, tp = 0, tv = 0;
#pragma unroll
      for (int w = 0; w < kBlock / 32; ++w) {
        wp += (w < warp) ? s_wc[w][j] : 0;
        wv += (w < warp) ? s_wl[w][j] : 0;
        tp += s_wc[w][j];
        tv += s_wl[w][j];
      }
      const long long i = tile * kOutTile + (long long)j * kPolyTile + threadIdx.x;
      const long long pb = bp + wp + s_xc[j][threadIdx.x];
      const long long vb = bv + wv + s_xl[j][threadIdx.x];
      bp += tp;
      bv += tv;
      const int pc = s_pc[j][threadIdx.x];
      const long long l = s_len[j][threadIdx.x];
      const long long c = pc == 0 ? 1 : pc;
      long long sj = -1;
      if (i < n) {
        if (pb + c > m || vb + l > 3 * m) {
          set_error(C, POLYLLA_ERR_LIMIT, 80);
        } else {
          if (obase) obase[i] = pb;
          if (pc == 0) {
            off[pb] = vb;
          } else {
            const long long fb = P.pbase[i];
            long long acc = 0;
            for (int r = 0; r < pc; ++r) {
              off[pb + r] = vb + acc;
              acc += F.len[fb + r];
            }
          }
          const long long src = s_src[j][threadIdx.x];
          if (src < 0 || src + l > pool.cap) set_error(C, POLYLLA_ERR_LIMIT, 81);
          else sj = src;
        }
      }
      const unsigned um = __ballot_sync(0xffffffffu, sj >= 0);
      const long long prev_end = __shfl_up_sync(0xffffffffu, sj + l, 1);
      const bool first = sj >= 0 && (lane == 0 || !((um >> (lane - 1)) & 1u) || prev_end != sj);
      unsigned starts = __ballot_sync(0xffffffffu, first);
      const unsigned breaks = starts | ~um;
      while (starts) {
        const int a = __ffs(starts) - 1;
        starts &= starts - 1;
        const unsigned above = breaks & ~((2u << a) - 1u);
        const int e = above ? __ffs(above) - 1 : 32;
        const long long s0 = __shfl_sync(0xffffffffu, sj, a);
        const long long d0 = __shfl_sync(0xffffffffu, vb, a);
        const long long s1 = __shfl_sync(0xffffffffu, sj + l, e - 1);
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
    if (s_clear) {  // every tile has finished its look-back
      for (long long q = threadIdx.x; q < ntiles; q += kBlock) status[q] = 0;
      if (threadIdx.x == 0) C->out_done = 0;
    }
    __syncthreads();
  }
}

cudaError_t launch_final_write(const PolyArrays& P, const FinalPieces& F, const Pool& pool,
                               unsigned long long* status, long long* off, int* vtx,
                               long long* obase, long long m, Counters* C, int grid,
                               cudaStream_t s) {
  static std::atomic<int> cap{0};
  grid = resident_grid(reinterpret_cast<const void*>(k_final_write), kBlock, 0, grid, &cap);
  k_final_write<<<grid, kBlock, 0, s>>>(P, F, pool, status, off, vtx, obase, m, C);
  return cudaGetLastError();
}

}  // namespace polylla
