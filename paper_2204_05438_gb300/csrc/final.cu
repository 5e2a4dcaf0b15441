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

// The unsplit polygons of a warp are copied together: the warp's 32 copy jobs are
// laid end to end and each lane moves every 32nd element, so reads and writes are
// coalesced (the 32 polygons of a warp were also pooled contiguously by k_walk).
// Split polygons' pieces are copied by their own thread.
__global__ void __launch_bounds__(kBlock) k_final_write(PolyArrays P, FinalPieces F, Pool pool,
                                                        const long long* __restrict__ tile_off,
                                                        long long* __restrict__ off,
                                                        int* __restrict__ vtx, long long m,
                                                        Counters* C) {
  __shared__ long long sh[kBlock / 32];
  __shared__ int s_incl[kBlock];
  __shared__ long long s_src[kBlock], s_dst[kBlock];
  const long long n = C->n_seeds;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  const int lane = threadIdx.x & 31;
  const int wbase = threadIdx.x & ~31;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    long long c = 0, l = 0;
    if (i < n) out_counts(P, i, &c, &l);
    long long t0, t1;
    const long long pb = tile_off[2 * tile] + block_exclusive_scan(c, &t0, sh);
    const long long vb = tile_off[2 * tile + 1] + block_exclusive_scan(l, &t1, sh);
    bool ok = i < n;
    if (ok && (pb + c > m || vb + l > 3 * m)) {
      set_error(C, POLYLLA_ERR_LIMIT, 80);
      ok = false;
    }
    const int pc = ok ? P.pcnt[i] : 0;
    // unsplit polygons: one offset, and a copy job for the warp
    int mine = 0;
    if (ok && pc == 0) {
      off[pb] = vb;
      mine = (int)l;
      s_src[threadIdx.x] = P.pos[i];
      s_dst[threadIdx.x] = vb;
    }
    int incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    s_incl[threadIdx.x] = incl;
    __syncwarp();
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int k = lane; k < total; k += 32) {
      int lo = 0, hi = 31;  // first lane whose inclusive sum exceeds k
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_incl[wbase + mid] > k) hi = mid;
        else lo = mid + 1;
      }
      const int excl = lo ? s_incl[wbase + lo - 1] : 0;
      const int rel = k - excl;
      vtx[s_dst[wbase + lo] + rel] = pool.v[s_src[wbase + lo] + rel];
    }
    __syncwarp();
    // split polygons: offsets and pieces by their own thread
    if (ok && pc > 0) {
      long long acc = 0;
      const long long fb = P.pbase[i];
      for (int r = 0; r < pc; ++r) {
        const int len = F.len[fb + r];
        off[pb + r] = vb + acc;
        const int* src = pool.v + F.pos[fb + r];
        for (int q = 0; q < len; ++q) vtx[vb + acc + q] = src[q];
        acc += len;
      }
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
