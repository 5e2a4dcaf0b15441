// Traversal phase (Section 3.2.2, Algorithms 3 and 4).
//
//   k_trav_count  one thread per seed: enter the seed's region, walk its boundary
//                 once, record the canonical start, the length, the barrier-edge
//                 tips and the tile's total length.
//   k_trav_write  one thread per seed: block scan of the lengths plus the tile
//                 offset gives the polygon's CSR offset (the paper's AtomicAdd on
//                 i_Gmesh / i_Gpos becomes this deterministic scan); walk again
//                 from the canonical start writing the origins.
#include "walk.cuh"

namespace polylla {

__global__ void __launch_bounds__(kBlock) k_trav_count(DevMesh M, const uint8_t* __restrict__ lab,
                                                       const int* __restrict__ seeds,
                                                       int* __restrict__ p_start,
                                                       int* __restrict__ p_len,
                                                       int* __restrict__ p_tip,
                                                       int* __restrict__ p_ntip,
                                                       long long* __restrict__ tile_sum,
                                                       Counters* C) {
  __shared__ long long sh[kBlock / 32];
  const long long n = C->n_seeds;
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  long long my_tips = 0, my_tip_polys = 0, my_len = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    long long len = 0;
    if (i < n) {
      const int s = seeds[i];
      WalkInfo w;
      w.ok = false;
      const int h0 = region_entry(M.twin, lab, s, H, limit);
      if (h0 >= 0) w = walk_cycle(M.tri, M.twin, lab, h0, H, limit);
      if (!w.ok) {
        set_error(C, POLYLLA_ERR_LIMIT, 20);
        w.start = 3 * s;
        w.len = 0;
        w.tip_h = -1;
        w.ntips = 0;
      }
      p_start[i] = w.start;
      p_len[i] = w.len;
      p_tip[i] = w.tip_h;
      p_ntip[i] = w.ntips;
      len = w.len;
      my_tips += w.ntips;
      my_tip_polys += (w.ntips > 0);
    }
    my_len += len;
    const long long tot = block_sum(len, sh);
    if (threadIdx.x == 0) {
      tile_sum[2 * tile] = tot;
      tile_sum[2 * tile + 1] = 0;
    }
  }
  // per-block statistics (three atomics per block)
  const long long a = block_sum(my_len, sh);
  const long long b = block_sum(my_tips, sh);
  const long long c = block_sum(my_tip_polys, sh);
  if (threadIdx.x == 0) {
    if (a) atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_vtx_trav), (unsigned long long)a);
    if (b) atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tips), (unsigned long long)b);
    if (c) atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tip_polys), (unsigned long long)c);
  }
}

cudaError_t launch_trav_count(const DevMesh& M, const uint8_t* lab, const int* seeds,
                              int* p_start, int* p_len, int* p_tip, int* p_ntip,
                              long long* tile_sum, Counters* C, int grid, cudaStream_t s) {
  k_trav_count<<<grid, kBlock, 0, s>>>(M, lab, seeds, p_start, p_len, p_tip, p_ntip, tile_sum, C);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock) k_trav_write(DevMesh M, const uint8_t* __restrict__ lab,
                                                       const int* __restrict__ p_start,
                                                       const int* __restrict__ p_len,
                                                       const long long* __restrict__ tile_off,
                                                       long long* __restrict__ off,
                                                       int* __restrict__ vtx, Counters* C) {
  __shared__ long long sh[kBlock / 32];
  const long long n = C->n_seeds;
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    const long long len = (i < n) ? p_len[i] : 0;
    long long tot;
    const long long pos = tile_off[2 * tile] + block_exclusive_scan(len, &tot, sh);
    if (i < n) {
      off[i] = pos;
      if (pos + len > (long long)H) {
        set_error(C, POLYLLA_ERR_LIMIT, 22);  // only possible on an inconsistent mesh
      } else if (len > 0 &&
                 !walk_write(M.tri, M.twin, lab, p_start[i], (int)len, H, limit, vtx + pos)) {
        set_error(C, POLYLLA_ERR_LIMIT, 21);
      }
    }
  }
}

cudaError_t launch_trav_write(const DevMesh& M, const uint8_t* lab, const int* p_start,
                              const int* p_len, const long long* tile_off, long long* off,
                              int* vtx, Counters* C, int grid, cudaStream_t s) {
  k_trav_write<<<grid, kBlock, 0, s>>>(M, lab, p_start, p_len, tile_off, off, vtx, C);
  return cudaGetLastError();
}

}  // namespace polylla
