// Reparation phase (Section 3.2.3, Algorithm 5, with the loop of Algorithm 1).
//
//   k_repair_split  one thread per polygon that has barrier-edge tips.  The
//                   polygon is kept as an ordered list of pieces; the first
//                   piece with a tip is split at its smallest tip vertex b: with
//                   o_0 = b->a the barrier half-edge leaving b, the k internal
//                   edges at b are o_j = twin(prev(o_{j-1})), j = 1..k (ccw), and
//                   o_ceil(k/2) becomes a frontier edge (both half-edges); the
//                   piece is replaced in place by the piece left of o_j followed
//                   by the piece left of twin(o_j).  Each split removes at least
//                   one tip and creates none, so a polygon with T tips ends in at
//                   most T + 1 pieces.  Splitting per polygon until no tip is left
//                   gives the same pieces in the same order as the paper's rounds
//                   (a tip's whole fan lies inside its own region, so polygons do
//                   not interact).  Also emits every polygon's final (count,
//                   length) tile sums for the output scan.
//   k_final_write   block scan of (count, length) + tile offsets gives each
//                   polygon's first output slot; polygons without tips are copied
//                   from the traversal CSR (or re-walked when it was not written),
//                   split ones are written piece by piece from their walks.
#include "walk.cuh"

namespace polylla {

__device__ __forceinline__ int rot_ccw(const int* __restrict__ twin, int o, int H) {
  const int p = he_prev(o);
  const int r = twin[p];
  return ((unsigned)r < (unsigned)H) ? r : -1;
}

__global__ void __launch_bounds__(kBlock) k_repair_split(
    DevMesh M, uint8_t* lab, const int* __restrict__ p_start, const int* __restrict__ p_len,
    const int* __restrict__ p_tip, const int* __restrict__ p_ntip, int* __restrict__ p_pbase,
    int* __restrict__ p_pcnt, int* __restrict__ piece_start, int* __restrict__ piece_len,
    long long piece_cap, long long* __restrict__ tile_sum, Counters* C) {
  __shared__ long long sh[kBlock / 32];
  const long long n = C->n_seeds;
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  long long my_splits = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    long long cnt = 0, tot_len = 0;
    if (i < n) {
      const int ntip = p_ntip[i];
      cnt = 1;
      tot_len = p_len[i];
      if (ntip > 0) {
        const int cap = ntip + 1;
        const long long base =
            (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&C->piece_alloc),
                                 (unsigned long long)cap);
        bool fail = base + cap > piece_cap;
        int count = 1;
        if (!fail) {
          int* ps = piece_start + base;
          int* pl = piece_len + base;
          ps[0] = p_start[i];
          // the traversal already walked piece 0: reuse its tip
          int cur_start = p_start[i], cur_len = p_len[i], cur_tip = p_tip[i];
          bool known = true;
          int j = 0;
          while (j < count) {
            if (!known) {
              const WalkInfo w = walk_cycle(M.tri, M.twin, lab, ps[j], H, limit);
              if (!w.ok) {
                fail = true;
                break;
              }
              cur_start = w.start;
              cur_len = w.len;
              cur_tip = w.tip_h;
            }
            known = false;
            if (cur_tip < 0) {
              ps[j] = cur_start;
              pl[j] = cur_len;
              ++j;
              continue;
            }
            // split at the tip: o_0 = twin(a->b) = b->a
            const int o0 = M.twin[cur_tip];
            if ((unsigned)o0 >= (unsigned)H || count + 1 > cap) {
              fail = true;
              break;
            }
            int k = 0;
            int r = rot_ccw(M.twin, o0, H);
            long long guard = 0;
            while (r != o0) {
              if (r < 0 || lab_frontier(lab, r) || ++guard > limit) {
                fail = true;
                break;
              }
              ++k;
              r = rot_ccw(M.twin, r, H);
            }
            if (fail || k < 2) {
              fail = true;
              break;
            }
            int oj = o0;
            for (int s = 0; s < (k + 1) / 2; ++s) oj = rot_ccw(M.twin, oj, H);
            const int tw = M.twin[oj];
            if ((unsigned)tw >= (unsigned)H) {
              fail = true;
              break;
            }
            const int ta = oj / 3, tb = tw / 3;
            lab[ta] = (uint8_t)(lab[ta] | (1u << (2 + oj - 3 * ta)));
            lab[tb] = (uint8_t)(lab[tb] | (1u << (2 + tw - 3 * tb)));
            for (int q = count; q > j + 1; --q) ps[q] = ps[q - 1];
            for (int q = count; q > j + 1; --q) pl[q] = pl[q - 1];
            ps[j] = oj;
            ps[j + 1] = tw;
            ++count;
            ++my_splits;
          }
        }
        if (fail) {
          set_error(C, POLYLLA_ERR_LIMIT, 30);
          count = 0;
        }
        p_pbase[i] = (int)base;
        p_pcnt[i] = count;
        cnt = count;
        tot_len = 0;
        for (int q = 0; q < count; ++q) tot_len += piece_len[base + q];
      }
    }
    const long long s0 = block_sum(cnt, sh);
    const long long s1 = block_sum(tot_len, sh);
    if (threadIdx.x == 0) {
      tile_sum[2 * tile] = s0;
      tile_sum[2 * tile + 1] = s1;
    }
  }
  const long long ss = block_sum(my_splits, sh);
  if (threadIdx.x == 0 && ss)
    atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_splits), (unsigned long long)ss);
}

cudaError_t launch_repair_split(const DevMesh& M, uint8_t* lab, const int* p_start,
                                const int* p_len, const int* p_tip, const int* p_ntip,
                                int* p_pbase, int* p_pcnt, int* piece_start, int* piece_len,
                                long long piece_cap, long long* tile_sum, Counters* C, int grid,
                                cudaStream_t s) {
  k_repair_split<<<grid, kBlock, 0, s>>>(M, lab, p_start, p_len, p_tip, p_ntip, p_pbase, p_pcnt,
                                         piece_start, piece_len, piece_cap, tile_sum, C);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock) k_final_write(
    DevMesh M, const uint8_t* __restrict__ lab, const int* __restrict__ p_start,
    const int* __restrict__ p_len, const int* __restrict__ p_ntip, const int* __restrict__ p_pbase,
    const int* __restrict__ p_pcnt, const int* __restrict__ piece_start,
    const int* __restrict__ piece_len, const long long* __restrict__ tile_off,
    const long long* __restrict__ off_trav, const int* __restrict__ vtx_trav,
    long long* __restrict__ off, int* __restrict__ vtx, Counters* C) {
  __shared__ long long sh[kBlock / 32];
  const long long n = C->n_seeds;
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    long long cnt = 0, len = 0;
    int ntip = 0, base = 0;
    if (i < n) {
      ntip = p_ntip[i];
      if (ntip == 0) {
        cnt = 1;
        len = p_len[i];
      } else {
        base = p_pbase[i];
        cnt = p_pcnt[i];
        for (int q = 0; q < cnt; ++q) len += piece_len[base + q];
      }
    }
    long long t0, t1;
    const long long pb = tile_off[2 * tile] + block_exclusive_scan(cnt, &t0, sh);
    const long long vb = tile_off[2 * tile + 1] + block_exclusive_scan(len, &t1, sh);
    if (i < n && (pb + cnt > M.m || vb + len > (long long)H)) {
      set_error(C, POLYLLA_ERR_LIMIT, 33);  // only possible on an inconsistent mesh
    } else if (i < n) {
      if (ntip == 0) {
        off[pb] = vb;
        if (off_trav) {
          const long long src = off_trav[i];
          for (long long q = 0; q < len; ++q) vtx[vb + q] = vtx_trav[src + q];
        } else if (len > 0 &&
                   !walk_write(M.tri, M.twin, lab, p_start[i], (int)len, H, limit, vtx + vb)) {
          set_error(C, POLYLLA_ERR_LIMIT, 31);
        }
      } else {
        long long acc = 0;
        for (int q = 0; q < cnt; ++q) {
          const int pl = piece_len[base + q];
          off[pb + q] = vb + acc;
          if (!walk_write(M.tri, M.twin, lab, piece_start[base + q], pl, H, limit, vtx + vb + acc))
            set_error(C, POLYLLA_ERR_LIMIT, 32);
          acc += pl;
        }
      }
    }
  }
}

cudaError_t launch_final_write(const DevMesh& M, const uint8_t* lab, const int* p_start,
                               const int* p_len, const int* p_ntip, const int* p_pbase,
                               const int* p_pcnt, const int* piece_start, const int* piece_len,
                               const long long* tile_off, const long long* off_trav,
                               const int* vtx_trav, long long* off, int* vtx, Counters* C,
                               int grid, cudaStream_t s) {
  k_final_write<<<grid, kBlock, 0, s>>>(M, lab, p_start, p_len, p_ntip, p_pbase, p_pcnt,
                                        piece_start, piece_len, tile_off, off_trav, vtx_trav, off,
                                        vtx, C);
  return cudaGetLastError();
}

}  // namespace polylla
