// Reparation phase (Section 3.2.3, Algorithm 5, with the loop of Algorithm 1),
// parallel over barrier-edge tips.
//
// The paper splits each non-simple polygon at one tip per round.  Its result,
// with the tip of smallest vertex id split first in every polygon, is computed
// here without rounds, from three facts:
//   * the split edge of tip b depends only on b's own fan: with o_0 = b->a the
//     barrier half-edge leaving b and o_j = twin(prev(o_{j-1})) the k internal
//     edges that follow ccw, it is o_ceil(k/2) = b->x;
//   * a split never creates a tip, and removes b -- and x, if x is a tip;
//   * two tips interact only when one's split edge ends at the other.
// So every tip is processed unless a processed tip with a smaller vertex id ends
// its split edge on it (k_tip_split finds those pairs, k_tip_resolve settles
// them), all processed split edges become frontier edges at once (k_tip_mark),
// and the boundary successors around their endpoints are recomputed
// (k_resucc).  The pieces are the cycles through the split half-edges
// (k_piece_walk); their output order is the paper's recursive in-place order
// (first split at the smallest tip, the half containing tip->x first), rebuilt per
// polygon from the tree of splits (k_poly_order).
#include "order.cuh"

namespace polylla {

__device__ __forceinline__ int rot_ccw(const int* __restrict__ twin, int o, int H) {
  const int r = twin[he_prev(o)];
  return ((unsigned)r < (unsigned)H) ? r : -1;
}

// R1: split edge of every tip, and the (smaller tip -> larger tip) pairs where the
// smaller tip's split edge ends on the larger tip.
__global__ void __launch_bounds__(kBlock) k_tip_split(DevMesh M, const uint8_t* __restrict__ lab,
                                                      TipArrays T, int epoch, Counters* C) {
  const long long nt = C->n_tips;
  const int H = (int)(3 * M.m);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nt;
       k += (long long)gridDim.x * blockDim.x) {
    T.state[k] = 1;
    T.o[k] = -1;
    const int g = T.h[k];
    const int o0 = M.twin[g];  // b -> a
    if ((unsigned)o0 >= (unsigned)H) {
      set_error(C, POLYLLA_ERR_LIMIT, 60);
      continue;
    }
    int cnt = 0;
    int r = rot_ccw(M.twin, o0, H);
    bool bad = false;
    while (r != o0) {
      if (r < 0 || lab_frontier(lab, r) || ++cnt > H) {
        bad = true;
        break;
      }
      r = rot_ccw(M.twin, r, H);
    }
    if (bad || cnt < 2) {
      set_error(C, POLYLLA_ERR_LIMIT, 61);
      continue;
    }
    int oj = o0;
    for (int s = 0; s < (cnt + 1) / 2; ++s) oj = rot_ccw(M.twin, oj, H);
    T.o[k] = oj;
    const int b = M.tri[o0];
    const int x = M.tri[he_next(oj)];
    const long long v = T.vtip[x];
    if ((int)(v >> 32) == epoch && b < x) {
      const long long p = (long long)atomicAdd(
          reinterpret_cast<unsigned long long*>(&C->n_pairs), 1ull);
      if (p < T.cap) {
        T.pair_src[p] = (int)k;
        T.pair_dst[p] = (int)(v & 0xffffffffll);
      } else {
        set_error(C, POLYLLA_ERR_LIMIT, 62);
      }
    }
  }
}

cudaError_t launch_tip_split(const DevMesh& M, const uint8_t* lab, const TipArrays& T, int epoch,
                             Counters* C, int grid, cudaStream_t s) {
  k_tip_split<<<grid, kBlock, 0, s>>>(M, lab, T, epoch, C);
  return cudaGetLastError();
}

// R2 (one block): a tip is cancelled iff a processed tip with a smaller vertex id
// ends its split edge on it.  The pairs form a DAG ordered by vertex id; Jacobi
// rounds reach its unique fixed point after (longest chain + 1) rounds.
__global__ void __launch_bounds__(1024) k_tip_resolve(TipArrays T, Counters* C) {
  __shared__ int changed;
  const long long np = min(C->n_pairs, T.cap);
  if (np == 0) return;
  for (long long p = threadIdx.x; p < np; p += blockDim.x) T.cancel_round[T.pair_dst[p]] = -1;
  __syncthreads();
  for (int round = 0; round <= np + 1; ++round) {
    for (long long p = threadIdx.x; p < np; p += blockDim.x)
      if (T.state[T.pair_src[p]] == 1) T.cancel_round[T.pair_dst[p]] = round;
    if (threadIdx.x == 0) changed = 0;
    __syncthreads();
    for (long long p = threadIdx.x; p < np; p += blockDim.x) {
      const int d = T.pair_dst[p];
      const int want = (T.cancel_round[d] == round) ? 0 : 1;
      if (T.state[d] != want) changed = 1;
    }
    __syncthreads();
    for (long long p = threadIdx.x; p < np; p += blockDim.x) {
      const int d = T.pair_dst[p];
      T.state[d] = (T.cancel_round[d] == round) ? 0 : 1;
    }
    __syncthreads();
    if (!changed) return;
    __syncthreads();
  }
  if (threadIdx.x == 0) set_error(C, POLYLLA_ERR_LIMIT, 63);
}

cudaError_t launch_tip_resolve(const TipArrays& T, Counters* C, cudaStream_t s) {
  k_tip_resolve<<<1, 1024, 0, s>>>(T, C);
  return cudaGetLastError();
}

__device__ __forceinline__ void lab_set_frontier(uint8_t* lab, int h) {
  const int t = h / 3;
  const unsigned bit = 1u << (2 + (h - 3 * t));
  // several split edges may touch one triangle: OR the byte inside its aligned word
  unsigned* word = reinterpret_cast<unsigned*>(lab + (t & ~3));
  atomicOr(word, bit << (8 * (t & 3)));
}

// R3: every processed split edge becomes a frontier edge (both half-edges).
__global__ void __launch_bounds__(kBlock) k_tip_mark(DevMesh M, uint8_t* lab, TipArrays T, int epoch,
                                                     Counters* C) {
  const long long nt = C->n_tips;
  long long my = 0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nt;
       k += (long long)gridDim.x * blockDim.x) {
    const int oj = T.o[k];
    if (T.state[k] != 1 || oj < 0) continue;
    const int tw = M.twin[oj];
    lab_set_frontier(lab, oj);
    lab_set_frontier(lab, tw);
    T.chord[oj] = ((long long)epoch << 32) | (unsigned)(2 * k);
    T.chord[tw] = ((long long)epoch << 32) | (unsigned)(2 * k + 1);
    ++my;
  }
  my = __reduce_add_sync(0xffffffffu, (unsigned)my);
  if ((threadIdx.x & 31) == 0 && my)
    atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_splits), (unsigned long long)my);
}

cudaError_t launch_tip_mark(const DevMesh& M, uint8_t* lab, const TipArrays& T, int epoch,
                            Counters* C, int grid, cudaStream_t s) {
  k_tip_mark<<<grid, kBlock, 0, s>>>(M, lab, T, epoch, C);
  return cudaGetLastError();
}

// Recompute succ for every frontier half-edge arriving at v (o_start leaves v).
__device__ void resucc_vertex(const DevMesh& M, const uint8_t* lab, int* succ, int o_start, int H,
                              long long limit, Counters* C) {
  int o = o_start;
  bool open = false;
  int guard = 0;
  do {  // ccw around v
    const int p = he_prev(o);
    if (lab_frontier(lab, p)) {
      const int g = turn_to_frontier(M.twin, lab, p, H, limit);
      if (g < 0) {
        set_error(C, POLYLLA_ERR_LIMIT, 64);
        return;
      }
      succ[p] = (g == M.twin[p]) ? (g | kTipFlag) : g;
    }
    o = rot_ccw(M.twin, o, H);
    if (o < 0) {
      open = true;
      break;
    }
  } while (o != o_start && ++guard < H);
  if (!open) return;
  o = o_start;
  for (;;) {  // border vertex: the rest of the fan, cw from the start
    const int tw = M.twin[o];
    if ((unsigned)tw >= (unsigned)H) break;
    o = he_next(tw);
    const int p = he_prev(o);
    if (lab_frontier(lab, p)) {
      const int g = turn_to_frontier(M.twin, lab, p, H, limit);
      if (g < 0) {
        set_error(C, POLYLLA_ERR_LIMIT, 65);
        return;
      }
      succ[p] = (g == M.twin[p]) ? (g | kTipFlag) : g;
    }
    if (++guard > H) break;
  }
}

// R4: successors around both endpoints of every processed split edge.
__global__ void __launch_bounds__(kBlock) k_resucc(DevMesh M, const uint8_t* __restrict__ lab,
                                                   int* succ, TipArrays T, Counters* C) {
  const long long nt = C->n_tips;
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nt;
       k += (long long)gridDim.x * blockDim.x) {
    const int oj = T.o[k];
    if (T.state[k] != 1 || oj < 0) continue;
    resucc_vertex(M, lab, succ, oj, H, limit, C);           // around the tip b
    resucc_vertex(M, lab, succ, M.twin[oj], H, limit, C);   // around x
  }
}

cudaError_t launch_resucc(const DevMesh& M, const uint8_t* lab, int* succ, const TipArrays& T,
                          Counters* C, int grid, cudaStream_t s) {
  k_resucc<<<grid, kBlock, 0, s>>>(M, lab, succ, T, C);
  return cudaGetLastError();
}

// R5: walk the piece on each side of every processed split edge.  A piece is
// named by the smallest split half-edge on its cycle (as its record 2k + side);
// the walker that starts on that half-edge records the piece's canonical start
// and length.
__global__ void __launch_bounds__(kBlock) k_piece_walk(DevMesh M, const int* __restrict__ succ,
                                                       PolyArrays P, TipArrays T, int epoch,
                                                       Counters* C) {
  const long long nt = C->n_tips;
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 2 * nt;
       q += (long long)gridDim.x * blockDim.x) {
    const long long k = q >> 1;
    const int oj = T.o[k];
    if (T.state[k] != 1 || oj < 0 || P.mode[T.poly[k]] == 3) continue;
    const int h0 = (q & 1) ? M.twin[oj] : oj;
    unsigned long long best = ~0ull;
    int leader = 0x7fffffff, leader_rec = -1;
    int len = 0, h = h0;
    long long steps = 0;
    bool ok = true;
    do {
      const unsigned long long key = he_key(M.tri, h);
      if (key < best) best = key;
      const long long tag = T.chord[h];
      if ((int)(tag >> 32) == epoch && h < leader) {
        leader = h;
        leader_rec = (int)(tag & 0xffffffffll);
      }
      const int s = succ[h];
      if (s & kTipFlag) ok = false;  // a tip survived: cannot happen on a valid mesh
      ++len;
      h = s & kSuccMask;
      if ((unsigned)h >= (unsigned)H || ++steps > limit) {
        ok = false;
        break;
      }
    } while (h != h0);
    if (!ok) {
      set_error(C, POLYLLA_ERR_LIMIT, 66);
      continue;
    }
    T.piece[q] = leader_rec;
    if (leader_rec == q) {
      T.rec_start[q] = (int)(best & 0xffffffffu);
      T.rec_len[q] = len;
    }
  }
}

cudaError_t launch_piece_walk(const DevMesh& M, const int* succ, const PolyArrays& P,
                              const TipArrays& T, int epoch, Counters* C, int grid,
                              cudaStream_t s) {
  k_piece_walk<<<grid, kBlock, 0, s>>>(M, succ, P, T, epoch, C);
  return cudaGetLastError();
}

// R6: per polygon with tips, its pieces in the paper's recursive order
// (order_pieces, order.cuh); long polygons are ordered by their block.
__global__ void __launch_bounds__(kBlock) k_poly_order(DevMesh M, PolyArrays P, TipArrays T,
                                                       FinalPieces F, Counters* C) {
  const long long n = C->n_seeds;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (P.ntip[i] == 0 || P.mode[i] == 3) continue;  // mode 3: ordered by k_long_repair
    order_pieces(M, P, T, F, C, i, T.scratch + 24ll * P.tipbase[i], 0);
  }
}

cudaError_t launch_poly_order(const DevMesh& M, const PolyArrays& P, const TipArrays& T,
                              const FinalPieces& F, Counters* C, int grid, cudaStream_t s) {
  k_poly_order<<<grid, kBlock, 0, s>>>(M, P, T, F, C);
  return cudaGetLastError();
}

// R7: per-tile sums of the final (polygon count, vertex count) of every traversal
// polygon (1 and its length if it has no tip, its pieces otherwise).
__global__ void __launch_bounds__(kBlock) k_final_tiles(PolyArrays P, long long* __restrict__ tile_sum,
                                                        Counters* C) {
  __shared__ long long sh[kBlock / 32];
  const long long n = C->n_seeds;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    long long c = 0, l = 0;
    if (i < n) {
      if (P.ntip[i] == 0) {
        c = 1;
        l = P.len[i];
      } else {
        c = P.pcnt[i];
        l = P.flen[i];
      }
    }
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

// R8: final CSR offsets: off[] for every output polygon, the output position of
// every untouched polygon (vb) and of every piece (F.off).
__global__ void __launch_bounds__(kBlock) k_final_offsets(PolyArrays P, FinalPieces F,
                                                          const long long* __restrict__ tile_off,
                                                          long long* __restrict__ off, long long m,
                                                          Counters* C) {
  __shared__ long long sh[kBlock / 32];
  const long long n = C->n_seeds;
  const long long ntiles = (n + kPolyTile - 1) / kPolyTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long i = tile * kPolyTile + threadIdx.x;
    long long c = 0, l = 0;
    const bool tip = (i < n) && P.ntip[i] > 0;
    if (i < n) {
      c = tip ? P.pcnt[i] : 1;
      l = tip ? P.flen[i] : P.len[i];
    }
    long long t0, t1;
    const long long pb = tile_off[2 * tile] + block_exclusive_scan(c, &t0, sh);
    const long long vb = tile_off[2 * tile + 1] + block_exclusive_scan(l, &t1, sh);
    if (i >= n) continue;
    if (pb + c > m || vb + l > 3 * m) {
      set_error(C, POLYLLA_ERR_LIMIT, 70);
      continue;
    }
    P.vb[i] = vb;
    if (!tip) {
      off[pb] = vb;
    } else {
      long long acc = 0;
      const long long base = P.pbase[i];
      for (int r = 0; r < c; ++r) {
        off[pb + r] = vb + acc;
        F.off[base + r] = vb + acc;
        acc += F.len[base + r];
      }
    }
  }
}

cudaError_t launch_final_offsets(const PolyArrays& P, const FinalPieces& F,
                                 const long long* tile_off, long long* off, long long m,
                                 Counters* C, int grid, cudaStream_t s) {
  k_final_offsets<<<grid, kBlock, 0, s>>>(P, F, tile_off, off, m, C);
  return cudaGetLastError();
}

// R9a: untouched polygons -- copied from the traversal CSR when it was written,
// walked again otherwise.
__global__ void __launch_bounds__(kBlock) k_final_write_polys(
    DevMesh M, const int* __restrict__ succ, PolyArrays P, const long long* __restrict__ off_trav,
    const int* __restrict__ vtx_trav, int* __restrict__ vtx, Counters* C) {
  const long long n = C->n_seeds;
  const int H = (int)(3 * M.m);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    if (P.ntip[i] != 0 || P.mode[i] == 1) continue;  // mode 1: written from member ranks
    const int L = P.len[i];
    const long long vb = P.vb[i];
    if (off_trav) {
      const long long src = off_trav[i];
      for (int q = 0; q < L; ++q) vtx[vb + q] = vtx_trav[src + q];
    } else if (L > 0 && !succ_write(M.tri, succ, P.start[i], L, H, vtx + vb)) {
      set_error(C, POLYLLA_ERR_LIMIT, 71);
    }
  }
}

cudaError_t launch_final_write_polys(const DevMesh& M, const int* succ, const PolyArrays& P,
                                     const long long* off_trav, const int* vtx_trav, int* vtx,
                                     Counters* C, int grid, cudaStream_t s) {
  k_final_write_polys<<<grid, kBlock, 0, s>>>(M, succ, P, off_trav, vtx_trav, vtx, C);
  return cudaGetLastError();
}

// R9b: every piece of a split polygon, one piece per thread.
__global__ void __launch_bounds__(kBlock) k_final_write_pieces(DevMesh M, const int* __restrict__ succ,
                                                               FinalPieces F, int* __restrict__ vtx,
                                                               Counters* C) {
  const long long np = min(C->piece_alloc, F.cap);
  const int H = (int)(3 * M.m);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < np;
       q += (long long)gridDim.x * blockDim.x) {
    const int L = F.len[q];
    if (F.src[q] != 0) continue;  // pieces of long polygons come from their member lists
    if (L > 0 && !succ_write(M.tri, succ, F.start[q], L, H, vtx + F.off[q]))
      set_error(C, POLYLLA_ERR_LIMIT, 72);
  }
}

cudaError_t launch_final_write_pieces(const DevMesh& M, const int* succ, const FinalPieces& F,
                                      int* vtx, Counters* C, int grid, cudaStream_t s) {
  k_final_write_pieces<<<grid, kBlock, 0, s>>>(M, succ, F, vtx, C);
  return cudaGetLastError();
}

}  // namespace polylla
