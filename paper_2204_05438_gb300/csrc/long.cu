// Long polygons: one thread block per polygon whose boundary has more than
// kWalkCap vertices.  A handful of regions per mesh are that large (on a
// 20M-triangle Gaussian-mixture mesh the largest polygon has over a thousand
// vertices); walking them one dependent load at a time would make each of them the
// critical path of its phase.  A block instead
//
//   * collects the region's frontier half-edges by a breadth-first search over
//     its triangles across non-frontier edges (tf words).  Every triangle reaches
//     its seed through its longest-edge links, so the search from the seed ends
//     after at most (longest-edge propagation depth + 1) levels;
//   * maps each half-edge's successor to a member index, finds the canonical start
//     (smallest (origin, id)) by a block reduction, and ranks the cycle from it by
//     pointer jumping (Wyllie) in shared memory: log2(length) rounds;
//   * writes the members in cycle order to a compact list, which k_long_write
//     scatters into the CSR once the offsets are known.
//
// k_long_repair does the reparation of a long polygon with tips in the same way:
// after the split edges are marked and the successors around them recomputed, the
// members (old frontier half-edges plus the split half-edges) fall into the pieces'
// cycles; pointer jumping labels every member with its cycle's smallest key (the
// piece's canonical start), the split half-edge that names the piece, and its rank;
// the pieces are then ordered as the recursive splitting emits them (the same
// chord-tree construction as k_poly_order).  A polygon that does not fit the shared
// memory budget falls back to the generic kernels (mode 2).
#include "order.cuh"

namespace polylla {

constexpr int kLongThreads = 512;
constexpr int kLongMaxMembers = 6144;  // frontier half-edges of one long polygon
constexpr int kLongMaxTri = 4096;      // BFS queue (triangles of one long region)

__device__ __forceinline__ int tf_twin(int x) { return x & 0x7fffffff; }

// Block-wide min of a 64-bit key (with the index that holds it).
__device__ void block_min_key(unsigned long long key, int idx, unsigned long long* s_key,
                              int* s_idx, unsigned long long* out_key, int* out_idx) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long ok = __shfl_down_sync(0xffffffffu, key, d);
    const int oi = __shfl_down_sync(0xffffffffu, idx, d);
    if (ok < key) {
      key = ok;
      idx = oi;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_key[warp] = key;
    s_idx[warp] = idx;
  }
  __syncthreads();
  if (warp == 0) {
    key = (lane < (int)(blockDim.x >> 5)) ? s_key[lane] : ~0ull;
    idx = (lane < (int)(blockDim.x >> 5)) ? s_idx[lane] : -1;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const unsigned long long ok = __shfl_down_sync(0xffffffffu, key, d);
      const int oi = __shfl_down_sync(0xffffffffu, idx, d);
      if (ok < key) {
        key = ok;
        idx = oi;
      }
    }
    if (lane == 0) {
      s_key[0] = key;
      s_idx[0] = idx;
    }
  }
  __syncthreads();
  *out_key = s_key[0];
  *out_idx = s_idx[0];
  __syncthreads();
}

// Pointer jumping on a functional graph given by nx[] (each node's successor;
// -1 ends a list): after the call, d[i] = number of hops from i to the end of
// its list.  Buffers a/b are swapped in place; returns the buffer holding d.
__device__ int* list_rank(int* nx0, int* nx1, int* d0, int* d1, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) d0[i] = (nx0[i] < 0) ? 0 : 1;
  __syncthreads();
  int rounds = 1;
  while ((1 << rounds) < n) ++rounds;
  for (int r = 0; r <= rounds; ++r) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int nn = nx0[i];
      if (nn >= 0) {
        d1[i] = d0[i] + d0[nn];
        nx1[i] = nx0[nn];
      } else {
        d1[i] = d0[i];
        nx1[i] = -1;
      }
    }
    __syncthreads();
    int* t = nx0; nx0 = nx1; nx1 = t;
    t = d0; d0 = d1; d1 = t;
  }
  return d0;
}

// ---------------------------------------------------------------- traversal
__global__ void __launch_bounds__(kLongThreads) k_long_trav(DevMesh M, const int* __restrict__ tf,
                                                            const int* __restrict__ seeds,
                                                            const int* __restrict__ succ,
                                                            PolyArrays P, TipArrays T, LongList Lg,
                                                            LongMembers LM, int* __restrict__ visit,
                                                            int* __restrict__ loc, int epoch,
                                                            Counters* C) {
  extern __shared__ int smem[];
  int* tq = smem;                       // kLongMaxTri
  int* mem = tq + kLongMaxTri;          // kLongMaxMembers
  int* nx0 = mem + kLongMaxMembers;
  int* nx1 = nx0 + kLongMaxMembers;
  int* d0 = nx1 + kLongMaxMembers;
  int* d1 = d0 + kLongMaxMembers;
  __shared__ int s_head, s_tail, s_nm, s_over, s_ntip, s_tipcur;
  __shared__ unsigned long long s_key[32];
  __shared__ int s_idx[32];
  __shared__ long long s_base;
  const int H = (int)(3 * M.m);
  const int stamp = 2 * epoch;
  const long long nl = min(C->n_long, Lg.cap);
  for (long long j = blockIdx.x; j < nl; j += gridDim.x) {
    const int i = Lg.poly[j];
    const int t0 = seeds[i];
    // 1. breadth-first search of the region
    if (threadIdx.x == 0) {
      s_head = 0;
      s_tail = 1;
      s_nm = 0;
      s_over = 0;
      tq[0] = t0;
      visit[t0] = stamp;
    }
    __syncthreads();
    for (;;) {
      const int lo = s_head, hi = s_tail;
      const int over = s_over;
      __syncthreads();
      if (lo >= hi || over) break;
      for (int q = lo + threadIdx.x; q < hi; q += blockDim.x) {
        const int t = tq[q];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int x = tf[3 * t + k];
          if (x < 0) {
            const int mi = atomicAdd(&s_nm, 1);
            if (mi < kLongMaxMembers) mem[mi] = 3 * t + k;
            else s_over = 1;
          } else {
            if (x >= H) {
              s_over = 2;
              continue;
            }
            const int nb = x / 3;
            if (atomicExch(visit + nb, stamp) != stamp) {
              const int p = atomicAdd(&s_tail, 1);
              if (p < kLongMaxTri) tq[p] = nb;
              else s_over = 1;
            }
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_head = hi;
      __syncthreads();
    }
    const int L = s_nm;
    if (s_over) {
      // too large for the shared-memory path: the generic walk takes it (mode 2)
      if (threadIdx.x == 0) {
        if (s_over == 2) set_error(C, POLYLLA_ERR_LIMIT, 100);
        P.mode[i] = 2;
        const long long limit = 3 * M.m + 3;
        const int e = region_entry_tf(tf, t0, H, limit);
        int len = 0, ntip = 0;
        unsigned long long best = ~0ull;
        int h = e;
        bool ok = e >= 0;
        while (ok) {
          const unsigned long long key = he_key(M.tri, h);
          if (key < best) best = key;
          const int sg = succ[h];
          ntip += (sg & kTipFlag) ? 1 : 0;
          ++len;
          h = sg & kSuccMask;
          if ((unsigned)h >= (unsigned)H || len > limit) ok = false;
          else if (h == e) break;
        }
        if (!ok) {
          set_error(C, POLYLLA_ERR_LIMIT, 101);
          len = 0;
          ntip = 0;
        }
        P.start[i] = (int)(best & 0xffffffffu);
        P.len[i] = len;
        P.ntip[i] = ntip;
        if (ntip > 0) {
          const long long base = (long long)atomicAdd(
              reinterpret_cast<unsigned long long*>(&C->n_tips), (unsigned long long)ntip);
          P.tipbase[i] = (int)base;
          int q = 0;
          h = e;
          for (int step = 0; step < len && base + q < T.cap; ++step) {
            const int sg = succ[h];
            if (sg & kTipFlag) {
              T.h[base + q] = h;
              T.poly[base + q] = i;
              T.vtip[M.tri[he_next(h)]] = ((long long)epoch << 32) | (unsigned)(base + q);
              ++q;
            }
            h = sg & kSuccMask;
          }
        }
        atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_vtx_trav), (unsigned long long)len);
        if (ntip) atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tip_polys), 1ull);
      }
      __syncthreads();
      continue;
    }
    // 2. successor of every member as a member index; canonical start
    for (int a = threadIdx.x; a < L; a += blockDim.x) loc[mem[a]] = a;
    __syncthreads();
    unsigned long long kbest = ~0ull;
    int ibest = -1;
    if (threadIdx.x == 0) {
      s_ntip = 0;
      s_tipcur = 0;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < L; a += blockDim.x) {
      const int h = mem[a];
      const int sg = succ[h];
      const int g = sg & kSuccMask;
      int b = ((unsigned)g < (unsigned)H) ? loc[g] : -1;
      if (b < 0 || b >= L || mem[b] != g) {
        set_error(C, POLYLLA_ERR_LIMIT, 102);
        b = a;
      }
      nx0[a] = b;
      if (sg & kTipFlag) atomicAdd(&s_ntip, 1);
      const unsigned long long key = he_key(M.tri, h);
      if (key < kbest) {
        kbest = key;
        ibest = a;
      }
    }
    unsigned long long kmin;
    int c;
    block_min_key(kbest, ibest, s_key, s_idx, &kmin, &c);
    // 3. rank from the canonical start: cut the cycle before it, then jump
    for (int a = threadIdx.x; a < L; a += blockDim.x)
      if (nx0[a] == c) nx0[a] = -1;
    __syncthreads();
    int* dist = list_rank(nx0, nx1, d0, d1, L);
    // 4. outputs: members in cycle order, polygon record, tips
    if (threadIdx.x == 0) {
      s_base = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&C->lm_alloc),
                                    (unsigned long long)L);
      const int ntip = s_ntip;
      P.start[i] = mem[c];
      P.len[i] = L;
      P.ntip[i] = ntip;
      if (ntip > 0) {
        const long long tb = (long long)atomicAdd(
            reinterpret_cast<unsigned long long*>(&C->n_tips), (unsigned long long)ntip);
        P.tipbase[i] = (int)tb;
        atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tip_polys), 1ull);
      }
      atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_vtx_trav), (unsigned long long)L);
    }
    __syncthreads();
    const long long base = s_base;
    if (threadIdx.x == 0) P.lmbase[i] = (base + L <= LM.cap) ? (int)base : -1;
    for (int a = threadIdx.x; a < L; a += blockDim.x) {
      const int r = L - 1 - dist[a];
      if (base + L <= LM.cap) {
        LM.h[base + r] = mem[a];
        LM.poly[base + r] = i;
      }
      const int h = mem[a];
      if (succ[h] & kTipFlag) {
        const int q = atomicAdd(&s_tipcur, 1);
        const long long slot = (long long)P.tipbase[i] + q;
        if (slot < T.cap) {
          T.h[slot] = h;
          T.poly[slot] = i;
          T.vtip[M.tri[he_next(h)]] = ((long long)epoch << 32) | (unsigned)slot;
        }
      }
    }
    if (threadIdx.x == 0 && base + L > LM.cap) set_error(C, POLYLLA_ERR_LIMIT, 103);
    __syncthreads();
  }
}

// Members of long polygons, in cycle order, into a CSR (traversal CSR: every long
// polygon; final CSR: long polygons without tips).
__global__ void __launch_bounds__(kBlock) k_long_write(DevMesh M, LongMembers LM, PolyArrays P,
                                                       const long long* __restrict__ off,
                                                       int* __restrict__ vtx, int final_pass,
                                                       Counters* C) {
  const long long nm = min(C->lm_alloc, LM.cap);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nm;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = LM.poly[e];
    if (P.mode[i] != 1) continue;
    if (final_pass && P.ntip[i] != 0) continue;  // its pieces are written elsewhere
    const long long r = e - P.lmbase[i];
    const long long dst = (final_pass ? P.vb[i] : off[i]) + r;
    vtx[dst] = M.tri[LM.h[e]];
  }
}

// ---------------------------------------------------------------- reparation
// Shared memory: mem[N] | A[N] | B[N] (ints) | K0[N] | K1[N] (64-bit), N <= kLongMaxMembers.
__global__ void __launch_bounds__(kLongThreads) k_long_repair(
    DevMesh M, const int* __restrict__ succ, PolyArrays P, TipArrays T, LongList Lg,
    LongMembers LM, LongMembers LM2, FinalPieces F, int* __restrict__ loc, int epoch, Counters* C) {
  extern __shared__ int smem[];
  int* mem = smem;
  int* A = mem + kLongMaxMembers;
  int* B = A + kLongMaxMembers;
  unsigned long long* K0 = reinterpret_cast<unsigned long long*>(B + kLongMaxMembers);
  unsigned long long* K1 = K0 + kLongMaxMembers;
  __shared__ int s_n;
  __shared__ long long s_base;
  const int H = (int)(3 * M.m);
  const long long nl = min(C->n_long, Lg.cap);
  for (long long j = blockIdx.x; j < nl; j += gridDim.x) {
    const int i = Lg.poly[j];
    if (P.mode[i] != 1 || P.ntip[i] == 0) continue;  // uniform across the block
    const int L = P.len[i];
    const long long lb = P.lmbase[i];
    const int nt = P.ntip[i];
    const long long tb = P.tipbase[i];
    // 1. members: the polygon's old frontier half-edges (in cycle order), then both
    //    half-edges of every processed split edge
    if (threadIdx.x == 0) {
      int w = L;
      for (int q = 0; q < nt; ++q) {
        const long long k = tb + q;
        if (T.state[k] != 1 || T.o[k] < 0) continue;
        if (w + 2 <= kLongMaxMembers) {
          mem[w] = T.o[k];
          mem[w + 1] = M.twin[T.o[k]];
        }
        w += 2;
      }
      s_n = w;
    }
    __syncthreads();
    const int N = s_n;
    if (N > kLongMaxMembers || lb < 0) {
      if (threadIdx.x == 0) P.mode[i] = 2;  // the generic kernels take this polygon
      __syncthreads();
      continue;
    }
    for (int a = threadIdx.x; a < L; a += blockDim.x) mem[a] = LM.h[lb + a];
    __syncthreads();
    for (int a = threadIdx.x; a < N; a += blockDim.x) loc[mem[a]] = a;
    __syncthreads();
    // 2. successors after the splits (A) and keys (K0)
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      const int g = succ[mem[a]] & kSuccMask;
      int b = ((unsigned)g < (unsigned)H) ? loc[g] : -1;
      if (b < 0 || b >= N || mem[b] != g) {
        set_error(C, POLYLLA_ERR_LIMIT, 110);
        b = a;
      }
      A[a] = b;
      K0[a] = he_key(M.tri, mem[a]);
    }
    __syncthreads();
    // 3. every member learns its cycle's smallest key by pointer jumping
    int rounds = 1;
    while ((1 << rounds) < N) ++rounds;
    {
      int *na = A, *nb = B;
      unsigned long long *ka = K0, *kb = K1;
      for (int r = 0; r <= rounds; ++r) {
        for (int a = threadIdx.x; a < N; a += blockDim.x) {
          const int n1 = na[a];
          const unsigned long long x = ka[n1];
          kb[a] = (x < ka[a]) ? x : ka[a];
          nb[a] = na[n1];
        }
        __syncthreads();
        int* t = na; na = nb; nb = t;
        unsigned long long* u = ka; ka = kb; kb = u;
      }
      if (ka != K0)
        for (int a = threadIdx.x; a < N; a += blockDim.x) K0[a] = ka[a];
      __syncthreads();
    }
    // A[a] = member index of a's piece's canonical start
    for (int a = threadIdx.x; a < N; a += blockDim.x) A[a] = loc[(int)(K0[a] & 0xffffffffu)];
    // 4. B[start] = smallest split record on the piece (names the piece)
    for (int a = threadIdx.x; a < N; a += blockDim.x) B[a] = 0x7fffffff;
    __syncthreads();
    for (int a = L + threadIdx.x; a < N; a += blockDim.x) {
      const long long tag = T.chord[mem[a]];
      if ((int)(tag >> 32) == epoch) atomicMin(B + A[a], (int)(tag & 0xffffffffll));
    }
    __syncthreads();
    // 5. ranks from each piece's canonical start (its cycle cut just before it)
    int* nx0 = reinterpret_cast<int*>(K1);
    int* nx1 = nx0 + kLongMaxMembers;
    int* d0 = reinterpret_cast<int*>(K0);
    int* d1 = d0 + kLongMaxMembers;
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      const int b = loc[succ[mem[a]] & kSuccMask];
      nx0[a] = (b == A[a]) ? -1 : b;
    }
    __syncthreads();
    const int* dist = list_rank(nx0, nx1, d0, d1, N);
    // 6. piece records of every split candidate; the naming ones get start / length
    for (int a = L + threadIdx.x; a < N; a += blockDim.x) {
      const long long tag = T.chord[mem[a]];
      if ((int)(tag >> 32) != epoch) continue;
      const int q = (int)(tag & 0xffffffffll);
      const int st = A[a];
      const int rec = B[st];
      T.piece[q] = rec;
      if (rec == q) {
        T.rec_start[q] = mem[st];
        T.rec_len[q] = dist[st] + 1;
      }
    }
    // 7. the pieces' members for the final write: (half-edge, rank, naming record)
    if (threadIdx.x == 0)
      s_base = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&C->lm2_alloc),
                                    (unsigned long long)N);
    __syncthreads();
    const long long base = s_base;
    if (base + N <= LM2.cap) {
      for (int a = threadIdx.x; a < N; a += blockDim.x) {
        const int st = A[a];
        LM2.h[base + a] = mem[a];
        LM2.poly[base + a] = B[st];
        LM2.rank[base + a] = dist[st] - dist[a];
      }
    } else if (threadIdx.x == 0) {
      set_error(C, POLYLLA_ERR_LIMIT, 111);
    }
    __syncthreads();
    // 8. order the pieces (shared memory is free again): one thread, as k_poly_order
    if (threadIdx.x == 0) {
      const bool fits = 24ll * nt + 8 <= 7ll * kLongMaxMembers;  // ints of shared memory
      order_pieces(M, P, T, F, C, i, fits ? smem : T.scratch + 24ll * tb, 1);
      P.mode[i] = 3;
    }
    __syncthreads();
  }
}

// Members of the pieces of long polygons into the final CSR.
__global__ void __launch_bounds__(kBlock) k_long_write_pieces(DevMesh M, LongMembers LM2,
                                                              TipArrays T, FinalPieces F,
                                                              int* __restrict__ vtx, Counters* C) {
  const long long nm = min(C->lm2_alloc, LM2.cap);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nm;
       e += (long long)gridDim.x * blockDim.x) {
    const int slot = T.rec_slot[LM2.poly[e]];
    if (slot < 0 || slot >= F.cap) {
      set_error(C, POLYLLA_ERR_LIMIT, 112);
      continue;
    }
    vtx[F.off[slot] + LM2.rank[e]] = M.tri[LM2.h[e]];
  }
}

cudaError_t launch_long_write_pieces(const DevMesh& M, const LongMembers& LM2, const TipArrays& T,
                                     const FinalPieces& F, int* vtx, Counters* C, int grid,
                                     cudaStream_t s) {
  k_long_write_pieces<<<grid, kBlock, 0, s>>>(M, LM2, T, F, vtx, C);
  return cudaGetLastError();
}

cudaError_t launch_long_trav(const DevMesh& M, const int* tf, const int* seeds, const int* succ,
                             const PolyArrays& P, const TipArrays& T, const LongList& Lg,
                             const LongMembers& LM, int* visit, int* loc, int epoch, Counters* C,
                             int grid, cudaStream_t s) {
  const size_t smem = sizeof(int) * (size_t)(kLongMaxTri + 5 * kLongMaxMembers);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_long_trav, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_long_trav<<<grid, kLongThreads, smem, s>>>(M, tf, seeds, succ, P, T, Lg, LM, visit, loc, epoch,
                                               C);
  return cudaGetLastError();
}

cudaError_t launch_long_write(const DevMesh& M, const LongMembers& LM, const PolyArrays& P,
                              const long long* off, int* vtx, int final_pass, Counters* C, int grid,
                              cudaStream_t s) {
  k_long_write<<<grid, kBlock, 0, s>>>(M, LM, P, off, vtx, final_pass, C);
  return cudaGetLastError();
}

cudaError_t launch_long_repair(const DevMesh& M, const int* succ, const PolyArrays& P,
                               const TipArrays& T, const LongList& Lg, const LongMembers& LM,
                               const LongMembers& LM2, const FinalPieces& F, int* loc, int epoch,
                               Counters* C, int grid, cudaStream_t s) {
  const size_t smem = sizeof(int) * (size_t)(3 * kLongMaxMembers) +
                      sizeof(unsigned long long) * (size_t)(2 * kLongMaxMembers);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_long_repair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_long_repair<<<grid, kLongThreads, smem, s>>>(M, succ, P, T, Lg, LM, LM2, F, loc, epoch, C);
  return cudaGetLastError();
}

}  // namespace polylla
