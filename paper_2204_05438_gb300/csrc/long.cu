// Long polygons: one thread block per polygon whose boundary has more than
// kWalkCap vertices.  A handful of regions per mesh are that large (on a
// 20M-triangle Gaussian-mixture mesh the largest polygon has over a thousand
// vertices and almost a hundred tips); walking or splitting them one dependent
// load at a time would make each of them the critical path of the run.  A block:
//
//   1. collects the region's frontier half-edges by a breadth-first search over
//      its triangles across non-frontier edges (tf words).  The non-frontier edges
//      form a tree (each triangle hangs from the neighbour across its longest
//      edge, Section 3.2.1's labels: a frontier edge is the longest edge of
//      neither of its triangles), so the search goes down it
//      from the seed without a visited set and ends after (longest-edge
//      propagation depth + 1) levels;
//   2. maps each half-edge's successor to a member index, finds the canonical
//      start by a block reduction;
//   3. without reparation (or tips): ranks the cycle from its start by pointer
//      jumping in shared memory (log2(length) rounds) and writes the members in
//      cycle order to the pool;
//   4. with reparation: computes every tip's split edge in parallel, settles in
//      increasing tip order which tips are removed by a smaller tip's split edge
//      ending on them (the result of the paper's rounds with the smallest tip
//      first), marks the split edges frontier, recomputes the successors that end
//      at their endpoints, finds the pieces as the cycles of the new successor
//      function (pointer jumping to each cycle's smallest key, which is the piece's
//      canonical start; a piece is named by its smallest split half-edge), ranks
//      them, orders them as the recursive splitting emits them (first the chord of
//      the smallest tip, the tip->x side first: merging pieces across chords in
//      decreasing tip order builds that tree, on one thread; the rest is parallel)
//      and writes them to the pool.
//
// A region too large for the shared-memory budget is handled by one thread of the
// block with the sequential code (long_fallback).
#include "walk.cuh"

namespace polylla {

// Two sizes of the block: a large one (4096 members, 4096 triangles, 512 threads,
// about 180 KB of shared memory: one block per SM) for any region, and a small
// one (512 members, 512 triangles, 128 threads, about 22 KB: several blocks per
// SM) that hands a region it cannot hold to the large one.
constexpr int kLongThreads = 512;
constexpr int kLM = 4096;  // members of one long polygon (with its split half-edges)
constexpr int kLT = 4096;  // BFS queue: triangles of one long region
constexpr int kSmallThreads = 128;
constexpr int kSmallLM = 512;
constexpr int kSmallLT = 512;
constexpr int kWarpLM = 128;  // one warp per polygon: up to 128 members and triangles
constexpr int kWarpLT = 128;

template <int LM, int LT>
constexpr int long_smem_ints() { return LT + 10 * LM; }

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

// Exclusive prefix sum of v over the block in thread order, for any block size
// (the shared helper assumes kBlock threads); *total gets the sum.  Every thread
// of the block calls it; s_wsum holds 33 ints.
__device__ __forceinline__ int block_scan_any(int v, int* s_wsum, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (int)(blockDim.x >> 5);
  int incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = lane < nw ? s_wsum[lane] : 0;
    int wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += y;
    }
    if (lane < nw) s_wsum[lane] = wi - w;
    if (lane == 31) s_wsum[32] = wi;
  }
  __syncthreads();
  const int r = s_wsum[warp] + incl - v;
  *total = s_wsum[32];
  __syncthreads();
  return r;
}

// Pointer jumping on successor lists (nx: successor, or -1 at a list's end):
// returns the buffer holding, for every node, its number of hops to the end.
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

__device__ __forceinline__ void heap_sift(int* key, int* val, int root, int n) {
  for (;;) {
    int c = 2 * root + 1;
    if (c >= n) return;
    if (c + 1 < n && key[c + 1] > key[c]) ++c;
    if (key[root] >= key[c]) return;
    int t = key[root]; key[root] = key[c]; key[c] = t;
    t = val[root]; val[root] = val[c]; val[c] = t;
    root = c;
  }
}

__device__ void heap_sort(int* key, int* val, int n) {
  for (int r = n / 2 - 1; r >= 0; --r) heap_sift(key, val, r, n);
  for (int e = n - 1; e > 0; --e) {
    int t = key[0]; key[0] = key[e]; key[e] = t;
    t = val[0]; val[0] = val[e]; val[e] = t;
    heap_sift(key, val, 0, e);
  }
}

// One thread: the sequential path for a region too large for shared memory.
__device__ void long_fallback(const DevMesh& M, uint8_t* lab, int* tf, int t0, long long i,
                              PolyArrays& P, FinalPieces& F, Pool& pool, int repair, Counters* C) {
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  P.pcnt[i] = 0;
  P.flen[i] = 0;
  atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_long_seq), 1ull);
  const int e = region_entry_tf(tf, t0, H, limit);
  if (e < 0) {
    set_error(C, POLYLLA_ERR_LIMIT, 100);
    return;
  }
  const Cyc c = cycle_tf(M.tri, tf, e, H, limit);
  if (!c.ok) {
    set_error(C, POLYLLA_ERR_LIMIT, 101);
    return;
  }
  P.start[i] = c.start;
  P.len[i] = c.len;
  P.ntip[i] = c.ntips;
  atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_vtx_trav), (unsigned long long)c.len);
  if (c.ntips) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tips), (unsigned long long)c.ntips);
    atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tip_polys), 1ull);
  }
  const bool split = repair && c.ntips > 0;
  const int need = split ? c.len + 2 * c.ntips : c.len;
  const long long off = (long long)atomicAdd(
      reinterpret_cast<unsigned long long*>(&C->pool_alloc), (unsigned long long)need);
  if (off + need > pool.cap) {
    set_error(C, POLYLLA_ERR_LIMIT, 102);
    return;
  }
  if (!split) {
    if (!write_tf(M.tri, tf, c.start, c.len, H, limit, pool.v + off))
      set_error(C, POLYLLA_ERR_LIMIT, 103);
    P.pos[i] = off;
    P.flen[i] = c.len;
    return;
  }
  const long long foff = (long long)atomicAdd(
      reinterpret_cast<unsigned long long*>(&C->fslot_alloc), (unsigned long long)(c.ntips + 1));
  if (foff + c.ntips + 1 > F.cap) {
    set_error(C, POLYLLA_ERR_LIMIT, 104);
    return;
  }
  const int cnt = repair_seq(M.tri, tf, lab, c, c.ntips + 1, H, limit, F.h + foff, F.pos + foff,
                             F.len + foff, pool.v + off, off, need);
  if (cnt < 0) {
    set_error(C, POLYLLA_ERR_LIMIT, 105);
    return;
  }
  P.pcnt[i] = cnt;
  P.pbase[i] = (int)foff;
  P.flen[i] = c.len + 2 * (cnt - 1);
  atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_splits), (unsigned long long)(cnt - 1));
}

// Lg / n: the polygons of this launch.  over (nullable): where a polygon too large
// for this block size goes (with the counter n_over) instead of the sequential path.
template <int THREADS, int LM, int LT>
__global__ void __launch_bounds__(THREADS, 1) k_long(DevMesh M, uint8_t* lab, int* tf,
                                                  const int* __restrict__ seeds,
                                                  const int* __restrict__ succ, PolyArrays P,
                                                  FinalPieces F, Pool pool, LongList Lg,
                                                  const long long* n_list, LongList over,
                                                  long long* n_over, int* __restrict__ loc,
                                                  int* __restrict__ vstamp, int epoch, int repair,
                                                  Counters* C) {
  constexpr int kLM = LM;
  constexpr int kLT = LT;
  extern __shared__ int smem[];
  int* RQ = smem;       // BFS queue; later the chord list and ordering counts
  int* mem = RQ + kLT;  // members
  int* const R0 = mem + 1 * kLM;
  int* const R1 = mem + 2 * kLM;
  int* const R2 = mem + 3 * kLM;
  int* const R3 = mem + 4 * kLM;
  int* const R4 = mem + 5 * kLM;
  int* const R5 = mem + 6 * kLM;
  int* const R6 = mem + 7 * kLM;
  int* const R7 = mem + 8 * kLM;
  int* const R8 = mem + 9 * kLM;
  __shared__ int s_cnt[3], s_ovf[3], s_nm, s_nt, s_ns, s_fail;
  __shared__ unsigned long long s_key[32];
  __shared__ int s_idx[32];
  __shared__ int s_wsum[33];
  __shared__ long long s_base, s_fbase;
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  const long long nl = min(*n_list, Lg.cap);
  for (long long j = blockIdx.x; j < nl; j += gridDim.x) {
    const long long i = Lg.poly[j];
    const int t0 = seeds[i];
    // ---- 1. the region's triangles, by a breadth-first search down its
    //         longest-edge tree: every non-frontier edge is the longest edge of one
    //         of its triangles, and every triangle but the seed's terminal pair hangs
    //         from the neighbour across its longest edge.  So from a triangle t the
    //         search crosses the non-frontier edges other than t's longest (from the
    //         seed, all of them: its longest edge leads to its terminal partner), and
    //         meets each triangle of the region once, without a visited set.  One
    //         barrier per level: the triangles found in level i go after the level's
    //         range, counted by s_cnt[i % 3] (overflow / error flag s_ovf[i % 3]);
    //         the count and flag of level i - 2 are cleared during level i, when
    //         every thread has read them.
    if (threadIdx.x == 0) {
      for (int c = 0; c < 3; ++c) {
        s_cnt[c] = 0;
        s_ovf[c] = 0;
      }
      s_nm = 0;
      RQ[0] = t0;
    }
    __syncthreads();
    int ovf = 0;
    for (int lvl = 0, lo = 0, hi = 1;; ++lvl) {
      const int c = lvl % 3;
      for (int q = lo + threadIdx.x; q < hi; q += blockDim.x) {
        const int t = RQ[q];
        int x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] = tf[3 * t + k];
        const int up = (t == t0) ? -1 : (int)(lab[t] & 3u);  // the longest edge
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          if (x[k] < 0) {
            const int mi = atomicAdd(&s_nm, 1);
            if (mi < kLM) mem[mi] = 3 * t + k;
            else s_ovf[c] = 1;
          } else if (x[k] >= H) {
            s_ovf[c] = 2;
          } else if (k != up) {
            const int nb = x[k] / 3;
            // the child's tf words and label byte to L1 now: the next level reads them
            asm volatile("prefetch.global.L1 [%0];" ::"l"(tf + 3 * nb));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(lab + nb));
            const int p = hi + atomicAdd(&s_cnt[c], 1);
            if (p < kLT) RQ[p] = nb;
            else s_ovf[c] = 1;
          }
        }
      }
      if (threadIdx.x == 0) {
        s_cnt[(lvl + 1) % 3] = 0;
        s_ovf[(lvl + 1) % 3] = 0;
      }
      __syncthreads();
      ovf = s_ovf[c];
      const int found = s_cnt[c];
      if (ovf || found == 0) break;
      lo = hi;
      hi += found;
    }
    const int L = s_nm;
    if (ovf) {
      if (threadIdx.x == 0) {
        if (ovf == 2) {
          set_error(C, POLYLLA_ERR_LIMIT, 106);
        } else if (over.poly) {  // too large for this block: the large blocks take it
          const long long q =
              (long long)atomicAdd(reinterpret_cast<unsigned long long*>(n_over), 1ull);
          if (q < over.cap) over.poly[q] = (int)i;
          else set_error(C, POLYLLA_ERR_LIMIT, 113);
        } else {
          long_fallback(M, lab, tf, t0, i, P, F, pool, repair, C);
        }
      }
      __syncthreads();
      continue;
    }
    // ---- 2. successors as member indices, tips, canonical start
    for (int a = threadIdx.x; a < L; a += blockDim.x) loc[mem[a]] = a;
    if (threadIdx.x == 0) {
      s_nt = 0;
      s_fail = 0;
    }
    __syncthreads();
    int* tip_bar = R4;
    unsigned long long kb = ~0ull;
    int ib = -1;
    for (int a = threadIdx.x; a < L; a += blockDim.x) {
      const int h = mem[a];
      const int sg = succ[h];
      const int g = sg & kSuccMask;
      int b = ((unsigned)g < (unsigned)H) ? loc[g] : -1;
      if (b < 0 || b >= L || mem[b] != g) {
        s_fail = 1;
        b = a;
      }
      R0[a] = b;
      if (sg & kTipFlag) tip_bar[atomicAdd(&s_nt, 1)] = h;
      const unsigned long long key = he_key(M.tri, h);
      if (key < kb) {
        kb = key;
        ib = a;
      }
    }
    unsigned long long kmin;
    int c;
    block_min_key(kb, ib, s_key, s_idx, &kmin, &c);
    const int nt = s_nt;
    if (s_fail) {
      if (threadIdx.x == 0) set_error(C, POLYLLA_ERR_LIMIT, 107);
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) {
      P.start[i] = mem[c];
      P.len[i] = L;
      P.ntip[i] = nt;
      P.pcnt[i] = 0;
      P.flen[i] = 0;
      atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_vtx_trav), (unsigned long long)L);
      if (nt) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tips), (unsigned long long)nt);
        atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tip_polys), 1ull);
      }
    }
    if (!repair || nt == 0) {
      // ---- 3. the polygon itself, in cycle order from its canonical start
      for (int a = threadIdx.x; a < L; a += blockDim.x)
        if (R0[a] == c) R0[a] = -1;
      __syncthreads();
      const int* dist = list_rank(R0, R1, R2, R3, L);
      if (threadIdx.x == 0)
        s_base = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&C->pool_alloc),
                                      (unsigned long long)L);
      __syncthreads();
      const long long base = s_base;
      if (base + L <= pool.cap) {
        for (int a = threadIdx.x; a < L; a += blockDim.x)
          pool.v[base + (L - 1 - dist[a])] = M.tri[mem[a]];
        if (threadIdx.x == 0) {
          P.pos[i] = base;
          P.flen[i] = L;
        }
      } else if (threadIdx.x == 0) {
        set_error(C, POLYLLA_ERR_LIMIT, 108);
      }
      __syncthreads();
      continue;
    }
    // ---- 4a. split edge of every tip (labels still as traversed)
    int* tip_b = R5;
    int* tip_o = R6;
    int* tip_x = R7;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
      const int g = tip_bar[t];
      const int oj = split_edge(tf, g, H);
      tip_b[t] = M.tri[tf_twin(tf[g])];  // origin of b->a
      tip_o[t] = oj;
      tip_x[t] = (oj >= 0) ? M.tri[he_next(oj)] : -1;
      if (oj < 0) s_fail = 1;
    }
    __syncthreads();
    // ---- 4b. which tips are split: in increasing tip order, a tip is removed when
    //          a split tip with a smaller id ends its split edge on it
    int* sb = R8;          // tip vertices, sorted
    int* st = R8 + kLM / 2;  // their tip indices (nt <= kLM / 2)
    int* cx = R2;          // sorted index of the larger tip at each split edge's end
    int* cancelled = R1;
    const bool sortable = !s_fail && 2 * nt <= kLM;
    if (sortable && nt <= 1024) {
      for (int t = threadIdx.x; t < nt; t += blockDim.x) {  // rank by counting
        const int b = tip_b[t];
        int r = 0;
        for (int u = 0; u < nt; ++u) r += tip_b[u] < b;
        sb[r] = b;
        st[r] = t;
      }
    } else if (sortable && threadIdx.x == 0) {
      for (int t = 0; t < nt; ++t) {
        sb[t] = tip_b[t];
        st[t] = t;
      }
      heap_sort(sb, st, nt);
    }
    __syncthreads();
    if (sortable) {
      for (int q = threadIdx.x; q < nt; q += blockDim.x) {
        cancelled[q] = 0;
        const int x = tip_x[st[q]];
        int hit = -1;
        if (x > sb[q]) {
          int lo = q + 1, hi = nt - 1;
          while (lo <= hi) {
            const int mid = (lo + hi) >> 1;
            if (sb[mid] < x) {
              lo = mid + 1;
            } else if (sb[mid] > x) {
              hi = mid - 1;
            } else {
              hit = mid;
              break;
            }
          }
        }
        cx[q] = hit;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int ns = 0;
      if (sortable) {
        for (int q = 0; q < nt; ++q) {
          if (cancelled[q]) continue;
          RQ[ns++] = st[q];  // chord list, increasing tip vertex
          if (cx[q] >= 0) cancelled[cx[q]] = 1;
        }
      } else {
        s_fail = 1;
      }
      s_ns = ns;
    }
    __syncthreads();
    const int ns = s_ns;
    const int N = L + 2 * ns;
    if (s_fail || N > kLM) {
      // no split edge has been marked yet: the large blocks, or the sequential path
      if (threadIdx.x == 0) {
        if (over.poly && !s_fail) {
          const long long q =
              (long long)atomicAdd(reinterpret_cast<unsigned long long*>(n_over), 1ull);
          if (q < over.cap) over.poly[q] = (int)i;
          else set_error(C, POLYLLA_ERR_LIMIT, 113);
        } else {
          long_fallback(M, lab, tf, t0, i, P, F, pool, repair, C);
        }
      }
      __syncthreads();
      continue;
    }
    // ---- 4c. mark the split edges; their endpoints' successors change
    const int vst = -1 - epoch;  // "endpoint of a split edge" stamp of this run
    for (int q = threadIdx.x; q < ns; q += blockDim.x) {
      const int t = RQ[q];
      const int oj = tip_o[t];
      const int tw = tf_twin(tf[oj]);
      set_frontier(lab, tf, oj);
      set_frontier(lab, tf, tw);
      vstamp[tip_b[t]] = vst;
      vstamp[tip_x[t]] = vst;
      mem[L + 2 * q] = oj;
      mem[L + 2 * q + 1] = tw;
    }
    __syncthreads();
    for (int a = L + threadIdx.x; a < N; a += blockDim.x) loc[mem[a]] = a;
    __syncthreads();
    // ---- 4d. new successors (kept in R6) and each member's cycle minimum key
    int* na = R0;
    int* nb = R1;
    unsigned long long* ka = reinterpret_cast<unsigned long long*>(R2);  // R2..R3
    unsigned long long* kb2 = reinterpret_cast<unsigned long long*>(R4); // R4..R5
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      const int h = mem[a];
      int g;
      if (vstamp[M.tri[he_next(h)]] == vst) {
        long long steps = 0;
        g = turn_tf(tf, h, H, steps, limit);
      } else {
        g = succ[h] & kSuccMask;
      }
      int b = ((unsigned)g < (unsigned)H) ? loc[g] : -1;
      if (b < 0 || b >= N || mem[b] != g) {
        s_fail = 1;
        b = a;
      }
      na[a] = b;
      R6[a] = b;
      ka[a] = he_key(M.tri, h);
    }
    __syncthreads();
    if (s_fail) {
      if (threadIdx.x == 0) set_error(C, POLYLLA_ERR_LIMIT, 109);
      __syncthreads();
      continue;
    }
    {
      int rounds = 1;
      while ((1 << rounds) < N) ++rounds;
      int *pa = na, *pb = nb;
      unsigned long long *qa = ka, *qb = kb2;
      for (int r = 0; r <= rounds; ++r) {
        for (int a = threadIdx.x; a < N; a += blockDim.x) {
          const int n1 = pa[a];
          const unsigned long long x = qa[n1];
          qb[a] = (x < qa[a]) ? x : qa[a];
          pb[a] = pa[n1];
        }
        __syncthreads();
        int* t = pa; pa = pb; pb = t;
        unsigned long long* u = qa; qa = qb; qb = u;
      }
      for (int a = threadIdx.x; a < N; a += blockDim.x)
        R7[a] = loc[(int)(qa[a] & 0xffffffffu)];
    }
    __syncthreads();
    int* A = R7;  // canonical start (member index) of each member's piece
    int* B = R8;  // piece name, at its start: the smallest split member on the piece
    for (int a = threadIdx.x; a < N; a += blockDim.x) B[a] = 0x7fffffff;
    __syncthreads();
    for (int a = L + threadIdx.x; a < N; a += blockDim.x) atomicMin(B + A[a], a);
    // ---- 4e. ranks in the pieces (each cycle cut just before its start)
    for (int a = threadIdx.x; a < N; a += blockDim.x) R0[a] = (R6[a] == A[a]) ? -1 : R6[a];
    __syncthreads();
    const int* dist = list_rank(R0, R1, R2, R3, N);
    int* pos = (dist == R2) ? R3 : R2;  // the free one of the ranking buffers
    int* nodeof = R0;                   // piece name - L -> leaf
    int* node_name = R1;
    int* uf = R4;
    int* left = R5;
    int* right = R6;
    int* cnt = RQ;
    // ---- 4f. the pieces' order.  Leaves: the pieces in increasing name order
    //          (member L + q names its piece when B[A[L + q]] == L + q; a block
    //          scan numbers them).  One thread merges the pieces across the chords
    //          in decreasing tip order into the chord tree and takes the leaves'
    //          positions from its subtree sizes; warp 0 turns the lengths in that
    //          order into offsets.
    int npieces = 0;
    {
      const int per = (2 * ns + (int)blockDim.x - 1) / (int)blockDim.x;
      const int q0 = (int)threadIdx.x * per;
      const int q1 = min(q0 + per, 2 * ns);
      int mine = 0;
      for (int q = q0; q < q1; ++q) {
        const int name = B[A[L + q]];
        if (name < L || name >= N) s_fail = 1;
        mine += name == L + q;
      }
      int id = block_scan_any(mine, s_wsum, &npieces);
      for (int q = q0; q < q1; ++q) {
        if (B[A[L + q]] == L + q) {
          nodeof[q] = id;
          node_name[id++] = L + q;
        }
      }
    }
    __syncthreads();
    if (s_fail || npieces != ns + 1) {
      if (threadIdx.x == 0) set_error(C, POLYLLA_ERR_LIMIT, 110);
      __syncthreads();
      continue;
    }
    // one thread merges, in decreasing tip order, the two trees the chord joins:
    // top[] is the tree of a representative leaf, cnt[] a tree's leaf count,
    // up[] a node's parent and inc[] what a leaf below its right child adds to its
    // position; the leaves then climb to the root in parallel
    int* top = pos;
    int* up = left;
    int* inc = right;
    int* ch = uf + npieces;  // the leaves on either side of chord q: ch[2q], ch[2q + 1]
    for (int v = threadIdx.x; v < npieces; v += blockDim.x) {
      uf[v] = v;
      top[v] = v;
      cnt[v] = 1;
    }
    for (int q = threadIdx.x; q < ns; q += blockDim.x) {
      ch[2 * q] = nodeof[B[A[L + 2 * q]] - L];
      ch[2 * q + 1] = nodeof[B[A[L + 2 * q + 1]] - L];
    }
    __syncthreads();
    if (threadIdx.x == (blockDim.x > 32 ? 32 : 0)) {  // beside the merging thread
      s_base = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&C->pool_alloc),
                                    (unsigned long long)N);
      s_fbase = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&C->fslot_alloc),
                                     (unsigned long long)npieces);
    }
    const int W = 2 * ns + 1;
    if (threadIdx.x == 0) {
      int nodes = npieces;
      for (int q = ns - 1; q >= 0; --q) {  // decreasing tip vertex
        int ra = ch[2 * q];
        int rb = ch[2 * q + 1];
        while (uf[ra] != ra) ra = uf[ra] = uf[uf[ra]];
        while (uf[rb] != rb) rb = uf[rb] = uf[uf[rb]];
        if (ra == rb || nodes >= W) {
          set_error(C, POLYLLA_ERR_LIMIT, 111);
          s_fail = 1;
          break;
        }
        const int u = nodes++;
        const int ta = top[ra], tb = top[rb];
        const int ca = cnt[ta];
        up[ta] = u;
        inc[ta] = 0;
        up[tb] = u;
        inc[tb] = ca;
        cnt[u] = ca + cnt[tb];
        uf[rb] = ra;
        top[ra] = u;
      }
      if (!s_fail) up[nodes - 1] = -1;  // the root
    }
    __syncthreads();
    const long long base = s_base, fb = s_fbase;
    if (s_fail || base + N > pool.cap || fb + npieces > F.cap) {
      if (threadIdx.x == 0 && !s_fail) set_error(C, POLYLLA_ERR_LIMIT, 112);
      __syncthreads();
      continue;
    }
    for (int v = threadIdx.x; v < npieces; v += blockDim.x) {  // position, then length there
      int p = 0;
      for (int x = v, k = 0; up[x] >= 0 && k < W; ++k) {
        p += inc[x];
        x = up[x];
      }
      if (p < npieces) {
        pos[v] = p;
        cnt[p] = dist[A[node_name[v]]] + 1;
      } else {
        s_fail = 1;
      }
    }
    __syncthreads();
    if (s_fail) {  // not a tree: left as an error (no record was written)
      if (threadIdx.x == 0) set_error(C, POLYLLA_ERR_LIMIT, 114);
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) {
      P.pcnt[i] = npieces;
      P.pbase[i] = (int)fb;
      P.flen[i] = N;
      atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_splits), (unsigned long long)ns);
    }
    if (threadIdx.x < 32) {  // offsets and piece records
      const int lane = threadIdx.x;
      int acc = 0;
      for (int p0 = 0; p0 < npieces; p0 += 32) {
        const int p = p0 + lane;
        const int l = p < npieces ? cnt[p] : 0;
        int incl = l;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += y;
        }
        if (p < npieces) {
          cnt[p] = acc + incl - l;
          F.pos[fb + p] = base + acc + incl - l;
          F.len[fb + p] = l;
        }
        acc += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    __syncthreads();
    // ---- 4g. members to the pool: piece offset + rank from the piece's start
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
      const int s0 = A[a];
      const int node = nodeof[B[s0] - L];
      pool.v[base + cnt[pos[node]] + (dist[s0] - dist[a])] = M.tri[mem[a]];
    }
    __syncthreads();
  }
}

template <int THREADS, int LM, int LT>
cudaError_t launch_long_t(const DevMesh& M, uint8_t* lab, int* tf, const int* seeds,
                          const int* succ, const PolyArrays& P, const FinalPieces& F,
                          const Pool& pool, const LongList& Lg, const long long* n_list,
                          const LongList& over, long long* n_over, int* loc, int* vstamp,
                          int epoch, int repair, Counters* C, int grid, cudaStream_t s) {
  const size_t smem = sizeof(int) * (size_t)long_smem_ints<LM, LT>();
  static std::atomic<bool> attr[kMaxDevices];
  const cudaError_t e =
      smem_limit_once(reinterpret_cast<const void*>(k_long<THREADS, LM, LT>), (int)smem, attr);
  if (e != cudaSuccess) return e;
  static std::atomic<int> cap{0};
  grid = resident_grid(reinterpret_cast<const void*>(k_long<THREADS, LM, LT>), THREADS, smem,
                       grid, &cap);
  k_long<THREADS, LM, LT><<<grid, THREADS, smem, s>>>(M, lab, tf, seeds, succ, P, F, pool, Lg,
                                                      n_list, over, n_over, loc, vstamp, epoch,
                                                      repair, C);
  return cudaGetLastError();
}

cudaError_t launch_long(const DevMesh& M, uint8_t* lab, int* tf, const int* seeds, const int* succ,
                        const PolyArrays& P, const FinalPieces& F, const Pool& pool,
                        const LongList& Lg, const LongList& Lg2, int* loc, int* vstamp, int epoch,
                        int repair, int mode, Counters* C, int sms, cudaStream_t s) {
  const LongList none{nullptr, 0};
  if (mode == 0)  // large blocks only
    return launch_long_t<kLongThreads, kLM, kLT>(M, lab, tf, seeds, succ, P, F, pool, Lg,
                                                 &C->n_long, none, nullptr, loc, vstamp, epoch,
                                                 repair, C, sms, s);
  // small blocks (mode 1) or one warp per polygon (mode 2) first; the regions
  // they cannot hold, in large blocks
  cudaError_t e =
      mode == 2 ? launch_long_t<32, kWarpLM, kWarpLT>(M, lab, tf, seeds, succ, P, F, pool, Lg,
                                                      &C->n_long, Lg2, &C->n_long2, loc, vstamp,
                                                      epoch, repair, C, 32 * sms, s)
                : launch_long_t<kSmallThreads, kSmallLM, kSmallLT>(
                      M, lab, tf, seeds, succ, P, F, pool, Lg, &C->n_long, Lg2, &C->n_long2, loc,
                      vstamp, epoch, repair, C, 16 * sms, s);
  if (e != cudaSuccess) return e;
  return launch_long_t<kLongThreads, kLM, kLT>(M, lab, tf, seeds, succ, P, F, pool, Lg2,
                                               &C->n_long2, none, nullptr, loc, vstamp, epoch,
                                               repair, C, sms, s);
}

}  // namespace polylla
