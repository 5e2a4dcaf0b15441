// Traversal (Section 3.2.2, Algorithms 3 and 4) and, for ordinary polygons,
// reparation (Section 3.2.3, Algorithm 5) in one pass.
//
//   k_succ  for each frontier half-edge, the next frontier half-edge of its
//           region's boundary (PolyConstruction's turn), with the barrier-edge
//           tip flag; each warp compacts the frontier half-edges of 256
//           triangles and turns them one per lane.
//   k_walk  one thread per seed: enter the region (at the entry half-edge the
//           seed kernel found), chase succ around the cycle (at most kWalkCap
//           vertices, staged in shared memory), note the canonical start and the
//           tips.  A polygon without tips (or any, when no reparation is asked
//           for) is copied, rotated to its canonical start, into the vertex pool,
//           whose space is handed out per warp.  A polygon
//           with tips is listed -- one tip (about 90% of them) or several -- so
//           that the dependent loads of a split do not stall the 31 other lanes of
//           its warp; a longer one is left to one thread block (long.cu).
//   k_repair_one    one thread per polygon with one tip: split it and cut the
//           two pieces out of the vertex sequence the walk left in the pool.
//   k_repair_multi  one thread per polygon with several tips: the cycle becomes
//           a linked list of nodes in shared memory, and each split (smallest tip
//           of the current piece first) adds two chord nodes and relinks four
//           pointers.
// The paper's AtomicAdd on i_Gmesh / i_Gpos is replaced by the output scan
// (final.cu); the pool order does not matter.
#include "walk.cuh"

namespace polylla {

// Each warp takes a chunk of 32 * PER consecutive triangles at a time (PER = 8
// on large meshes): their frontier half-edges (label bits 2-4, PER triangles per
// lane) are compacted into the warp's list in shared memory by a warp scan, in
// increasing order, and then turned 32 at a time, one per lane: no lane idles on a
// half-edge that is not frontier, and the 32 turns of a round start at
// neighbouring half-edges.  On a mesh with fewer 256-triangle chunks than the
// grid has warps, smaller chunks (PER = 4, 2, 1) give every warp work, so a warp
// turns fewer rounds one after another.
template <int PER>
__device__ __forceinline__ unsigned long long load_lab(const uint8_t* __restrict__ lab,
                                                       long long t0, long long m) {
  unsigned long long v = 0;
  if (t0 + PER <= m && (reinterpret_cast<uintptr_t>(lab + t0) & (PER - 1)) == 0) {
    if (PER == 8) {
      const uint2 w = __ldg(reinterpret_cast<const uint2*>(lab + t0));
      v = (unsigned long long)w.x | ((unsigned long long)w.y << 32);
    } else if (PER == 4) {
      v = __ldg(reinterpret_cast<const unsigned*>(lab + t0));
    } else if (PER == 2) {
      v = __ldg(reinterpret_cast<const unsigned short*>(lab + t0));
    } else {
      v = __ldg(lab + t0);
    }
  } else {
    for (int i = 0; i < PER && t0 + i < m; ++i)
      v |= (unsigned long long)__ldg(lab + t0 + i) << (8 * i);
  }
  return v;
}

template <int PER>
__global__ void __launch_bounds__(kBlock) k_succ(DevMesh M, const uint8_t* __restrict__ lab,
                                                 const int* __restrict__ tf,
                                                 int* __restrict__ succ, Counters* C) {
  constexpr int kChunk = 32 * PER;
  // half-edge offsets inside the chunk (< 3 * kChunk): 16 bits leave the L1 the
  // turns read from
  __shared__ unsigned short s_list[kBlock / 32][3 * kChunk];
  pdl_wait();  // the label bytes and tf words
  pdl_launch_dependents();
  const long long m = M.m;
  const int H = (int)(3 * m);
  const int lane = threadIdx.x & 31;
  unsigned short* list = s_list[threadIdx.x >> 5];
  const long long nchunks = (m + kChunk - 1) / kChunk;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  // the label bytes of this lane's PER triangles of chunk ch (loaded one chunk ahead)
  auto load = [&](long long ch) -> unsigned long long {
    if (ch >= nchunks) return 0;
    return load_lab<PER>(lab, ch * kChunk + (long long)lane * PER, m);
  };
  long long ch = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
  unsigned long long next = load(ch);
  for (; ch < nchunks; ch += nwarps) {
    const unsigned long long bytes = next;
    next = load(ch + nwarps);
    // bit 3i + k: half-edge k of the lane's triangle i is frontier
    unsigned mask = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) mask |= (unsigned)((bytes >> (8 * i + 2)) & 7u) << (3 * i);
    const int c = __popc(mask);
    int incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    int pos = incl - c;
    const int o0 = 3 * PER * lane;  // this lane's first half-edge in the chunk
    while (mask) {
      const int s = __ffs(mask) - 1;
      mask &= mask - 1;
      list[pos++] = (unsigned short)(o0 + s);
    }
    __syncwarp();
    const int hc = (int)(3 * ch * kChunk);  // the chunk's first half-edge
    for (int j = lane; j < total; j += 32) {
      const int h = hc + list[j];
      const int x = __ldg(tf + h);
      int cur = he_next(h);
      int y = __ldg(tf + cur);
      for (int steps = 0; y >= 0;) {
        if (y >= H || ++steps > H) {
          set_error(C, POLYLLA_ERR_LIMIT, 50);
          cur = h;
          break;
        }
        cur = he_next(y);
        y = __ldg(tf + cur);
      }
      succ[h] = (cur == tf_twin(x)) ? (cur | kTipFlag) : cur;
    }
    __syncwarp();
  }
}

template <int PER>
cudaError_t launch_succ_t(const DevMesh& M, const uint8_t* lab, const int* tf, int* succ,
                          Counters* C, int grid, cudaStream_t s, bool pdl) {
  static std::atomic<int> cap{0};
  grid = resident_grid(reinterpret_cast<const void*>(k_succ<PER>), kBlock, 0, grid, &cap);
  return launch_chain(k_succ<PER>, grid, kBlock, 0, s, pdl, M, lab, tf, succ, C);
}

cudaError_t launch_succ(const DevMesh& M, const uint8_t* lab, const int* tf, int* succ,
                        Counters* C, int grid, cudaStream_t s, bool pdl) {
  // the largest chunk that still gives every warp of the grid at least one
  const long long warps = (long long)grid * (kBlock / 32);
  if (M.m >= 256 * warps) return launch_succ_t<8>(M, lab, tf, succ, C, grid, s, pdl);
  if (M.m >= 128 * warps) return launch_succ_t<4>(M, lab, tf, succ, C, grid, s, pdl);
  if (M.m >= 64 * warps) return launch_succ_t<2>(M, lab, tf, succ, C, grid, s, pdl);
  return launch_succ_t<1>(M, lab, tf, succ, C, grid, s, pdl);
}

// Warp-aggregated allocation: each lane asks for `need` entries; one atomic per
// warp.  All 32 lanes must call it.
__device__ __forceinline__ long long warp_alloc(long long* counter, int need) {
  const int lane = threadIdx.x & 31;
  int incl = need;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total > 0)
    base = atomicAdd(reinterpret_cast<unsigned long long*>(counter), (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return (long long)base + incl - need;
}


// Polygons with more tips than this are split by one thread re-walking its pieces
// (repair_seq); those with 2..kRsMaxSplit tips get the walk's tip records and the
// several-tip kernel's node list.
constexpr int kRsMaxSplit = 8;

// Warp-aggregated list append: each lane with `want` gets its own slot of the
// list counted by `counter` (one atomic per warp, slots in lane order), the
// others -1.  All 32 lanes must call it.
__device__ __forceinline__ long long warp_append(long long* counter, bool want) {
  const unsigned b = __ballot_sync(0xffffffffu, want);
  if (b == 0) return -1;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(b) - 1;
  unsigned long long base = 0;
  if (lane == leader)
    base = atomicAdd(reinterpret_cast<unsigned long long*>(counter), (unsigned long long)__popc(b));
  base = __shfl_sync(0xffffffffu, base, leader);
  return want ? (long long)base + __popc(b & ((1u << lane) - 1u)) : -1;
}

// Triangle of a seed's entry word (3t + k, or -1 - t)
__device__ __forceinline__ long long entry_tri(int e) { return e >= 0 ? e / 3 : -1 - (long long)e; }

// L2 prefetch of the whole 128-byte lines inside [p, p + bytes) (the partial
// lines at either end are left out, so no address outside the range is touched),
// spread over the block
__device__ __forceinline__ void prefetch_l2(const void* p, long long bytes) {
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(p) + 127) & ~(uintptr_t)127;
  const uintptr_t hi = (reinterpret_cast<uintptr_t>(p) + (uintptr_t)bytes) & ~(uintptr_t)127;
  for (uintptr_t c = lo + 128 * (uintptr_t)threadIdx.x; c < hi; c += 128 * (uintptr_t)blockDim.x)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c));
}


__global__ void __launch_bounds__(kWalkThreads) k_walk(DevMesh M, int* tf,
                                                       const int* __restrict__ entry,
                                                       const int* __restrict__ succ, PolyArrays P,
                                                       Pool pool, LongList Lg, LongList D1,
                                                       LongList Dm, int cap, int repair,
                                                       int tips_to_long, Counters* C) {
  // staging transposed (word q of thread x at q * blockDim + x): the lanes of a
  // warp, writing the same position in lockstep, hit 32 different banks
  extern __shared__ int sbuf[];
  pdl_wait();  // the successors, seeds and entries
  int* my = sbuf + threadIdx.x;
  const long long n = C->n_seeds;
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  unsigned st_len = 0, st_tips = 0, st_tippolys = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += stride) {
    const long long i = base + threadIdx.x;
    // the next iteration's seeds lie in one run of triangles (seeds ascend): the
    // successor words of that run go to L2 now, while this iteration walks (the
    // same for tri, or with a margin around the run, was slower)
    if (base + stride < n) {
      const long long nb = base + stride;
      const long long ne = (nb + blockDim.x < n ? nb + blockDim.x : n) - 1;
      const long long t0 = entry_tri(__ldg(entry + nb));
      long long t1 = entry_tri(__ldg(entry + ne));
      t1 = t1 >= M.m ? M.m - 1 : t1;
      if (t1 >= t0) {
        prefetch_l2(succ + 3 * t0, 12 * (t1 - t0 + 1));
      }
    }
    int len = 0, ntips = 0, tip_h = -1, tip_s = 0, rank0 = 0, start = 0;
    bool closed = false, is_long = false;
    if (i < n) {
      int e = entry[i];
      if (e < 0) e = region_entry_tf(tf, -1 - e, H, limit);
      if (e < 0) {
        set_error(C, POLYLLA_ERR_LIMIT, 51);
      } else {
        unsigned long long best = ~0ull;
        int tipv = 0x7fffffff;
        int h = e;
        bool ok = true;
        do {
          const int o = M.tri[h];
          my[len * kWalkThreads] = o;
          const unsigned long long key = ((unsigned long long)(unsigned)o << 32) | (unsigned)h;
          if (key < best) {
            best = key;
            rank0 = len;
          }
          const int sg = succ[h];
          const int g = sg & kSuccMask;
          if (sg & kTipFlag) {
            ++ntips;
            // tip record k (its half-edge and step), staged from the top while
            // the origins below have not reached it
            if (ntips <= kRsMaxSplit && cap - 2 * ntips > len) {
              my[(cap - 2 * ntips) * kWalkThreads] = h;
              my[(cap - 2 * ntips + 1) * kWalkThreads] = len;
            }
            const int b = M.tri[g];  // dest(h) = origin(twin(h))
            if (b < tipv) {
              tipv = b;
              tip_h = h;
              tip_s = len;
            }
          }
          ++len;
          if ((unsigned)g >= (unsigned)H) {
            ok = false;
            break;
          }
          h = g;
        } while (h != e && len < cap);
        closed = ok && h == e;
        is_long = ok && !closed;
        // several tips on a small mesh: the block kernel splits them in parallel
        if (closed && repair && tips_to_long > 0 && ntips >= tips_to_long) {
          closed = false;
          is_long = true;
        }
        if (!ok) set_error(C, POLYLLA_ERR_LIMIT, 52);
        start = (int)(best & 0xffffffffu);
      }
    }
    const bool split = closed && repair && ntips > 0;
    // a one-tip polygon's vertex sequence goes to the pool too: its split cuts
    // the two pieces out of it
    const bool seq = split && ntips == 1;
    // a polygon with 2..kRsMaxSplit tips whose records all stayed above its
    // origins: the sequence and the records (rotated tip index, tip half-edge)
    // go to the pool, where the several-tip kernel also writes its pieces
    const bool rec = split && ntips >= 2 && ntips <= kRsMaxSplit && len + 2 * ntips <= cap;
    const int need = (closed && (!split || seq)) ? len : (rec ? len + 2 * ntips : 0);
    const long long off = warp_alloc(&C->pool_alloc, need);
    // list slots, one atomic per warp and list
    const long long jl = warp_append(&C->n_long, i < n && is_long);
    const long long j1 = warp_append(&C->n_defer, i < n && split && ntips == 1);
    const long long jm = warp_append(&C->n_multi, i < n && split && ntips > 1);
    if (i >= n) continue;
    if (is_long) {
      P.pcnt[i] = 0;
      P.flen[i] = 0;
      if (jl < Lg.cap) Lg.poly[jl] = (int)i;
      continue;
    }
    // start, length and tips are read only by the reparation kernels
    P.pcnt[i] = 0;
    P.flen[i] = 0;
    if (!closed) continue;
    st_len += len;
    st_tips += ntips;
    st_tippolys += ntips > 0;
    if (need) {  // the sequence, rotated to the canonical start
      if (off + need > pool.cap) {
        set_error(C, POLYLLA_ERR_LIMIT, 53);
        // its list slot is taken: a record the split kernels skip
        if (seq && j1 < D1.cap) {
          P.len[i] = 0;
          D1.poly[j1] = (int)i;
        }
        if (rec && jm < Dm.cap) {
          P.len[i] = 0;
          Dm.poly[jm] = (int)i;
        }
        continue;
      }
      int* out = pool.v + off;
      int r = rank0;
      for (int q = 0; q < len; ++q) {
        out[q] = my[r * kWalkThreads];
        if (++r == len) r = 0;
      }
      for (int k = 1; rec && k <= ntips; ++k) {
        const int st = my[(cap - 2 * k + 1) * kWalkThreads];
        out[len + 2 * (k - 1)] = st >= rank0 ? st - rank0 : st - rank0 + len;
        out[len + 2 * (k - 1) + 1] = my[(cap - 2 * k) * kWalkThreads];
      }
      P.pos[i] = off;
    }
    if (split) {
      P.start[i] = start;
      P.len[i] = len;
      P.ntip[i] = ntips;
      P.tip_h[i] = tip_h;
      if (seq) P.pbase[i] = tip_s >= rank0 ? tip_s - rank0 : tip_s - rank0 + len;
      else P.pbase[i] = rec ? 1 : 0;  // several tips: records at pos, or none
      LongList& D = (ntips == 1) ? D1 : Dm;
      const long long d = (ntips == 1) ? j1 : jm;
      if (d < D.cap) D.poly[d] = (int)i;
      else set_error(C, POLYLLA_ERR_LIMIT, 55);
      continue;
    }
    P.flen[i] = len;
  }
  st_len = __reduce_add_sync(0xffffffffu, st_len);
  st_tips = __reduce_add_sync(0xffffffffu, st_tips);
  st_tippolys = __reduce_add_sync(0xffffffffu, st_tippolys);
  if ((threadIdx.x & 31) == 0) {
    if (st_len) atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_vtx_trav), (unsigned long long)st_len);
    if (st_tips) atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tips), (unsigned long long)st_tips);
    if (st_tippolys)
      atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_tip_polys), (unsigned long long)st_tippolys);
  }
}

cudaError_t launch_walk(const DevMesh& M, int* tf, const int* entry, const int* succ,
                        const PolyArrays& P, const Pool& pool, const LongList& Lg,
                        const LongList& D1, const LongList& Dm, int cap, int repair,
                        int tips_to_long, Counters* C, int grid, cudaStream_t s, bool pdl) {
  if (cap < 16 || cap > kWalkCap || cap % 16) return cudaErrorInvalidValue;
  const size_t smem = sizeof(int) * (size_t)kWalkThreads * cap;
  static std::atomic<bool> attr[kMaxDevices];
  const cudaError_t e = smem_limit_once(reinterpret_cast<const void*>(k_walk),
                                        (int)(sizeof(int) * kWalkThreads * kWalkCap), attr);
  if (e != cudaSuccess) return e;
  static std::atomic<int> resident[kWalkCap / 16 + 1] = {};
  grid = resident_grid(reinterpret_cast<const void*>(k_walk), kWalkThreads, smem, grid,
                       &resident[cap / 16]);
  return launch_chain(k_walk, grid, kWalkThreads, smem, s, pdl, M, tf, entry, succ, P, pool, Lg, D1,
                      Dm, cap, repair, tips_to_long, C);
}

__device__ __forceinline__ unsigned long long vkey(int origin, int h) {
  return ((unsigned long long)(unsigned)origin << 32) | (unsigned)h;
}

constexpr int kSeqChunk = 4;  // sequence entries loaded at a time by the split kernels

// One tip p = a->b, split along oj = b->x (tw = x->b), with q = turn(oj) and
// pn = twin(p) = b->a.  The two pieces are
//     oj, q, succ(q), ..., p          and          tw, pn, succ(pn), ..., pred(q)
// (the boundary walk with oj, tw frontier); the other frontier half-edges keep
// their turns.  The walk left the polygon's vertex sequence v (from its canonical
// start) in the pool and the tip's index t in it (v[t] = a, v[t+1] = b).  When x
// occurs once in v, at u, q is the half-edge leaving x there, and the pieces are
//     b, v[u], ..., v[t]          and          x, v[t+1], ..., v[u-1]
// (indices cyclic); each is written from its smallest vertex when that vertex
// occurs once in it (then it is the canonical start).  Otherwise (x, or a piece's
// smallest vertex, repeated: the canonical start needs half-edge ids) the two arcs
// of the cycle are chased along succ at once, staged over v (arc 1 from the
// front, arc 2 from the back), and each piece is copied from its canonical start.
// Pool space: L + 2 for the pieces.
__global__ void __launch_bounds__(kBlock) k_repair_one(DevMesh M, uint8_t* lab, int* tf,
                                                       const int* __restrict__ succ, PolyArrays P,
                                                       FinalPieces F, Pool pool, LongList D1,
                                                       int rare, Counters* C) {
  pdl_wait();  // the walk's lists, records and sequences
  const long long nd = min(C->n_defer, D1.cap);
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  unsigned st_bad = 0, st_chase = 0;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nd;
       base += (long long)gridDim.x * blockDim.x) {
    const long long d = base + threadIdx.x;
    const long long i = (d < nd) ? D1.poly[d] : -1;
    const int L = (i >= 0) ? P.len[i] : 0;
    const long long off = warp_alloc(&C->pool_alloc, i >= 0 ? L + 2 : 0);
    const long long foff = warp_alloc(&C->fslot_alloc, i >= 0 ? 2 : 0);
    if (i < 0) continue;
    if (off + L + 2 > pool.cap || foff + 2 > F.cap || L < 3) {
      set_error(C, POLYLLA_ERR_LIMIT, 56);
      continue;
    }
    const int tp = P.tip_h[i];
    const int t = P.pbase[i];
    const long long vpos = P.pos[i];
    if ((unsigned)tp >= (unsigned)H || (unsigned)t >= (unsigned)L || vpos < 0 ||
        vpos + L > pool.cap) {
      set_error(C, POLYLLA_ERR_LIMIT, 57);
      continue;
    }
    int* v = pool.v + vpos;
    const int pn = tf_twin(tf[tp]);
    const int b = M.tri[he_next(tp)];
    const int oj = split_edge(tf, tp, H);
    if (oj < 0 || pn >= H) {
      set_error(C, POLYLLA_ERR_LIMIT, 54);
      continue;
    }
    const int tw = tf_twin(tf[oj]);
    const int x = M.tri[he_next(oj)];
    if (tw >= H) {
      set_error(C, POLYLLA_ERR_LIMIT, 54);
      continue;
    }
    set_frontier(lab, tf, oj);
    set_frontier(lab, tf, tw);
    int* out = pool.v + off;
    // the passes over the sequence load kSeqChunk entries at a time, so that
    // their latencies overlap
    int u = -1, nx = 0;
    for (int q0 = 0; q0 < L; q0 += kSeqChunk) {
      int w[kSeqChunk];
#pragma unroll
      for (int k = 0; k < kSeqChunk; ++k) w[k] = (q0 + k < L) ? v[q0 + k] : -1;
#pragma unroll
      for (int k = 0; k < kSeqChunk; ++k) {
        if (w[k] == x) {
          u = q0 + k;
          ++nx;
        }
      }
    }
    bool fast = nx == 1 && !rare;
    int l1 = 0, l2 = 0, r1 = 0, r2 = 0;
    if (fast) {
      const int n1 = (t >= u ? t - u : t - u + L) + 1;  // v[u..t]
      l1 = n1 + 1;
      l2 = L - n1 + 1;
      int m1 = b, c1 = 1, m2 = x, c2 = 1;
      for (int j0 = 0; j0 < L; j0 += kSeqChunk) {  // v[u + j], j = 0..L-1
        int w[kSeqChunk];
#pragma unroll
        for (int k = 0; k < kSeqChunk; ++k) {
          int q = u + j0 + k;
          if (q >= L) q -= L;
          w[k] = (j0 + k < L) ? v[q] : 0;
        }
#pragma unroll
        for (int k = 0; k < kSeqChunk; ++k) {
          const int j = j0 + k, o = w[k];
          if (j >= L) break;
          if (j < n1) {
            if (o < m1) {
              m1 = o;
              c1 = 1;
              r1 = 1 + j;
            } else if (o == m1) {
              ++c1;
            }
          } else if (o < m2) {
            m2 = o;
            c2 = 1;
            r2 = 1 + j - n1;
          } else if (o == m2) {
            ++c2;
          }
        }
      }
      fast = c1 == 1 && c2 == 1;
      if (fast) {
        // piece 1: index k >= 1 is v[u + k - 1]; piece 2: index k >= 1 is v[t + k]
        for (int q0 = 0; q0 < l1 + l2; q0 += kSeqChunk) {
          int w[kSeqChunk];
#pragma unroll
          for (int c = 0; c < kSeqChunk; ++c) {
            const int q = q0 + c;
            int val = 0;
            if (q < l1) {
              int k = r1 + q;
              if (k >= l1) k -= l1;
              int z = u + k - 1;
              if (z >= L) z -= L;
              val = k ? v[z] : b;
            } else if (q < l1 + l2) {
              int k = r2 + (q - l1);
              if (k >= l2) k -= l2;
              int z = t + k;
              if (z >= L) z -= L;
              val = k ? v[z] : x;
            }
            w[c] = val;
          }
#pragma unroll
          for (int c = 0; c < kSeqChunk; ++c)
            if (q0 + c < l1 + l2) out[q0 + c] = w[c];
        }
      }
    }
    if (!fast) {
      ++st_chase;
      long long steps = 0;
      const int g = turn_tf(tf, oj, H, steps, limit);
      if (g < 0 || g == tw || g == pn) {
        set_error(C, POLYLLA_ERR_LIMIT, 54);
        continue;
      }
      int* stage = v;  // the sequence is not read again
      int c1 = g, c2 = pn, n1 = 0, n2 = 0;
      bool a1 = true, a2 = true;
      unsigned long long b1 = vkey(b, oj), b2 = vkey(x, tw);
      for (int it = 0; (a1 || a2) && it < L; ++it) {
        const int o1 = a1 ? M.tri[c1] : 0;
        const int s1 = a1 ? succ[c1] : 0;
        const int o2 = a2 ? M.tri[c2] : 0;
        const int s2 = a2 ? succ[c2] : 0;
        if (a1) {
          stage[n1] = o1;
          const unsigned long long k = vkey(o1, c1);
          ++n1;
          if (k < b1) {
            b1 = k;
            r1 = n1;
          }
          if (c1 == tp) a1 = false;
          else c1 = s1 & kSuccMask;
        }
        if (a2) {
          ++n2;
          stage[L - n2] = o2;
          const unsigned long long k = vkey(o2, c2);
          if (k < b2) {
            b2 = k;
            r2 = n2;
          }
          c2 = s2 & kSuccMask;
          if (c2 == g) a2 = false;
        }
        if ((unsigned)c1 >= (unsigned)H || (unsigned)c2 >= (unsigned)H) break;
      }
      if (a1 || a2 || n1 + n2 != L) {
        ++st_bad;
        continue;
      }
      // piece 1 = [b, stage[0..n1)], piece 2 = [x, stage[L-1], ..., stage[L-n2]]
      l1 = n1 + 1;
      l2 = n2 + 1;
      int k = r1;
      for (int q = 0; q < l1; ++q) {
        out[q] = k ? stage[k - 1] : b;
        if (++k == l1) k = 0;
      }
      k = r2;
      for (int q = 0; q < l2; ++q) {
        out[l1 + q] = k ? stage[L - k] : x;
        if (++k == l2) k = 0;
      }
    }
    F.pos[foff] = off;
    F.len[foff] = l1;
    F.pos[foff + 1] = off + l1;
    F.len[foff + 1] = l2;
    P.pcnt[i] = 2;
    P.pbase[i] = (int)foff;
    P.flen[i] = L + 2;
  }
  if (st_bad) set_error(C, POLYLLA_ERR_LIMIT, 58);
  st_chase = __reduce_add_sync(0xffffffffu, st_chase);
  if ((threadIdx.x & 31) == 0 && st_chase)
    atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_one_chase), (unsigned long long)st_chase);
  // one split per polygon of this list
  if (blockIdx.x == 0 && threadIdx.x == 0 && nd > 0)
    atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_splits), (unsigned long long)nd);
}

// Linked-list reparation of one polygon with several tips per thread.
//
// Nodes 0..L-1 are the polygon's frontier half-edges in boundary order from its
// canonical start (bit 31 set on a barrier-edge tip a->b, i.e. the node followed
// by twin(a->b)); nodes kWalkCap.. are chord half-edges added by splits.  Each
// node keeps its half-edge, its origin vertex and next/prev links, all in shared
// memory, transposed ([node][thread]) so that lanes at the same step hit distinct
// banks.  The pieces form an ordered list of start nodes, as in repair_seq: the
// first piece with a tip is split at its smallest tip b (the destination of tip
// node p) along oj = split_edge(), and is replaced by the piece from oj (b->x)
// followed by the piece from tw = twin(oj) (x->b).  With q the node of turn(oj)
// -- the first frontier half-edge after oj around x -- and qp its predecessor:
//     p -> oj -> q   and   qp -> tw -> next(p),
// which is the boundary that walking the region with the new frontier edge gives.
// A split removes the tip at p, and the one at qp if x was a tip, and creates
// none (x always has a frontier edge of the region besides the chord), so only
// those two flags change.
//
// The node list comes from the walk's records when it left them (the origins
// from the canonical start, and each tip's index and half-edge): the other
// nodes' half-edges stay unknown (kSuccMask) unless needed.  q is the piece's
// only node with origin x; when x occurs more than once in the piece, q is the
// one whose successor's origin is dest(turn(oj)) (a directed edge occurs once in
// a boundary).  A finished piece starts at its smallest vertex; when that vertex
// occurs more than once, the piece's half-edges are found by turning from a node
// whose half-edge is known (a chord), and the smallest (origin, half-edge) key
// decides.  Without records the list is built by chasing the successors.  The
// pieces are written over the records (as long as the polygon and its tip
// records, at least its final length).
constexpr int kRsThreads = 64;
constexpr int kRsNodes = kWalkCap + 2 * kRsMaxSplit;
constexpr int kRsList = kRsMaxSplit + 2;
constexpr size_t kRsSmem =
    (size_t)kRsThreads * (kRsNodes * (2 * sizeof(int) + 2) + kRsList);

__global__ void __launch_bounds__(kRsThreads) k_repair_multi(DevMesh M, uint8_t* lab, int* tf,
                                                             const int* __restrict__ succ,
                                                             PolyArrays P, FinalPieces F,
                                                             Pool pool, LongList Dm, int rare,
                                                             Counters* C) {
  extern __shared__ int rs_smem[];
  int* nh = rs_smem;                                   // [kRsNodes][kRsThreads]
  int* no = nh + kRsNodes * kRsThreads;                // origins
  uint8_t* nx = reinterpret_cast<uint8_t*>(no + kRsNodes * kRsThreads);
  uint8_t* pv = nx + kRsNodes * kRsThreads;
  uint8_t* ps = pv + kRsNodes * kRsThreads;            // [kRsList][kRsThreads]
  const int t = threadIdx.x;
#define NH(j) nh[(j) * kRsThreads + t]
#define NO(j) no[(j) * kRsThreads + t]
#define NX(j) nx[(j) * kRsThreads + t]
#define PV(j) pv[(j) * kRsThreads + t]
#define PS(j) ps[(j) * kRsThreads + t]
  const long long nd = min(C->n_multi, Dm.cap);
  const int H = (int)(3 * M.m);
  const long long limit = 3 * M.m + 3;
  unsigned st_splits = 0, st_seq = 0, st_turn = 0;
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nd;
       base += (long long)gridDim.x * blockDim.x) {
    const long long d = base + t;
    const long long i = (d < nd) ? Dm.poly[d] : -1;
    const int L = (i >= 0) ? P.len[i] : 0;
    const int nt = (i >= 0) ? P.ntip[i] : 0;
    const bool listed = nt <= kRsMaxSplit && L <= kWalkCap;
    const bool rec = i >= 0 && listed && nt >= 2 && L >= 3 && P.pbase[i] == 1;
    const long long off0 = warp_alloc(&C->pool_alloc, i >= 0 && !rec ? L + 2 * nt : 0);
    const long long foff = warp_alloc(&C->fslot_alloc, i >= 0 ? nt + 1 : 0);
    if (i < 0) continue;
    const long long off = rec ? P.pos[i] : off0;
    if (L < 3 || off < 0 || off + L + 2 * nt > pool.cap || foff + nt + 1 > F.cap) {
      set_error(C, POLYLLA_ERR_LIMIT, 56);
      continue;
    }
    int cnt;
    if (!listed) {
      ++st_seq;
      const Cyc first{P.start[i], L, P.tip_h[i], nt, true};
      cnt = repair_seq(M.tri, tf, lab, first, nt + 1, H, limit, F.h + foff, F.pos + foff,
                       F.len + foff, pool.v + off, off, L + 2 * nt);
    } else {
      cnt = -1;
      bool bad = false;
      if (rec) {  // the walk's records
        const int* rv = pool.v + off;
        for (int j0 = 0; j0 < L; j0 += kSeqChunk) {
          int w[kSeqChunk];
#pragma unroll
          for (int k = 0; k < kSeqChunk; ++k) w[k] = (j0 + k < L) ? rv[j0 + k] : 0;
#pragma unroll
          for (int k = 0; k < kSeqChunk; ++k) {
            const int j = j0 + k;
            if (j >= L) break;
            NH(j) = kSuccMask;
            NO(j) = w[k];
            NX(j) = (uint8_t)(j + 1 == L ? 0 : j + 1);
            PV(j) = (uint8_t)(j == 0 ? L - 1 : j - 1);
          }
        }
        for (int k = 0; k < nt; ++k) {
          const int ix = rv[L + 2 * k], hh = rv[L + 2 * k + 1];
          if ((unsigned)ix >= (unsigned)L || (unsigned)hh >= (unsigned)H) {
            bad = true;
            break;
          }
          NH(ix) = hh | kTipFlag;
        }
      } else {  // chase the successors from the canonical start
        int h = P.start[i];
        for (int j = 0; j < L; ++j) {
          if ((unsigned)h >= (unsigned)H) {
            bad = true;
            break;
          }
          const int sg = succ[h];
          NH(j) = h | (sg & kTipFlag);
          NO(j) = M.tri[h];
          NX(j) = (uint8_t)(j + 1 == L ? 0 : j + 1);
          PV(j) = (uint8_t)(j == 0 ? L - 1 : j - 1);
          h = sg & kSuccMask;
        }
        if (h != P.start[i]) bad = true;
      }
      int nn = kWalkCap;  // next chord node
      int count = 1;
      PS(0) = 0;
      long long acc = 0;
      int j = 0;
      while (!bad && j < count) {
        const int s0 = PS(j);
        // the piece: its smallest tip, its smallest vertex and how often it occurs
        int tb = 0x7fffffff, tipn = -1, mo = 0x7fffffff, mn = s0, mc = 0, len = 0;
        int v = s0;
        do {
          const int x = NH(v);
          const int nv = NX(v);
          if (x < 0) {
            const int b = NO(nv);
            if (b < tb) {
              tb = b;
              tipn = v;
            }
          }
          const int o = NO(v);
          if (o < mo) {
            mo = o;
            mn = v;
            mc = 1;
          } else if (o == mo) {
            ++mc;
          }
          ++len;
          v = nv;
        } while (v != s0 && len <= kRsNodes);
        if (len > kRsNodes) {
          bad = true;
          break;
        }
        if (tipn < 0) {  // finished piece: its origins from the canonical start
          if (mc > 1 || rare) {  // the smallest vertex repeats: compare (origin, half-edge)
            ++st_turn;
            int c0 = -1;
            v = s0;
            for (int k = 0; k < len && c0 < 0; ++k, v = NX(v))
              if ((NH(v) & kSuccMask) != kSuccMask) c0 = v;
            if (c0 < 0) {
              bad = true;
              break;
            }
            v = c0;
            for (int k = 0; k + 1 < len && !bad; ++k) {  // unknown half-edges by turning
              const int nv = NX(v);
              if ((NH(nv) & kSuccMask) == kSuccMask) {
                long long steps = 0;
                const int g = turn_tf(tf, NH(v) & kSuccMask, H, steps, limit);
                if (g < 0) bad = true;
                else NH(nv) = g;
              }
              v = nv;
            }
            if (bad) break;
            unsigned long long best = ~0ull;
            v = s0;
            for (int k = 0; k < len; ++k, v = NX(v)) {
              const unsigned long long key = vkey(NO(v), NH(v) & kSuccMask);
              if (key < best) {
                best = key;
                mn = v;
              }
            }
          }
          int* out = pool.v + off + acc;
          v = mn;
          for (int k = 0; k < len; ++k) {
            out[k] = NO(v);
            v = NX(v);
          }
          F.pos[foff + j] = off + acc;
          F.len[foff + j] = len;
          acc += len;
          ++j;
          continue;
        }
        if (count + 1 > nt + 1 || nn + 2 > kRsNodes) {
          bad = true;
          break;
        }
        const int oj = split_edge(tf, NH(tipn) & kSuccMask, H);
        if (oj < 0) {
          bad = true;
          break;
        }
        const int tw = tf_twin(tf[oj]);
        if (tw >= H) {
          bad = true;
          break;
        }
        set_frontier(lab, tf, oj);
        set_frontier(lab, tf, tw);
        const int x = M.tri[tw];  // origin of tw = dest(oj)
        // q: the piece's node leaving x at turn(oj)
        int q = -1, nq = 0;
        v = s0;
        for (int k = 0; k < len; ++k, v = NX(v)) {
          if (NO(v) == x) {
            q = v;
            ++nq;
          }
        }
        if (nq != 1 || rare) {  // x repeats: the node whose edge is x -> dest(turn(oj))
          long long steps = 0;
          const int g = turn_tf(tf, oj, H, steps, limit);
          if (g < 0 || g == tw) {
            bad = true;
            break;
          }
          const int y = M.tri[he_next(g)];
          q = -1;
          v = s0;
          for (int k = 0; k < len; ++k, v = NX(v))
            if (NO(v) == x && NO(NX(v)) == y) q = v;
          if (q < 0) {
            bad = true;
            break;
          }
          if ((NH(q) & kSuccMask) == kSuccMask) NH(q) = g;
        }
        const int qp = PV(q);
        const int pn = NX(tipn);
        const int u = nn, w = nn + 1;
        nn += 2;
        NH(u) = oj;
        NO(u) = tb;
        NH(w) = tw;
        NO(w) = x;
        NX(tipn) = (uint8_t)u;
        PV(u) = (uint8_t)tipn;
        NX(u) = (uint8_t)q;
        PV(q) = (uint8_t)u;
        NX(qp) = (uint8_t)w;
        PV(w) = (uint8_t)qp;
        NX(w) = (uint8_t)pn;
        PV(pn) = (uint8_t)w;
        NH(tipn) &= kSuccMask;
        NH(qp) &= kSuccMask;
        for (int k = count; k > j + 1; --k) PS(k) = PS(k - 1);
        PS(j) = (uint8_t)u;
        PS(j + 1) = (uint8_t)w;
        ++count;
      }
      if (!bad) cnt = count;
    }
#undef NH
#undef NO
#undef NX
#undef PV
#undef PS
    if (cnt < 0) {
      set_error(C, POLYLLA_ERR_LIMIT, 54);
      continue;
    }
    P.pcnt[i] = cnt;
    P.pbase[i] = (int)foff;
    P.flen[i] = L + 2 * (cnt - 1);
    st_splits += cnt - 1;
  }
  st_splits = __reduce_add_sync(0xffffffffu, st_splits);
  st_seq = __reduce_add_sync(0xffffffffu, st_seq);
  if ((threadIdx.x & 31) == 0 && st_splits)
    atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_splits), (unsigned long long)st_splits);
  if ((threadIdx.x & 31) == 0 && st_seq)
    atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_multi_seq), (unsigned long long)st_seq);
  st_turn = __reduce_add_sync(0xffffffffu, st_turn);
  if ((threadIdx.x & 31) == 0 && st_turn)
    atomicAdd(reinterpret_cast<unsigned long long*>(&C->n_multi_turn), (unsigned long long)st_turn);
}

cudaError_t launch_repair_one(const DevMesh& M, uint8_t* lab, int* tf, const int* succ,
                              const PolyArrays& P, const FinalPieces& F, const Pool& pool,
                              const LongList& D1, int rare, Counters* C, int sms,
                              cudaStream_t s, bool pdl) {
  static std::atomic<int> cap{0};
  const int grid = resident_grid(reinterpret_cast<const void*>(k_repair_one), kBlock, 0,
                                 (long long)sms * 8, &cap);
  return launch_chain(k_repair_one, grid, kBlock, 0, s, pdl, M, lab, tf, succ, P, F, pool, D1, rare,
                      C);
}

cudaError_t launch_repair_multi(const DevMesh& M, uint8_t* lab, int* tf, const int* succ,
                                const PolyArrays& P, const FinalPieces& F, const Pool& pool,
                                const LongList& Dm, int rare, Counters* C, int sms,
                                cudaStream_t s) {
  static std::atomic<bool> attr[kMaxDevices];
  const cudaError_t e =
      smem_limit_once(reinterpret_cast<const void*>(k_repair_multi), (int)kRsSmem, attr);
  if (e != cudaSuccess) return e;
  const int per_sm = (int)((220 * 1024) / (kRsSmem + 1024));
  const int grid = sms * (per_sm < 1 ? 1 : per_sm);
  k_repair_multi<<<grid, kRsThreads, kRsSmem, s>>>(M, lab, tf, succ, P, F, pool, Dm, rare, C);
  return cudaGetLastError();
}

}  // namespace polylla
