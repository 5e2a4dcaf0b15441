// Label phase (Section 3.2.1, Algorithm 2) and seed compaction.
//
//   k_label_max    LabelMax: per triangle, the index of its longest edge.
//   k_label_class  LabelSeed + LabelFrontier fused: per triangle, the frontier
//                  flag of each edge, "longest edge is terminal" and the seed
//                  flag.
//   k_seed_write   the Seed array compacted in ascending order, the tile
//                  offsets by a decoupled look-back in the same pass.
//
// All three are HBM streams over the triangle arrays (tri / twin: 12 bytes per
// triangle each, read as 3 x int4 per thread of 4 triangles) with gathers of
// vertex coordinates (LabelMax) or of neighbour label bytes (LabelSeed /
// LabelFrontier) that hit L2 on spatially ordered meshes.  Every id read from the
// input is range-checked before it is dereferenced; a bad id sets the handle's
// error word and the element is skipped.
#include "polylla_internal.cuh"

namespace polylla {

// ------------------------------------------------------------------ validation
__global__ void __launch_bounds__(kBlock) k_validate(DevMesh M, Counters* C) {
  const long long n = M.n, m = M.m, H = 3 * m;
  const long long lim = n > H ? n : H;
  const long long kMaxCoord = 1ll << 30;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < lim;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < n) {
      const long long x = M.xy[2 * i], y = M.xy[2 * i + 1];
      if (x < 0 || x >= kMaxCoord || y < 0 || y >= kMaxCoord) set_error(C, POLYLLA_ERR_RANGE, 1);
    }
    if (i < H) {
      const int h = (int)i;
      const int v = M.tri[h];
      const int w = M.tri[he_next(h)];
      if (v < 0 || v >= n) {
        set_error(C, POLYLLA_ERR_RANGE, 2);
      }
      const int g = M.twin[h];
      if (g < -1 || g >= H) {
        set_error(C, POLYLLA_ERR_RANGE, 3);
      } else if (g >= 0) {
        if (g == h || M.twin[g] != h || M.tri[g] != w || M.tri[he_next(g)] != v)
          set_error(C, POLYLLA_ERR_TOPOLOGY, 4);
      }
    }
    if (i < m) {
      const int a = M.tri[3 * i], b = M.tri[3 * i + 1], c = M.tri[3 * i + 2];
      if (a < 0 || a >= n || b < 0 || b >= n || c < 0 || c >= n) continue;  // reported above
      const long long ax = M.xy[2 * a], ay = M.xy[2 * a + 1];
      const long long bx = M.xy[2 * b], by = M.xy[2 * b + 1];
      const long long cx = M.xy[2 * c], cy = M.xy[2 * c + 1];
      if (ax < 0 || ax >= kMaxCoord || ay < 0 || ay >= kMaxCoord || bx < 0 || bx >= kMaxCoord ||
          by < 0 || by >= kMaxCoord || cx < 0 || cx >= kMaxCoord || cy < 0 || cy >= kMaxCoord)
        continue;  // reported by the vertex check
      const long long orient = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
      if (orient <= 0) set_error(C, POLYLLA_ERR_TOPOLOGY, 5);
    }
  }
}

cudaError_t launch_validate(const DevMesh& M, Counters* C, int grid, cudaStream_t s) {
  k_validate<<<grid, kBlock, 0, s>>>(M, C);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ loads
// The 12 ints of triangles 4g .. 4g+3 (3 x int4 when the group is complete;
// scalar loads, zero-filled, for the ragged last group).
__device__ __forceinline__ void load_tri_group(const int* __restrict__ a, long long g, long long m,
                                               int v[12]) {
  const long long t0 = 4 * g;
  if (t0 + 4 <= m) {
    const int4* p = reinterpret_cast<const int4*>(a) + 3 * g;
    const int4 x = __ldg(p), y = __ldg(p + 1), z = __ldg(p + 2);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
    v[8] = z.x; v[9] = z.y; v[10] = z.z; v[11] = z.w;
  } else {
#pragma unroll
    for (int j = 0; j < 12; ++j) v[j] = (3 * t0 + j < 3 * m) ? __ldg(a + 3 * t0 + j) : 0;
  }
}

__device__ __forceinline__ long long sqdist(longlong2 p, longlong2 q) {
  const long long dx = q.x - p.x, dy = q.y - p.y;
  return dx * dx + dy * dy;
}

// ------------------------------------------------------------------ LabelMax
// Longest edge by (exact squared length, then lower undirected id min(h, twin(h))).
// The twin array is read only for triangles whose longest length is tied.
__global__ void __launch_bounds__(kBlock, 6) k_label_max(DevMesh M, uint8_t* __restrict__ lab,
                                                      Counters* C) {
  pdl_launch_dependents();
  const long long m = M.m, n = M.n;
  const long long ngroups = (m + 3) / 4;
  const longlong2* __restrict__ xy2 = reinterpret_cast<const longlong2*>(M.xy);
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ngroups;
       g += (long long)gridDim.x * blockDim.x) {
    int v[12];
    load_tri_group(M.tri, g, m, v);
    unsigned packed = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long t = 4 * g + j;
      if (t >= m) break;
      const int a = v[3 * j], b = v[3 * j + 1], c = v[3 * j + 2];
      if ((unsigned)a >= (unsigned long long)n || (unsigned)b >= (unsigned long long)n ||
          (unsigned)c >= (unsigned long long)n) {
        set_error(C, POLYLLA_ERR_RANGE, 10);
        continue;
      }
      const longlong2 pa = __ldg(xy2 + a), pb = __ldg(xy2 + b), pc = __ldg(xy2 + c);
      const long long l0 = sqdist(pa, pb), l1 = sqdist(pb, pc), l2 = sqdist(pc, pa);
      const long long lmax = max(l0, max(l1, l2));
      const int cnt = (l0 == lmax) + (l1 == lmax) + (l2 == lmax);
      int k;
      if (cnt == 1) {
        k = (l0 == lmax) ? 0 : ((l1 == lmax) ? 1 : 2);
      } else {
        // tie at the maximum: the lower undirected edge id wins
        const long long l[3] = {l0, l1, l2};
        int best_e = 0x7fffffff;
        k = 0;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          if (l[e] != lmax) continue;
          const int h = (int)(3 * t + e);
          const int tw = __ldg(M.twin + h);
          const int eid = (tw >= 0 && tw < h) ? tw : h;
          if (eid < best_e) {
            best_e = eid;
            k = e;
          }
        }
      }
      packed |= (unsigned)k << (8 * j);
    }
    const long long t0 = 4 * g;
    if (t0 + 4 <= m) {
      reinterpret_cast<unsigned*>(lab)[g] = packed;
    } else {
      for (int j = 0; t0 + j < m; ++j) lab[t0 + j] = (uint8_t)(packed >> (8 * j));
    }
  }
}

cudaError_t launch_label_max(const DevMesh& M, uint8_t* lab, Counters* C, int grid,
                             cudaStream_t s) {
  static std::atomic<int> cap{0};
  grid = resident_grid(reinterpret_cast<const void*>(k_label_max), kBlock, 0, grid, &cap);
  k_label_max<<<grid, kBlock, 0, s>>>(M, lab, C);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ LabelSeed + LabelFrontier
// Per triangle t with longest edge k* and twins g_k:
//   frontier(k)  <=> g_k < 0  or  (k != k*  and  edge g_k is not the longest of its triangle)
//   terminal     <=> g_k* < 0 or  edge g_k* is the longest of its triangle
//   seed         <=> terminal and (g_k* < 0 or t < triangle(g_k*))
// Neighbour label bytes are read while other threads rewrite them; only their
// bits 0-1 (the Max array, written by the previous kernel) are used, and every
// rewrite keeps those bits, so any version of a byte gives the same answer.
// When tf is given, also writes tf[h] = twin(h) with bit 31 set iff h is frontier
// (0x7fffffff as the twin of a border half-edge): one load then tells both
// whether a walk stops at h and where it turns next.  No barrier: each thread's 4
// triangles are independent.
__global__ void __launch_bounds__(kBlock, 5) k_label_class(DevMesh M, uint8_t* lab,
                                                           int* __restrict__ tf, Counters* C) {
  pdl_wait();  // the Max array
  pdl_launch_dependents();
  const long long m = M.m;
  const long long H = 3 * m;
  const long long ntiles = (m + kTriTile - 1) / kTriTile;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long g = tile * kBlock + threadIdx.x;  // group of 4 triangles
    const long long t0 = 4 * g;
    if (t0 < m) {
      int tw[12];
      load_tri_group(M.twin, g, m, tw);
      const bool full = t0 + 4 <= m;
      unsigned own = 0;
      if (full) {
        own = *reinterpret_cast<const unsigned*>(lab + t0);
      } else {
        for (int j = 0; t0 + j < m; ++j) own |= (unsigned)lab[t0 + j] << (8 * j);
      }
      unsigned out = 0;
      int tfo[12];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long long t = t0 + j;
        if (t >= m) break;
        const int kst = (own >> (8 * j)) & 3;
        unsigned byte = (unsigned)kst;
        unsigned nbm = 0;  // bit k: edge k is also the longest edge of the neighbour
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int gk = tw[3 * j + k];
          if (gk >= 0) {
            if (gk >= H) {
              set_error(C, POLYLLA_ERR_RANGE, 11);
              continue;
            }
            const int gt = gk / 3;
            const int nb = lab[gt] & 3;
            nbm |= (unsigned)(nb == gk - 3 * gt) << k;
          }
          const bool fr = (gk < 0) || (k != kst && !((nbm >> k) & 1u));
          byte |= (unsigned)fr << (2 + k);
          tfo[3 * j + k] = (gk & 0x7fffffff) | (fr ? (int)0x80000000u : 0);
        }
        const int gs = (kst == 0) ? tw[3 * j] : ((kst == 1) ? tw[3 * j + 1] : tw[3 * j + 2]);
        const bool terminal = (gs < 0) || ((nbm >> kst) & 1u);
        const bool seed = terminal && (gs < 0 || t < gs / 3);
        byte |= (unsigned)terminal << 6;
        byte |= (unsigned)seed << 5;
        out |= byte << (8 * j);
      }
      if (full) {
        *reinterpret_cast<unsigned*>(lab + t0) = out;
        if (tf) {
          int4* q = reinterpret_cast<int4*>(tf) + 3 * g;
          q[0] = make_int4(tfo[0], tfo[1], tfo[2], tfo[3]);
          q[1] = make_int4(tfo[4], tfo[5], tfo[6], tfo[7]);
          q[2] = make_int4(tfo[8], tfo[9], tfo[10], tfo[11]);
        }
      } else {
        for (int j = 0; t0 + j < m; ++j) {
          lab[t0 + j] = (uint8_t)(out >> (8 * j));
          if (tf)
            for (int k = 0; k < 3; ++k) tf[3 * (t0 + j) + k] = tfo[3 * j + k];
        }
      }
    }
  }
}

cudaError_t launch_label_class(const DevMesh& M, uint8_t* lab, int* tf, Counters* C, int grid,
                               cudaStream_t s, bool pdl) {
  static std::atomic<int> cap{0};
  grid = resident_grid(reinterpret_cast<const void*>(k_label_class), kBlock, 0, grid, &cap);
  return launch_chain(k_label_class, grid, kBlock, 0, s, pdl, M, lab, tf, C);
}

// ------------------------------------------------------------------ seed compaction
// The Seed array compacted in ascending order in one pass: a block takes, in
// ticket order, tiles of kSeedSub sub-tiles of kSeedSpan triangles (16 per thread
// and sub-tile, one 16-byte label load each), counts their seeds (label bit 5),
// gets the tile's offset by a decoupled look-back over `status` (one word per
// tile), and writes each sub-tile's seeds -- staged in shared memory -- coalesced.
// The last tile writes the seed count to C->n_seeds.  The status words clean
// themselves: the block that completes the last look-back (C->seed_done counts
// them) clears them and the count, so nothing has to be zeroed before the next
// run; the ticket counter C->seed_ticket starts at zero with the label phase's
// counters.
// With `entry` non-null, also the entry half-edge of each seed's region for the
// walk: 3t + k for the first frontier edge k of t (label bits 2-4), or -1 - t when
// t has no frontier edge (the walk then turns around t's first vertex).
constexpr int kSeedPer = 16;
constexpr int kSeedSpan = kBlock * kSeedPer;   // triangles per sub-tile
constexpr int kSeedSub = 4;                    // sub-tiles per look-back tile
constexpr int kSeedTile = kSeedSub * kSeedSpan;

__global__ void __launch_bounds__(kBlock) k_seed_write(const uint8_t* __restrict__ lab, long long m,
                                                       unsigned long long* status,
                                                       int* __restrict__ seeds,
                                                       int* __restrict__ entry, Counters* C) {
  __shared__ int sw[kSeedSub][kBlock / 32];
  __shared__ int s_seed[kSeedSpan], s_entry[kSeedSpan];
  __shared__ long long s_tile, s_base;
  __shared__ int s_clear;
  pdl_wait();  // the label bytes
  pdl_launch_dependents();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long nbt = (m + kSeedTile - 1) / kSeedTile;
  const bool aligned16 = (reinterpret_cast<uintptr_t>(lab) & 15u) == 0;
  for (;;) {
    if (threadIdx.x == 0)
      s_tile = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&C->seed_ticket), 1ull);
    __syncthreads();
    const long long bt = s_tile;
    if (bt >= nbt) break;
    // this thread's 16 label bytes of each sub-tile (every load issued first)
    unsigned w[kSeedSub][4];
    unsigned smask[kSeedSub];
    int incl[kSeedSub], cnt[kSeedSub];
#pragma unroll
    for (int j = 0; j < kSeedSub; ++j) {
      const long long t0 = ((bt * kSeedSub + j) * kBlock + threadIdx.x) * kSeedPer;
      w[j][0] = w[j][1] = w[j][2] = w[j][3] = 0;
      if (t0 + kSeedPer <= m && aligned16) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(lab) + (t0 / kSeedPer));
        w[j][0] = v.x;
        w[j][1] = v.y;
        w[j][2] = v.z;
        w[j][3] = v.w;
      } else if (t0 + kSeedPer <= m) {  // a caller's label array aligned to 4 bytes only
        const unsigned* l4 = reinterpret_cast<const unsigned*>(lab + t0);
#pragma unroll
        for (int q = 0; q < 4; ++q) w[j][q] = __ldg(l4 + q);
      } else {
        for (int i = 0; i < kSeedPer && t0 + i < m; ++i)
          w[j][i >> 2] |= (unsigned)__ldg(lab + t0 + i) << (8 * (i & 3));
      }
    }
#pragma unroll
    for (int j = 0; j < kSeedSub; ++j) {
      unsigned sm = 0;  // bit i: triangle t0 + i is a seed
#pragma unroll
      for (int i = 0; i < kSeedPer; ++i) sm |= ((w[j][i >> 2] >> (8 * (i & 3) + 5)) & 1u) << i;
      smask[j] = sm;
      cnt[j] = __popc(sm);
      int x = cnt[j];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
      }
      incl[j] = x;
      if (lane == 31) sw[j][warp] = x;
    }
    __syncthreads();
    int sub_total[kSeedSub];
    int total = 0;
#pragma unroll
    for (int j = 0; j < kSeedSub; ++j) {
      int t = 0;
#pragma unroll
      for (int v = 0; v < kBlock / 32; ++v) t += sw[j][v];
      sub_total[j] = t;
      total += t;
    }
    if (warp == 0) {
      const long long ex = lookback_warp(status, bt, total, C);
      if (lane == 0) {
        s_base = ex;
        if (bt == nbt - 1) C->n_seeds = ex + total;
        // the last look-back to complete clears the status words for the next run
        const unsigned long long done =
            atomicAdd(reinterpret_cast<unsigned long long*>(&C->seed_done), 1ull);
        s_clear = done == (unsigned long long)(nbt - 1);
      }
    }
    __syncthreads();
    long long base = s_base;
#pragma unroll
    for (int j = 0; j < kSeedSub; ++j) {
      const long long t0 = ((bt * kSeedSub + j) * kBlock + threadIdx.x) * kSeedPer;
      int before = 0;
#pragma unroll
      for (int v = 0; v < kBlock / 32; ++v) before += (v < warp) ? sw[j][v] : 0;
      int pos = before + incl[j] - cnt[j];
      unsigned sm = smask[j];
      while (sm) {  // the seeds only, in increasing order
        const int i = __ffs(sm) - 1;
        sm &= sm - 1;
        const unsigned wq = i < 8 ? (i < 4 ? w[j][0] : w[j][1]) : (i < 12 ? w[j][2] : w[j][3]);
        const unsigned fr = (wq >> (8 * (i & 3) + 2)) & 7u;
        const int t = (int)(t0 + i);
        s_seed[pos] = t;
        s_entry[pos] = fr ? 3 * t + (__ffs(fr) - 1) : -1 - t;
        ++pos;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < sub_total[j]; k += kBlock) {
        seeds[base + k] = s_seed[k];
        if (entry) entry[base + k] = s_entry[k];
      }
      base += sub_total[j];
      __syncthreads();
    }
    if (s_clear) {  // every tile has finished its look-back
      for (long long q = threadIdx.x; q < nbt; q += kBlock) status[q] = 0;
      if (threadIdx.x == 0) C->seed_done = 0;
    }
    __syncthreads();
  }
}

cudaError_t launch_seed_write(const uint8_t* lab, long long m, unsigned long long* status,
                              int* seeds, int* entry, Counters* C, int grid, cudaStream_t s,
                              bool pdl) {
  static std::atomic<int> cap{0};
  grid = resident_grid(reinterpret_cast<const void*>(k_seed_write), kBlock, 0, grid, &cap);
  return launch_chain(k_seed_write, grid, kBlock, 0, s, pdl, lab, m, status, seeds, entry, C);
}

long long seed_tiles(long long m) { return (m + kSeedTile - 1) / kSeedTile; }

// ------------------------------------------------------------------ tile scan
// Exclusive scan of the per-tile pairs by up to kScanBlocks blocks, none waiting
// for another: block b owns a contiguous range of tiles, first sums every tile
// before its range (coalesced, the carry), then scans its range (thread i a
// contiguous run of it).  The last block writes the totals and the optional CSR
// end marker.  Reads: at most kScanBlocks / 2 times the tile array.
constexpr int kScanBlocks = 64;

__device__ __forceinline__ int scan_blocks_for(long long ntiles) {
  const long long b = (ntiles + kScanThreads - 1) / kScanThreads;
  return (int)(b < 1 ? 1 : (b > kScanBlocks ? kScanBlocks : b));
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(
    const long long* __restrict__ tile_sum, long long* __restrict__ tile_off, long long n_host,
    const long long* n_dev, int tile, long long* tot0, long long* tot1, long long* end,
    int end_mode, long long end_cap, Counters* C) {
  __shared__ long long sh0[32], sh1[32];
  const long long n = n_dev ? *n_dev : n_host;
  const long long ntiles = (n + tile - 1) / tile;
  const int nb = scan_blocks_for(ntiles);
  if ((int)blockIdx.x >= nb) return;
  const long long per_block = (ntiles + nb - 1) / nb;
  const long long b0 = (long long)blockIdx.x * per_block;
  const long long b1 = min(b0 + per_block, ntiles);
  const longlong2* ts = reinterpret_cast<const longlong2*>(tile_sum);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // carry: every tile before this block's range
  long long c0 = 0, c1 = 0;
#pragma unroll 4
  for (long long i = threadIdx.x; i < b0; i += kScanThreads) {
    const longlong2 v = ts[i];
    c0 += v.x;
    c1 += v.y;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    c0 += __shfl_xor_sync(0xffffffffu, c0, d);
    c1 += __shfl_xor_sync(0xffffffffu, c1, d);
  }
  if (lane == 0) {
    sh0[warp] = c0;
    sh1[warp] = c1;
  }
  __syncthreads();
  c0 = 0;
  c1 = 0;
  for (int w = 0; w < kScanThreads / 32; ++w) {
    c0 += sh0[w];
    c1 += sh1[w];
  }
  __syncthreads();
  // this block's range: thread i owns a contiguous run
  const long long per = (b1 - b0 + kScanThreads - 1) / kScanThreads;
  const long long lo = min(b0 + threadIdx.x * per, b1);
  const long long hi = min(lo + per, b1);
  long long s0 = 0, s1 = 0;
#pragma unroll 8
  for (long long i = lo; i < hi; ++i) {
    const longlong2 v = ts[i];
    s0 += v.x;
    s1 += v.y;
  }
  long long x0 = s0, x1 = s1;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    long long y0 = __shfl_up_sync(0xffffffffu, x0, d), y1 = __shfl_up_sync(0xffffffffu, x1, d);
    if (lane >= d) {
      x0 += y0;
      x1 += y1;
    }
  }
  if (lane == 31) {
    sh0[warp] = x0;
    sh1[warp] = x1;
  }
  __syncthreads();
  if (warp == 0) {
    long long w0 = sh0[lane], w1 = sh1[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      long long y0 = __shfl_up_sync(0xffffffffu, w0, d), y1 = __shfl_up_sync(0xffffffffu, w1, d);
      if (lane >= d) {
        w0 += y0;
        w1 += y1;
      }
    }
    sh0[lane] = w0;
    sh1[lane] = w1;
  }
  __syncthreads();
  long long p0 = c0 + (warp ? sh0[warp - 1] : 0) + x0 - s0;
  long long p1 = c1 + (warp ? sh1[warp - 1] : 0) + x1 - s1;
  longlong2* to = reinterpret_cast<longlong2*>(tile_off);
#pragma unroll 8
  for (long long i = lo; i < hi; ++i) {
    const longlong2 v = ts[i];
    to[i] = make_longlong2(p0, p1);
    p0 += v.x;
    p1 += v.y;
  }
  if ((int)blockIdx.x == nb - 1 && threadIdx.x == kScanThreads - 1) {
    const long long t0 = c0 + sh0[31], t1 = c1 + sh1[31];
    if (tot0) *tot0 = t0;
    if (tot1) *tot1 = t1;
    const long long at = (end_mode == 1) ? n : t0;
    const long long val = (end_mode == 1) ? t0 : t1;
    if (end_mode != 0) {
      if (at >= 0 && at <= end_cap) {
        end[at] = val;
      } else {
        set_error(C, POLYLLA_ERR_LIMIT, 40);
      }
    }
  }
}

cudaError_t launch_scan_tiles(const long long* tile_sum, long long* tile_off, long long n_host,
                              const long long* n_dev, long long n_bound, int tile,
                              long long* tot0, long long* tot1, long long* end, int end_mode,
                              long long end_cap, Counters* C, cudaStream_t s) {
  const long long tiles = (n_bound + tile - 1) / tile;
  long long b = (tiles + kScanThreads - 1) / kScanThreads;
  if (b < 1) b = 1;
  if (b > kScanBlocks) b = kScanBlocks;
  k_scan_tiles<<<(int)b, kScanThreads, 0, s>>>(tile_sum, tile_off, n_host, n_dev, tile, tot0, tot1,
                                               end, end_mode, end_cap, C);
  return cudaGetLastError();
}

}  // namespace polylla
