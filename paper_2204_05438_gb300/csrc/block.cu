// The whole path for one small triangulation in one thread block.
//
// A mesh of at most kBlockMeshMax triangles is meshed by a single block of
// kMeshThreads threads, with its half-edge state in shared memory:
//   LabelMax (Algorithm 2)          per triangle: the longest edge by exact squared
//                                   length, ties to the lower undirected edge id;
//   LabelSeed + LabelFrontier       per triangle: frontier bits, terminal and seed
//                                   flags, and the tf words (twin | frontier);
//   successors                      per frontier half-edge: its boundary successor
//                                   (PolyConstruction's turn, bounded) and whether
//                                   it ends at a barrier-edge tip, 16 bits each;
//   Seed array, compacted           ascending, by a block scan;
//   traversal (Algorithms 3, 4)     one thread per seed follows the successors
//                                   around its region's boundary, noting the
//                                   canonical start and listing the tips;
//   reparation (Algorithm 5)        one warp per polygon with tips: the split edges
//                                   of its tips a lane each, the splits applied in
//                                   increasing tip order by one lane on the
//                                   successor array (split edges made frontier,
//                                   four successors relinked per split), the
//                                   pieces walked a lane per split-edge side and
//                                   listed in the rule's order;
//   CSR output                      one block scan of (pieces, vertices) per seed,
//                                   then every piece written from its canonical
//                                   start along the successors.
// The result is the multi-kernel path's, bit for bit: the same label bytes (after
// reparation), seed list and final CSR in seed order.  One launch replaces the
// label, seed, successor, walk, split and output kernels, the counter memset and
// the side-stream fork and join, whose fixed latency dominates a small mesh.
#include "walk.cuh"

namespace polylla {

namespace {

// Exclusive scan of two values over the kMeshThreads threads of the block; the
// totals go to *ta and *tb.  `sh` holds 2 * 32 entries.  Contains barriers.
__device__ __forceinline__ void mesh_scan2(long long& a, long long& b, long long* ta,
                                           long long* tb, long long* sh) {
  constexpr int kWarps = kMeshThreads / 32;
  static_assert(kMeshThreads % 32 == 0 && kWarps <= 32, "one warp scans the warp totals");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long xa = a, xb = b;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const long long ya = __shfl_up_sync(0xffffffffu, xa, d);
    const long long yb = __shfl_up_sync(0xffffffffu, xb, d);
    if (lane >= d) {
      xa += ya;
      xb += yb;
    }
  }
  if (lane == 31) {
    sh[warp] = xa;
    sh[32 + warp] = xb;
  }
  __syncthreads();
  if (warp == 0) {
    long long wa = lane < kWarps ? sh[lane] : 0, wb = lane < kWarps ? sh[32 + lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long ya = __shfl_up_sync(0xffffffffu, wa, d);
      const long long yb = __shfl_up_sync(0xffffffffu, wb, d);
      if (lane >= d) {
        wa += ya;
        wb += yb;
      }
    }
    sh[lane] = wa;
    sh[32 + lane] = wb;
  }
  __syncthreads();
  const long long ba = warp ? sh[warp - 1] : 0, bb = warp ? sh[31 + warp] : 0;
  *ta = sh[kWarps - 1];
  *tb = sh[32 + kWarps - 1];
  a = ba + xa - a;
  b = bb + xb - b;
  __syncthreads();  // sh may be reused
}

__device__ __forceinline__ long long sqlen(longlong2 p, longlong2 q) {
  const long long dx = q.x - p.x, dy = q.y - p.y;
  return dx * dx + dy * dy;
}

}  // namespace

// Shared memory of a mesh of m triangles (16-bit fields hold half-edge ids and
// lengths, below 3 * kBlockMeshMax < 2^14, and triangle ids):
//   tf, tri            int[3m] each
//   succ               uint16[3m]: boundary successor of each frontier half-edge;
//                      bit 15: its end is a barrier-edge tip; bit 14: a split edge
//   Max, label bytes   uint8[m4] each (m rounded up to 4)
//   per seed           uint16[m] x 3: the seed (until its walk), then the canonical
//                      start or first piece record; output length; output polygons
//                      (bit 15: split)
//   piece records      uint16[2m + 4] x 2: a piece's start half-edge and length
//                      (a polygon with k tips has at most k + 1 pieces, and the
//                      tips of all polygons are distinct vertices: at most m + 2)
//   polygons with tips uint16[m]: their seed indices, for the split pass
//   split scratch      uint16[kSplitScratch]: tip lists and piece trees of the
//                      polygons split in increasing tip order
//   tip list           uint16[kTipList] x 2: (seed, barrier half-edge) of every tip
//                      the walks met
constexpr long long kPieceSlack = 4;
constexpr int kSplitScratch = 8192;
constexpr int kTipList = 4096;
static_assert(3 * kBlockMeshMax < (1 << 14), "half-edge ids and lengths fit 14 bits");
static_assert(2 * kBlockMeshMax + kPieceSlack < (1 << 15) && kSplitScratch < (1 << 16),
              "piece-record and scratch positions fit 16 bits");
size_t mesh_block_smem(long long m) {
  const long long m4 = (m + 3) & ~3ll;
  const long long h2 = (3 * m + 1) & ~1ll;  // uint16 arrays padded to 4 bytes
  const long long m2 = (m + 1) & ~1ll;
  const long long p2 = (2 * m + kPieceSlack + 1) & ~1ll;
  return (size_t)(4 * 6 * m + 2 * h2 + 2 * m4 + 2 * 4 * m2 + 2 * 2 * p2 + 2 * kSplitScratch +
                  2 * 2 * kTipList);
}

namespace {

constexpr unsigned kSuccTip = 0x8000u;
constexpr unsigned kSuccChord = 0x4000u;
constexpr unsigned kSuccVal = 0x3fffu;
constexpr unsigned kSuccBad = 0x3fffu;  // a turn that did not end: every walk through it stops
constexpr unsigned kNone = 0xffffu;
constexpr unsigned kSplitFlag = 0x8000u;

// The frontier half-edge arriving at origin(q) whose turn is q: the inverse of
// turn_tf, rotating the other way around origin(q).  -1 on a bound violation.
__device__ __forceinline__ int rturn_tf(const int* tf, int q, int H, long long limit) {
  int g = he_prev(q);
  long long steps = 0;
  for (int x = tf[g]; x >= 0; x = tf[g]) {
    if (x >= H || ++steps > limit) return -1;
    g = he_prev(x);
  }
  return g;
}

struct Piece {
  int start;  // frontier half-edge with the smallest (origin, id)
  int len;
  int tip;    // barrier half-edge a->b ending at the smallest tip b, or -1
  int ntips;
  bool ok;
};

// One cycle of the successor array from h0: its canonical start, length and
// smallest tip (tips flagged in succ).  With tl_n, every tip's barrier half-edge
// is also appended with `seed` to the list tl_seed / tl_h (kTipList entries; the
// count goes on past a full list, whose polygons are then split without it).
__device__ __forceinline__ Piece chase(const int* tri, const uint16_t* succ, int h0, int H,
                                       int seed = 0, uint16_t* tl_seed = nullptr,
                                       uint16_t* tl_h = nullptr, int* tl_n = nullptr) {
  Piece p{h0, 0, -1, 0, false};
  unsigned long long best = ~0ull;
  int tipv = 0x7fffffff;
  int h = h0;
  do {
    const unsigned sg = succ[h];
    const int g = (int)(sg & kSuccVal);
    const int o = tri[h];
    const unsigned long long key = ((unsigned long long)(unsigned)o << 32) | (unsigned)h;
    if (key < best) best = key;
    if (g >= H) return p;
    if (sg & kSuccTip) {
      ++p.ntips;
      if (tl_n) {
        const int j = atomicAdd(tl_n, 1);
        if (j < kTipList) {
          tl_seed[j] = (uint16_t)seed;
          tl_h[j] = (uint16_t)h;
        }
      }
      const int b = tri[g];  // dest(h) = origin of its successor twin(h)
      if (b < tipv) {
        tipv = b;
        p.tip = h;
      }
    }
    h = g;
    if (++p.len > H) return p;
  } while (h != h0);
  p.start = (int)(best & 0xffffffffu);
  p.ok = true;
  return p;
}

// The split of tip p = a->b (Section 3.2.3) on the successor array along its
// split edge oj = b->x (the middle internal edge of b's fan; tw = x->b), with
// q = turn(oj) and pq the frontier half-edge whose turn was q: p -> oj -> q and
// pq -> tw -> twin(p) afterwards.  A tip flag on pq (x was a tip) drops with the
// rewrite; split-edge marks stay.  Returns oj, or -1 on a bound violation.
__device__ __forceinline__ int apply_split(int* tf, uint8_t* lab, uint16_t* succ, int p, int oj,
                                           int H, long long limit) {
  const int pn = (int)(succ[p] & kSuccVal);  // twin(p) = b->a
  if (oj < 0 || oj >= H || pn >= H) return -1;
  const int tw = tf_twin(tf[oj]);
  if (tw >= H) return -1;
  long long steps = 0;
  const int q = turn_tf(tf, oj, H, steps, limit);
  const int pq = q >= 0 ? rturn_tf(tf, q, H, limit) : -1;  // before oj is frontier
  if (pq < 0) return -1;
  set_frontier(lab, tf, oj);
  set_frontier(lab, tf, tw);
  succ[p] = (uint16_t)oj;
  succ[oj] = (uint16_t)(q | kSuccChord);
  succ[pq] = (uint16_t)(tw | (succ[pq] & kSuccChord));
  succ[tw] = (uint16_t)(pn | kSuccChord);
  return oj;
}

// Reparation of one polygon by one thread, as the sequential rule does it: the
// pieces are listed in order, and the first piece with a tip is split at its
// smallest tip and replaced by the piece through oj followed by the piece
// through tw, until no piece has a tip.  Each split re-walks the piece it splits.
// Pieces go to ps[0 .. cap) / pl[]; returns their number, or -1.
__device__ int repair_by_pieces(const int* tri, int* tf, uint8_t* lab, uint16_t* succ, int start,
                                int cap, int H, long long limit, uint16_t* ps, uint16_t* pl,
                                long long* total) {
  int count = 1, j = 0;
  ps[0] = (uint16_t)start;
  *total = 0;
  while (j < count) {
    const Piece c = chase(tri, succ, ps[j], H);
    if (!c.ok) return -1;
    if (c.tip < 0) {
      ps[j] = (uint16_t)c.start;
      pl[j] = (uint16_t)c.len;
      *total += c.len;
      ++j;
      continue;
    }
    if (count + 1 > cap) return -1;
    const int oj = apply_split(tf, lab, succ, c.tip, split_edge(tf, c.tip, H), H, limit);
    if (oj < 0) return -1;
    for (int r = count; r > j + 1; --r) ps[r] = ps[r - 1];
    ps[j] = (uint16_t)oj;
    ps[j + 1] = (uint16_t)tf_twin(tf[oj]);
    ++count;
  }
  return count;
}

// The same reparation by the 32 lanes of a warp, without re-walking a piece per
// split.  Within one piece the rule splits tips in increasing vertex order; a
// split only changes its own tip's fan and cancels x if x is a tip of the same
// piece, and tips of different pieces never meet, so splitting all of the
// polygon's tips in increasing order (skipping those a smaller tip's split edge
// cancelled) makes the same split edges.  A tip's fan changes only by a split
// edge that ends at the tip, which cancels it, so every tip's split edge is found
// at once from the labels before any split (a lane per tip); the splits are then
// applied in order by one lane.  The pieces are the cycles of the successor
// array: a lane per side of each split edge walks its piece, which is named by
// its smallest split half-edge, and the lane that started there records it.  The
// rule emits the pieces as a tree of splits (the smallest tip's split at the
// root, the piece through oj on the left), rebuilt by joining the two sides of
// each split in decreasing tip order.  The polygon's tips come from the list the
// walks made (tl_seed / tl_h, ntl entries).  Scratch (13 nt + 4 (nt + 1)
// entries at sc): the tips sorted by tip vertex, their split edges (oj, tw), the
// pieces on either side, per side its piece's name, number, canonical start and
// length, per piece its group's parent, head and tail and the next piece.  Every lane of the warp calls it and
// gets the same result: the number of pieces, -1 on an error, or -2 when the
// list lacks some of the polygon's tips (nothing changed yet).
__device__ int repair_by_tips_warp(const int* tri, int* tf, uint8_t* lab, uint16_t* succ, int seed,
                                   int nt, int H, long long limit, const uint16_t* tl_seed,
                                   const uint16_t* tl_h, int ntl, uint16_t* ps, uint16_t* pl,
                                   uint16_t* sc, long long* total) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int cap = nt + 1;
  uint16_t* tp = sc;            // barrier half-edge a->b of each tip, by increasing b
  uint16_t* toj = tp + nt;      // its split edge oj, or kNone if cancelled
  uint16_t* ttw = toj + nt;     // tw
  uint16_t* tpo = ttw + nt;     // the piece through oj, through tw
  uint16_t* tpt = tpo + nt;
  uint16_t* sname = tpt + nt;   // per side 2k + d: its piece's smallest split half-edge
  uint16_t* snum = sname + 2 * nt;  // per side: its piece's number
  uint16_t* sstart = snum + 2 * nt;  // per side: its piece's canonical start, length
  uint16_t* slen = sstart + 2 * nt;
  uint16_t* upar = slen + 2 * nt;   // per piece: group parent, head, tail, next
  uint16_t* uhead = upar + cap;
  uint16_t* utail = uhead + cap;
  uint16_t* unext = utail + cap;
  // the polygon's tips from the walks' list, then sorted by tip vertex (ranks)
  uint16_t* raw = sname;
  int got = 0;
  for (int j0 = 0; j0 < ntl; j0 += 32) {
    const int j = j0 + lane;
    const bool mine = j < ntl && tl_seed[j] == seed;
    const unsigned b = __ballot_sync(full, mine);
    if (mine) {
      const int pos = got + __popc(b & ((1u << lane) - 1u));
      if (pos < nt) raw[pos] = tl_h[j];
    }
    got += __popc(b);
  }
  for (int k = lane; k < nt; k += 32) tp[k] = (uint16_t)kNone;
  __syncwarp();
  if (got != nt) return -2;
  for (int k = lane; k < nt; k += 32) {
    const int h = raw[k];
    const int b = tri[he_next(h)];
    int rank = 0;
    for (int r = 0; r < nt; ++r) rank += tri[he_next(raw[r])] < b;
    tp[rank] = (uint16_t)h;
  }
  __syncwarp();
  // every tip's split edge, from the labels as they are (a tip vertex met twice,
  // on a corrupt mesh, leaves a rank empty)
  for (int k = lane; k < nt; k += 32) {
    const int oj = tp[k] < H ? split_edge(tf, tp[k], H) : -1;
    toj[k] = (uint16_t)(oj < 0 ? kNone : oj);
    tpo[k] = tpt[k] = (uint16_t)kNone;
  }
  __syncwarp();
  // the splits, in increasing tip order, by one lane
  int splits = 0, bad = 0;
  if (lane == 0) {
    for (int k = 0; k < nt; ++k) {
      const int p = tp[k];
      if (p >= H) {
        bad = 1;
        break;
      }
      if (!(succ[p] & kSuccTip)) {  // cancelled by a smaller tip's split edge
        toj[k] = (uint16_t)kNone;
        continue;
      }
      const int oj = toj[k] == kNone ? -1 : (int)toj[k];
      if (apply_split(tf, lab, succ, p, oj, H, limit) < 0) {
        bad = 1;
        break;
      }
      ttw[k] = (uint16_t)tf_twin(tf[oj]);
      ++splits;
    }
  }
  splits = __shfl_sync(full, splits, 0);
  if (__shfl_sync(full, bad, 0) || splits + 1 > cap) return -1;
  __syncwarp();
  // the pieces: a lane per side of each split edge
  const int ns2 = 2 * nt;
  for (int s0 = 0; s0 < ns2; s0 += 32) {
    const int sd = s0 + lane;
    const bool live = sd < ns2 && toj[sd >> 1] != kNone;
    int h0 = 0, name = 0x7fffffff, len = 0;
    if (live) {
      h0 = (sd & 1) ? ttw[sd >> 1] : toj[sd >> 1];
      unsigned long long best = ~0ull;
      int h = h0;
      do {
        const unsigned sg = succ[h];
        const unsigned long long key = ((unsigned long long)(unsigned)tri[h] << 32) | (unsigned)h;
        if (key < best) best = key;
        if ((sg & kSuccChord) && h < name) name = h;
        h = (int)(sg & kSuccVal);
        if (h >= H || ++len > H) {
          name = -1;
          break;
        }
      } while (h != h0);
      sname[sd] = (uint16_t)(name < 0 ? kNone : name);
      sstart[sd] = (uint16_t)(best & 0xffffffffu);
      slen[sd] = (uint16_t)len;
    }
    if (__any_sync(full, live && name < 0)) return -1;
  }
  __syncwarp();
  // the lanes whose side names its piece number the pieces and record them
  int np = 0;
  long long tot = 0;
  for (int s0 = 0; s0 < ns2; s0 += 32) {
    const int sd = s0 + lane;
    const bool live = sd < ns2 && toj[sd >> 1] != kNone;
    const int h0 = live ? ((sd & 1) ? ttw[sd >> 1] : toj[sd >> 1]) : 0;
    const bool owner = live && sname[sd] == h0;
    const unsigned b = __ballot_sync(full, owner);
    if (owner) {
      const int num = np + __popc(b & ((1u << lane) - 1u));
      snum[sd] = (uint16_t)num;
      if (num < cap) {
        ps[num] = sstart[sd];
        pl[num] = slen[sd];
        tot += slen[sd];
        upar[num] = uhead[num] = utail[num] = (uint16_t)num;
        unext[num] = (uint16_t)kNone;
      }
    }
    np += __popc(b);
  }
  if (np != splits + 1) return -1;
  __syncwarp();
  // every side's piece number, from the side that names its piece
  for (int sd = lane; sd < ns2; sd += 32) {
    if (toj[sd >> 1] == kNone) continue;
    const int name = sname[sd];
    int num = kNone;
    for (int r = 0; r < ns2; ++r) {
      if (toj[r >> 1] == kNone) continue;
      if (((r & 1) ? ttw[r >> 1] : toj[r >> 1]) == name) {
        num = snum[r];
        break;
      }
    }
    if (sd & 1) tpt[sd >> 1] = (uint16_t)num;
    else tpo[sd >> 1] = (uint16_t)num;
  }
  __syncwarp();
  // the split tree: the two sides of each split joined, largest tip first
  for (int d = 16; d > 0; d >>= 1) tot += __shfl_xor_sync(full, tot, d);
  *total = tot;
  int ok = 1;
  if (lane == 0) {
    for (int k = nt - 1; k >= 0 && ok; --k) {
      if (toj[k] == kNone) continue;
      int a = tpo[k], b = tpt[k];
      if (a >= np || b >= np) {
        ok = 0;
        break;
      }
      while (upar[a] != a) a = upar[a];  // a forest: each join hangs one root under another
      while (upar[b] != b) b = upar[b];
      if (a == b) {
        ok = 0;
        break;
      }
      unext[utail[a]] = uhead[b];
      utail[a] = utail[b];
      upar[b] = (uint16_t)a;
    }
    if (ok) {
      int r0 = 0;
      while (upar[r0] != r0) r0 = upar[r0];
      // the pieces in that order (the group arrays are free now)
      for (int i = 0; i < np; ++i) {
        upar[i] = ps[i];
        utail[i] = pl[i];
      }
      for (int i = uhead[r0], j = 0; j < np; ++j) {
        if (i == (int)kNone) {
          ok = 0;
          break;
        }
        ps[j] = upar[i];
        pl[j] = utail[i];
        i = unext[i];
      }
    }
  }
  ok = __shfl_sync(full, ok, 0);
  __syncwarp();
  return ok ? np : -1;
}

}  // namespace

__global__ void __launch_bounds__(kMeshThreads, 1) k_mesh_block(DevMesh M, MeshBlockOut O,
                                                                int by_pieces, Counters* C) {
  extern __shared__ __align__(16) int mb_smem[];
  __shared__ long long s_scan[64];
  __shared__ unsigned long long s_stat[4];  // traversal length, tips, polygons with tips, splits
  __shared__ int s_piece, s_scratch, s_ntipped, s_ntl;
  const int tid = threadIdx.x, lane = tid & 31;
  const int m = (int)M.m;
  const long long n = M.n;
  const int H = 3 * m;
  const long long limit = 3 * (long long)m + 3;
  const int m4 = (m + 3) & ~3;
  const int h2 = (H + 1) & ~1, m2 = (m + 1) & ~1;
  const int pcap = 2 * m + (int)kPieceSlack, p2 = (pcap + 1) & ~1;
  int* tf = mb_smem;      // twin, then twin | frontier bit
  int* tri = tf + H;      // origins
  uint16_t* succ = reinterpret_cast<uint16_t*>(tri + H);
  uint8_t* mx = reinterpret_cast<uint8_t*>(succ + h2);  // the Max array
  uint8_t* lab = mx + m4;                               // label bytes (4-byte aligned)
  uint16_t* r_start = reinterpret_cast<uint16_t*>(lab + m4);  // seed, then start / record
  uint16_t* r_len = r_start + m2;  // output length
  uint16_t* r_cnt = r_len + m2;    // output polygons (0 after an error) | kSplitFlag
  uint16_t* tipped = r_cnt + m2;   // seeds whose polygons have tips
  uint16_t* pc_h = tipped + m2;    // piece records: start half-edge
  uint16_t* pc_len = pc_h + p2;    //                length
  uint16_t* scratch = pc_len + p2;
  uint16_t* tl_seed = scratch + kSplitScratch;  // the tips the walks met
  uint16_t* tl_h = tl_seed + kTipList;

  // this launch is the whole run: its counters start at zero, as the label
  // phase's memset leaves them for the multi-kernel path
  static_assert(sizeof(Counters) % sizeof(long long) == 0, "counters clear as 64-bit words");
  constexpr int kWords = (int)(sizeof(Counters) / sizeof(long long));
  if (tid < kWords) reinterpret_cast<long long*>(C)[tid] = 0;
  if (tid < 4) s_stat[tid] = 0;
  if (tid == 0) {
    s_piece = 0;
    s_scratch = 0;
    s_ntipped = 0;
    s_ntl = 0;
  }
  for (int i = tid; i < H; i += kMeshThreads) {
    tri[i] = __ldg(M.tri + i);
    tf[i] = __ldg(M.twin + i);
  }
  __syncthreads();

  // LabelMax
  const longlong2* __restrict__ xy2 = reinterpret_cast<const longlong2*>(M.xy);
  for (int t = tid; t < m; t += kMeshThreads) {
    const int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    int k = 0;
    if ((unsigned)a >= (unsigned long long)n || (unsigned)b >= (unsigned long long)n ||
        (unsigned)c >= (unsigned long long)n) {
      set_error(C, POLYLLA_ERR_RANGE, 140);
    } else {
      const longlong2 pa = __ldg(xy2 + a), pb = __ldg(xy2 + b), pc = __ldg(xy2 + c);
      const long long l[3] = {sqlen(pa, pb), sqlen(pb, pc), sqlen(pc, pa)};
      // longest first; among equal lengths the lower undirected id min(h, twin(h))
      int best_e = 0x7fffffff;
      long long best_l = -1;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int h = 3 * t + e;
        const int tw = tf[h];
        const int eid = (tw >= 0 && tw < h) ? tw : h;
        if (l[e] > best_l || (l[e] == best_l && eid < best_e)) {
          best_l = l[e];
          best_e = eid;
          k = e;
        }
      }
    }
    mx[t] = (uint8_t)k;
  }
  __syncthreads();

  // LabelSeed + LabelFrontier; the tf words replace the twins in place (a thread
  // reads and writes only its own triangle's words; neighbours' Max bytes come
  // from the separate Max array)
  for (int t = tid; t < m; t += kMeshThreads) {
    const int kst = mx[t];
    int g[3], w[3];
    unsigned byte = (unsigned)kst, nbm = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      g[k] = tf[3 * t + k];
      w[k] = g[k];
      if (g[k] >= 0) {
        if (g[k] >= H) {  // a border edge from here on: every tf word is frontier or a twin
          set_error(C, POLYLLA_ERR_RANGE, 141);
          byte |= 1u << (2 + k);
          w[k] = -1;
          continue;
        }
        const int gt = g[k] / 3;
        nbm |= (unsigned)(mx[gt] == g[k] - 3 * gt) << k;
      }
      const bool fr = (g[k] < 0) || (k != kst && !((nbm >> k) & 1u));
      byte |= (unsigned)fr << (2 + k);
      w[k] = (g[k] & 0x7fffffff) | (fr ? (int)0x80000000u : 0);
    }
    const int gs = g[kst];
    const bool terminal = (gs < 0) || ((nbm >> kst) & 1u);
    const bool seed = terminal && (gs < 0 || t < gs / 3);
    byte |= (unsigned)terminal << 6;
    byte |= (unsigned)seed << 5;
    lab[t] = (uint8_t)byte;
#pragma unroll
    for (int k = 0; k < 3; ++k) tf[3 * t + k] = w[k];
  }
  __syncthreads();

  // the successor of every frontier half-edge (PolyConstruction's turn) with the
  // tip flag (the turn comes straight back along the twin), and the seeds in
  // ascending order
  for (int h = tid; h < H; h += kMeshThreads) {
    const int x = tf[h];
    if (x < 0) {
      long long steps = 0;
      const int g = turn_tf(tf, h, H, steps, limit);
      if (g < 0) {
        set_error(C, POLYLLA_ERR_LIMIT, 142);
        succ[h] = (uint16_t)kSuccBad;
      } else {
        succ[h] = (uint16_t)(g | (g == tf_twin(x) ? kSuccTip : 0u));
      }
    }
  }
  const int per_t = (m + kMeshThreads - 1) / kMeshThreads;
  const int t0 = min(tid * per_t, m), t1 = min(t0 + per_t, m);
  long long ns_mine = 0, unused = 0;
  for (int t = t0; t < t1; ++t) ns_mine += (lab[t] >> 5) & 1;
  long long ns = 0, unused_tot = 0;
  long long sb = ns_mine;
  mesh_scan2(sb, unused, &ns, &unused_tot, s_scan);  // barriers: the successors are complete
  for (int t = t0; t < t1; ++t)
    if ((lab[t] >> 5) & 1) {
      r_start[sb] = (uint16_t)t;
      O.seeds[sb] = t;
      ++sb;
    }
  __syncthreads();

  // traversal, one thread per seed: the walk follows succ and lists the tips it
  // meets; a polygon without tips is done, one with tips is listed for the split
  // pass with its canonical start, length and tip count
  unsigned long long st_len = 0, st_tips = 0, st_tp = 0, st_splits = 0;
  for (int i = tid; i < (int)ns; i += kMeshThreads) {
    const int t = r_start[i];
    int cnt = 0, len = 0, head = 0;
    const int e = region_entry_tf(tf, t, H, limit);
    Piece c{0, 0, -1, 0, false};
    if (e < 0) {
      set_error(C, POLYLLA_ERR_LIMIT, 143);
    } else {
      c = chase(tri, succ, e, H, i, tl_seed, tl_h, &s_ntl);
      if (!c.ok) set_error(C, POLYLLA_ERR_LIMIT, 144);
    }
    if (c.ok) {
      st_len += c.len;
      st_tips += c.ntips;
      st_tp += c.ntips > 0;
      head = c.start;
      len = c.len;
      if (c.tip < 0) {
        cnt = 1;
      } else {
        cnt = c.ntips;
        tipped[atomicAdd(&s_ntipped, 1)] = (uint16_t)i;
      }
    }
    r_start[i] = (uint16_t)head;
    r_len[i] = (uint16_t)len;
    r_cnt[i] = (uint16_t)cnt;
  }
  __syncthreads();

  // reparation, one warp per polygon with tips (only its region's half-edges
  // change): the warp splits its tips in increasing order when the scratch and
  // the tip list hold them, else its first lane splits it piece by piece.
  const int warp = tid >> 5;
  const int ntl = min(s_ntl, kTipList);
  for (int k = warp; k < s_ntipped; k += kMeshThreads / 32) {
    const int i = tipped[k];
    const int start = r_start[i];
    const int nt = r_cnt[i];  // the walk's tip count
    const int cap = nt + 1;
    const int need = 13 * nt + 4 * cap;
    int pb = 0, sb0 = 0;
    if (lane == 0) {
      pb = atomicAdd(&s_piece, cap);
      sb0 = by_pieces ? kSplitScratch : atomicAdd(&s_scratch, need);
    }
    pb = __shfl_sync(0xffffffffu, pb, 0);
    sb0 = __shfl_sync(0xffffffffu, sb0, 0);
    long long total = 0;
    int r = -1;
    if (pb + cap <= pcap) {
      r = -2;
      if (sb0 + need <= kSplitScratch)
        r = repair_by_tips_warp(tri, tf, lab, succ, i, nt, H, limit, tl_seed, tl_h, ntl,
                                pc_h + pb, pc_len + pb, scratch + sb0, &total);
      if (r == -2) {
        if (lane == 0)
          r = repair_by_pieces(tri, tf, lab, succ, start, cap, H, limit, pc_h + pb, pc_len + pb,
                               &total);
        r = __shfl_sync(0xffffffffu, r, 0);
        total = __shfl_sync(0xffffffffu, total, 0);
      }
    }
    if (lane == 0) {
      if (r < 1) {
        set_error(C, POLYLLA_ERR_LIMIT, 146);
        r_cnt[i] = 0;
        r_len[i] = 0;
      } else {
        r_start[i] = (uint16_t)pb;
        r_cnt[i] = (uint16_t)(r | (int)kSplitFlag);
        r_len[i] = (uint16_t)total;
        st_splits += r - 1;
      }
    }
  }
  // per-warp sums, one shared atomic per warp and statistic
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    st_len += __shfl_xor_sync(0xffffffffu, st_len, d);
    st_tips += __shfl_xor_sync(0xffffffffu, st_tips, d);
    st_tp += __shfl_xor_sync(0xffffffffu, st_tp, d);
    st_splits += __shfl_xor_sync(0xffffffffu, st_splits, d);
  }
  if (lane == 0 && (st_len | st_tips | st_tp | st_splits)) {
    atomicAdd(&s_stat[0], st_len);
    atomicAdd(&s_stat[1], st_tips);
    atomicAdd(&s_stat[2], st_tp);
    atomicAdd(&s_stat[3], st_splits);
  }
  __syncthreads();

  // the labels after reparation
  for (int t = tid; t < m; t += kMeshThreads) O.lab[t] = lab[t];

  // offsets: each thread takes a contiguous run of seeds
  const int per_s = ((int)ns + kMeshThreads - 1) / kMeshThreads;
  const int i0 = min(tid * per_s, (int)ns), i1 = min(i0 + per_s, (int)ns);
  long long pbase = 0, vbase = 0;
  for (int i = i0; i < i1; ++i) {
    pbase += r_cnt[i] & ~kSplitFlag;
    vbase += r_len[i];
  }
  long long np = 0, nv = 0;
  mesh_scan2(pbase, vbase, &np, &nv, s_scan);
  const bool fits = np <= m && nv <= H;  // at most one polygon per triangle, one vertex per half-edge
  if (!fits && tid == 0) set_error(C, POLYLLA_ERR_LIMIT, 147);
  for (int i = i0; fits && i < i1; ++i) {
    const bool split = r_cnt[i] & kSplitFlag;
    const int cnt = r_cnt[i] & ~kSplitFlag;
    for (int j = 0; j < cnt; ++j) {
      const int pr = r_start[i] + j;
      int h = split ? pc_h[pr] : r_start[i];
      const int len = split ? pc_len[pr] : r_len[i];
      O.off[pbase] = vbase;
      for (int q = 0; q < len; ++q) {
        O.vtx[vbase + q] = tri[h];
        h = (int)(succ[h] & kSuccVal);
        if (h >= H) {
          set_error(C, POLYLLA_ERR_LIMIT, 148);
          break;
        }
      }
      ++pbase;
      vbase += len;
    }
  }
  if (tid == 0) {
    if (fits) O.off[np] = nv;
    C->n_seeds = ns;
    C->n_vtx_trav = (long long)s_stat[0];
    C->n_tips = (long long)s_stat[1];
    C->n_tip_polys = (long long)s_stat[2];
    C->n_splits = (long long)s_stat[3];
    C->n_poly = fits ? np : 0;
    C->n_vtx = fits ? nv : 0;
    C->fslot_alloc = s_piece;
    C->scratch0 = s_scratch;
    C->n_block = ns;
  }
}

cudaError_t launch_mesh_block(const DevMesh& M, const MeshBlockOut& O, int by_pieces,
                              Counters* C, cudaStream_t s) {
  if (M.m < 1 || M.m > kBlockMeshMax) return cudaErrorInvalidValue;
  static std::atomic<bool> attr[kMaxDevices];
  const cudaError_t e = smem_limit_once(reinterpret_cast<const void*>(k_mesh_block),
                                        (int)mesh_block_smem(kBlockMeshMax), attr);
  if (e != cudaSuccess) return e;
  k_mesh_block<<<1, kMeshThreads, mesh_block_smem(M.m), s>>>(M, O, by_pieces, C);
  return cudaGetLastError();
}

}  // namespace polylla
