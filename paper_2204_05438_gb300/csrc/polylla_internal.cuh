// Internal declarations of the GB300 mesher library: device-side data, half-edge
// helpers, block-level scans and the launchers of every kernel.
//
// Mesh layout (Section 2 of the paper, with an explicit half-edge twin): half-edge
// h = 3t+k of triangle t runs from tri[h] to tri[3t+(k+1)%3]; twin[h] is the
// opposite half-edge or -1.  The label byte of triangle t packs the Max array
// (bits 0-1), the frontier flag of each edge (bits 2-4), the Seed array (bit 5)
// and "the longest edge is terminal" (bit 6).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "polylla.h"

namespace polylla {

constexpr int kBlock = 256;                    // threads per block, every kernel
constexpr int kTriPerThread = 4;               // label kernels: 4 triangles = 3 x int4
constexpr int kTriTile = kBlock * kTriPerThread;  // 1024 triangles per seed-count tile
constexpr int kPolyTile = kBlock;              // per-polygon scans: one polygon per thread
constexpr int kScanThreads = 1024;

// Device-resident counters of one pipeline run (zeroed by the label phase).
struct Counters {
  long long n_seeds;
  long long n_vtx_trav;   // total length of the traversal polygons
  long long n_tip_polys;  // polygons with >= 1 barrier-edge tip
  long long n_tips;
  long long n_splits;
  long long n_poly;       // final polygons
  long long n_vtx;        // final total length
  long long piece_alloc;  // final piece slots handed out
  long long n_pairs;      // (tip -> tip) split-edge pairs found by reparation
  long long n_long;       // polygons longer than the walk cap
  long long lm_alloc;     // members of long polygons written
  long long lm2_alloc;    // members of long polygons' pieces written
  long long scratch0;     // scan totals that are not reported
  long long scratch1;
  int error;              // first device error (polylla_status), 0 if none
  int err_info;
};

struct DevMesh {
  const long long* xy;  // 2n
  const int* tri;       // 3m
  const int* twin;      // 3m
  long long n, m;
};

// ----------------------------------------------------------------- half-edges
__device__ __forceinline__ int he_tri(int h) { return h / 3; }
__device__ __forceinline__ int he_next(int h) {
  const int t3 = 3 * (h / 3);
  return (h - t3 == 2) ? t3 : h + 1;
}
__device__ __forceinline__ int he_prev(int h) {
  const int t3 = 3 * (h / 3);
  return (h == t3) ? t3 + 2 : h - 1;
}
// Frontier flag of half-edge h read from the label byte of its triangle.  Plain
// loads: reparation updates label bytes inside the same kernel.
__device__ __forceinline__ bool lab_frontier(const uint8_t* lab, int h) {
  const int t = h / 3;
  return (lab[t] >> (2 + (h - 3 * t))) & 1;
}

__device__ __forceinline__ void set_error(Counters* c, int code, int info) {
  if (atomicCAS(&c->error, 0, code) == 0) c->err_info = info;
}

// ----------------------------------------------------------------- block scans
// Exclusive scan over the kBlock threads of a block; returns the thread's prefix
// and writes the block total.  `sh` needs kBlock/32 entries.  Contains barriers:
// every thread of the block must call it.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total, T* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = (lane < kBlock / 32) ? sh[lane] : T(0);
#pragma unroll
    for (int d = 1; d < kBlock / 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < kBlock / 32) sh[lane] = w;
  }
  __syncthreads();
  const T before = warp ? sh[warp - 1] : T(0);
  *total = sh[kBlock / 32 - 1];
  __syncthreads();
  return before + x - v;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  T tot;
  block_exclusive_scan(v, &tot, sh);
  return tot;
}

// ----------------------------------------------------------------- launchers
// Every launcher enqueues one kernel on `s` and returns the launch error.
cudaError_t launch_validate(const DevMesh& M, Counters* C, int grid, cudaStream_t s);
cudaError_t launch_label_max(const DevMesh& M, uint8_t* lab, Counters* C, int grid,
                             cudaStream_t s);
cudaError_t launch_label_class(const DevMesh& M, uint8_t* lab, long long* tile_sum, int* tf,
                               Counters* C, int grid, cudaStream_t s);
cudaError_t launch_seed_write(const uint8_t* lab, long long m, const long long* tile_off,
                              int* seeds, int grid, cudaStream_t s);
// Exclusive scan of per-tile pairs.  Tile count = ceil(n / tile) with n = *n_dev if
// n_dev, else n_host.  Totals go to *tot0, *tot1.  end_mode 1: end[n] = total0;
// end_mode 2: end[total0] = total1 (index checked against end_cap).
cudaError_t launch_scan_tiles(const long long* tile_sum, long long* tile_off, long long n_host,
                              const long long* n_dev, int tile, long long* tot0, long long* tot1,
                              long long* end, int end_mode, long long end_cap, Counters* C,
                              cudaStream_t s);
// Per traversal polygon (index = seed order), capacity m.
struct PolyArrays {
  int* start;     // canonical start half-edge
  int* len;       // traversal length
  int* ntip;      // barrier-edge tips on the cycle
  int* tipbase;   // first entry of its tips in the tip list
  int* pbase;     // first final piece slot (polygons with tips)
  int* pcnt;      // final pieces
  int* flen;      // total length of the final pieces
  long long* vb;  // output vertex offset
  int* mode;      // 0 walked by one thread; 1 long (one block); 2 long, generic
                  // kernels; 3 long with pieces from the block's reparation
  int* lmbase;    // first entry of a long polygon's members (cycle order)
};

// Polygons longer than the walk cap (capacity m).
struct LongList {
  int* poly;
  long long cap;
};

// Members of long polygons (or of their pieces): half-edge, owner, rank.
struct LongMembers {
  int* h;
  int* poly;  // polygon (traversal) or naming record (pieces)
  int* rank;  // rank in the piece (pieces only)
  long long cap;
};

// Barrier-edge tips (capacity = n vertices), grouped by polygon.
struct TipArrays {
  int* h;              // barrier half-edge a->b ending at the tip b
  int* poly;           // polygon of the tip
  int* o;              // split half-edge b->x, or -1
  int* state;          // 1 processed, 0 cancelled
  int* piece;          // [2 per tip] record naming the piece on each side
  int* rec_start;      // [2 per tip] canonical start of the named piece
  int* rec_len;        // [2 per tip] its length
  int* rec_slot;       // [2 per tip] final piece slot of a naming record
  int* pair_src;       // (tip -> tip) pairs
  int* pair_dst;
  int* cancel_round;
  int* scratch;        // [24 per tip] per-polygon ordering scratch
  long long* vtip;     // [n] (epoch << 32 | tip entry) of the vertex's tip
  long long* chord;    // [3m] (epoch << 32 | record) of split half-edges
  long long cap;
};

// Final pieces of split polygons (capacity m + 1).
struct FinalPieces {
  int* start;
  int* len;
  long long* off;
  int* src;  // 0 written by a walk, 1 from a long polygon's member list
  long long cap;
};

cudaError_t launch_succ(const DevMesh& M, const int* tf, int* succ, Counters* C, int grid,
                        cudaStream_t s);
cudaError_t launch_trav_count(const DevMesh& M, const uint8_t* lab, const int* seeds,
                              const int* succ, const PolyArrays& P, const TipArrays& T,
                              const LongList& Lg, int epoch, Counters* C, int grid,
                              cudaStream_t s);
cudaError_t launch_long_trav(const DevMesh& M, const int* tf, const int* seeds, const int* succ,
                             const PolyArrays& P, const TipArrays& T, const LongList& Lg,
                             const LongMembers& LM, int* visit, int* loc, int epoch, Counters* C,
                             int grid, cudaStream_t s);
cudaError_t launch_long_write(const DevMesh& M, const LongMembers& LM, const PolyArrays& P,
                              const long long* off, int* vtx, int final_pass, Counters* C, int grid,
                              cudaStream_t s);
cudaError_t launch_long_repair(const DevMesh& M, const int* succ, const PolyArrays& P,
                               const TipArrays& T, const LongList& Lg, const LongMembers& LM,
                               const LongMembers& LM2, const FinalPieces& F, int* loc, int epoch,
                               Counters* C, int grid, cudaStream_t s);
cudaError_t launch_long_write_pieces(const DevMesh& M, const LongMembers& LM2, const TipArrays& T,
                                     const FinalPieces& F, int* vtx, Counters* C, int grid,
                                     cudaStream_t s);
cudaError_t launch_len_tiles(const int* len, long long* tile_sum, Counters* C, int grid,
                             cudaStream_t s);
cudaError_t launch_offsets(const int* len, const long long* tile_off, long long* off, Counters* C,
                           int grid, cudaStream_t s);
cudaError_t launch_trav_write(const DevMesh& M, const int* succ, const int* start, const int* len,
                              const int* mode, const long long* off, int* vtx, Counters* C,
                              int grid, cudaStream_t s);
cudaError_t launch_tip_split(const DevMesh& M, const uint8_t* lab, const TipArrays& T, int epoch,
                             Counters* C, int grid, cudaStream_t s);
cudaError_t launch_tip_resolve(const TipArrays& T, Counters* C, cudaStream_t s);
cudaError_t launch_tip_mark(const DevMesh& M, uint8_t* lab, const TipArrays& T, int epoch,
                            Counters* C, int grid, cudaStream_t s);
cudaError_t launch_resucc(const DevMesh& M, const uint8_t* lab, int* succ, const TipArrays& T,
                          Counters* C, int grid, cudaStream_t s);
cudaError_t launch_piece_walk(const DevMesh& M, const int* succ, const PolyArrays& P,
                              const TipArrays& T, int epoch, Counters* C, int grid,
                              cudaStream_t s);
cudaError_t launch_poly_order(const DevMesh& M, const PolyArrays& P, const TipArrays& T,
                              const FinalPieces& F, Counters* C, int grid, cudaStream_t s);
cudaError_t launch_final_tiles(const PolyArrays& P, long long* tile_sum, Counters* C, int grid,
                               cudaStream_t s);
cudaError_t launch_final_offsets(const PolyArrays& P, const FinalPieces& F,
                                 const long long* tile_off, long long* off, long long m,
                                 Counters* C, int grid, cudaStream_t s);
cudaError_t launch_final_write_polys(const DevMesh& M, const int* succ, const PolyArrays& P,
                                     const long long* off_trav, const int* vtx_trav, int* vtx,
                                     Counters* C, int grid, cudaStream_t s);
cudaError_t launch_final_write_pieces(const DevMesh& M, const int* succ, const FinalPieces& F,
                                      int* vtx, Counters* C, int grid, cudaStream_t s);

}  // namespace polylla
