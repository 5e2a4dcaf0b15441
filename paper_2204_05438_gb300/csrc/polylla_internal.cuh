// Internal declarations of the GB300 mesher library: device-side data, half-edge
// helpers, block-level scans and the launchers of every kernel.
//
// Mesh layout (Section 2 of the paper, with an explicit half-edge twin): half-edge
// h = 3t+k of triangle t runs from tri[h] to tri[3t+(k+1)%3]; twin[h] is the
// opposite half-edge or -1.  The label byte of triangle t packs the Max array
// (bits 0-1), the frontier flag of each edge (bits 2-4), the Seed array (bit 5)
// and "the longest edge is terminal" (bit 6).
#pragma once
#include <atomic>

#include <cuda_runtime.h>
#include <stdint.h>

#include "polylla.h"

namespace polylla {

constexpr int kBlock = 256;                    // threads per block, every kernel
constexpr int kTriPerThread = 4;               // label kernels: 4 triangles = 3 x int4
constexpr int kTriTile = kBlock * kTriPerThread;  // 1024 triangles per seed-count tile
// Mesh size limits: half-edge ids fit int32, and the output scan packs a tile
// prefix's polygon count (< 2^29) and vertex count (< 3m + 2n < 2^33) in one word.
constexpr long long kMaxTriangles = 1ll << 29;
constexpr long long kMaxVertices = 1ll << 30;
constexpr int kWalkThreads = 256;  // k_walk block
constexpr int kWalkCap = 64;       // longer polygons go to one thread block each (long.cu)
constexpr int kPolyTile = kBlock;              // per-polygon scans: one polygon per thread
constexpr int kScanThreads = 1024;

// Device-resident counters of one pipeline run (zeroed by the label phase).
struct Counters {
  long long n_seeds;
  long long n_vtx_trav;   // total length of the traversal polygons
  long long n_tip_polys;  // polygons with >= 1 barrier-edge tip
  long long n_tips;
  long long n_splits;
  long long n_poly;       // output polygons
  long long n_vtx;        // output total length
  long long pool_alloc;   // vertex pool entries handed out
  long long fslot_alloc;  // piece records handed out
  long long n_long;       // polygons longer than the walk cap
  long long n_defer;      // polygons with one tip, left to k_repair_one
  long long n_multi;      // polygons with several tips, left to k_repair_multi
  long long ticket;       // tile tickets of the single-pass (look-back) scans
  long long n_long2;      // long polygons handed from the small blocks to the large ones
  long long n_long_seq;   // long regions too large for a block, walked by one thread
  long long n_multi_seq;  // several-tip polygons with more tips than the node list holds
  long long n_one_chase;  // one-tip polygons split by chasing (a repeated vertex)
  long long n_multi_turn; // several-tip pieces with a repeated smallest vertex
  long long seed_ticket;  // tile tickets of the seed compaction's look-back
  long long seed_done;    // its completed look-backs (the last one clears the status)
  long long out_done;     // the output pass's completed look-backs (likewise)
  long long scratch0;     // scan totals that are not reported
  long long scratch1;
  long long n_block;      // polygons meshed by the one-block path (block.cu)
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

// ------------------------------------------------------------ look-back scan
// Single-pass prefix sums over tiles (decoupled look-back): tiles are taken in
// ticket order, so every predecessor of a tile is already running; each tile
// publishes its aggregate, then sums its predecessors' words back to the nearest
// inclusive prefix, then publishes its own.  A status word holds the flag in bits
// 62-63 (0: not yet, 1: aggregate, 2: inclusive prefix) and the value in bits
// 0-61, so one 64-bit store publishes both.  The array starts zeroed.
constexpr unsigned long long kLbAgg = 1ull << 62;
constexpr unsigned long long kLbPre = 2ull << 62;
constexpr unsigned long long kLbVal = (1ull << 62) - 1;
constexpr long long kLbSpin = 1ll << 20;  // polls of one word before giving up

// Warp 0 of the block owning `tile` (aggregate `agg`, the same on every lane):
// returns the exclusive prefix on every lane and publishes the inclusive one.  A
// predecessor that never publishes (it cannot, while the tickets are honoured)
// ends the wait after kLbSpin polls with an error.
__device__ __forceinline__ long long lookback_warp(unsigned long long* status, long long tile,
                                                   long long agg, Counters* C) {
  const int lane = threadIdx.x & 31;
  volatile unsigned long long* vs = status;
  if (lane == 0) vs[tile] = (tile == 0 ? kLbPre : kLbAgg) | (unsigned long long)agg;
  long long excl = 0;
  for (long long j = tile - 1; j >= 0; j -= 32) {
    const long long idx = j - lane;
    unsigned long long w = kLbPre;  // before the first tile: a prefix of 0
    if (idx >= 0) {
      long long spins = 0;
      do {
        w = vs[idx];
      } while ((w >> 62) == 0 && ++spins < kLbSpin);
      if ((w >> 62) == 0) {
        set_error(C, POLYLLA_ERR_LIMIT, 90);
        w = kLbPre;
      }
    }
    const unsigned pm = __ballot_sync(0xffffffffu, (w >> 62) == 2);
    const int last = pm ? __ffs(pm) - 1 : 31;  // lanes 0..last are summed
    long long v = (lane <= last) ? (long long)(w & kLbVal) : 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    excl += v;
    if (pm) break;
  }
  if (lane == 0 && tile > 0) vs[tile] = kLbPre | (unsigned long long)(excl + agg);
  return excl;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  T tot;
  block_exclusive_scan(v, &tot, sh);
  return tot;
}

// ---------------------------------------------- programmatic dependent launch
// The kernels of the chain label_max -> label_class -> seed_write -> succ -> walk
// run back to back on one stream.  A chain kernel may be launched with
// programmatic stream serialization (launch_chain, pdl = true) when the previous
// operation on the stream is a kernel: its launch is then processed while the
// previous kernel finishes, instead of after.  Every chain kernel waits
// (pdl_wait) before it touches anything earlier work wrote -- a no-op when it was
// launched normally -- and lets its own dependent launch (pdl_launch_dependents)
// once all of its blocks have started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_chain(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                         bool pdl, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// ----------------------------------------------------------------- grid sizing
// Grid-stride kernels launch at most one full wave: the blocks that fit on all
// SMs at once (from the occupancy calculator, cached per kernel in *cache),
// and no more than `want` blocks.  A second, partial wave would leave its blocks
// with as many iterations as the first wave's, after it.
// cache: one per launcher (a function-local static), written once with the same
// value by whichever thread launches first
inline int resident_grid(const void* kernel, int threads, size_t smem, long long want,
                         std::atomic<int>* cache) {
  int cached = cache->load(std::memory_order_relaxed);
  if (cached <= 0) {
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
      sms = 1;
    cached = per_sm * sms;
    cache->store(cached, std::memory_order_relaxed);
  }
  long long g = want < cached ? want : cached;
  return (int)(g < 1 ? 1 : g);
}

// A kernel's dynamic shared-memory limit raised to `bytes`, once per device: the
// attribute belongs to the device's context, so a process that launches on several
// devices sets it on each.  done: one flag per device (a launcher's static array).
constexpr int kMaxDevices = 64;
inline cudaError_t smem_limit_once(const void* kernel, int bytes, std::atomic<bool>* done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cached = dev >= 0 && dev < kMaxDevices;
  if (cached && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && cached) done[dev].store(true, std::memory_order_release);
  return e;
}

// ----------------------------------------------------------------- launchers
// Every launcher enqueues one kernel on `s` and returns the launch error.
cudaError_t launch_validate(const DevMesh& M, Counters* C, int grid, cudaStream_t s);
cudaError_t launch_label_max(const DevMesh& M, uint8_t* lab, Counters* C, int grid,
                             cudaStream_t s);
// pdl: launch with programmatic stream serialization (the previous operation on
// the stream is a kernel)
cudaError_t launch_label_class(const DevMesh& M, uint8_t* lab, int* tf, Counters* C, int grid,
                               cudaStream_t s, bool pdl);
// The ascending seed list (and entries, if non-null) and C->n_seeds in one pass:
// look-back over `status` (seed_tiles(m) words, zero at the first use; left zero)
// with tickets from C->seed_ticket (zero at the start).
cudaError_t launch_seed_write(const uint8_t* lab, long long m, unsigned long long* status,
                              int* seeds, int* entry, Counters* C, int grid, cudaStream_t s,
                              bool pdl);
long long seed_tiles(long long m);
// Exclusive scan of per-tile pairs.  Tile count = ceil(n / tile) with n = *n_dev if
// n_dev, else n_host.  Totals go to *tot0, *tot1.  end_mode 1: end[n] = total0;
// end_mode 2: end[total0] = total1 (index checked against end_cap).
// n_bound: an upper bound of the element count (n_host, or *n_dev on the device).
cudaError_t launch_scan_tiles(const long long* tile_sum, long long* tile_off, long long n_host,
                              const long long* n_dev, long long n_bound, int tile,
                              long long* tot0, long long* tot1, long long* end, int end_mode,
                              long long end_cap, Counters* C, cudaStream_t s);
// Per polygon of the traversal (index = seed order), capacity m.
struct PolyArrays {
  int* start;     // canonical start half-edge of the traversal polygon
  int* len;       // traversal length
  int* ntip;      // barrier-edge tips
  int* tip_h;     // barrier half-edge ending at the smallest tip vertex, or -1
  int* pcnt;      // output pieces: 0 = the polygon itself, at pos; else records at pbase
  int* pbase;     // first piece record (of a one-tip polygon, until its split: the
                  // tip's index in the vertex sequence at pos)
  int* flen;      // total output length
  long long* pos; // pool position of an unsplit polygon (or of a one-tip polygon's
                  // sequence, before its split)
};

// Output pieces of split polygons: pool position and length (capacity n + m).
struct FinalPieces {
  long long* pos;
  int* len;
  int* h;  // start half-edges while a polygon is being split
  long long cap;
};

// Vertex pool: every output polygon is written here first, in its final order and
// contiguously (a split polygon's pieces back to back), by the thread or block
// that walked or split it; the CSR is a copy.  Capacity 6m + 2n: the output (at
// most 3m + 2n) and the staging of one-tip polygons (at most 3m).
struct Pool {
  int* v;
  long long cap;
};

// Polygons longer than the walk cap (capacity m).
struct LongList {
  int* poly;
  long long cap;
};

// lab: the label bytes (their frontier bits select the half-edges to turn)
cudaError_t launch_succ(const DevMesh& M, const uint8_t* lab, const int* tf, int* succ,
                        Counters* C, int grid, cudaStream_t s, bool pdl);
// One thread per seed: walk (<= kWalkCap) and, if `repair`, list polygons with
// tips.  cap: polygons longer than cap (16, 32, 48 or 64) go to the long-polygon
// blocks; with tips_to_long > 0 (small meshes), so do polygons with that many tips
// or more when `repair` (the block splits their tips in parallel; one thread would
// split them one after another).
constexpr long long kSmallMeshTri = 1ll << 16;  // meshes below this: tips_to_long = 3
cudaError_t launch_walk(const DevMesh& M, int* tf, const int* entry, const int* succ,
                        const PolyArrays& P, const Pool& pool, const LongList& Lg,
                        const LongList& D1, const LongList& Dm, int cap, int repair,
                        int tips_to_long, Counters* C, int grid, cudaStream_t s, bool pdl);
// One thread per polygon with one tip / with several tips (listed by k_walk).
cudaError_t launch_repair_one(const DevMesh& M, uint8_t* lab, int* tf, const int* succ,
                              const PolyArrays& P, const FinalPieces& F, const Pool& pool,
                              const LongList& D1, int rare, Counters* C, int sms,
                              cudaStream_t s, bool pdl);
cudaError_t launch_repair_multi(const DevMesh& M, uint8_t* lab, int* tf, const int* succ,
                                const PolyArrays& P, const FinalPieces& F, const Pool& pool,
                                const LongList& Dm, int rare, Counters* C, int sms,
                                cudaStream_t s);
// One block per long polygon: gather, rank and, if `repair`, split.  mode 0:
// large blocks only; mode 1: small blocks first, the regions they cannot hold
// (listed in Lg2) then in large blocks; mode 2: the same with one-warp blocks
// first.
cudaError_t launch_long(const DevMesh& M, uint8_t* lab, int* tf, const int* seeds, const int* succ,
                        const PolyArrays& P, const FinalPieces& F, const Pool& pool,
                        const LongList& Lg, const LongList& Lg2, int* loc, int* vstamp, int epoch,
                        int repair, int mode, Counters* C, int sms, cudaStream_t s);
// Output: the CSR offsets (a look-back scan over `status`, one word per
// 1024-polygon tile, zero at the first use and left zero) and the copy; also
// C->n_poly, C->n_vtx and off[n_poly].
// obase (nullable): per traversal polygon, the index of its first output polygon.
cudaError_t launch_final_write(const PolyArrays& P, const FinalPieces& F, const Pool& pool,
                               unsigned long long* status, long long* off, int* vtx,
                               long long* obase, long long m, Counters* C, int grid,
                               cudaStream_t s);
// The twin array from tri (scratch: cnt n, start n + 1, adj 3m pairs; the tile words).
cudaError_t launch_build_twin(const int* tri, long long m, long long n, int* twin, int* cnt,
                              int* start, int2* adj, long long* tile_sum, long long* tile_off,
                              Counters* C, int sms, cudaStream_t s);
// The twin array from a Neighbor array (convention 0: nb[3t+j] across the edge
// opposite vertex j; 1: across the edge from vertex j to vertex j+1).
cudaError_t launch_twin_from_neighbor(const int* tri, const int* nb, long long m, int convention,
                                      int* twin, Counters* C, int grid, cudaStream_t s);
// Trivertex: per vertex the smallest half-edge leaving it, or -1 (clears tv first).
cudaError_t launch_trivertex(const int* tri, long long m, long long n, int* tv, Counters* C,
                             int grid, cudaStream_t s);
// Longest-edge propagation paths: per triangle its region's seed and the path length.
cudaError_t launch_lepp(const DevMesh& M, const uint8_t* lab, int* region, int* depth, Counters* C,
                        int grid, cudaStream_t s);
// The whole path for one mesh of at most kBlockMeshMax triangles in one block of
// kMeshThreads threads (block.cu): labels, seeds, walks, splits and the CSR.
constexpr int kMeshThreads = 1024;
constexpr long long kBlockMeshMax = 4096;
struct MeshBlockOut {
  uint8_t* lab;    // m label bytes (after reparation)
  int* seeds;      // the ascending seed list
  long long* off;  // final CSR offsets (capacity m + 1)
  int* vtx;        // final CSR vertices (capacity 3m)
};
size_t mesh_block_smem(long long m);
// by_pieces != 0: every polygon with tips is split piece by piece (the rule as
// stated), never by the increasing-tip-order form (a test switch)
cudaError_t launch_mesh_block(const DevMesh& M, const MeshBlockOut& O, int by_pieces,
                              Counters* C, cudaStream_t s);
// Batches: union ids from per-mesh local ids, and each mesh's first output polygon.
cudaError_t launch_batch_globalize(const int* tri, const int* twin, const long long* tri_off,
                                   const long long* vtx_off, long long n_meshes, long long m,
                                   int* tri_g, int* twin_g, Counters* C, int grid,
                                   cudaStream_t s);
cudaError_t launch_batch_first(const int* seeds, const long long* tri_off, long long n_meshes,
                               const long long* obase, long long* pfirst, Counters* C,
                               cudaStream_t s);

}  // namespace polylla
