// C ABI of the mesher (declared in include/polylla.h): handle, buffers, phase
// sequencing, getters, host-buffer entry point and per-kernel timing.
//
// Every buffer is allocated once by polylla_mesh_create (sizes are bounded by the
// triangle count m: at most m seeds and polygons, at most 3m polygon vertices, at
// most m reparation pieces), so no phase allocates, synchronises or copies to the
// host; phases only enqueue kernels on the caller's stream.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "polylla_internal.cuh"

using namespace polylla;

namespace polylla {
int64_t host_repair(int64_t n, int64_t m, const int32_t* tri, const int32_t* twin, uint8_t* lab,
                    const int64_t* off, const int32_t* vtx, int64_t n_poly, int64_t* out_off,
                    int32_t* out_vtx, int64_t* out_np, int64_t* out_nv);
}

namespace {

enum Phase { kCreated = 0, kLabeled, kSeeded, kTraversed, kRepaired };

struct TimingRec {
  const char* name;
  cudaEvent_t a, b;
};

}  // namespace

struct polylla_mesh {
  DevMesh M;
  long long n_cap = 0, m_cap = 0;  // sizes the buffers were allocated for
  int device = 0;
  int sms = 148;
  bool owns_inputs = false;
  bool owns_twin = false;      // twin built on the device (handle-owned)
  int* tw_cnt = nullptr;       // twin construction scratch: per-vertex counts,
  int* tw_start = nullptr;     // first slots (n + 1),
  int2* tw_adj = nullptr;      // outgoing half-edges with their destinations (3m)
  int phase = kCreated;
  int latest_csr = -1;  // 0: traversal CSR, 1: final CSR
  cudaStream_t last_stream = nullptr;

  uint8_t* lab = nullptr;
  int* seeds = nullptr;
  int* entry = nullptr;   // per seed: entry half-edge of its region (or -1 - t)
  int* lepp_region = nullptr;  // per triangle: seed of its longest-edge path's end
  int* lepp_depth = nullptr;   // per triangle: links of that path
  int* trivertex = nullptr;    // per vertex: smallest half-edge leaving it, or -1
  bool trivertex_valid = false;
  int* succ = nullptr;    // per frontier half-edge: boundary successor | tip flag
  int* tf = nullptr;      // twin | frontier bit, per half-edge (written by the label phase)
  int* loc = nullptr;     // per half-edge: member index inside a long-polygon block
  int* vstamp = nullptr;  // per vertex: "endpoint of a split edge" stamp
  LongList Lg{};
  LongList Dl{};          // polygons with one tip
  PolyArrays P{};
  FinalPieces F{};
  Pool pool{};
  LongList Dm{};          // polygons with several tips
  LongList Lg2{};         // long polygons the small blocks hand to the large ones
  int epoch = 0;
  long long* tile_sum = nullptr;  // twin construction: per-tile counts and offsets
  long long* tile_off = nullptr;
  unsigned long long* seed_status = nullptr;  // look-back words of the seed pass
  unsigned long long* out_status = nullptr;   // look-back words of the output pass
  long long* off_trav = nullptr;
  int* vtx_trav = nullptr;
  long long* off_final = nullptr;
  int* vtx_final = nullptr;
  Counters* C = nullptr;

  // the three kernels after the walk touch disjoint polygons: fork to two side
  // streams and join back (sequential in timing mode, for per-kernel times)
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};

  // schedule: the walk's thread-per-seed cap and the long-polygon mode
  int walk_cap = kWalkCap;
  bool overlap = true;  // the kernels after the walk on side streams
  bool rare_paths = false;  // polylla_debug_rare_paths
  int long_mode = 0;
  // polylla_run meshes a mesh of at most this many triangles in one thread block
  long long block_max = kBlockMeshMax;
  int block_by_pieces = 0;  // polylla_debug_split_by_pieces
  bool lepp_valid = false;
  long long* obase = nullptr;  // batches: output index of each traversal polygon

  // host copies for polylla_repair_host (sized on first use)
  std::vector<int32_t> h_tri, h_twin, h_vtx, h_out_vtx;
  std::vector<uint8_t> h_lab;
  std::vector<int64_t> h_off, h_out_off;

  bool timing = false;
  std::vector<TimingRec> recs;
  std::vector<cudaEvent_t> event_pool;
  long long launches = 0;
};

namespace {

polylla_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return POLYLLA_OK;
  if (e == cudaErrorMemoryAllocation) return POLYLLA_ERR_OOM;
  return POLYLLA_ERR_CUDA;
}

cudaEvent_t take_event(polylla_mesh* h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch one kernel through `fn`, bracketed by events when timing is on.
template <class F>
polylla_status launch(polylla_mesh* h, const char* name, cudaStream_t s, F fn) {
  TimingRec r{name, nullptr, nullptr};
  if (h->timing) {
    r.a = take_event(h);
    r.b = take_event(h);
    if (r.a) cudaEventRecord(r.a, s);
  }
  cudaError_t e = fn();
  ++h->launches;
  if (h->timing) {
    if (r.b) cudaEventRecord(r.b, s);
    if (r.a && r.b) h->recs.push_back(r);
  }
  return cuda_status(e);
}

#define POLY_TRY(expr)                        \
  do {                                        \
    polylla_status _st = (expr);              \
    if (_st != POLYLLA_OK) return _st;        \
  } while (0)

int grid_for(const polylla_mesh* h, long long units, int per_block) {
  long long blocks = (units + per_block - 1) / per_block;
  long long cap = (long long)h->sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

// failure injection (polylla_debug_fail_alloc): allocations left before the one
// that fails; 0 when off
std::atomic<long long> g_fail_alloc{0};

template <class T>
cudaError_t dalloc(T** p, long long count) {
  if (g_fail_alloc.load(std::memory_order_relaxed) > 0 && g_fail_alloc.fetch_sub(1) == 1) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  if (count < 1) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (size_t)count);
}

// NVTX range over one phase (seen by profilers; a no-op without one)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

void free_all(polylla_mesh* h) {
  void* ptrs[] = {h->lab,      h->seeds,     h->succ,      h->tf,
                  h->loc,      h->vstamp,    h->Lg.poly,   h->P.start,    h->P.len,
                  h->P.ntip,   h->P.pcnt,    h->P.pbase,    h->P.flen,
                  h->P.pos,    h->F.pos,     h->F.len,     h->F.h,        h->pool.v,
                  h->tile_sum, h->tile_off,  h->off_trav,  h->vtx_trav,   h->off_final,
                  h->seed_status, h->out_status,
                  h->vtx_final, h->C,         h->Dl.poly,   h->P.tip_h,
                  h->Dm.poly,   h->entry,     h->Lg2.poly,
                  h->lepp_region, h->lepp_depth, h->trivertex};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->owns_twin && !h->owns_inputs) cudaFree(const_cast<int*>(h->M.twin));
  for (void* p : {(void*)h->tw_cnt, (void*)h->tw_start, (void*)h->tw_adj})
    if (p) cudaFree(p);
  if (h->owns_inputs) {
    cudaFree(const_cast<long long*>(h->M.xy));
    cudaFree(const_cast<int*>(h->M.tri));
    cudaFree(const_cast<int*>(h->M.twin));
  }
  for (auto& r : h->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : h->event_pool) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k) {
    if (h->side[k]) cudaStreamDestroy(h->side[k]);
    if (h->join[k]) cudaEventDestroy(h->join[k]);
  }
  if (h->fork) cudaEventDestroy(h->fork);
}

// Device bytes of a handle's derived buffers for n vertices and m triangles (as
// allocated by alloc_derived; each allocation rounded up to 512 bytes).
long long derived_bytes(long long n, long long m);

polylla_status alloc_derived(polylla_mesh* h) {
  h->n_cap = h->M.n;
  h->m_cap = h->M.m;
  const long long m = h->M.m, n = h->M.n;
  for (int k = 0; k < 2; ++k) {
    if (cudaStreamCreateWithFlags(&h->side[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->join[k], cudaEventDisableTiming) != cudaSuccess)
      return POLYLLA_ERR_CUDA;
  }
  if (cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess)
    return POLYLLA_ERR_CUDA;
  const long long ntiles_tri = (m + kTriTile - 1) / kTriTile;
  const long long ntiles_poly = (m + kPolyTile - 1) / kPolyTile;
  const long long ntiles = ntiles_tri > ntiles_poly ? ntiles_tri : ntiles_poly;
  // bounds: at most m polygons and 3m polygon vertices after reparation; the pool
  // also holds the up to 2 extra slots per tip a splitting thread reserves, and
  // there is at most one piece record per tip plus one per polygon
  h->Lg.cap = m;
  h->Dl.cap = m;
  h->F.cap = n + m;
  h->pool.cap = 6 * m + 2 * n;
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, cnt) \
  if (e == cudaSuccess) e = dalloc(&(ptr), (cnt))
  ALLOC(h->lab, m + 4);
  ALLOC(h->seeds, m);
  ALLOC(h->succ, 3 * m);
  ALLOC(h->entry, m);
  ALLOC(h->lepp_region, m);
  ALLOC(h->lepp_depth, m);
  ALLOC(h->trivertex, n);
  ALLOC(h->tf, 3 * m);
  ALLOC(h->loc, 3 * m);
  ALLOC(h->vstamp, n);
  ALLOC(h->Lg.poly, m);
  ALLOC(h->Dl.poly, m);
  ALLOC(h->P.tip_h, m);
  h->Dm.cap = m;
  ALLOC(h->Dm.poly, m);
  h->Lg2.cap = m;
  ALLOC(h->Lg2.poly, m);
  ALLOC(h->P.start, m);
  ALLOC(h->P.len, m);
  ALLOC(h->P.ntip, m);
  ALLOC(h->P.pcnt, m);
  ALLOC(h->P.pbase, m);
  ALLOC(h->P.flen, m);
  ALLOC(h->P.pos, m);
  ALLOC(h->F.pos, h->F.cap);
  ALLOC(h->F.len, h->F.cap);
  ALLOC(h->F.h, h->F.cap);
  ALLOC(h->pool.v, h->pool.cap);
  ALLOC(h->tile_sum, 2 * ntiles);
  ALLOC(h->tile_off, 2 * ntiles);
  ALLOC(h->seed_status, seed_tiles(m) + 1);
  ALLOC(h->out_status, ntiles + 1);
  ALLOC(h->off_trav, m + 1);
  ALLOC(h->vtx_trav, 3 * m);
  ALLOC(h->off_final, m + 1);
  ALLOC(h->vtx_final, 3 * m);
  ALLOC(h->C, 1);
#undef ALLOC
  // stamped arrays start empty (run stamps are never 0)
  if (e == cudaSuccess) e = cudaMemset(h->vstamp, 0, sizeof(int) * (size_t)n);
  // look-back words start zero (each pass leaves them zero)
  if (e == cudaSuccess)
    e = cudaMemset(h->seed_status, 0, sizeof(unsigned long long) * (size_t)(seed_tiles(m) + 1));
  if (e == cudaSuccess)
    e = cudaMemset(h->out_status, 0, sizeof(unsigned long long) * (size_t)(ntiles + 1));
  if (e == cudaSuccess) e = cudaMemset(h->C, 0, sizeof(Counters));
  return cuda_status(e);
}

long long derived_bytes(long long n, long long m) {
  polylla_mesh c;  // only for the member types and capacities
  const long long ntiles_tri = (m + kTriTile - 1) / kTriTile;
  const long long ntiles_poly = (m + kPolyTile - 1) / kPolyTile;
  const long long ntiles = ntiles_tri > ntiles_poly ? ntiles_tri : ntiles_poly;
  c.F.cap = n + m;
  c.pool.cap = 6 * m + 2 * n;
  long long bytes = 0;
#define COUNT(ptr, cnt) \
  bytes += ((long long)sizeof(*(ptr)) * ((cnt) < 1 ? 1 : (long long)(cnt)) + 511) / 512 * 512
  COUNT(c.lab, m + 4);
  COUNT(c.seeds, m);
  COUNT(c.succ, 3 * m);
  COUNT(c.entry, m);
  COUNT(c.tf, 3 * m);
  COUNT(c.loc, 3 * m);
  COUNT(c.vstamp, n);
  COUNT(c.Lg.poly, m);
  COUNT(c.Dl.poly, m);
  COUNT(c.P.tip_h, m);
  c.Dm.cap = m;
  COUNT(c.Dm.poly, m);
  COUNT(c.Lg2.poly, m);
  COUNT(c.lepp_region, m);
  COUNT(c.lepp_depth, m);
  COUNT(c.trivertex, n);
  COUNT(c.P.start, m);
  COUNT(c.P.len, m);
  COUNT(c.P.ntip, m);
  COUNT(c.P.pcnt, m);
  COUNT(c.P.pbase, m);
  COUNT(c.P.flen, m);
  COUNT(c.P.pos, m);
  COUNT(c.F.pos, c.F.cap);
  COUNT(c.F.len, c.F.cap);
  COUNT(c.F.h, c.F.cap);
  COUNT(c.pool.v, c.pool.cap);
  COUNT(c.tile_sum, 2 * ntiles);
  COUNT(c.tile_off, 2 * ntiles);
  COUNT(c.seed_status, seed_tiles(m) + 1);
  COUNT(c.out_status, ntiles + 1);
  COUNT(c.off_trav, m + 1);
  COUNT(c.vtx_trav, 3 * m);
  COUNT(c.off_final, m + 1);
  COUNT(c.vtx_final, 3 * m);
  COUNT(c.C, 1);
#undef COUNT
  return bytes;
}

polylla_status read_counters(polylla_mesh* h, Counters* out) {
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  if (e == cudaSuccess) e = cudaMemcpy(out, h->C, sizeof(Counters), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  if (out->error) return (polylla_status)out->error;
  return POLYLLA_OK;
}

polylla_status check_handle(polylla_mesh* h) {
  if (!h) return POLYLLA_ERR_INVALID_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return POLYLLA_ERR_CUDA;
  if (cur != h->device && cudaSetDevice(h->device) != cudaSuccess) return POLYLLA_ERR_CUDA;
  return POLYLLA_OK;
}

// ---------------------------------------------------------------- phases
polylla_status do_label(polylla_mesh* h, cudaStream_t s) {
  const Range range("polylla label");
  const DevMesh& M = h->M;
  if (h->epoch >= 0x3ffffff0) {  // stamps: wrap around once in 2^30 runs
    POLY_TRY(cuda_status(cudaMemsetAsync(h->vstamp, 0, sizeof(int) * (size_t)M.n, s)));
    h->epoch = 0;
  }
  ++h->epoch;
  POLY_TRY(cuda_status(cudaMemsetAsync(h->C, 0, sizeof(Counters), s)));
  const int g1 = grid_for(h, (M.m + 3) / 4, kBlock);
  POLY_TRY(launch(h, "label_max", s, [&] { return launch_label_max(M, h->lab, h->C, g1, s); }));
  const int g2 = grid_for(h, M.m, kTriTile);
  POLY_TRY(launch(h, "label_class", s, [&] {
    return launch_label_class(M, h->lab, h->tf, h->C, g2, s, !h->timing);
  }));
  h->phase = kLabeled;
  h->lepp_valid = false;
  h->latest_csr = -1;
  return POLYLLA_OK;
}

polylla_status do_seeds(polylla_mesh* h, cudaStream_t s) {
  const Range range("polylla seeds");
  const DevMesh& M = h->M;
  const int g = grid_for(h, M.m, 16 * kTriTile);
  POLY_TRY(launch(h, "seed_write", s, [&] {
    return launch_seed_write(h->lab, M.m, h->seed_status, h->seeds, h->entry, h->C, g, s,
                             !h->timing && h->phase == kLabeled);
  }));
  h->phase = kSeeded;
  return POLYLLA_OK;
}

// Walk every polygon (one thread, or one block for a long one) into the pool,
// splitting those with tips when `repair`; then the CSR.
polylla_status do_polygons(polylla_mesh* h, cudaStream_t s, int repair, long long* off, int* vtx) {
  const Range range(repair ? "polylla repair" : "polylla traverse");
  const DevMesh& M = h->M;
  // counters of this pass start at zero: right after the seeds they are (the label
  // phase cleared them); after a traversal pass they are cleared here
  // the kernel chain continues without a gap where the previous operation on the
  // stream is its predecessor kernel: succ right after the seeds, the walk right
  // after succ (not in timing mode, where events sit between the kernels)
  const bool pdl = !h->timing && h->phase == kSeeded;
  const bool succ_runs = repair == 0 || h->phase < kTraversed;
  if (h->phase != kSeeded) {
    const size_t first = offsetof(Counters, n_vtx_trav);
    const size_t last = offsetof(Counters, seed_ticket);
    POLY_TRY(cuda_status(cudaMemsetAsync(reinterpret_cast<char*>(h->C) + first, 0, last - first, s)));
  }
  if (succ_runs) {
    const int gt = grid_for(h, M.m, kBlock);
    POLY_TRY(launch(h, "succ", s, [&] {
      return launch_succ(M, h->lab, h->tf, h->succ, h->C, gt, s, pdl);
    }));
  }
  const int gw = grid_for(h, M.m, 4 * 256);
  POLY_TRY(launch(h, "walk", s, [&] {
    return launch_walk(M, h->tf, h->entry, h->succ, h->P, h->pool, h->Lg, h->Dl, h->Dm,
                       h->walk_cap, repair, M.m < kSmallMeshTri ? 3 : 0, h->C, gw, s,
                       !h->timing && succ_runs);
  }));
  // repair_one (this stream), repair_multi and long (side streams) at once
  const bool fork = !h->timing && h->overlap;
  cudaStream_t s1 = s, s2 = s;
  if (fork) {
    POLY_TRY(cuda_status(cudaEventRecord(h->fork, s)));
    for (int k = 0; k < 2; ++k)
      POLY_TRY(cuda_status(cudaStreamWaitEvent(h->side[k], h->fork, 0)));
    s1 = h->side[0];
    s2 = h->side[1];
  }
  POLY_TRY(launch(h, "long", s1, [&] {
    return launch_long(M, h->lab, h->tf, h->seeds, h->succ, h->P, h->F, h->pool, h->Lg, h->Lg2,
                       h->loc, h->vstamp, 2 * h->epoch + repair, repair, h->long_mode, h->C,
                       h->sms, s1);
  }));
  if (repair) {
    POLY_TRY(launch(h, "repair_multi", s2, [&] {
      return launch_repair_multi(M, h->lab, h->tf, h->succ, h->P, h->F, h->pool, h->Dm,
                                 h->rare_paths, h->C,
                                 h->sms, s2);
    }));
    POLY_TRY(launch(h, "repair_one", s, [&] {
      return launch_repair_one(M, h->lab, h->tf, h->succ, h->P, h->F, h->pool, h->Dl,
                               h->rare_paths, h->C, h->sms, s, !h->timing);
    }));
  }
  if (fork) {
    for (int k = 0; k < 2; ++k) {
      POLY_TRY(cuda_status(cudaEventRecord(h->join[k], h->side[k])));
      POLY_TRY(cuda_status(cudaStreamWaitEvent(s, h->join[k], 0)));
    }
  }
  // one pass: offsets by look-back (the status words are zero; the ticket counter
  // starts at zero with the pass's counters)
  const int gt = grid_for(h, M.m, kPolyTile);
  return launch(h, "out_write", s, [&] {
    return launch_final_write(h->P, h->F, h->pool, h->out_status, off, vtx, h->obase, M.m, h->C,
                              gt, s);
  });
}

// The whole path in one launch of one thread block (small meshes).
polylla_status do_block(polylla_mesh* h, cudaStream_t s) {
  const Range range("polylla run (one block)");
  const MeshBlockOut O{h->lab, h->seeds, h->off_final, h->vtx_final};
  POLY_TRY(launch(h, "mesh_block", s, [&] {
    return launch_mesh_block(h->M, O, h->block_by_pieces, h->C, s);
  }));
  h->phase = kRepaired;
  h->latest_csr = 1;
  h->lepp_valid = false;
  return POLYLLA_OK;
}

polylla_status do_traverse(polylla_mesh* h, cudaStream_t s) {
  POLY_TRY(do_polygons(h, s, 0, h->off_trav, h->vtx_trav));
  h->phase = kTraversed;
  h->latest_csr = 0;
  return POLYLLA_OK;
}

polylla_status do_repair(polylla_mesh* h, cudaStream_t s) {
  POLY_TRY(do_polygons(h, s, 1, h->off_final, h->vtx_final));
  h->phase = kRepaired;
  h->latest_csr = 1;
  return POLYLLA_OK;
}

// Scratch of the twin construction, for handles that may build their twin.
polylla_status alloc_twin_scratch(polylla_mesh* h) {
  const long long m = h->M.m, n = h->M.n;
  const long long have = (m + kPolyTile - 1) / kPolyTile;  // tile words allocated
  if ((n + kTriTile - 1) / kTriTile > have) return POLYLLA_ERR_INVALID_ARG;
  cudaError_t e = dalloc(&h->tw_cnt, n);
  if (e == cudaSuccess) e = dalloc(&h->tw_start, n + 1);
  if (e == cudaSuccess) e = dalloc(&h->tw_adj, 3 * m);
  return cuda_status(e);
}

polylla_status do_build_twin(polylla_mesh* h, cudaStream_t s) {
  if (!h->tw_adj || !(h->owns_twin || h->owns_inputs)) return POLYLLA_ERR_STATE;
  h->phase = kCreated;
  h->latest_csr = -1;
  h->lepp_valid = false;
  return launch(h, "build_twin", s, [&] {
    return launch_build_twin(h->M.tri, h->M.m, h->M.n, const_cast<int*>(h->M.twin), h->tw_cnt,
                             h->tw_start, h->tw_adj, h->tile_sum, h->tile_off, h->C, h->sms, s);
  });
}

// neigh (nullable): a Neighbor array (with its convention) the owned twin array is
// built from, instead of from tri alone
polylla_status create_common(polylla_mesh* h, cudaStream_t s, uint32_t flags,
                             const int* neigh = nullptr, int convention = 0) {
  if (cudaGetDevice(&h->device) != cudaSuccess) return POLYLLA_ERR_CUDA;
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  POLY_TRY(alloc_derived(h));
  h->last_stream = s;
  if (h->owns_twin || h->owns_inputs) POLY_TRY(alloc_twin_scratch(h));
  if (h->owns_twin && neigh) {  // converted from the Neighbor array now, and checked
    const int g = grid_for(h, h->M.m, kBlock);
    POLY_TRY(launch(h, "twin_from_neighbor", s, [&] {
      return launch_twin_from_neighbor(h->M.tri, neigh, h->M.m, convention,
                                       const_cast<int*>(h->M.twin), h->C, g, s);
    }));
    Counters c;
    POLY_TRY(read_counters(h, &c));
  } else if (h->owns_twin) {  // built from tri now, and checked
    POLY_TRY(do_build_twin(h, s));
    Counters c;
    POLY_TRY(read_counters(h, &c));
  }
  if (flags & POLYLLA_VALIDATE) {
    const int g = grid_for(h, (h->M.n > 3 * h->M.m ? h->M.n : 3 * h->M.m), kBlock);
    POLY_TRY(launch(h, "validate", s, [&] { return launch_validate(h->M, h->C, g, s); }));
    Counters c;
    polylla_status st = read_counters(h, &c);
    if (st != POLYLLA_OK) return st;
  }
  return POLYLLA_OK;
}

// ---------------------------------------------------------------- batches
// Schedules a batch can be run with: the walk's thread-per-seed cap, the
// long-polygon mode (0: large blocks only; 1: small blocks first; 2: one warp per
// polygon first), and whether the three kernels after the walk overlap on side
// streams (1) or run one after another (0: each one-wave grid then has the whole
// GPU to itself).
constexpr int kSchedules = 12;
constexpr int kSchedCap[kSchedules] = {64, 64, 32, 48, 64, 64, 32, 48, 16, 32, 16, 32};
constexpr int kSchedLong[kSchedules] = {0, 1, 1, 1, 0, 1, 1, 1, 2, 2, 2, 2};
constexpr int kSchedOverlap[kSchedules] = {1, 1, 1, 1, 0, 0, 0, 0, 1, 1, 0, 0};

}  // namespace

struct polylla_batch {
  polylla_mesh* mesh = nullptr;  // the union of the meshes
  int* tri_g = nullptr;          // union ids
  int* twin_g = nullptr;
  long long n_meshes = 0;
  long long* d_tri_off = nullptr;
  long long* d_vtx_off = nullptr;
  long long* d_pfirst = nullptr;
  long long* d_obase = nullptr;
  std::vector<long long> pfirst;  // host copy, read after a run
  bool pfirst_valid = false;
  int tuned = -1;
  cudaGraphExec_t exec[kSchedules] = {};
  // graphs are captured and replayed on this stream (the caller's may be the
  // legacy default stream, which cannot be captured), joined to the caller's
  cudaStream_t gs = nullptr;
  cudaEvent_t in = nullptr, out = nullptr;
};

namespace {

void batch_free(polylla_batch* b) {
  for (int k = 0; k < kSchedules; ++k)
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
  if (b->gs) cudaStreamDestroy(b->gs);
  if (b->in) cudaEventDestroy(b->in);
  if (b->out) cudaEventDestroy(b->out);
  if (b->mesh) {
    free_all(b->mesh);
    delete b->mesh;
  }
  void* ptrs[] = {b->tri_g, b->twin_g, b->d_tri_off, b->d_vtx_off, b->d_pfirst, b->d_obase};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// The whole path over the union plus the per-mesh table, enqueued on s.
polylla_status batch_body(polylla_batch* b, cudaStream_t s) {
  polylla_mesh* h = b->mesh;
  h->last_stream = s;
  POLY_TRY(do_label(h, s));
  POLY_TRY(do_seeds(h, s));
  POLY_TRY(do_repair(h, s));
  return launch(h, "batch_first", s, [&] {
    return launch_batch_first(h->seeds, b->d_tri_off, b->n_meshes, b->d_obase, b->d_pfirst, h->C,
                              s);
  });
}

// Run schedule k: the first time eagerly (kernel attributes and occupancy caches
// are set up outside a capture), then captured into a CUDA graph that later runs
// replay.  With per-kernel timing on, always eagerly.
polylla_status batch_run_sched(polylla_batch* b, int k, cudaStream_t s) {
  polylla_mesh* h = b->mesh;
  h->walk_cap = kSchedCap[k];
  h->long_mode = kSchedLong[k];
  h->overlap = kSchedOverlap[k] != 0;
  b->pfirst_valid = false;
  if (h->timing) return batch_body(b, s);
  if (!b->exec[k]) {
    POLY_TRY(batch_body(b, s));
    // capture on the batch's own stream (nothing runs during a capture)
    cudaGraph_t g = nullptr;
    POLY_TRY(cuda_status(cudaStreamBeginCapture(b->gs, cudaStreamCaptureModeThreadLocal)));
    polylla_status st = batch_body(b, b->gs);
    cudaError_t e = cudaStreamEndCapture(b->gs, &g);
    h->last_stream = s;
    if (st != POLYLLA_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    POLY_TRY(cuda_status(e));
    e = cudaGraphInstantiate(&b->exec[k], g, 0);
    cudaGraphDestroy(g);
    POLY_TRY(cuda_status(e));
    return POLYLLA_OK;  // the captured launches did not run; the eager ones did
  }
  POLY_TRY(cuda_status(cudaEventRecord(b->in, s)));
  POLY_TRY(cuda_status(cudaStreamWaitEvent(b->gs, b->in, 0)));
  POLY_TRY(cuda_status(cudaGraphLaunch(b->exec[k], b->gs)));
  POLY_TRY(cuda_status(cudaEventRecord(b->out, b->gs)));
  POLY_TRY(cuda_status(cudaStreamWaitEvent(s, b->out, 0)));
  h->last_stream = s;
  h->phase = kRepaired;
  h->latest_csr = 1;
  ++h->launches;
  return POLYLLA_OK;
}

polylla_status batch_table(polylla_batch* b) {
  if (b->pfirst_valid) return POLYLLA_OK;
  polylla_mesh* h = b->mesh;
  if (h->phase != kRepaired) return POLYLLA_ERR_STATE;
  Counters c;
  POLY_TRY(read_counters(h, &c));  // syncs and reports device errors
  b->pfirst.assign((size_t)b->n_meshes + 1, 0);
  POLY_TRY(cuda_status(cudaMemcpy(b->pfirst.data(), b->d_pfirst,
                                  sizeof(long long) * (size_t)(b->n_meshes + 1),
                                  cudaMemcpyDeviceToHost)));
  b->pfirst_valid = true;
  return POLYLLA_OK;
}

}  // namespace

extern "C" {

void polylla_debug_fail_alloc(int64_t k) { g_fail_alloc.store(k > 0 ? k : 0); }

polylla_status polylla_debug_rare_paths(polylla_mesh_t h, int enable) {
  if (!h) return POLYLLA_ERR_INVALID_ARG;
  h->rare_paths = enable != 0;
  return POLYLLA_OK;
}

polylla_status polylla_debug_split_by_pieces(polylla_mesh_t h, int enable) {
  if (!h) return POLYLLA_ERR_INVALID_ARG;
  h->block_by_pieces = enable != 0;
  return POLYLLA_OK;
}

const char* polylla_status_str(polylla_status st) {
  switch (st) {
    case POLYLLA_OK: return "POLYLLA_OK";
    case POLYLLA_ERR_INVALID_ARG: return "POLYLLA_ERR_INVALID_ARG";
    case POLYLLA_ERR_RANGE: return "POLYLLA_ERR_RANGE";
    case POLYLLA_ERR_TOPOLOGY: return "POLYLLA_ERR_TOPOLOGY";
    case POLYLLA_ERR_OOM: return "POLYLLA_ERR_OOM";
    case POLYLLA_ERR_CUDA: return "POLYLLA_ERR_CUDA";
    case POLYLLA_ERR_LIMIT: return "POLYLLA_ERR_LIMIT";
    case POLYLLA_ERR_STATE: return "POLYLLA_ERR_STATE";
    case POLYLLA_ERR_CANCELLED: return "POLYLLA_ERR_CANCELLED";
  }
  return "POLYLLA_ERR_UNKNOWN";
}

polylla_status polylla_mesh_create(const int64_t* d_xy, int64_t n_vertices, const int32_t* d_tri,
                                   int64_t n_tri, const int32_t* d_twin, uint32_t flags,
                                   void* stream, polylla_mesh_t* out) {
  if (!out) return POLYLLA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d_xy || !d_tri) return POLYLLA_ERR_INVALID_ARG;
  if (n_vertices < 3 || n_vertices >= kMaxVertices || n_tri < 1 || n_tri >= kMaxTriangles)
    return POLYLLA_ERR_INVALID_ARG;
  if ((flags & ~POLYLLA_VALIDATE) != 0) return POLYLLA_ERR_INVALID_ARG;
  if (((uintptr_t)d_xy | (uintptr_t)d_tri | (uintptr_t)d_twin) & 15u) return POLYLLA_ERR_INVALID_ARG;
  polylla_mesh* h = new (std::nothrow) polylla_mesh();
  if (!h) return POLYLLA_ERR_OOM;
  h->M.xy = reinterpret_cast<const long long*>(d_xy);
  h->M.tri = d_tri;
  h->M.twin = d_twin;
  h->M.n = n_vertices;
  h->M.m = n_tri;
  polylla_status st = POLYLLA_OK;
  if (!d_twin) {  // built on the device from tri
    int* tw = nullptr;
    st = cuda_status(dalloc(&tw, 3 * n_tri));
    h->M.twin = tw;
    h->owns_twin = true;
  }
  if (st == POLYLLA_OK) st = create_common(h, (cudaStream_t)stream, flags);
  if (st != POLYLLA_OK) {
    free_all(h);
    delete h;
    return st;
  }
  *out = h;
  return POLYLLA_OK;
}

polylla_status polylla_mesh_create_neighbors(const int64_t* d_xy, int64_t n_vertices,
                                             const int32_t* d_tri, int64_t n_tri,
                                             const int32_t* d_neighbor, int convention,
                                             uint32_t flags, void* stream, polylla_mesh_t* out) {
  if (!out) return POLYLLA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d_xy || !d_tri || !d_neighbor) return POLYLLA_ERR_INVALID_ARG;
  if (convention != POLYLLA_NEIGHBOR_OPPOSITE && convention != POLYLLA_NEIGHBOR_EDGE)
    return POLYLLA_ERR_INVALID_ARG;
  if (n_vertices < 3 || n_vertices >= kMaxVertices || n_tri < 1 || n_tri >= kMaxTriangles)
    return POLYLLA_ERR_INVALID_ARG;
  if ((flags & ~POLYLLA_VALIDATE) != 0) return POLYLLA_ERR_INVALID_ARG;
  if (((uintptr_t)d_xy | (uintptr_t)d_tri) & 15u) return POLYLLA_ERR_INVALID_ARG;
  if ((uintptr_t)d_neighbor & 3u) return POLYLLA_ERR_INVALID_ARG;
  polylla_mesh* h = new (std::nothrow) polylla_mesh();
  if (!h) return POLYLLA_ERR_OOM;
  h->M.xy = reinterpret_cast<const long long*>(d_xy);
  h->M.tri = d_tri;
  h->M.n = n_vertices;
  h->M.m = n_tri;
  int* tw = nullptr;
  polylla_status st = cuda_status(dalloc(&tw, 3 * n_tri));
  h->M.twin = tw;
  h->owns_twin = true;
  if (st == POLYLLA_OK)
    st = create_common(h, (cudaStream_t)stream, flags, d_neighbor, convention);
  if (st != POLYLLA_OK) {
    free_all(h);
    delete h;
    return st;
  }
  *out = h;
  return POLYLLA_OK;
}

polylla_status polylla_get_twin(polylla_mesh_t h, const int32_t** d_twin) {
  POLY_TRY(check_handle(h));
  if (!d_twin) return POLYLLA_ERR_INVALID_ARG;
  *d_twin = h->M.twin;
  return POLYLLA_OK;
}

polylla_status polylla_trivertex(polylla_mesh_t h, void* stream) {
  POLY_TRY(check_handle(h));
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  const int g = grid_for(h, 3 * h->M.m, kBlock);
  POLY_TRY(launch(h, "trivertex", s, [&] {
    return launch_trivertex(h->M.tri, h->M.m, h->M.n, h->trivertex, h->C, g, s);
  }));
  h->trivertex_valid = true;
  return POLYLLA_OK;
}

polylla_status polylla_get_trivertex(polylla_mesh_t h, const int32_t** d_trivertex) {
  POLY_TRY(check_handle(h));
  if (!d_trivertex) return POLYLLA_ERR_INVALID_ARG;
  if (!h->trivertex_valid) return POLYLLA_ERR_STATE;
  Counters c;
  POLY_TRY(read_counters(h, &c));  // syncs; reports an id out of range
  *d_trivertex = h->trivertex;
  return POLYLLA_OK;
}

polylla_status polylla_mesh_create_host(int64_t n_vertices, int64_t n_tri, polylla_mesh_t* out) {
  if (!out) return POLYLLA_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_vertices < 3 || n_vertices >= kMaxVertices || n_tri < 1 || n_tri >= kMaxTriangles)
    return POLYLLA_ERR_INVALID_ARG;
  polylla_mesh* h = new (std::nothrow) polylla_mesh();
  if (!h) return POLYLLA_ERR_OOM;
  long long* xy = nullptr;
  int *tri = nullptr, *twin = nullptr;
  cudaError_t e = dalloc(&xy, 2 * n_vertices);
  if (e == cudaSuccess) e = dalloc(&tri, 3 * n_tri);
  if (e == cudaSuccess) e = dalloc(&twin, 3 * n_tri);
  h->owns_inputs = true;
  h->M.xy = xy;
  h->M.tri = tri;
  h->M.twin = twin;
  h->M.n = n_vertices;
  h->M.m = n_tri;
  polylla_status st = cuda_status(e);
  if (st == POLYLLA_OK) st = create_common(h, nullptr, 0);
  if (st != POLYLLA_OK) {
    free_all(h);
    delete h;
    return st;
  }
  *out = h;
  return POLYLLA_OK;
}

polylla_status polylla_label(polylla_mesh_t h, void* stream) {
  POLY_TRY(check_handle(h));
  h->last_stream = (cudaStream_t)stream;
  return do_label(h, (cudaStream_t)stream);
}

polylla_status polylla_seeds(polylla_mesh_t h, void* stream) {
  POLY_TRY(check_handle(h));
  if (h->phase != kLabeled) return POLYLLA_ERR_STATE;
  h->last_stream = (cudaStream_t)stream;
  return do_seeds(h, (cudaStream_t)stream);
}

polylla_status polylla_traverse(polylla_mesh_t h, void* stream) {
  POLY_TRY(check_handle(h));
  if (h->phase != kSeeded) return POLYLLA_ERR_STATE;
  h->last_stream = (cudaStream_t)stream;
  return do_traverse(h, (cudaStream_t)stream);
}

polylla_status polylla_repair(polylla_mesh_t h, void* stream) {
  POLY_TRY(check_handle(h));
  if (h->phase != kTraversed) return POLYLLA_ERR_STATE;
  h->last_stream = (cudaStream_t)stream;
  return do_repair(h, (cudaStream_t)stream);
}

polylla_status polylla_repair_host(polylla_mesh_t h, void* stream) {
  POLY_TRY(check_handle(h));
  if (h->phase != kTraversed) return POLYLLA_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  Counters c;
  POLY_TRY(read_counters(h, &c));  // syncs; the traversal's errors first
  const long long n = h->M.n, m = h->M.m, np = c.n_seeds, nv = c.n_vtx_trav;
  try {
    h->h_tri.resize((size_t)(3 * m));
    h->h_twin.resize((size_t)(3 * m));
    h->h_lab.resize((size_t)m);
    h->h_off.resize((size_t)(np + 1));
    h->h_vtx.resize((size_t)(nv > 0 ? nv : 1));
    h->h_out_off.resize((size_t)(m + 1));
    h->h_out_vtx.resize((size_t)(3 * m));
  } catch (...) {
    return POLYLLA_ERR_OOM;
  }
  cudaError_t e = cudaMemcpy(h->h_tri.data(), h->M.tri, sizeof(int) * 3 * m, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->h_twin.data(), h->M.twin, sizeof(int) * 3 * m, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h->h_lab.data(), h->lab, (size_t)m, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->h_off.data(), h->off_trav, sizeof(long long) * (np + 1), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && nv > 0)
    e = cudaMemcpy(h->h_vtx.data(), h->vtx_trav, sizeof(int) * nv, cudaMemcpyDeviceToHost);
  POLY_TRY(cuda_status(e));
  int64_t out_np = 0, out_nv = 0;
  const int64_t splits =
      host_repair(n, m, h->h_tri.data(), h->h_twin.data(), h->h_lab.data(), h->h_off.data(),
                  h->h_vtx.data(), np, h->h_out_off.data(), h->h_out_vtx.data(), &out_np, &out_nv);
  if (splits < 0) return POLYLLA_ERR_LIMIT;
  e = cudaMemcpy(h->lab, h->h_lab.data(), (size_t)m, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->off_final, h->h_out_off.data(), sizeof(long long) * (out_np + 1),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && out_nv > 0)
    e = cudaMemcpy(h->vtx_final, h->h_out_vtx.data(), sizeof(int) * out_nv, cudaMemcpyHostToDevice);
  // the counters the getters report: splits, final polygons and their length
  const long long cnt[3] = {splits, out_np, out_nv};
  static_assert(offsetof(Counters, n_poly) == offsetof(Counters, n_splits) + sizeof(long long) &&
                    offsetof(Counters, n_vtx) == offsetof(Counters, n_poly) + sizeof(long long),
                "n_splits, n_poly and n_vtx are adjacent");
  if (e == cudaSuccess) e = cudaMemcpy(&h->C->n_splits, cnt, sizeof(cnt), cudaMemcpyHostToDevice);
  POLY_TRY(cuda_status(e));
  h->phase = kRepaired;
  h->latest_csr = 1;
  return POLYLLA_OK;
}

polylla_status polylla_run(polylla_mesh_t h, void* stream) {
  POLY_TRY(check_handle(h));
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  if (h->M.m <= h->block_max && !h->rare_paths) return do_block(h, s);
  POLY_TRY(do_label(h, s));
  POLY_TRY(do_seeds(h, s));
  return do_repair(h, s);
}

polylla_status polylla_set_one_block(polylla_mesh_t h, int64_t max_tri) {
  if (!h) return POLYLLA_ERR_INVALID_ARG;
  if (max_tri < 0 || max_tri > kBlockMeshMax) return POLYLLA_ERR_INVALID_ARG;
  h->block_max = max_tri;
  return POLYLLA_OK;
}

int64_t polylla_one_block_limit(void) { return kBlockMeshMax; }

polylla_status polylla_get_labels(polylla_mesh_t h, const uint8_t** d_lab) {
  POLY_TRY(check_handle(h));
  if (!d_lab) return POLYLLA_ERR_INVALID_ARG;
  if (h->phase < kLabeled) return POLYLLA_ERR_STATE;
  *d_lab = h->lab;
  return POLYLLA_OK;
}

polylla_status polylla_get_seeds(polylla_mesh_t h, const int32_t** d_seeds, int64_t* n_seeds) {
  POLY_TRY(check_handle(h));
  if (!d_seeds || !n_seeds) return POLYLLA_ERR_INVALID_ARG;
  if (h->phase < kSeeded) return POLYLLA_ERR_STATE;
  Counters c;
  POLY_TRY(read_counters(h, &c));
  *d_seeds = h->seeds;
  *n_seeds = c.n_seeds;
  return POLYLLA_OK;
}

polylla_status polylla_get_polygons(polylla_mesh_t h, const int64_t** d_off, const int32_t** d_vtx,
                                    int64_t* n_poly, int64_t* n_vtx) {
  POLY_TRY(check_handle(h));
  if (!d_off || !d_vtx || !n_poly || !n_vtx) return POLYLLA_ERR_INVALID_ARG;
  if (h->latest_csr < 0) return POLYLLA_ERR_STATE;
  Counters c;
  POLY_TRY(read_counters(h, &c));
  if (h->latest_csr == 0) {
    *d_off = reinterpret_cast<const int64_t*>(h->off_trav);
    *d_vtx = h->vtx_trav;
    *n_poly = c.n_seeds;
    *n_vtx = c.n_vtx_trav;
  } else {
    *d_off = reinterpret_cast<const int64_t*>(h->off_final);
    *d_vtx = h->vtx_final;
    *n_poly = c.n_poly;
    *n_vtx = c.n_vtx;
  }
  return POLYLLA_OK;
}

polylla_status polylla_get_stats(polylla_mesh_t h, polylla_stats* out) {
  POLY_TRY(check_handle(h));
  if (!out) return POLYLLA_ERR_INVALID_ARG;
  Counters c;
  POLY_TRY(read_counters(h, &c));
  std::memset(out, 0, sizeof(*out));
  if (h->phase >= kSeeded) out->n_seeds = c.n_seeds;
  if (h->phase >= kTraversed || h->latest_csr == 1) {
    out->n_poly_trav = c.n_seeds;
    out->n_vtx_trav = c.n_vtx_trav;
    out->n_tip_polygons = c.n_tip_polys;
    out->n_tips = c.n_tips;
  }
  if (h->phase >= kTraversed || h->latest_csr == 1) {
    out->n_long = c.n_long;
    out->n_long_handoff = c.n_long2;
    out->n_long_seq = c.n_long_seq;
  }
  if (h->phase >= kRepaired) {
    out->n_splits = c.n_splits;
    out->n_poly = c.n_poly;
    out->n_vtx = c.n_vtx;
    out->n_one_tip = c.n_defer;
    out->n_multi_tip = c.n_multi;
    out->n_multi_seq = c.n_multi_seq;
    out->n_one_chase = c.n_one_chase;
    out->n_multi_turn = c.n_multi_turn;
    out->n_one_block = c.n_block;
  }
  return POLYLLA_OK;
}

polylla_status polylla_mesh_destroy(polylla_mesh_t h) {
  if (!h) return POLYLLA_ERR_INVALID_ARG;
  POLY_TRY(check_handle(h));
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return POLYLLA_OK;
}

polylla_status polylla_run_host(polylla_mesh_t h, const int64_t* h_xy, const int32_t* h_tri,
                                const int32_t* h_twin, int64_t* h_off, int32_t* h_vtx,
                                int64_t* n_poly, int64_t* n_vtx, void* stream) {
  POLY_TRY(check_handle(h));
  if (!h->owns_inputs) return POLYLLA_ERR_STATE;
  if (!h_xy || !h_tri || !h_off || !h_vtx || !n_poly || !n_vtx) return POLYLLA_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = h->M.n, m = h->M.m;
  h->trivertex_valid = false;
  cudaError_t e =
      cudaMemcpyAsync(const_cast<long long*>(h->M.xy), h_xy, sizeof(long long) * 2 * n,
                      cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(const_cast<int*>(h->M.tri), h_tri, sizeof(int) * 3 * m,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && h_twin)
    e = cudaMemcpyAsync(const_cast<int*>(h->M.twin), h_twin, sizeof(int) * 3 * m,
                        cudaMemcpyHostToDevice, s);
  POLY_TRY(cuda_status(e));
  if (!h_twin) POLY_TRY(do_build_twin(h, s));  // from tri, on the device
  POLY_TRY(polylla_run(h, stream));
  Counters c;
  POLY_TRY(read_counters(h, &c));
  e = cudaMemcpyAsync(h_off, h->off_final, sizeof(long long) * (size_t)(c.n_poly + 1),
                      cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h_vtx, h->vtx_final, sizeof(int) * (size_t)c.n_vtx, cudaMemcpyDeviceToHost,
                        s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  POLY_TRY(cuda_status(e));
  *n_poly = c.n_poly;
  *n_vtx = c.n_vtx;
  return POLYLLA_OK;
}

polylla_status polylla_set_timing(polylla_mesh_t h, int enable) {
  POLY_TRY(check_handle(h));
  h->timing = enable != 0;
  return POLYLLA_OK;
}

int64_t polylla_kernel_times(polylla_mesh_t h, const char** names, float* ms, int64_t cap,
                             int reset) {
  if (check_handle(h) != POLYLLA_OK) return -1;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return -1;
  const int64_t n = (int64_t)h->recs.size();
  for (int64_t i = 0; i < n && i < cap; ++i) {
    if (names) names[i] = h->recs[(size_t)i].name;
    if (ms) {
      float t = 0.f;
      cudaEventElapsedTime(&t, h->recs[(size_t)i].a, h->recs[(size_t)i].b);
      ms[i] = t;
    }
  }
  if (reset) {
    for (auto& r : h->recs) {
      h->event_pool.push_back(r.a);
      h->event_pool.push_back(r.b);
    }
    h->recs.clear();
  }
  return n;
}

int64_t polylla_launch_count(polylla_mesh_t h) { return h ? h->launches : -1; }

polylla_status polylla_lepp(polylla_mesh_t h, void* stream) {
  POLY_TRY(check_handle(h));
  if (h->phase < kLabeled) return POLYLLA_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  const int g = grid_for(h, h->M.m, kBlock);
  POLY_TRY(launch(h, "lepp", s, [&] {
    return launch_lepp(h->M, h->lab, h->lepp_region, h->lepp_depth, h->C, g, s);
  }));
  h->lepp_valid = true;
  return POLYLLA_OK;
}

polylla_status polylla_get_lepp(polylla_mesh_t h, const int32_t** d_region,
                                const int32_t** d_depth) {
  POLY_TRY(check_handle(h));
  if (!d_region || !d_depth) return POLYLLA_ERR_INVALID_ARG;
  if (!h->lepp_valid) return POLYLLA_ERR_STATE;
  Counters c;
  POLY_TRY(read_counters(h, &c));  // syncs; reports a path error
  *d_region = h->lepp_region;
  *d_depth = h->lepp_depth;
  return POLYLLA_OK;
}

int64_t polylla_mesh_footprint(int64_t n_vertices, int64_t n_tri, int owns_inputs) {
  if (n_vertices < 3 || n_tri < 1) return -1;
  long long b = derived_bytes(n_vertices, n_tri);
  if (owns_inputs) b += 16 * n_vertices + 24 * n_tri + 8 * n_vertices + 4 + 24 * n_tri;
  return b;
}

polylla_status polylla_mesh_build_twin(polylla_mesh_t h, void* stream) {
  POLY_TRY(check_handle(h));
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  return do_build_twin(h, s);
}

polylla_status polylla_mesh_set_size(polylla_mesh_t h, int64_t n_vertices, int64_t n_tri) {
  POLY_TRY(check_handle(h));
  if (!h->owns_inputs) return POLYLLA_ERR_STATE;
  if (n_vertices < 3 || n_tri < 1 || n_vertices > h->n_cap || n_tri > h->m_cap)
    return POLYLLA_ERR_INVALID_ARG;
  h->M.n = n_vertices;
  h->M.m = n_tri;
  h->phase = kCreated;
  h->latest_csr = -1;
  h->lepp_valid = false;
  h->trivertex_valid = false;
  return POLYLLA_OK;
}

polylla_status polylla_mesh_inputs(polylla_mesh_t h, int64_t** d_xy, int32_t** d_tri,
                                   int32_t** d_twin) {
  POLY_TRY(check_handle(h));
  if (!d_xy || !d_tri || !d_twin) return POLYLLA_ERR_INVALID_ARG;
  if (!h->owns_inputs) return POLYLLA_ERR_STATE;
  *d_xy = reinterpret_cast<int64_t*>(const_cast<long long*>(h->M.xy));
  *d_tri = const_cast<int32_t*>(h->M.tri);
  *d_twin = const_cast<int32_t*>(h->M.twin);
  return POLYLLA_OK;
}

polylla_status polylla_get_polygons_async(polylla_mesh_t h, const int64_t** d_off,
                                          const int32_t** d_vtx, const int64_t** d_counts,
                                          const int32_t** d_error) {
  POLY_TRY(check_handle(h));
  if (!d_off || !d_vtx || !d_counts || !d_error) return POLYLLA_ERR_INVALID_ARG;
  if (h->latest_csr < 0) return POLYLLA_ERR_STATE;
  *d_off = reinterpret_cast<const int64_t*>(h->latest_csr == 1 ? h->off_final : h->off_trav);
  *d_vtx = h->latest_csr == 1 ? h->vtx_final : h->vtx_trav;
  static_assert(offsetof(Counters, n_vtx) == offsetof(Counters, n_poly) + sizeof(long long),
                "n_poly and n_vtx are adjacent");
  *d_counts = reinterpret_cast<const int64_t*>(&h->C->n_poly);
  *d_error = &h->C->error;
  return POLYLLA_OK;
}

polylla_status polylla_batch_create(const int64_t* d_xy, const int64_t* d_vtx_off,
                                    const int32_t* d_tri, const int32_t* d_twin,
                                    const int64_t* d_tri_off, int64_t n_meshes, uint32_t flags,
                                    void* stream, polylla_batch_t* out) {
  if (!out) return POLYLLA_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d_xy || !d_vtx_off || !d_tri || !d_twin || !d_tri_off || n_meshes < 1)
    return POLYLLA_ERR_INVALID_ARG;
  if ((flags & ~POLYLLA_VALIDATE) != 0) return POLYLLA_ERR_INVALID_ARG;
  if (((uintptr_t)d_xy | (uintptr_t)d_tri | (uintptr_t)d_twin) & 15u) return POLYLLA_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<long long> to((size_t)n_meshes + 1), vo((size_t)n_meshes + 1);
  if (cudaMemcpy(to.data(), d_tri_off, sizeof(long long) * to.size(), cudaMemcpyDeviceToHost) !=
          cudaSuccess ||
      cudaMemcpy(vo.data(), d_vtx_off, sizeof(long long) * vo.size(), cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return POLYLLA_ERR_CUDA;
  if (to[0] != 0 || vo[0] != 0) return POLYLLA_ERR_INVALID_ARG;
  for (int64_t j = 0; j < n_meshes; ++j)
    if (to[(size_t)j + 1] - to[(size_t)j] < 1 || vo[(size_t)j + 1] - vo[(size_t)j] < 3)
      return POLYLLA_ERR_INVALID_ARG;
  const long long m = to[(size_t)n_meshes], n = vo[(size_t)n_meshes];
  if (m >= kMaxTriangles || n >= kMaxVertices) return POLYLLA_ERR_INVALID_ARG;
  polylla_batch* b = new (std::nothrow) polylla_batch();
  if (!b) return POLYLLA_ERR_OOM;
  b->n_meshes = n_meshes;
  polylla_mesh* h = new (std::nothrow) polylla_mesh();
  if (!h) {
    delete b;
    return POLYLLA_ERR_OOM;
  }
  b->mesh = h;
  cudaError_t e = dalloc(&b->tri_g, 3 * m);
  if (e == cudaSuccess) e = dalloc(&b->twin_g, 3 * m);
  if (e == cudaSuccess) e = dalloc(&b->d_tri_off, n_meshes + 1);
  if (e == cudaSuccess) e = dalloc(&b->d_vtx_off, n_meshes + 1);
  if (e == cudaSuccess) e = dalloc(&b->d_pfirst, n_meshes + 1);
  if (e == cudaSuccess) e = dalloc(&b->d_obase, m);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->out, cudaEventDisableTiming);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_tri_off, to.data(), sizeof(long long) * to.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_vtx_off, vo.data(), sizeof(long long) * vo.size(), cudaMemcpyHostToDevice);
  polylla_status st = cuda_status(e);
  if (st == POLYLLA_OK) {
    h->M.xy = reinterpret_cast<const long long*>(d_xy);
    h->M.tri = b->tri_g;
    h->M.twin = b->twin_g;
    h->M.n = n;
    h->M.m = m;
    h->obase = b->d_obase;
    st = create_common(h, s, 0);
  }
  if (st == POLYLLA_OK) {
    const int g = grid_for(h, m, kBlock);
    st = launch(h, "batch_globalize", s, [&] {
      return launch_batch_globalize(d_tri, d_twin, b->d_tri_off, b->d_vtx_off, n_meshes, m,
                                    b->tri_g, b->twin_g, h->C, g, s);
    });
  }
  if (st == POLYLLA_OK && (flags & POLYLLA_VALIDATE)) {
    const int g = grid_for(h, (n > 3 * m ? n : 3 * m), kBlock);
    st = launch(h, "validate", s, [&] { return launch_validate(h->M, h->C, g, s); });
  }
  if (st == POLYLLA_OK) {
    Counters c;
    st = read_counters(h, &c);  // range errors of the local ids, validation
  }
  if (st != POLYLLA_OK) {
    batch_free(b);
    delete b;
    return st;
  }
  *out = b;
  return POLYLLA_OK;
}

int polylla_batch_schedules(void) { return kSchedules; }

polylla_status polylla_batch_schedule_info(int schedule, int* walk_cap, int* long_mode,
                                           int* overlap) {
  if (schedule < 0 || schedule >= kSchedules) return POLYLLA_ERR_INVALID_ARG;
  if (walk_cap) *walk_cap = kSchedCap[schedule];
  if (long_mode) *long_mode = kSchedLong[schedule];
  if (overlap) *overlap = kSchedOverlap[schedule];
  return POLYLLA_OK;
}

polylla_status polylla_batch_tune(polylla_batch_t b, int reps, void* stream, int* best,
                                  float* ms) {
  if (!b || reps < 1) return POLYLLA_ERR_INVALID_ARG;
  POLY_TRY(check_handle(b->mesh));
  if (b->mesh->timing) return POLYLLA_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return POLYLLA_ERR_CUDA;
  }
  polylla_status st = POLYLLA_OK;
  float best_ms = 0.f;
  int arg = 0;
  for (int k = 0; k < kSchedules && st == POLYLLA_OK; ++k) {
    st = batch_run_sched(b, k, s);                         // builds the graph
    if (st == POLYLLA_OK) st = batch_run_sched(b, k, s);  // one warm replay
    if (st != POLYLLA_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == POLYLLA_OK; ++r) st = batch_run_sched(b, k, s);
    cudaEventRecord(e1, s);
    if (st == POLYLLA_OK) st = cuda_status(cudaEventSynchronize(e1));
    float t = 0.f;
    if (st == POLYLLA_OK) st = cuda_status(cudaEventElapsedTime(&t, e0, e1));
    t /= (float)reps;
    if (ms) ms[k] = t;
    if (k == 0 || t < best_ms) {
      best_ms = t;
      arg = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != POLYLLA_OK) return st;
  Counters c;
  POLY_TRY(read_counters(b->mesh, &c));  // device errors of the timed runs
  b->tuned = arg;
  if (best) *best = arg;
  return POLYLLA_OK;
}

polylla_status polylla_batch_run(polylla_batch_t b, int schedule, void* stream) {
  if (!b) return POLYLLA_ERR_INVALID_ARG;
  POLY_TRY(check_handle(b->mesh));
  if (schedule == POLYLLA_SCHEDULE_TUNED) {
    if (b->tuned < 0) POLY_TRY(polylla_batch_tune(b, 3, stream, nullptr, nullptr));
    schedule = b->tuned;
  }
  if (schedule < 0 || schedule >= kSchedules) return POLYLLA_ERR_INVALID_ARG;
  return batch_run_sched(b, schedule, (cudaStream_t)stream);
}

polylla_status polylla_batch_get(polylla_batch_t b, int64_t mesh, const int64_t** d_off,
                                 const int32_t** d_vtx, int64_t* n_poly, int64_t* n_vtx) {
  if (!b || !d_off || !d_vtx || !n_poly || !n_vtx) return POLYLLA_ERR_INVALID_ARG;
  POLY_TRY(check_handle(b->mesh));
  if (mesh < 0 || mesh >= b->n_meshes) return POLYLLA_ERR_INVALID_ARG;
  POLY_TRY(batch_table(b));
  const long long p0 = b->pfirst[(size_t)mesh], p1 = b->pfirst[(size_t)mesh + 1];
  long long v[2] = {0, 0};
  const long long* off = b->mesh->off_final;
  if (cudaMemcpy(&v[0], off + p0, sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&v[1], off + p1, sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess)
    return POLYLLA_ERR_CUDA;
  *d_off = reinterpret_cast<const int64_t*>(off + p0);
  *d_vtx = b->mesh->vtx_final;
  *n_poly = p1 - p0;
  *n_vtx = v[1] - v[0];
  return POLYLLA_OK;
}

polylla_status polylla_batch_get_all(polylla_batch_t b, const int64_t** d_off,
                                     const int32_t** d_vtx, const int64_t** d_mesh_first,
                                     int64_t* n_poly, int64_t* n_vtx) {
  if (!b || !d_off || !d_vtx || !d_mesh_first || !n_poly || !n_vtx) return POLYLLA_ERR_INVALID_ARG;
  POLY_TRY(check_handle(b->mesh));
  POLY_TRY(batch_table(b));
  Counters c;
  POLY_TRY(read_counters(b->mesh, &c));
  *d_off = reinterpret_cast<const int64_t*>(b->mesh->off_final);
  *d_vtx = b->mesh->vtx_final;
  *d_mesh_first = reinterpret_cast<const int64_t*>(b->d_pfirst);
  *n_poly = c.n_poly;
  *n_vtx = c.n_vtx;
  return POLYLLA_OK;
}

polylla_status polylla_batch_stats(polylla_batch_t b, polylla_stats* out) {
  if (!b) return POLYLLA_ERR_INVALID_ARG;
  return polylla_get_stats(b->mesh, out);
}

polylla_mesh_t polylla_batch_mesh(polylla_batch_t b) { return b ? b->mesh : nullptr; }

polylla_status polylla_batch_destroy(polylla_batch_t b) {
  if (!b) return POLYLLA_ERR_INVALID_ARG;
  POLY_TRY(check_handle(b->mesh));
  cudaDeviceSynchronize();
  batch_free(b);
  delete b;
  return POLYLLA_OK;
}

}  // extern "C"
