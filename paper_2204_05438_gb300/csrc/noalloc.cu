// polylla_label_seeds_noalloc: the label phase and the seed compaction for callers
// that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a host application that carves
// all of its device memory out of one arena at start-up and forbids further
// allocation, code that runs where a cudaMalloc / cudaFree would implicitly
// synchronise the device and stall other work, or a plugin whose host owns the
// device heap.  The handle-based entry points allocate their scratch in
// polylla_mesh_create, so they are closed to such callers.  This entry point takes
// the same computation (LabelMax, the fused LabelSeed / LabelFrontier pass and the
// ordered seed compaction) and keeps its only scratch -- the look-back words of
// the seed compaction and the counters with the error word -- in a file-scope
// __device__ array of fixed size, so it allocates nothing.  The caller passes the mesh (inputs) and
// the label bytes, seed list and seed count (outputs).
//
// Limits and sharing:
//   * at most kNoAllocMaxTri = 2^26 triangles; larger meshes are rejected with
//     POLYLLA_ERR_INVALID_ARG before anything is launched;
//   * the scratch array (about 33 KiB) belongs to this file's device module.  The
//     CUDA runtime loads modules lazily by default, so the array and the kernels
//     are placed on a device by the first call on that device (its
//     cudaGetSymbolAddress, or its first launch): that first call allocates the
//     module's device memory and may synchronise the device.  A caller that
//     reserves all device memory for its own arena makes one call (any small mesh)
//     on each device before reserving it; after that no call allocates.  The module then stays loaded on that device until
//     the process exits (or the caller resets the device);
//   * every call on a device uses the same array and leaves its contents behind;
//     the parts that must start at zero (the error word, the counters and the
//     look-back words) are cleared at the start of each call, so
//     consecutive calls are independent, but calls that overlap on the GPU (two
//     streams, or two host threads at once) race on it and must be serialised by
//     the caller;
//   * the array's device address is looked up on every call, with the calling
//     device current (a lookup, once the module is loaded), so a caller's
//     cudaDeviceReset leaves no stale address behind;
//   * each call waits for `stream` to finish its work before returning, to report
//     errors that the kernels found on the device.
#include "polylla_internal.cuh"

using namespace polylla;

namespace {

constexpr long long kNoAllocMaxTri = 1ll << 26;
// look-back words of the seed compaction: one per 16384-triangle tile, and one spare
constexpr long long kNoAllocTiles = kNoAllocMaxTri / 16384 + 1;
constexpr size_t kStatusBytes = sizeof(unsigned long long) * (size_t)kNoAllocTiles;
constexpr size_t kCountersOffset = (kStatusBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCountersOffset + ((sizeof(Counters) + 255) / 256) * 256;

// The whole scratch of this entry point: look-back words, counters.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array on the current device.  The host-side
// symbol g_noalloc_scratch is not a device address and is never passed to a
// kernel; cudaGetSymbolAddress gives the address in the current device's context.
cudaError_t scratch_for(int dev, unsigned char** out, int* sms) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

int grid_of(int sms, long long units, long long per_block) {
  long long b = (units + per_block - 1) / per_block;
  const long long cap = 8ll * sms;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

extern "C" polylla_status polylla_label_seeds_noalloc(const int64_t* d_xy, int64_t n_vertices,
                                                      const int32_t* d_tri, const int32_t* d_twin,
                                                      int64_t n_tri, uint8_t* d_lab,
                                                      int32_t* d_seeds, int64_t* d_n_seeds,
                                                      void* stream) {
  if (!d_xy || !d_tri || !d_twin || !d_lab || !d_seeds || !d_n_seeds)
    return POLYLLA_ERR_INVALID_ARG;
  if (n_vertices < 3 || n_vertices > 0x7fffffffll || n_tri < 1) return POLYLLA_ERR_INVALID_ARG;
  if (n_tri > kNoAllocMaxTri) return POLYLLA_ERR_INVALID_ARG;  // beyond the fixed scratch
  if (((uintptr_t)d_xy | (uintptr_t)d_tri | (uintptr_t)d_twin) & 15u) return POLYLLA_ERR_INVALID_ARG;
  if (((uintptr_t)d_lab & 3u) || ((uintptr_t)d_n_seeds & 7u)) return POLYLLA_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return POLYLLA_ERR_CUDA;
  unsigned char* base = nullptr;
  int sms = 0;
  if (scratch_for(dev, &base, &sms) != cudaSuccess) return POLYLLA_ERR_CUDA;
  unsigned long long* status = reinterpret_cast<unsigned long long*>(base);
  Counters* C = reinterpret_cast<Counters*>(base + kCountersOffset);
  cudaStream_t s = (cudaStream_t)stream;

  DevMesh M;
  M.xy = reinterpret_cast<const long long*>(d_xy);
  M.tri = d_tri;
  M.twin = d_twin;
  M.n = n_vertices;
  M.m = n_tri;
  // the error word, counters and look-back words start at zero
  if (seed_tiles(n_tri) + 1 > kNoAllocTiles) return POLYLLA_ERR_INVALID_ARG;
  cudaError_t e = cudaMemsetAsync(C, 0, sizeof(Counters), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(status, 0, sizeof(unsigned long long) * (size_t)(seed_tiles(n_tri) + 1), s);
  if (e == cudaSuccess) e = launch_label_max(M, d_lab, C, grid_of(sms, (n_tri + 3) / 4, kBlock), s);
  if (e == cudaSuccess)
    e = launch_label_class(M, d_lab, nullptr, C, grid_of(sms, n_tri, kTriTile), s, true);
  if (e == cudaSuccess)
    e = launch_seed_write(d_lab, n_tri, status, d_seeds, nullptr, C,
                          grid_of(sms, n_tri, 16 * kTriTile), s, true);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_n_seeds, &C->n_seeds, sizeof(long long), cudaMemcpyDeviceToDevice, s);
  int err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &C->error, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return POLYLLA_ERR_CUDA;
  return (polylla_status)err;
}
