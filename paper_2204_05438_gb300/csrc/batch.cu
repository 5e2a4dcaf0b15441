// Batches of independent meshes (no counterpart in the paper, which meshes one
// triangulation at a time).
//
// A batch is run as one disjoint union mesh: mesh j's vertex ids are offset by
// vtx_off[j] and its half-edge ids by 3 * tri_off[j].  No half-edge has a twin in
// another mesh, so no region, walk or split crosses meshes, and the single-mesh
// path runs unchanged over all of them at once; its polygons come out in seed
// order, which is mesh order, so each mesh's polygons are one contiguous run of
// the union's CSR.
//
//   k_batch_globalize  per triangle of the union: its mesh (binary search over
//                      tri_off), local ids range-checked against that mesh's
//                      vertex and triangle counts, rewritten as union ids.
//   k_batch_first      per mesh: its first output polygon (the first seed at or
//                      after tri_off[j], mapped through obase), and the total.
#include "polylla_internal.cuh"

namespace polylla {

__device__ __forceinline__ long long mesh_of(const long long* __restrict__ tri_off, long long n,
                                             long long t) {
  long long lo = 0, hi = n - 1;  // last j with tri_off[j] <= t
  while (lo < hi) {
    const long long mid = (lo + hi + 1) >> 1;
    if (__ldg(tri_off + mid) <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kBlock) k_batch_globalize(
    const int* __restrict__ tri, const int* __restrict__ twin, const long long* __restrict__ tri_off,
    const long long* __restrict__ vtx_off, long long n_meshes, long long m, int* __restrict__ tri_g,
    int* __restrict__ twin_g, Counters* C) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x) {
    const long long j = mesh_of(tri_off, n_meshes, t);
    const long long v0 = __ldg(vtx_off + j), nv = __ldg(vtx_off + j + 1) - v0;
    const long long h0 = 3 * __ldg(tri_off + j);
    const long long nh = 3 * __ldg(tri_off + j + 1) - h0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const long long h = 3 * t + k;
      const int v = __ldg(tri + h);
      const int g = __ldg(twin + h);
      if (v < 0 || v >= nv) {
        set_error(C, POLYLLA_ERR_RANGE, 120);
        tri_g[h] = 0;
      } else {
        tri_g[h] = (int)(v0 + v);
      }
      if (g >= nh || g < -1) {
        set_error(C, POLYLLA_ERR_RANGE, 121);
        twin_g[h] = -1;
      } else {
        twin_g[h] = g < 0 ? -1 : (int)(h0 + g);
      }
    }
  }
}

cudaError_t launch_batch_globalize(const int* tri, const int* twin, const long long* tri_off,
                                   const long long* vtx_off, long long n_meshes, long long m,
                                   int* tri_g, int* twin_g, Counters* C, int grid,
                                   cudaStream_t s) {
  static std::atomic<int> cap{0};
  grid = resident_grid(reinterpret_cast<const void*>(k_batch_globalize), kBlock, 0, grid, &cap);
  k_batch_globalize<<<grid, kBlock, 0, s>>>(tri, twin, tri_off, vtx_off, n_meshes, m, tri_g,
                                            twin_g, C);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock) k_batch_first(const int* __restrict__ seeds,
                                                        const long long* __restrict__ tri_off,
                                                        long long n_meshes,
                                                        const long long* __restrict__ obase,
                                                        long long* __restrict__ pfirst,
                                                        Counters* C) {
  const long long ns = C->n_seeds;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j <= n_meshes;
       j += (long long)gridDim.x * blockDim.x) {
    if (j == n_meshes) {
      pfirst[j] = C->n_poly;
      continue;
    }
    const long long t = tri_off[j];
    long long lo = 0, hi = ns;  // first seed >= t
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (seeds[mid] < t) lo = mid + 1;
      else hi = mid;
    }
    if (lo >= ns || seeds[lo] >= tri_off[j + 1]) {  // every mesh has a seed
      set_error(C, POLYLLA_ERR_LIMIT, 122);
      pfirst[j] = C->n_poly;
    } else {
      pfirst[j] = obase[lo];
    }
  }
}

cudaError_t launch_batch_first(const int* seeds, const long long* tri_off, long long n_meshes,
                               const long long* obase, long long* pfirst, Counters* C,
                               cudaStream_t s) {
  const long long blocks = (n_meshes + 1 + kBlock - 1) / kBlock;
  k_batch_first<<<(int)(blocks < 1024 ? blocks : 1024), kBlock, 0, s>>>(seeds, tri_off, n_meshes,
                                                                        obase, pfirst, C);
  return cudaGetLastError();
}

}  // namespace polylla
