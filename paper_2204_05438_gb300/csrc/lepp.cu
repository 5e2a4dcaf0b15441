// Longest-edge propagation paths (the Lepp that defines terminal-edge regions,
// Section 2; Lepp-based kernels are the paper's future work, Section 5), reusing
// the label step's Max array.
//
//   k_lepp  per triangle t: follow the neighbour across the longest edge until
//           that edge is the longest edge of both its triangles or a border edge
//           (a terminal edge).  region[t] = the seed of that terminal edge (its
//           lower triangle, or the border triangle), depth[t] = links followed.
// Lanes of a warp start at consecutive triangles, whose paths run through the same
// neighbourhood.  Each link is two dependent loads (the twin, then the
// neighbour's label byte); a path longer than m links is an error.
#include "polylla_internal.cuh"

namespace polylla {

__global__ void __launch_bounds__(kBlock) k_lepp(DevMesh M, const uint8_t* __restrict__ lab,
                                                 int* __restrict__ region,
                                                 int* __restrict__ depth, Counters* C) {
  const long long m = M.m;
  const int H = (int)(3 * m);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m;
       t += (long long)gridDim.x * blockDim.x) {
    int u = (int)t, d = 0, reg = -1;
    int mx = __ldg(lab + u) & 3;
    for (;;) {
      const int g = __ldg(M.twin + 3 * u + mx);
      if (g < 0) {  // a border terminal edge
        reg = u;
        break;
      }
      if (g >= H) {
        set_error(C, POLYLLA_ERR_RANGE, 130);
        break;
      }
      const int gt = g / 3;
      const int gm = __ldg(lab + gt) & 3;
      if (gm == g - 3 * gt) {  // the longest edge of both triangles
        reg = u < gt ? u : gt;
        break;
      }
      u = gt;
      mx = gm;
      if (++d > m) {
        set_error(C, POLYLLA_ERR_LIMIT, 131);
        break;
      }
    }
    region[t] = reg;
    depth[t] = d;
  }
}

cudaError_t launch_lepp(const DevMesh& M, const uint8_t* lab, int* region, int* depth, Counters* C,
                        int grid, cudaStream_t s) {
  static std::atomic<int> cap{0};
  grid = resident_grid(reinterpret_cast<const void*>(k_lepp), kBlock, 0, grid, &cap);
  k_lepp<<<grid, kBlock, 0, s>>>(M, lab, region, depth, C);
  return cudaGetLastError();
}

}  // namespace polylla
