// Legendre-Gauss node set: the layout of the device table of the Gauss basis
// and the line indexing shared by the Gauss-node kernels and their adjoint.
#pragma once

#include "dg_stage.cuh"

namespace dg {

// Device table of the Gauss basis (doubles), n = N + 1.
struct GaussTab {
  // [r][m] = (w_m / w_r) D_{m r}, D_{m r} = l_r'(x_m): the weak derivative
  __host__ __device__ static constexpr int Dw(int) { return 0; }
  __host__ __device__ static constexpr int lmw(int n) { return n * n; }           // l_i(-1) / w_i
  __host__ __device__ static constexpr int lpw(int n) { return n * n + n; }       // l_i(+1) / w_i
  __host__ __device__ static constexpr int lm(int n) { return n * n + 2 * n; }    // l_i(-1)
  __host__ __device__ static constexpr int lp(int n) { return n * n + 3 * n; }    // l_i(+1)
  __host__ __device__ static constexpr int V(int n) { return n * n + 4 * n; }     // [i][j]: LGL l_j at Gauss x_i
  __host__ __device__ static constexpr int w(int n) { return 2 * n * n + 4 * n; } // Gauss weights
  __host__ __device__ static constexpr int size(int n) { return 2 * n * n + 5 * n; }
};

// Volume node with index i along direction d and face-local indices (p, q)
// along the two other directions in increasing order (the face_node order).
template <int n>
__device__ __forceinline__ int line_node(int d, int i, int p, int q) {
  return d == 0 ? vidx<n>(i, p, q) : (d == 1 ? vidx<n>(p, i, q) : vidx<n>(p, q, i));
}

}  // namespace dg
