// Mortar maps shared by the mortar kernels and their adjoint (GALAEXI Sec.
// 3.2.2, Algorithm 1): a big face split into four quadrants k = a + 2 b, the
// interpolation of the big face's values to the quadrant nodes and the
// projection back with the node set's quadrature, both as two one-direction
// sweeps through shared memory.  One block per mortar, a thread per quadrant
// node.
#pragma once

#include "dg_stage.cuh"

namespace dg {

template <int N>
struct MortarShape {
  static constexpr int n = N + 1, P = n * n * n, NN = n * n, THREADS = 4 * NN;
};

// Where the values of side (e, f) at its face point (p, q) start, and the
// stride between their fields: the volume nodes (LGL, the face points are
// nodes) or the face values [E][6][NF][NN] (Gauss nodes).
template <int n, bool FACE, int NF, typename T>
__device__ __forceinline__ const T* side_ptr(const T* base, int e, int f, int p, int q, int& st) {
  constexpr int NN = n * n, P = n * n * n;
  if constexpr (FACE) {
    st = NN;
    return base + ((size_t)e * 6 + f) * NF * NN + p + n * q;
  } else {
    st = P;
    return base + (size_t)e * NF * P + face_node<n>(f, p, q);
  }
}

// Both kernels work in tensor-product sweeps (one direction at a time) over
// shared memory.  Tables, from the interpolation I_h[x][j] and the weights w:
//   sI [h][x][j] = I_h[x][j]        (second sweep of the interpolation)
//   sIT[h][j][x] = I_h[x][j]        (first sweep: consecutive threads, consecutive x)
//   sW [h][x][j] = w_x I_h[x][j]    (both sweeps of the projection)
template <int n>
__device__ __forceinline__ void mortar_tables(const double* __restrict__ tab, double* sI, double* sIT, double* sW,
                                              double* sw, int t, int nthr) {
  constexpr int NN = n * n;
  for (int x = t; x < 2 * NN; x += nthr) {
    const int h = x / NN, r = x - h * NN, a = r / n, j = r - a * n;   // r = a n + j
    const double v = tab[x];
    sI[x] = v;
    sIT[h * NN + j * n + a] = v;
    sW[x] = tab[2 * NN + a] * v;
  }
  for (int x = t; x < n; x += nthr) sw[x] = tab[2 * NN + x];
}

// First interpolation sweep, along the big face's first direction:
//   T[h][f][pp + n j] = sum_i I_h[pp][i] B[f][i + n j]   for both halves h.
template <int n, int NF>
__device__ __forceinline__ void mortar_sweep1(const double* sIT, const double* B, double* T, int t, int nthr) {
  constexpr int NN = n * n;
  for (int o = t; o < 2 * NF * NN; o += nthr) {
    const int h = o / (NF * NN), r = o - h * NF * NN, f = r / NN, pj = r - f * NN, pp = pj % n, j = pj / n;
    const double* it = sIT + h * NN + pp;
    const double* b = B + f * NN + j * n;
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < n; ++i) s = fma(it[i * n], b[i], s);
    T[o] = s;
  }
}

// Second sweep for quadrant k = a + 2 b at its node (pp, qq):
//   out[f] = sum_j I_b[qq][j] T[a][f][pp + n j].
template <int n, int NF>
__device__ __forceinline__ void mortar_sweep2(const double* sI, const double* T, int k, int pp, int qq,
                                              double out[NF]) {
  constexpr int NN = n * n;
  const double* ib = sI + (k >> 1) * NN + qq * n;
  const double* tr = T + (k & 1) * NF * NN + pp;
#pragma unroll
  for (int f = 0; f < NF; ++f) out[f] = 0.0;
#pragma unroll
  for (int j = 0; j < n; ++j) {
    const double c = ib[j];
#pragma unroll
    for (int f = 0; f < NF; ++f) out[f] = fma(c, tr[f * NN + j * n], out[f]);
  }
}

// The projection's first sweep, along the quadrants' second direction:
//   S[k][f][pp + n j] = sum_qq w_qq I_b[qq][j] Q[k][f][pp + n qq].
template <int n, int NF>
__device__ __forceinline__ void mortar_proj1(const double* sW, const double* Q, double* S, int t, int nthr) {
  constexpr int NN = n * n;
  for (int o = t; o < 4 * NF * NN; o += nthr) {
    const int k = o / (NF * NN), r = o - k * NF * NN, f = r / NN, pj = r - f * NN, pp = pj % n, j = pj / n;
    const double* wb = sW + (k >> 1) * NN + j;
    const double* q = Q + (k * NF + f) * NN + pp;
    double s = 0.0;
#pragma unroll
    for (int qq = 0; qq < n; ++qq) s = fma(wb[qq * n], q[qq * n], s);
    S[o] = s;
  }
}

// Second sweep, summed over the quadrants, at big-face node (i, j):
//   sum_k sum_pp w_pp I_a[pp][i] S[k][f][pp + n j].
template <int n, int NF>
__device__ __forceinline__ double mortar_proj2(const double* sW, const double* S, int f, int i, int j) {
  constexpr int NN = n * n;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double* wa = sW + (k & 1) * NN + i;
    const double* sr = S + (k * NF + f) * NN + j * n;
#pragma unroll
    for (int pp = 0; pp < n; ++pp) s = fma(wa[pp * n], sr[pp], s);
  }
  return s;
}

// (u, v, w, T) of a conservative state (FP64 or FP32 values), in FP64; E_off
// is added to the energy (E_ref for FP32 face values that carry E - E_ref)
template <typename T>
__device__ __forceinline__ void lift_vars(const T* q, int st, const Gas& g, double ph[4], double E_off = 0.0) {
  const double q0 = q[0], q1 = q[st], q2 = q[2 * st], q3 = q[3 * st], q4 = (double)q[4 * st] + E_off;
  const double ir = 1.0 / q0;
  const double u = q1 * ir, v = q2 * ir, w = q3 * ir;
  const double p = g.gm1 * (q4 - 0.5 * (q1 * u + q2 * v + q3 * w));
  ph[0] = u;
  ph[1] = v;
  ph[2] = w;
  ph[3] = p * ir * g.inv_R;
}

// the conservative state with density 1 whose lifting variables are ph
__device__ __forceinline__ void encode_vars(const double ph[4], const Gas& g, double* o, int st) {
  o[0] = 1.0;
  o[st] = ph[0];
  o[2 * st] = ph[1];
  o[3 * st] = ph[2];
  o[4 * st] = g.R * ph[3] * g.inv_gm1 + 0.5 * (ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2]);
}

}  // namespace dg
