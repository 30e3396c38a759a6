// Modal troubled-cell indicator of Persson & Peraire (2006), the detector that
// marks DG elements for the FV sub-cell shock capturing (GALAEXI Sec. 3.1).
//
// The indicator quantity q (rho, p or rho p) of an element is expanded in the
// orthonormal Legendre basis Lt_m = sqrt((2m+1)/2) P_m per direction, and
//   eta_e = sum_{max(a,b,c) = N} qh_abc^2 / sum_abc qh_abc^2,
// the share of the L2 energy that the truncation to degree N-1 in every
// direction removes.  The modes come from the node set's quadrature: on Gauss
// nodes (exact to degree 2N+1) qh_m = sum_i w_i Lt_m(x_i) q_i exactly; on LGL
// nodes (exact to 2N-1) the same sum is exact for m < N and the top mode's
// discrete norm is sum_i w_i Lt_N(x_i)^2 = (2N+1)/N, divided out.  One block
// per element (several for small N), the three directions as line sums of
// the n x n transform through shared memory, FP64 throughout (eta decides the
// flag), a fixed-order reduction per element.
//
// Automatic DG/FV switching (switch_mask): the flag array is the FV mask of
// the context, updated before each evaluation of R(U): an element becomes an
// FV element where log10 eta > the upper threshold or where its nodal state
// is not admissible (density or pressure not positive at some node), a DG
// element where log10 eta < the lower threshold and every node is admissible,
// and otherwise keeps its representation.  The nodal polynomial of an FV
// element's sub-cell means can leave the admissible states where the means do
// not; the rule keeps such an element off the DG operator.
#include <cmath>
#include <vector>

#include "dg_stage.cuh"

namespace dg {

// Orthonormal Legendre value sqrt((2m+1)/2) P_m(x).
static double lt_value(int m, double x) {
  double a = 1.0, b = x;
  if (m == 0) return std::sqrt(0.5);
  for (int k = 1; k < m; ++k) {
    const double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
    a = b;
    b = c;
  }
  return std::sqrt((2.0 * m + 1.0) / 2.0) * b;
}

// Host table T[m][i]: qh_m = sum_i T[m][i] q_i for the node set (x, w).
void modal_table(int N, const std::vector<double>& x, const std::vector<double>& w, bool lobatto,
                 std::vector<double>& T) {
  const int n = N + 1;
  T.assign((size_t)n * n, 0.0);
  for (int m = 0; m < n; ++m) {
    const double g = (lobatto && m == N) ? (2.0 * N + 1.0) / N : 1.0;
    for (int i = 0; i < n; ++i) T[(size_t)m * n + i] = w[i] * lt_value(m, x[i]) / g;
  }
}

template <int N>
__global__ void __launch_bounds__(Shape<N>::THREADS)
k_indicator(const double* __restrict__ U, const double* __restrict__ T, int E, Gas g, int var, double log_thresh,
            double* __restrict__ eta, int* __restrict__ flag, bool switch_mask, double log_low,
            const int* __restrict__ pin) {
  using S = Shape<N>;
  constexpr int n = S::n, P = S::P, EPB = S::EPB;
  __shared__ double sT[n * n];
  __shared__ double s0[EPB * P], s1[EPB * P];
  __shared__ int s_bad[EPB];
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  const int e = blockIdx.x * EPB + le;
  const bool active = e < E;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sT[t] = T[t];
  if (id == 0) s_bad[le] = 0;
  double q = 0.0;
  bool bad = false;
  if (active) {
    const double* u = U + (size_t)e * 5 * P + id;
    const double rho = u[0], ir = rcp_op(rho);
    const double p = g.gm1 * (u[4 * P] - 0.5 * ir * (u[P] * u[P] + u[2 * P] * u[2 * P] + u[3 * P] * u[3 * P]));
    q = var == 0 ? rho : (var == 1 ? p : rho * p);
    bad = !(rho > 0.0 && p > 0.0);
  }
  __syncthreads();   // s_bad cleared
  if (bad) s_bad[le] = 1;
  double* q0 = s0 + le * P;
  double* q1 = s1 + le * P;
  q0[id] = q;
  __syncthreads();
  const int i = id % n, j = (id / n) % n, k = id / (n * n);
  // xi: (a = i, j, k) <- sum_i' T[a][i'] q(i', j, k)
  double t = 0.0;
#pragma unroll
  for (int m = 0; m < n; ++m) t = fma(sT[i * n + m], q0[m + n * (j + n * k)], t);
  q1[id] = t;
  __syncthreads();
  t = 0.0;
#pragma unroll
  for (int m = 0; m < n; ++m) t = fma(sT[j * n + m], q1[i + n * (m + n * k)], t);
  q0[id] = t;
  __syncthreads();
  t = 0.0;
#pragma unroll
  for (int m = 0; m < n; ++m) t = fma(sT[k * n + m], q0[i + n * (j + n * m)], t);
  // mode (a, b, c) = (i, j, k): its energy, and the same where the truncation
  // to degree N-1 removes it; per element a tree sum in a fixed order
  __syncthreads();
  q0[id] = active ? t * t : 0.0;
  q1[id] = (active && (i == N || j == N || k == N)) ? t * t : 0.0;
  __syncthreads();
  constexpr int H = P <= 1 ? 1 : (P <= 2 ? 1 : (P <= 4 ? 2 : (P <= 8 ? 4 : (P <= 16 ? 8 : (P <= 32 ? 16 :
                    (P <= 64 ? 32 : (P <= 128 ? 64 : (P <= 256 ? 128 : (P <= 512 ? 256 : 512)))))))));
#pragma unroll 1
  for (int h = H; h > 0; h >>= 1) {
    if (id < h && id + h < P) {
      q0[id] += q0[id + h];
      q1[id] += q1[id + h];
    }
    __syncthreads();
  }
  if (active && id == 0) {
    const double sa = q0[0], st = q1[0];
    const double r = sa > 0.0 ? st / sa : 0.0;
    if (eta) eta[e] = r;
    const double l = r > 0.0 ? log10(r) : -HUGE_VAL;
    if (switch_mask) {
      if (pin && pin[e]) flag[e] = 0;   // an element with a mortar face stays DG
      else if (l > log_thresh || s_bad[le]) flag[e] = 1;
      else if (l < log_low) flag[e] = 0;
    } else if (flag) {
      flag[e] = l > log_thresh ? 1 : 0;
    }
  }
}

template <int N>
static cudaError_t indicator_N(const Ctx& c, const double* U, const double* T, int var, double log_thresh,
                               double* eta, int* flag, cudaStream_t s, bool switch_mask, double log_low) {
  using S = Shape<N>;
  const int blocks = (c.E + S::EPB - 1) / S::EPB;
  k_indicator<N><<<blocks, S::THREADS, 0, s>>>(U, T, c.E, c.gas, var, log_thresh, eta, flag, switch_mask,
                                                log_low, switch_mask ? c.d_fv_pin : nullptr);
  return cudaGetLastError();
}

cudaError_t launch_indicator(const Ctx& c, const double* U, int var, double log_thresh, double* eta, int* flag,
                             cudaStream_t s, bool switch_mask, double log_low) {
  switch (c.N) {
#define DG_IND_CASE(K) \
    case K: return indicator_N<K>(c, U, c.d_modal, var, log_thresh, eta, flag, s, switch_mask, log_low);
    DG_IND_CASE(1) DG_IND_CASE(2) DG_IND_CASE(3) DG_IND_CASE(4) DG_IND_CASE(5)
    DG_IND_CASE(6) DG_IND_CASE(7) DG_IND_CASE(8) DG_IND_CASE(9)
#undef DG_IND_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fv_switch(const Ctx& c, const double* U, cudaStream_t s) {
  if (!c.fv_switch) return cudaSuccess;
  cudaError_t e = launch_indicator(c, U, c.fv_sw_var, c.fv_sw_up, nullptr, c.d_fv_mask, s, true, c.fv_sw_low);
  if (e == cudaSuccess) e = launch_fv_lists(c, s);
  return e;
}

}  // namespace dg
