// Diagnostics and set-up kernels: LGL-quadrature volume integrals (GALAEXI
// Sec. 4.2: kinetic energy, dissipation from the vorticity), the explicit time
// step of Sec. 3.1 (CFL and viscous limits), built-in initial states, clock.
// Reductions are two-pass and deterministic: fixed-size blocks write partials,
// one block folds them in a fixed order.
#include "dg_physics.cuh"

namespace dg {

constexpr int kRedThreads = 256;
constexpr int kRedVals = kRedValues;   // 5 conserved totals, volume, sum rho|u|^2, sum |omega|^2, min p

template <int THREADS, int V>
__device__ void block_reduce(double (&v)[V], const bool (&is_min)[V], double* out) {
  __shared__ double sh[V][THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < V; ++a) {
    double x = v[a];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = is_min[a] ? fmin(x, y) : x + y;
    }
    if (lane == 0) sh[a][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < V; ++a) {
      double x = sh[a][0];
      for (int w = 1; w < THREADS / 32; ++w) x = is_min[a] ? fmin(x, sh[a][w]) : x + sh[a][w];
      out[a] = x;
    }
  }
}

template <int N>
__global__ void __launch_bounds__(kRedThreads)
k_integrals(const double* __restrict__ U, const double* __restrict__ J, const double* __restrict__ grad,
            const double* __restrict__ w, double* __restrict__ part, int E, Gas gas) {
  const double gm1 = gas.gm1;
  constexpr int n = N + 1, P = n * n * n;
  double v[kRedVals] = {0, 0, 0, 0, 0, 0, 0, 0, 1e300};
  const bool is_min[kRedVals] = {false, false, false, false, false, false, false, false, true};
  const long total = (long)E * P;
  for (long t = (long)blockIdx.x * kRedThreads + threadIdx.x; t < total; t += (long)gridDim.x * kRedThreads) {
    const int e = (int)(t / P), id = (int)(t % P);
    const int i = id % n, j = (id / n) % n, k = id / (n * n);
    const double wq = w[i] * w[j] * w[k] * J[t];
    double q[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) q[c] = U[((size_t)e * 5 + c) * P + id];
#pragma unroll
    for (int c = 0; c < 5; ++c) v[c] += wq * q[c];
    v[5] += wq;
    const double ir = 1.0 / q[0];
    const double m2 = q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    v[6] += wq * m2 * ir;
    const double* g = grad + (size_t)e * 12 * P + id;
    const double o0 = g[7 * P] - g[5 * P];   // dw/dy - dv/dz
    const double o1 = g[2 * P] - g[6 * P];   // du/dz - dw/dx
    const double o2 = g[3 * P] - g[1 * P];   // dv/dx - du/dy
    const double p = gm1 * (q[4] - 0.5 * m2 * ir);
    // mu(T) / mu_ref; Sutherland's law needs T > 0: a node with T <= 0 (only
    // inside an FV element, whose nodal polynomial of admissible sub-cell
    // means may leave the admissible states) adds nothing; NaN stays NaN
    const double Tn = p * ir * gas.inv_R;
    const double sf = (gas.visc_law == DG_VISC_SUTHERLAND && Tn <= 0.0) ? 0.0 : visc_factor<double>(gas, Tn);
    v[7] += wq * sf * (o0 * o0 + o1 * o1 + o2 * o2);
    v[8] = fmin(v[8], p);
  }
  block_reduce<kRedThreads, kRedVals>(v, is_min, part + (size_t)blockIdx.x * kRedVals);
}

__global__ void __launch_bounds__(kRedThreads) k_fold(double* part, int nblk, int nval, const int* min_mask) {
  // one block folds nblk rows of nval values; row nblk receives the result
  __shared__ double sh[kRedThreads];
  for (int a = 0; a < nval; ++a) {
    const bool mn = (min_mask[0] >> a) & 1;
    double x = mn ? 1e300 : 0.0;
    for (int b = threadIdx.x; b < nblk; b += kRedThreads) {
      const double y = part[(size_t)b * nval + a];
      x = mn ? fmin(x, y) : x + y;
    }
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] = mn ? fmin(sh[threadIdx.x], sh[threadIdx.x + o]) : sh[threadIdx.x] + sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)nblk * nval + a] = sh[0];
    __syncthreads();
  }
}

// Per-node explicit-time-step limits: convective sum_d (|u . Ja^d| + c |Ja^d|)/J
// and viscous mu_eff sum_d |Ja^d|^2 / J^2, maxima over all nodes.
template <int N>
__global__ void __launch_bounds__(kRedThreads)
k_dt(const double* __restrict__ U, const double* __restrict__ metrics, double* __restrict__ part, int E, Gas g,
     const int* __restrict__ fv_mask) {
  constexpr int n = N + 1, P = n * n * n;
  double v[2] = {0.0, 0.0};
  const bool is_min[2] = {false, false};
  const long total = (long)E * P;
  for (long t = (long)blockIdx.x * kRedThreads + threadIdx.x; t < total; t += (long)gridDim.x * kRedThreads) {
    const int e = (int)(t / P), id = (int)(t % P);
    double q[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) q[c] = U[((size_t)e * 5 + c) * P + id];
    const double ir = 1.0 / q[0];
    const double u = q[1] * ir, vv = q[2] * ir, w = q[3] * ir;
    const double p = g.gm1 * (q[4] - 0.5 * (q[1] * u + q[2] * vv + q[3] * w));
    // an FV element's nodes hold the polynomial of its sub-cell means, which
    // may leave the admissible states where the means do not: such nodes do
    // not enter (the DG bound used here is below the sub-cells' own one)
    if (fv_mask && fv_mask[e] && !(q[0] > 0.0 && p > 0.0)) continue;
    const double cs = sqrt(g.gamma * p * ir);
    const double* mt = metrics + (size_t)e * 10 * P + id;
    const double iJ = mt[9 * P];
    double lc = 0.0, lv = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double a0 = mt[(d * 3) * P], a1 = mt[(d * 3 + 1) * P], a2 = mt[(d * 3 + 2) * P];
      const double a2n = a0 * a0 + a1 * a1 + a2 * a2;
      lc += (fabs(u * a0 + vv * a1 + w * a2) + cs * sqrt(a2n)) * iJ;
      lv += a2n * iJ * iJ;
    }
    const double mu_eff = fmax(4.0 / 3.0, g.gamma / g.Pr) * g.mu * visc_factor<double>(g, p * ir * g.inv_R) * ir;
    // fmax drops NaN operands: a non-finite node (or a negative pressure,
    // whose sound speed is NaN) enters as +Inf so that the host sees it
    const double vl = mu_eff * lv;
    v[0] = fmax(v[0], isnan(lc) ? HUGE_VAL : lc);
    v[1] = fmax(v[1], isnan(vl) ? HUGE_VAL : vl);
  }
  // max-reduce through the generic block reducer (sum slots reused as max)
  __shared__ double sh[2][kRedThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int a = 0; a < 2; ++a) {
    double x = v[a];
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if (lane == 0) sh[a][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int a = 0; a < 2; ++a) {
      double x = sh[a][0];
      for (int w2 = 1; w2 < kRedThreads / 32; ++w2) x = fmax(x, sh[a][w2]);
      part[(size_t)blockIdx.x * 2 + a] = x;
    }
  (void)is_min;
}

__global__ void k_fold_max(double* part, int nblk) {
  __shared__ double sh[2][kRedThreads];
  double a = 0.0, b = 0.0;
  for (int t = threadIdx.x; t < nblk; t += kRedThreads) {
    a = fmax(a, part[(size_t)t * 2]);
    b = fmax(b, part[(size_t)t * 2 + 1]);
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  __syncthreads();
  for (int o = kRedThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + o]);
      sh[1][threadIdx.x] = fmax(sh[1][threadIdx.x], sh[1][threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { part[(size_t)nblk * 2] = sh[0][0]; part[(size_t)nblk * 2 + 1] = sh[1][0]; }
}

// Taylor-Green vortex (Sec. 4.2, Eq. 6) in rho0 = U0 = L = R = 1 units and the
// density-wave manufactured solution.
__global__ void k_initial(const double* __restrict__ X, double* __restrict__ U, int E, int P, int kind,
                          double prm0, Gas g) {
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)E * P) return;
  const int e = (int)(t / P), id = (int)(t % P);
  const double x = X[((size_t)e * 3 + 0) * P + id], y = X[((size_t)e * 3 + 1) * P + id],
               z = X[((size_t)e * 3 + 2) * P + id];
  double rho, u, v, w, p;
  if (kind == DG_IC_TGV) {
    const double p0 = prm0;
    u = sin(x) * cos(y) * cos(z);
    v = -cos(x) * sin(y) * cos(z);
    w = 0.0;
    p = p0 + (cos(2.0 * x) + cos(2.0 * y)) * (2.0 + cos(2.0 * z)) / 16.0;
    rho = p / (g.R * p0);
  } else {
    rho = 2.0 + g.mms_amp * sinpi(x + y + z - prm0);
    u = v = w = 1.0;
    p = 1.0;
  }
  double* o = U + (size_t)e * 5 * P + id;
  o[0] = rho;
  o[P] = rho * u;
  o[2 * P] = rho * v;
  o[3 * P] = rho * w;
  o[4 * P] = p * g.inv_gm1 + 0.5 * rho * (u * u + v * v + w * w);
}

// sin and cos of pi (x + y + z) at every node, for the manufactured source.
__global__ void k_mms_phase(const double* __restrict__ X, double* __restrict__ ph, int E, int P) {
  const long tot = (long)E * P;
  for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (long)gridDim.x * blockDim.x) {
    const long e = t / P, id = t - e * P;
    const double s = X[(e * 3 + 0) * P + id] + X[(e * 3 + 1) * P + id] + X[(e * 3 + 2) * P + id];
    sincospi(s, &ph[(e * 2) * P + id], &ph[(e * 2 + 1) * P + id]);
  }
}

__global__ void k_set_clock(double* clock, double t, double dt) { clock[0] = t; clock[1] = dt; }
__global__ void k_clock_advance(double* clock) { clock[0] += clock[1]; }

static int red_blocks(const Ctx& c) {
  const long total = (long)c.E * c.P;
  long b = (total + kRedThreads - 1) / kRedThreads;
  return (int)(b < c.red_len ? b : c.red_len);
}

template <int N>
static cudaError_t integrals_N(Ctx& c, const double* U, double* d_w, cudaStream_t s) {
  const int nb = red_blocks(c);
  k_integrals<N><<<nb, kRedThreads, 0, s>>>(U, c.d_J, (const double*)c.d_grad, d_w, c.d_red, c.E, c.gas);
  return cudaGetLastError();
}

template <int N>
static cudaError_t dt_N(Ctx& c, const double* U, cudaStream_t s) {
  const int nb = red_blocks(c);
  k_dt<N><<<nb, kRedThreads, 0, s>>>(U, c.d_metrics, c.d_red, c.E, c.gas, c.fv_on ? c.d_fv_mask : nullptr);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_fold_max<<<1, kRedThreads, 0, s>>>(c.d_red, nb);
  return cudaGetLastError();
}

cudaError_t launch_integrals(Ctx& c, const double* U, cudaStream_t s) {
  cudaError_t err = launch_lift_fp64(c, U, s);   // diagnostics stay FP64 on every path
  if (err != cudaSuccess) return err;
  double* d_w = c.d_w;
  switch (c.N) {
    case 1: err = integrals_N<1>(c, U, d_w, s); break;
    case 2: err = integrals_N<2>(c, U, d_w, s); break;
    case 3: err = integrals_N<3>(c, U, d_w, s); break;
    case 4: err = integrals_N<4>(c, U, d_w, s); break;
    case 5: err = integrals_N<5>(c, U, d_w, s); break;
    case 6: err = integrals_N<6>(c, U, d_w, s); break;
    case 7: err = integrals_N<7>(c, U, d_w, s); break;
    case 8: err = integrals_N<8>(c, U, d_w, s); break;
    case 9: err = integrals_N<9>(c, U, d_w, s); break;
    default: err = cudaErrorInvalidValue;
  }
  if (err != cudaSuccess) return err;
  k_fold<<<1, kRedThreads, 0, s>>>(c.d_red, red_blocks(c), kRedVals, c.d_minmask);
  return cudaGetLastError();
}

cudaError_t launch_max_dt(Ctx& c, const double* U, double, double, cudaStream_t s) {
  switch (c.N) {
    case 1: return dt_N<1>(c, U, s);
    case 2: return dt_N<2>(c, U, s);
    case 3: return dt_N<3>(c, U, s);
    case 4: return dt_N<4>(c, U, s);
    case 5: return dt_N<5>(c, U, s);
    case 6: return dt_N<6>(c, U, s);
    case 7: return dt_N<7>(c, U, s);
    case 8: return dt_N<8>(c, U, s);
    case 9: return dt_N<9>(c, U, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_initial_state(Ctx& c, int kind, double prm0, double* U, cudaStream_t s) {
  const long tot = (long)c.E * c.P;
  k_initial<<<(int)((tot + 255) / 256), 256, 0, s>>>(c.d_X, U, c.E, c.P, kind, prm0, c.gas);
  return cudaGetLastError();
}

cudaError_t launch_mms_phase(Ctx& c, cudaStream_t s) {
  const long tot = (long)c.E * c.P;
  const long blocks = (tot + 255) / 256;
  k_mms_phase<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(c.d_X, c.d_mms, c.E, c.P);
  return cudaGetLastError();
}

cudaError_t launch_set_clock(double* clock, double t, double dt, cudaStream_t s) {
  k_set_clock<<<1, 1, 0, s>>>(clock, t, dt);
  return cudaGetLastError();
}

cudaError_t launch_clock_advance(double* clock, cudaStream_t s) {
  k_clock_advance<<<1, 1, 0, s>>>(clock);
  return cudaGetLastError();
}

int reduction_rows(const Ctx& c) { return red_blocks(c); }

}  // namespace dg
