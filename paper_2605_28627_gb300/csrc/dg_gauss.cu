// Legendre-Gauss node set (GALAEXI Sec. 3.1: the weak form, Eq. 2, and the
// weak BR1 lifting, Eq. 3, collocated at the N+1 Gauss points per direction):
// the standard DGSEM without a split form.  Per stage four kernels:
//   k_prolong_lg  face values of U, from each element's own nodes,
//   k_lift_lg     weak lifting -> g at the nodes and its face values,
//   k_face_lg     Riemann flux and BR1 viscous average at the Gauss face points,
//   k_volume_lg   weak volume and surface terms, 1/J, source, LSERK update.
// No node lies on a face: every node receives a surface term from each of the
// six faces, weighted by l_i(+-1)/w_i along its line.
//
// Geometry: the curl-form metric terms of degree N are built on the LGL nodes
// (k_geometry), then this polynomial is evaluated at the Gauss nodes and at the
// Gauss points of each face.  Both sides of a face see the same face values of
// the polynomial, and its discrete metric identities keep a uniform flow
// uniform.  FP64 only.
#include "dg_gauss.cuh"

#include <cmath>

namespace dg {

// P_n(x) and P_n'(x) for |x| < 1 by the three-term recurrence.
static void legendre_pn(int n, double x, double& p, double& dp) {
  double a = 1.0, b = x;
  for (int k = 2; k <= n; ++k) {
    const double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  p = n == 0 ? 1.0 : b;
  dp = n == 0 ? 0.0 : n * (a - x * b) / (1.0 - x * x);
}

// Host table of the Gauss basis of degree N; xl are the LGL nodes of degree N.
void gauss_table(int N, const std::vector<double>& xl, std::vector<double>& tab, std::vector<double>* gx,
                 std::vector<double>* gw) {
  const int n = N + 1;
  std::vector<double> x(n), w(n), D((size_t)n * n), c(n), lm(n), lp(n);
  for (int k = 0; k < (n + 1) / 2; ++k) {
    // k-th largest root of P_n, Newton from the standard trigonometric guess
    double t = std::cos(M_PI * (k + 0.75) / (n + 0.5));
    for (int it = 0; it < 60; ++it) {
      double p, dp;
      legendre_pn(n, t, p, dp);
      const double step = p / dp;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    x[n - 1 - k] = t;
    x[k] = -t;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
  for (int j = 0; j < n; ++j) {
    double p, dp;
    legendre_pn(n, x[j], p, dp);
    w[j] = 2.0 / ((1.0 - x[j] * x[j]) * dp * dp);
    c[j] = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) c[j] *= x[j] - x[k];
  }
  for (int i = 0; i < n; ++i) {
    double row = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const double dij = c[i] / (c[j] * (x[i] - x[j]));
      D[(size_t)i * n + j] = dij;
      row += dij;
    }
    D[(size_t)i * n + i] = -row;
  }
  for (int j = 0; j < n; ++j) {
    double a = 1.0, b = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) {
        a *= (-1.0 - x[k]) / (x[j] - x[k]);
        b *= (1.0 - x[k]) / (x[j] - x[k]);
      }
    lm[j] = a;
    lp[j] = b;
  }
  if (gx) *gx = x;
  if (gw) *gw = w;
  tab.assign(GaussTab::size(n), 0.0);
  for (int r = 0; r < n; ++r)
    for (int m = 0; m < n; ++m) tab[GaussTab::Dw(n) + r * n + m] = (w[m] / w[r]) * D[(size_t)m * n + r];
  for (int i = 0; i < n; ++i) {
    tab[GaussTab::lmw(n) + i] = lm[i] / w[i];
    tab[GaussTab::lpw(n) + i] = lp[i] / w[i];
    tab[GaussTab::lm(n) + i] = lm[i];
    tab[GaussTab::lp(n) + i] = lp[i];
    tab[GaussTab::w(n) + i] = w[i];
    for (int j = 0; j < n; ++j) {
      double l = 1.0;
      for (int k = 0; k < n; ++k)
        if (k != j) l *= (x[i] - xl[k]) / (xl[j] - xl[k]);
      tab[GaussTab::V(n) + i * n + j] = l;
    }
  }
}

// Spectral radius of the 1-D upwind DG operator of u_t + u_x = 0 on K periodic
// elements of reference length 2, weak form with the node set's own
// quadrature: du_i/dt = sum_m (w_m/w_i) D_mi u_m - (l_i(1) u_R - l_i(-1) u_L^-)/w_i.
// Estimated from the growth rate of A^k x (Gelfand's formula) after a
// transient, which converges for the complex-conjugate dominant pairs of this
// operator where plain power iteration oscillates.
static double dg1d_spectral_radius(int n, const std::vector<double>& w, const std::vector<double>& D,
                                   const std::vector<double>& lm, const std::vector<double>& lp) {
  const int K = 8, M = n * K;
  std::vector<double> A((size_t)M * M, 0.0);
  for (int e = 0; e < K; ++e) {
    const int el = (e + K - 1) % K;
    for (int i = 0; i < n; ++i)
      for (int m = 0; m < n; ++m) {
        double* row = &A[(size_t)(e * n + i) * M];
        row[e * n + m] += (w[m] / w[i]) * D[(size_t)m * n + i] - lp[i] / w[i] * lp[m];
        row[el * n + m] += lm[i] / w[i] * lp[m];
      }
  }
  std::vector<double> x(M), y(M);
  for (int a = 0; a < M; ++a) x[a] = 1.0 + 0.37 * std::sin(1.3 * a + 0.2);   // generic start
  double logsum = 0.0;
  const int k0 = 300, k1 = 1500;
  for (int k = 0; k < k1; ++k) {
    double nrm = 0.0;
    for (int a = 0; a < M; ++a) {
      double s = 0.0;
      for (int b = 0; b < M; ++b) s += A[(size_t)a * M + b] * x[b];
      y[a] = s;
      nrm += s * s;
    }
    nrm = std::sqrt(nrm);
    if (k >= k0) logsum += std::log(nrm);
    for (int a = 0; a < M; ++a) x[a] = y[a] / nrm;
  }
  return std::exp(logsum / (k1 - k0));
}

// Factor on the time step of the Gauss-node operator: the bound of max_dt
// (set for LGL nodes) times rho_LGL / rho_LG of the 1-D operators, so that both
// node sets keep the same stability margin at the same CFL number (about 0.37
// at N = 1 rising to 0.57 at N = 9; without it the Gauss operator is unstable
// at CFL 0.9 for high N).
double gauss_dt_factor(int N, const std::vector<double>& xl, const std::vector<double>& wl,
                       const std::vector<double>& Dl, const std::vector<double>& tab) {
  const int n = N + 1;
  std::vector<double> lmL(n, 0.0), lpL(n, 0.0);
  lmL[0] = 1.0;
  lpL[N] = 1.0;
  std::vector<double> wG(n), DG((size_t)n * n), lmG(n), lpG(n);
  for (int i = 0; i < n; ++i) {
    wG[i] = tab[GaussTab::w(n) + i];
    lmG[i] = tab[GaussTab::lm(n) + i];
    lpG[i] = tab[GaussTab::lp(n) + i];
  }
  // D_{m r} back from the weak table (w_m / w_r) D_{m r}
  for (int r = 0; r < n; ++r)
    for (int m = 0; m < n; ++m) DG[(size_t)m * n + r] = tab[GaussTab::Dw(n) + r * n + m] * wG[r] / wG[m];
  (void)xl;
  return dg1d_spectral_radius(n, wl, Dl, lmL, lpL) / dg1d_spectral_radius(n, wG, DG, lmG, lpG);
}

// ---------------------------------------------------------------------------
// Geometry on Gauss points

// Master-side unit normal and surface element at the Gauss face points:
// n sJ = (2s-1) J a^d of the LGL polynomial at (p, q), interpolated from the
// LGL nodes of the face.  Reads the LGL metrics, so it runs before they are
// replaced by their Gauss values.
template <int N>
__global__ void k_face_geometry_lg(const FaceInfo* __restrict__ faces, const double* __restrict__ metrics,
                                   const double* __restrict__ tab, double* __restrict__ facegeo, int F, int E) {
  constexpr int n = N + 1, P = n * n * n, NN = n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)F * NN) return;
  const int f = (int)(gid / NN), pq = (int)(gid % NN);
  const int p = pq % n, q = pq / n;
  const FaceInfo fi = faces[f];
  const int e = dg_idx(fi.master >> 3, E, kSiteGaussFace), lf = fi.master & 7, d = lf >> 1;
  const double sg = (lf & 1) ? 1.0 : -1.0;
  const double* V = tab + GaussTab::V(n);
  double nv[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < n; ++a) {
      const double wab = V[p * n + a] * V[q * n + b];
      const double* mt = metrics + (size_t)e * 10 * P + face_node<n>(lf, a, b);
      for (int l = 0; l < 3; ++l) nv[l] = fma(wab, mt[(d * 3 + l) * P], nv[l]);
    }
  const double nx = sg * nv[0], ny = sg * nv[1], nz = sg * nv[2];
  const double sJ = sqrt(nx * nx + ny * ny + nz * nz);
  double* fg = facegeo + (size_t)f * 4 * NN + pq;
  fg[0] = nx / sJ;
  fg[NN] = ny / sJ;
  fg[2 * NN] = nz / sJ;
  fg[3 * NN] = sJ;
}

// One field of an element from LGL to Gauss nodes: three sweeps of V through
// shared memory (a -> b -> a -> b); the result is left in b.
template <int n>
__device__ __forceinline__ void to_gauss_3d(const double* __restrict__ V, double* a, double* b, int id) {
  constexpr int P = n * n * n;
  const int i = id % n, j = (id / n) % n, k = id / (n * n);
  double s = 0.0;
  if (id < P)
    for (int m = 0; m < n; ++m) s = fma(V[i * n + m], a[vidx<n>(m, j, k)], s);
  __syncthreads();
  if (id < P) b[id] = s;
  __syncthreads();
  s = 0.0;
  if (id < P)
    for (int m = 0; m < n; ++m) s = fma(V[j * n + m], b[vidx<n>(i, m, k)], s);
  __syncthreads();
  if (id < P) a[id] = s;
  __syncthreads();
  s = 0.0;
  if (id < P)
    for (int m = 0; m < n; ++m) s = fma(V[k * n + m], a[vidx<n>(i, j, m)], s);
  __syncthreads();
  if (id < P) b[id] = s;
  __syncthreads();
}

// In place: node positions, metric terms and Jacobian of each element from
// the LGL nodes to the Gauss nodes (the Jacobian from the interpolated
// derivatives of the LGL geometry, taken on coordinates relative to the
// element's first node).  One block of P threads per element.
template <int N>
__global__ void __launch_bounds__((N + 1) * (N + 1) * (N + 1))
k_geometry_to_gauss(double* __restrict__ X, double* __restrict__ metrics, double* __restrict__ Jout,
                    const double* __restrict__ Dl, const double* __restrict__ tab, int* __restrict__ bad, int E) {
  constexpr int n = N + 1, P = n * n * n;
  extern __shared__ double sm[];
  double* sX = sm;            // [3][P] LGL positions, relative to the first node
  double* sA = sX + 3 * P;    // sweep buffers
  double* sB = sA + P;
  __shared__ double sV[n * n], sD[n * n];
  const int e = blockIdx.x, id = threadIdx.x;
  const int i = id % n, j = (id / n) % n, k = id / (n * n);
  for (int t = id; t < n * n; t += blockDim.x) {
    sV[t] = tab[GaussTab::V(n) + t];
    sD[t] = Dl[t];
  }
  double x0[3];
  for (int c = 0; c < 3; ++c) {
    x0[c] = X[((size_t)e * 3 + c) * P];
    sX[c * P + id] = X[((size_t)e * 3 + c) * P + id] - x0[c];
  }
  __syncthreads();
  // positions
  for (int c = 0; c < 3; ++c) {
    sA[id] = sX[c * P + id];
    __syncthreads();
    to_gauss_3d<n>(sV, sA, sB, id);
    X[((size_t)e * 3 + c) * P + id] = sB[id] + x0[c];
  }
  // metric terms (rows 0..8); row 9 (1/J) is written below
  for (int r = 0; r < 9; ++r) {
    sA[id] = metrics[((size_t)e * 10 + r) * P + id];
    __syncthreads();
    to_gauss_3d<n>(sV, sA, sB, id);
    metrics[((size_t)e * 10 + r) * P + id] = sB[id];
  }
  // Jacobian: derivatives of the LGL interpolant, evaluated at the Gauss nodes
  double A[3][3];
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      const int r = d == 0 ? i : (d == 1 ? j : k);
      double s = 0.0;
      for (int m = 0; m < n; ++m) {
        const int mid = d == 0 ? vidx<n>(m, j, k) : (d == 1 ? vidx<n>(i, m, k) : vidx<n>(i, j, m));
        s = fma(sD[r * n + m], sX[c * P + mid], s);
      }
      sA[id] = s;
      __syncthreads();
      to_gauss_3d<n>(sV, sA, sB, id);
      A[c][d] = sB[id];
    }
  const double Jv = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                    A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                    A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (!(Jv > 0.0)) atomicExch(bad, 1);
  Jout[(size_t)e * P + id] = Jv;
  metrics[((size_t)e * 10 + 9) * P + id] = 1.0 / Jv;
}

// ---------------------------------------------------------------------------
// Stage kernels

// Face values of U: Uf[e][f][v][p + n q] = sum_i l_i(+-1) U(line of (p, q)),
// in the operator type R (the FP32 operator prolongs FP32 values: an FP64
// prolongation would take the FP64 pipe for more than the whole FP32 stage).
// The FP32 operator prolongs the energy as E - E_ref (E_ref = p_ref/(gamma-1),
// the difference taken in FP64 per node), so that the face values keep the
// digits of the pressure fluctuation at low Mach numbers; its readers add
// E_ref back where they need the whole energy.
template <int N, int EPB, typename R = double>
__global__ void __launch_bounds__(Shape<N, EPB>::THREADS)
k_prolong_lg(const double* __restrict__ U, const double* __restrict__ tab, R* __restrict__ Uf, int E, double E_off) {
  using S = Shape<N, EPB>;
  constexpr int n = S::n, P = S::P, NN = n * n;
  extern __shared__ __align__(16) unsigned char prolong_raw[];
  R* sm = reinterpret_cast<R*>(prolong_raw);   // [EPB][5][P]
  __shared__ R sl[2 * n];                       // l_i(-1), l_i(+1)
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  const int e = blockIdx.x * EPB + le;
  for (int t = threadIdx.x; t < 2 * n; t += blockDim.x) sl[t] = to_op<R>(tab[GaussTab::lm(n) + t]);
  if (e < E)
    for (int v = 0; v < 5; ++v) sm[(le * 5 + v) * P + id] = to_op<R>(U[((size_t)e * 5 + v) * P + id] - (v == 4 ? E_off : 0.0));
  __syncthreads();
  if (e >= E) return;
  for (int o = id; o < 30 * NN; o += P) {
    const int f = o / (5 * NN), r = o - f * 5 * NN, v = r / NN, pq = r - v * NN;
    const int p = pq % n, q = pq / n, d = f >> 1;
    const R* l = sl + (f & 1) * n;
    const R* u = sm + (le * 5 + v) * P;
    R s = R(0);
#pragma unroll
    for (int i = 0; i < n; ++i) s = fma(l[i], u[line_node<n>(d, i, p, q)], s);
    Uf[((size_t)e * 6 + f) * 5 * NN + (size_t)v * NN + pq] = s;
  }
}

// Lifting variables (u, v, w, T) of a state given with stride st, in R; p_off
// is added to the pressure (p_ref for face values that carry E - E_ref).
template <typename R, typename Q>
__device__ __forceinline__ void state_phi(const Q* q, int st, const Gas& g, R ph[4], R p_off = R(0)) {
  const R rho = to_op<R>(q[0]), ir = rcp_op(rho);
  const R m0 = to_op<R>(q[st]), m1 = to_op<R>(q[2 * st]), m2 = to_op<R>(q[3 * st]);
  const R u = m0 * ir, v = m1 * ir, w = m2 * ir;
  const R p = p_off + gsel<R>(g.gm1, g.f_gm1) * (to_op<R>(q[4 * st]) - R(0.5) * (m0 * u + m1 * v + m2 * w));
  ph[0] = u;
  ph[1] = v;
  ph[2] = w;
  ph[3] = p * ir * gsel<R>(g.inv_R, g.f_inv_R);
}

template <int N, int EPB, typename R = double>
constexpr size_t lift_lg_smem() {
  constexpr int n = N + 1, P = n * n * n, NN = n * n;
  return sizeof(R) * EPB * (16 * P + 72 * NN);
}

// Weak BR1 lifting (Eq. 3): J g_l,i = sum_faces l_{i_d}(+-1)/w_{i_d} phi* (n_l sJ)
//   - sum_d sum_m (w_m/w_{i_d}) D_{m i_d} (phi Ja^d_l)_m, phi* the face average;
// then the face values of g for the face kernel.  R: the operator type (the
// face values Uf, the metric terms, face geometry, g and its face values gf).
// MORTAR: a face whose neighbour entry is negative is a mortar side,
// whose neighbour face state is mvirt[-1 - entry][5][NN] in its own point order.
template <int N, int EPB, bool MORTAR = false, typename R = double>
__global__ void __launch_bounds__(Shape<N, EPB>::THREADS)
k_lift_lg(const double* __restrict__ U, const R* __restrict__ Uf, const R* __restrict__ metrics,
          const R* __restrict__ facegeo, const int* __restrict__ elem_face, const int* __restrict__ elem_nbr,
          const double* __restrict__ tab, R* __restrict__ grad, R* __restrict__ gf, int E, int F, Gas g,
          const double* __restrict__ mvirt, int n_mortar) {
  using S = Shape<N, EPB>;
  constexpr int n = S::n, P = S::P, NN = n * n, PER = 16 * P + 72 * NN;
  extern __shared__ __align__(16) unsigned char lift_lg_raw[];
  R* sm = reinterpret_cast<R*>(lift_lg_raw);
  __shared__ R sDw[n * n], sT[4 * n];   // weak D; l(-1)/w, l(+1)/w, l(-1), l(+1)
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  const int e = blockIdx.x * EPB + le;
  const bool active = e < E;
  R* sphi = sm + le * PER;     // [4][P]
  R* sprod = sphi + 4 * P;     // [12][P]
  R* sS = sprod + 12 * P;      // [6][12][NN]: phi* (n_l sJ) with the outward normal
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sDw[t] = to_op<R>(tab[GaussTab::Dw(n) + t]);
  for (int t = threadIdx.x; t < 4 * n; t += blockDim.x) sT[t] = to_op<R>(tab[GaussTab::lmw(n) + t]);
  R Ja[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, iJ = R(0);
  if (active) {
    R ph[4];
    state_phi<R>(U + (size_t)e * 5 * P + id, P, g, ph);
    for (int a = 0; a < 4; ++a) sphi[a * P + id] = ph[a];
    const R* mt = metrics + (size_t)e * 10 * P + id;
#pragma unroll
    for (int r = 0; r < 9; ++r) Ja[r] = mt[r * P];
    iJ = mt[9 * P];
    for (int o = id; o < 6 * NN; o += P) {
      const int f = o / NN, pq = o - f * NN, p = pq % n, q = pq / n;
      const int code = elem_face[e * 6 + f], nb = elem_nbr[e * 6 + f];
      const int fid = dg_idx(code >> 4, F, kSiteGaussLift);
      int p2, q2;
      apply_flip<n>(code & 7, p, q, p2, q2);
      const int pq2 = p2 + n * q2;
      R pm[4], pn[4];
      const R poff = sizeof(R) == 4 ? gsel<R>(g.p_ref, g.f_p_ref) : R(0);   // face values carry E - E_ref
      state_phi<R>(Uf + ((size_t)e * 6 + f) * 5 * NN + pq, NN, g, pm, poff);
      bool done = false;
      if constexpr (MORTAR) {
        if (nb < 0) {
          state_phi<R>(mvirt + (size_t)dg_idx(-1 - nb, 5L * n_mortar, kSiteMortar) * 5 * NN + pq, NN, g, pn);
          done = true;
        }
      }
      if (!done) {
        const int e2 = dg_idx(nb >> 3, E, kSiteGaussLift), f2 = nb & 7;
        state_phi<R>(Uf + ((size_t)e2 * 6 + f2) * 5 * NN + pq2, NN, g, pn, poff);
      }
      const bool master = code & 8;
      const R* fg = facegeo + (size_t)fid * 4 * NN + (master ? pq : pq2);
      const R sJ = master ? fg[3 * NN] : -fg[3 * NN];
      const R ns[3] = {sJ * fg[0], sJ * fg[NN], sJ * fg[2 * NN]};
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const R star = R(0.5) * (pm[a] + pn[a]);
#pragma unroll
        for (int l = 0; l < 3; ++l) sS[(f * 12 + a * 3 + l) * NN + pq] = star * ns[l];
      }
    }
  }
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  R acc[12];
#pragma unroll
  for (int r = 0; r < 12; ++r) acc[r] = R(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    __syncthreads();
    if (active)
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int l = 0; l < 3; ++l) sprod[(a * 3 + l) * P + id] = sphi[a * P + id] * Ja[d * 3 + l];
    __syncthreads();
    if (active) {
      const int r = ijk[d];
      const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
      const int line0 = id - r * stride;
      for (int m = 0; m < n; ++m) {
        const R c = sDw[r * n + m];
        const int mid = line0 + m * stride;
#pragma unroll
        for (int al = 0; al < 12; ++al) acc[al] = fma(-c, sprod[al * P + mid], acc[al]);
      }
    }
  }
  if (active) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int r = ijk[d];
      const int pq = d == 0 ? j + n * k : (d == 1 ? i + n * k : i + n * j);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const R c = sT[s * n + r];
        const R* src = sS + ((2 * d + s) * 12) * NN + pq;
#pragma unroll
        for (int al = 0; al < 12; ++al) acc[al] = fma(c, src[al * NN], acc[al]);
      }
    }
  }
  __syncthreads();   // every thread is done with sprod
  if (active) {
    R* go = grad + (size_t)e * 12 * P + id;
#pragma unroll
    for (int al = 0; al < 12; ++al) {
      const R gv = acc[al] * iJ;
      go[al * P] = gv;
      sprod[al * P + id] = gv;
    }
  }
  __syncthreads();
  if (!active) return;
  for (int o = id; o < 72 * NN; o += P) {
    const int f = o / (12 * NN), r = o - f * 12 * NN, al = r / NN, pq = r - al * NN;
    const int p = pq % n, q = pq / n, d = f >> 1;
    const R* l = sT + (2 + (f & 1)) * n;
    R s = R(0);
#pragma unroll
    for (int m = 0; m < n; ++m) s = fma(l[m], sprod[al * P + line_node<n>(d, m, p, q)], s);
    gf[((size_t)e * 6 + f) * 12 * NN + (size_t)al * NN + pq] = s;
  }
}

// Surface flux at the Gauss face points of each master face, from both sides'
// face values of the state and of the lifted gradients.
// FVSKIP: faces with an FV sub-cell element on either side are left to the FV
// face kernel (fv_mask: [E], 1 for an FV element).
template <int N, bool FVSKIP, typename R = double>
__global__ void __launch_bounds__(128)
k_face_lg(const R* __restrict__ Uf, const R* __restrict__ gf, const FaceInfo* __restrict__ faces,
          const R* __restrict__ facegeo, R* __restrict__ fstar, int F, int E, Gas g,
          const int* __restrict__ fv_mask) {
  constexpr int n = N + 1, NN = n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)F * NN) return;
  const int f = (int)(gid / NN), pq = (int)(gid % NN);
  const int p = pq % n, q = pq / n;
  const FaceInfo fi = faces[f];
  const int eM = dg_idx(fi.master >> 3, E, kSiteGaussFace), fM = fi.master & 7;
  const int eS = dg_idx(fi.slave >> 3, E, kSiteGaussFace), fS = fi.slave & 7;
  if constexpr (FVSKIP) {
    if (fv_mask[eM] || fv_mask[eS]) return;
  }
  int p2, q2;
  apply_flip<n>(fi.flip, p, q, p2, q2);
  const int pq2 = p2 + n * q2;
  // the face states enter the flux core as FP64 values (exact widening of FP32
  // face values with the FP32 operator)
  double dL[5], dR[5];
  R gL[12], gR[12];
  const R* uM = Uf + ((size_t)eM * 6 + fM) * 5 * NN + pq;
  const R* uS = Uf + ((size_t)eS * 6 + fS) * 5 * NN + pq2;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    dL[v] = to_f64(uM[v * NN]);
    dR[v] = to_f64(uS[v * NN]);
  }
  if constexpr (sizeof(R) == 4) {   // the FP32 face values carry E - E_ref
    dL[4] += g.E_ref;
    dR[4] += g.E_ref;
  }
  const R* gM = gf + ((size_t)eM * 6 + fM) * 12 * NN + pq;
  const R* gS = gf + ((size_t)eS * 6 + fS) * 12 * NN + pq2;
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    gL[r] = gM[r * NN];
    gR[r] = gS[r * NN];
  }
  const R* fg = facegeo + (size_t)f * 4 * NN + pq;
  face_flux_core<R>(dL, dR, gL, gR, fg[0], fg[NN], fg[2 * NN], fg[3 * NN], g, fstar + (size_t)f * 5 * NN + pq, NN);
}

template <int N, int EPB, typename R = double>
constexpr size_t volume_lg_smem() {
  constexpr int n = N + 1, P = n * n * n, NN = n * n;
  return sizeof(R) * EPB * (15 * P + 30 * NN);
}

// Weak volume and surface terms (Eq. 2):
//   J U_t,i = - sum_faces l_{i_d}(+-1)/w_{i_d} F*_out + sum_d sum_m (w_m/w_{i_d}) D_{m i_d} Ft^d_m,
// Ft^d = (f - f_v)(q, g) . Ja^d; then 1/J, the source and the LSERK update.
// LIST: the element slots come from a.list (the DG elements when FV sub-cell
// elements exist), idle past its end.
// R: the operator type (metric terms, gradients, surface fluxes and the
// arithmetic of the residual); the state, 1/J of the final scaling and the RK
// update are FP64 (metrics64: the FP64 metric array, row 9 = 1/J).
template <int N, int EPB, bool LIST, typename R = double>
__global__ void __launch_bounds__(Shape<N, EPB>::THREADS)
k_volume_lg(StageArgs a, const R* __restrict__ metrics, const double* __restrict__ metrics64,
            const R* __restrict__ grad, const R* __restrict__ fstar, const int* __restrict__ elem_face,
            const double* __restrict__ mms, const double* __restrict__ tab, int E, Gas g) {
  using S = Shape<N, EPB>;
  constexpr int n = S::n, P = S::P, NN = n * n, PER = 15 * P + 30 * NN;
  extern __shared__ __align__(16) unsigned char volume_lg_raw[];
  R* sm = reinterpret_cast<R*>(volume_lg_raw);
  __shared__ R sDw[n * n], sT[2 * n];       // weak D; l(-1)/w, l(+1)/w
  __shared__ double s_tc[2];                 // sin, cos of pi t (manufactured source)
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  int e = blockIdx.x * EPB + le;
  if constexpr (LIST) {
    const int nslot = *a.list_len;
    e = e < nslot ? a.list[e] : E;
    if constexpr (EPB == 1) {
      if (e >= E) return;   // the whole block, before any barrier
    }
  }
  const bool active = e < E;
  R* sF = sm + le * PER;   // [3][5][P] contravariant fluxes
  R* sFs = sF + 15 * P;    // [6][5][NN] outward surface fluxes
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sDw[t] = to_op<R>(tab[GaussTab::Dw(n) + t]);
  for (int t = threadIdx.x; t < 2 * n; t += blockDim.x) sT[t] = to_op<R>(tab[GaussTab::lmw(n) + t]);
  if (threadIdx.x == 0 && g.source == DG_SOURCE_MMS)
    sincospi(a.clock[0] + a.c_stage * a.clock[1], &s_tc[0], &s_tc[1]);
  double q[5] = {0, 0, 0, 0, 0}, iJ = 0.0;
  if (active) {
    const R* mt = metrics + (size_t)e * 10 * P + id;
#pragma unroll
    for (int v = 0; v < 5; ++v) q[v] = a.U[((size_t)e * 5 + v) * P + id];
    R gr[12];
#pragma unroll
    for (int r = 0; r < 12; ++r) gr[r] = grad[((size_t)e * 12 + r) * P + id];
    iJ = metrics64[((size_t)e * 10 + 9) * P + id];
    R qo[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) qo[v] = to_op<R>(q[v]);
    const R ir = rcp_op(qo[0]);
    const R u = qo[1] * ir, v = qo[2] * ir, w = qo[3] * ir;
    const R p = gsel<R>(g.gm1, g.f_gm1) * (qo[4] - R(0.5) * (qo[1] * u + qo[2] * v + qo[3] * w));
    R pmom = p;
    if constexpr (sizeof(R) == 4)
      pmom = g.f_gm1 * (to_op<R>(q[4] - g.E_ref) - R(0.5) * (qo[1] * u + qo[2] * v + qo[3] * w));
    R mu = gsel<R>(g.mu, g.f_mu), lam = gsel<R>(g.mu * g.kappa, g.f_lam);
    if (g.visc_law == DG_VISC_SUTHERLAND) {
      const R sf = visc_factor<R>(g, p * ir * gsel<R>(g.inv_R, g.f_inv_R));
      mu *= sf;
      lam *= sf;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const R nx = mt[(d * 3) * P], ny = mt[(d * 3 + 1) * P], nz = mt[(d * 3 + 2) * P];
      R fa[5], fv[4];
      if constexpr (sizeof(R) == 4)   // p - p_ref in the momentum flux, from the FP64 energy difference
        euler_flux_pm<R>(qo, u, v, w, p, pmom, nx, ny, nz, fa);
      else
        euler_flux<R>(qo, u, v, w, p, nx, ny, nz, fa);
      visc_flux<R>(gr, u, v, w, mu, lam, nx, ny, nz, fv);
      sF[(d * 5) * P + id] = fa[0];
#pragma unroll
      for (int c = 0; c < 4; ++c) sF[(d * 5 + 1 + c) * P + id] = fa[1 + c] - fv[c];
    }
    for (int o = id; o < 30 * NN; o += P) {
      const int f = o / (5 * NN), r = o - f * 5 * NN, v2 = r / NN, pq = r - v2 * NN;
      const int code = elem_face[e * 6 + f], fid = dg_idx(code >> 4, a.nfaces > 0 ? a.nfaces : 3L * E, kSiteGaussVol);
      R val;
      if (code & 8) {
        val = fstar[((size_t)fid * 5 + v2) * NN + pq];
      } else {
        int p2, q2;
        apply_flip<n>(code & 7, pq % n, pq / n, p2, q2);
        val = -fstar[((size_t)fid * 5 + v2) * NN + p2 + n * q2];
      }
      sFs[(f * 5 + v2) * NN + pq] = val;
    }
  }
  __syncthreads();
  if (!active) return;
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  R acc[5] = {0, 0, 0, 0, 0};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int r = ijk[d];
    const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
    const int line0 = id - r * stride;
    for (int m = 0; m < n; ++m) {
      const R c = sDw[r * n + m];
      const int mid = line0 + m * stride;
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] = fma(-c, sF[(d * 5 + v) * P + mid], acc[v]);
    }
    const int pq = d == 0 ? j + n * k : (d == 1 ? i + n * k : i + n * j);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const R c = sT[s * n + r];
#pragma unroll
      for (int v = 0; v < 5; ++v) acc[v] = fma(c, sFs[((2 * d + s) * 5 + v) * NN + pq], acc[v]);
    }
  }
  // the manufactured source (density wave, see volume_body), in R
  R srcr[5] = {0, 0, 0, 0, 0};
  if (g.source == DG_SOURCE_MMS) mms_source<R>(g, mms, e, P, id, s_tc[0], s_tc[1], srcr);
  double src[5], accd[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    src[c] = to_f64(srcr[c]);
    accd[c] = to_f64(acc[c]);
  }
  const size_t o0 = (size_t)e * 5 * P + id;
  if (a.mode == 0) {
#pragma unroll
    for (int c = 0; c < 5; ++c) a.Ut[o0 + (size_t)c * P] = fma(-accd[c], iJ, src[c]);
  } else {
    const double dt = a.clock[1];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const size_t o = o0 + (size_t)c * P;
      const double gk = fma(a.A, a.Gk[o], dt * fma(-accd[c], iJ, src[c]));
      a.Gk[o] = gk;
      a.Uw[o] = fma(a.B, gk, q[c]);
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers

template <int N, typename R>
static cudaError_t setup_lg_NR() {
  using S = Shape<N>;
  cudaError_t e = cudaFuncSetAttribute(k_lift_lg<N, S::EPB, false, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)lift_lg_smem<N, S::EPB, R>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lift_lg<N, S::EPB, true, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lift_lg_smem<N, S::EPB, R>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_volume_lg<N, S::EPB, false, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)volume_lg_smem<N, S::EPB, R>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_volume_lg<N, S::EPB, true, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)volume_lg_smem<N, S::EPB, R>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_prolong_lg<N, S::EPB, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(R) * S::EPB * 5 * S::P));
  return e;
}

template <int N>
static cudaError_t setup_lg_N() {
  cudaError_t e = setup_lg_NR<N, double>();
  if (e == cudaSuccess) e = setup_lg_NR<N, float>();
  constexpr int P = (N + 1) * (N + 1) * (N + 1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_geometry_to_gauss<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * 5 * P));
  return e;
}

template <int N>
static cudaError_t geometry_lg_N(Ctx& c, int* d_bad, cudaStream_t s) {
  constexpr int n = N + 1, P = n * n * n;
  const long tot = (long)c.nfaces * n * n;
  k_face_geometry_lg<N><<<(int)((tot + 127) / 128), 128, 0, s>>>(c.d_faces, c.d_metrics, c.d_lgb, c.d_facegeo,
                                                                c.nfaces, c.E);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_geometry_to_gauss<N><<<c.E, P, sizeof(double) * 5 * P, s>>>(c.d_X, c.d_metrics, c.d_J, c.d_D, c.d_lgb, d_bad,
                                                                 c.E);
  return cudaGetLastError();
}

// The operator type's metric terms and face geometry.
template <typename R>
static const R* metrics_of(const Ctx& c) {
  return sizeof(R) == 8 ? (const R*)c.d_metrics : (const R*)c.d_metrics_f;
}
template <typename R>
static const R* facegeo_of(const Ctx& c) {
  return sizeof(R) == 8 ? (const R*)c.d_facegeo : (const R*)c.d_facegeo_f;
}

template <int N, typename R>
static cudaError_t lift_lg_NR(const Ctx& c, const double* U, cudaStream_t s) {
  using S = Shape<N>;
  const int blocks = (c.E + S::EPB - 1) / S::EPB;
  R* Uf = reinterpret_cast<R*>(c.d_Uf);
  R* gf = reinterpret_cast<R*>(c.d_gf);
  k_prolong_lg<N, S::EPB, R><<<blocks, S::THREADS, sizeof(R) * S::EPB * 5 * S::P, s>>>(
      U, c.d_lgb, Uf, c.E, sizeof(R) == 4 ? c.gas.E_ref : 0.0);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  if (c.M > 0) {   // the mortar sides' neighbour face states first
    err = launch_mortar_lift(c, U, s);
    if (err != cudaSuccess) return err;
    k_lift_lg<N, S::EPB, true, R><<<blocks, S::THREADS, lift_lg_smem<N, S::EPB, R>(), s>>>(
        U, Uf, metrics_of<R>(c), facegeo_of<R>(c), c.d_elem_face, c.d_elem_nbr, c.d_lgb, (R*)c.d_grad, gf, c.E,
        c.nfaces, c.gas, c.d_mortar_virt, c.M);
    return cudaGetLastError();
  }
  k_lift_lg<N, S::EPB, false, R><<<blocks, S::THREADS, lift_lg_smem<N, S::EPB, R>(), s>>>(
      U, Uf, metrics_of<R>(c), facegeo_of<R>(c), c.d_elem_face, c.d_elem_nbr, c.d_lgb, (R*)c.d_grad, gf, c.E,
      c.nfaces, c.gas, nullptr, 0);
  return cudaGetLastError();
}

template <int N>
static cudaError_t lift_lg_N(const Ctx& c, const double* U, cudaStream_t s, bool fp64) {
  return (fp64 || c.prm.precision != DG_FP32OP) ? lift_lg_NR<N, double>(c, U, s) : lift_lg_NR<N, float>(c, U, s);
}

template <int N, typename R>
static cudaError_t face_lg_NR(const Ctx& c, cudaStream_t s) {
  // the conforming faces (the mortars' slots follow them)
  const long tot = (long)c.nfaces_conf * (N + 1) * (N + 1);
  const R* Uf = reinterpret_cast<const R*>(c.d_Uf);
  const R* gf = reinterpret_cast<const R*>(c.d_gf);
  if (tot > 0) {
    if (c.fv_on)
      k_face_lg<N, true, R><<<(int)((tot + 127) / 128), 128, 0, s>>>(
          Uf, gf, c.d_faces, facegeo_of<R>(c), (R*)c.d_fstar, c.nfaces_conf, c.E, c.gas, c.d_fv_mask);
    else
      k_face_lg<N, false, R><<<(int)((tot + 127) / 128), 128, 0, s>>>(
          Uf, gf, c.d_faces, facegeo_of<R>(c), (R*)c.d_fstar, c.nfaces_conf, c.E, c.gas, nullptr);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && c.M > 0) e = launch_mortar_flux(c, nullptr, s);
  return e;
}

template <int N>
static cudaError_t face_lg_N(const Ctx& c, cudaStream_t s) {
  return c.prm.precision == DG_FP32OP ? face_lg_NR<N, float>(c, s) : face_lg_NR<N, double>(c, s);
}

template <int N, typename R>
static cudaError_t volume_lg_NR(const Ctx& c, const StageArgs& a0, cudaStream_t s) {
  using S = Shape<N>;
  StageArgs a = a0;
  a.nfaces = c.nfaces;
  const int blocks = (c.E + S::EPB - 1) / S::EPB;
  if (a.list != nullptr)
    k_volume_lg<N, S::EPB, true, R><<<blocks, S::THREADS, volume_lg_smem<N, S::EPB, R>(), s>>>(
        a, metrics_of<R>(c), c.d_metrics, (const R*)c.d_grad, (const R*)c.d_fstar, c.d_elem_face, c.d_mms, c.d_lgb,
        c.E, c.gas);
  else
    k_volume_lg<N, S::EPB, false, R><<<blocks, S::THREADS, volume_lg_smem<N, S::EPB, R>(), s>>>(
        a, metrics_of<R>(c), c.d_metrics, (const R*)c.d_grad, (const R*)c.d_fstar, c.d_elem_face, c.d_mms, c.d_lgb,
        c.E, c.gas);
  return cudaGetLastError();
}

template <int N>
static cudaError_t volume_lg_N(const Ctx& c, const StageArgs& a, cudaStream_t s) {
  return c.prm.precision == DG_FP32OP ? volume_lg_NR<N, float>(c, a, s) : volume_lg_NR<N, double>(c, a, s);
}

#define DG_LG_DISPATCH(FN, ...)              \
  switch (c.N) {                             \
    case 1: return FN<1>(__VA_ARGS__);       \
    case 2: return FN<2>(__VA_ARGS__);       \
    case 3: return FN<3>(__VA_ARGS__);       \
    case 4: return FN<4>(__VA_ARGS__);       \
    case 5: return FN<5>(__VA_ARGS__);       \
    case 6: return FN<6>(__VA_ARGS__);       \
    case 7: return FN<7>(__VA_ARGS__);       \
    case 8: return FN<8>(__VA_ARGS__);       \
    case 9: return FN<9>(__VA_ARGS__);       \
    default: return cudaErrorInvalidValue;   \
  }

cudaError_t setup_gauss(int N) {
  switch (N) {
    case 1: return setup_lg_N<1>();
    case 2: return setup_lg_N<2>();
    case 3: return setup_lg_N<3>();
    case 4: return setup_lg_N<4>();
    case 5: return setup_lg_N<5>();
    case 6: return setup_lg_N<6>();
    case 7: return setup_lg_N<7>();
    case 8: return setup_lg_N<8>();
    case 9: return setup_lg_N<9>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t gauss_geometry(Ctx& c, int* d_bad, cudaStream_t s) { DG_LG_DISPATCH(geometry_lg_N, c, d_bad, s) }
cudaError_t launch_lift_lg(const Ctx& c, const double* U, cudaStream_t s, bool fp64) {
  DG_LG_DISPATCH(lift_lg_N, c, U, s, fp64)
}
cudaError_t launch_face_lg(const Ctx& c, cudaStream_t s) { DG_LG_DISPATCH(face_lg_N, c, s) }
cudaError_t launch_volume_lg(const Ctx& c, const StageArgs& a, cudaStream_t s) {
  DG_LG_DISPATCH(volume_lg_N, c, a, s)
}

// Host reader of this file's bounds-check error word (0 in normal builds).
DG_BOUNDS_READER(bounds_word_gauss)

}  // namespace dg
