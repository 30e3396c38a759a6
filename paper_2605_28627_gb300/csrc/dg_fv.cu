// FV sub-cell operator of the shock capturing (GALAEXI Sec. 3.1: a second-order
// finite-volume scheme on (N+1)^3 integral means per DG element, switched on
// for the elements a troubled-cell indicator selects).
//
// The scheme, as built here (FP64, on either node set):
//  * sub-cells: the (N+1)^3 equal sub-cubes of the reference element, width
//    h = 2/(N+1), indexed like the nodes; sub-faces like the face nodes;
//  * unknowns: J-weighted sub-cell means of the nodal interpolant,
//    ub = V3 (J u) / V3 J, V[a][j] = mean over sub-interval a of the Lagrange
//    polynomial j, V3 = V (x) V (x) V (invertible: nodal values and means map
//    one to one, and the element integrals agree);
//  * sub-face area vectors S = integral of J a^d over the sub-face, exact for
//    the metric polynomial, so every sub-cell's surface closes and free
//    streams are kept;
//  * reconstruction: primitive variables of the means, per reference
//    direction a minmod-limited slope of the two one-sided differences (across
//    an element face the neighbour's sub-cell), face values w +- slope/2;
//  * sub-face flux: local Lax-Friedrichs in S/|S| of the two reconstructed
//    states minus the average of the two sub-cells' viscous fluxes (means of
//    the state and of the BR1 gradients), times |S|; each sub-cell's viscous
//    flux tensor is formed once, in the means kernel;
//  * residual: J R at the nodes = V3^-1 (-(outward sub-face fluxes) / h^3),
//    then 1/J, the source and the RK update like a DG element;
//  * faces between a DG and an FV element are evaluated on sub-faces: the DG
//    side enters with the means of its trace over each sub-face and takes the
//    nodal form F* = (V (x) V)^-1 (Fb / h^2) of the sub-face fluxes, whose
//    face integral is their sum (conservation); the flux so acts on the DG
//    face values themselves, as an upwind DG face flux does.
//
// Per stage (all on the caller's stream, after the lifting and face kernels):
//   k_fv_means   sub-cell means of U (as primitives) for FV elements and
//                their face neighbours, of the lifted gradients (as viscous
//                flux tensors) for FV elements;
//   k_fv_face    sub-face fluxes of faces with an FV side; nodal F* for the
//                DG side of mixed faces (overwrites the DG face flux);
//   DG volume    over the list of the DG elements;
//   k_fv_volume  the FV residual of each FV element and its RK update.
// k_fv_lists builds the two element lists when the mask is set.
// k_fv_geom computes 1 / Jb (Jb = V3 J) and the area vectors once per context.
#include <cmath>
#include <vector>

#include "dg_stage.cuh"

namespace dg {

// Layout of the table d_fv_tab: V [n][n], V^-1 [n][n], L [n+1][n] (Lagrange
// polynomial m at the sub-cell plane -1 + pl h).
template <int N>
struct FvShape {
  static constexpr int n = N + 1, P = n * n * n, NN = n * n, NP = (n + 1) * n * n;
  static constexpr int TAB = 2 * NN + (n + 1) * n;
  // faces per block of the sub-face kernel (one thread per sub-face)
  static constexpr int FPB = NN >= 128 ? 1 : 128 / NN;
  static constexpr int FACE_THREADS = FPB * NN;
  static constexpr double h = 2.0 / n;
};

// Sub-cell (or node) at position m along direction d, transverse indices (p, q)
// in increasing direction order (the face-node convention).
template <int n>
__device__ __forceinline__ int line_cell(int d, int m, int p, int q) {
  return d == 0 ? vidx<n>(m, p, q) : (d == 1 ? vidx<n>(p, m, q) : vidx<n>(p, q, m));
}

// minmod(x, y): 0 where the signs differ, else the argument of smaller
// magnitude.  Decided on the bit patterns in integer instructions (for
// magnitudes the integer order is the floating-point order), so it costs no
// FP64 instruction; a zero argument gives a zero (of either sign).
__device__ __forceinline__ double minmod(double x, double y) {
  const long long bx = __double_as_longlong(x), by = __double_as_longlong(y);
  if ((bx ^ by) < 0) return 0.0;
  return (bx & 0x7fffffffffffffffll) < (by & 0x7fffffffffffffffll) ? x : y;
}

// Sub-face flux through a sub-face of area A and unit normal (nx, ny, nz) from
// the two sides' primitive states wL, wR (rho, u, v, w, p) and viscous flux
// tensors vL, vR (12 values, vsL / vsR apart: row l*4 + c = component c
// (momentum x, y, z, energy) of the flux in direction x_l).
__device__ __forceinline__ void fv_subface_flux(const double wL[5], const double wR[5], const double* vL, int vsL,
                                                const double* vR, int vsR, double nx, double ny, double nz, double A,
                                                const Gas& g, double out[5]) {
  double qL[5], qR[5], fL[5], fR[5];
  qL[0] = wL[0]; qL[1] = wL[0] * wL[1]; qL[2] = wL[0] * wL[2]; qL[3] = wL[0] * wL[3];
  qL[4] = wL[4] * g.inv_gm1 + 0.5 * (qL[1] * wL[1] + qL[2] * wL[2] + qL[3] * wL[3]);
  qR[0] = wR[0]; qR[1] = wR[0] * wR[1]; qR[2] = wR[0] * wR[2]; qR[3] = wR[0] * wR[3];
  qR[4] = wR[4] * g.inv_gm1 + 0.5 * (qR[1] * wR[1] + qR[2] * wR[2] + qR[3] * wR[3]);
  euler_flux<double>(qL, wL[1], wL[2], wL[3], wL[4], nx, ny, nz, fL);
  euler_flux<double>(qR, wR[1], wR[2], wR[3], wR[4], nx, ny, nz, fR);
  // sound speeds sqrt(gamma p / rho) = gamma p / sqrt(gamma p rho): one root, no divide
  const double gpL = g.gamma * wL[4], gpR = g.gamma * wR[4];
  const double lL = fabs(wL[1] * nx + wL[2] * ny + wL[3] * nz) + gpL * rsqrt(gpL * wL[0]);
  const double lR = fabs(wR[1] * nx + wR[2] * ny + wR[3] * nz) + gpR * rsqrt(gpR * wR[0]);
  const double hl = 0.5 * fmax(lL, lR);
  out[0] = (0.5 * (fL[0] + fR[0]) - hl * (qR[0] - qL[0])) * A;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double fv = nx * (vL[c * vsL] + vR[c * vsR]) + ny * (vL[(4 + c) * vsL] + vR[(4 + c) * vsR]) +
                      nz * (vL[(8 + c) * vsL] + vR[(8 + c) * vsR]);
    out[1 + c] = (0.5 * (fL[1 + c] + fR[1 + c]) - hl * (qR[1 + c] - qL[1 + c]) - 0.5 * fv) * A;
  }
}

// Viscous flux tensor (Newtonian stress with Stokes' hypothesis, Fourier heat
// flux) of the state (u, v, w, p/rho) with gradients gm[phi*3 + l] = d phi /
// d x_l, phi = (u, v, w, T): out[l*4 + c], c = momentum x, y, z, energy.
__device__ __forceinline__ void visc_tensor(const Gas& g, double u, double v, double w, double p_over_rho,
                                            const double gm[12], double out[12]) {
  double mu = g.mu, lam = g.mu * g.kappa;
  if (g.visc_law == DG_VISC_SUTHERLAND) {
    const double sf = visc_factor<double>(g, p_over_rho * g.inv_R);
    mu *= sf;
    lam *= sf;
  }
  const double div = gm[0] + gm[4] + gm[8];
  double tau[3][3];
#pragma unroll
  for (int a2 = 0; a2 < 3; ++a2)
#pragma unroll
    for (int b2 = 0; b2 < 3; ++b2)
      tau[a2][b2] = a2 == b2 ? mu * (2.0 * gm[a2 * 4] - (2.0 / 3.0) * div) : mu * (gm[a2 * 3 + b2] + gm[b2 * 3 + a2]);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    out[l * 4] = tau[l][0];
    out[l * 4 + 1] = tau[l][1];
    out[l * 4 + 2] = tau[l][2];
    out[l * 4 + 3] = tau[l][0] * u + tau[l][1] * v + tau[l][2] * w + lam * gm[9 + l];
  }
}

// One sweep of a tensor-product operator M along direction d on an n^3 field:
// out[node] = sum_m M[idx_d][m] in[node with idx_d -> m].
template <int n>
__device__ __forceinline__ double sweep(const double* __restrict__ M, const double* in, int d, int i, int j, int k) {
  double s = 0.0;
  const int r = d == 0 ? i : (d == 1 ? j : k);
#pragma unroll
  for (int m = 0; m < n; ++m) {
    const int id = d == 0 ? vidx<n>(m, j, k) : (d == 1 ? vidx<n>(i, m, k) : vidx<n>(i, j, m));
    s = fma(M[r * n + m], in[id], s);
  }
  return s;
}

// ---------------------------------------------------------------------------
// Once per context: 1 / Jb (Jb = V3 J) and the sub-face area vectors
// S [E][3][n+1][NN][4] (direction, plane, sub-face; unit normal, area).
template <int N>
__global__ void __launch_bounds__(FvShape<N>::P)
k_fv_geom(const double* __restrict__ metrics, const double* __restrict__ J, const double* __restrict__ tab,
          double* __restrict__ Jb, double* __restrict__ S, int E) {
  using F = FvShape<N>;
  constexpr int n = F::n, P = F::P, NN = F::NN, NP = F::NP;
  extern __shared__ __align__(16) double fsm[];
  double* sV = fsm;
  double* sL = sV + NN;
  double* A = sL + (n + 1) * n;
  double* B = A + P;
  double* C = B + NP;
  const int e = blockIdx.x, id = threadIdx.x;
  const int i = id % n, j = (id / n) % n, k = id / NN;
  for (int t = id; t < NN; t += P) sV[t] = tab[t];
  for (int t = id; t < (n + 1) * n; t += P) sL[t] = tab[2 * NN + t];
  A[id] = J[(size_t)e * P + id];
  __syncthreads();
  B[id] = sweep<n>(sV, A, 0, i, j, k);
  __syncthreads();
  A[id] = sweep<n>(sV, B, 1, i, j, k);
  __syncthreads();
  Jb[(size_t)e * P + id] = 1.0 / sweep<n>(sV, A, 2, i, j, k);
  const double h2 = F::h * F::h;
  for (int d = 0; d < 3; ++d)
    for (int l = 0; l < 3; ++l) {
      __syncthreads();
      A[id] = metrics[((size_t)e * 10 + d * 3 + l) * P + id];
      __syncthreads();
      // the metric polynomial on each plane pl along d
      for (int t = id; t < NP; t += P) {
        const int pl = t / NN, pq = t % NN, p = pq % n, q = pq / n;
        double s = 0.0;
        for (int m = 0; m < n; ++m) s = fma(sL[pl * n + m], A[line_cell<n>(d, m, p, q)], s);
        B[t] = s;
      }
      __syncthreads();
      // means across: first transverse direction, then the second
      for (int t = id; t < NP; t += P) {
        const int pl = t / NN, pq = t % NN, a = pq % n, q = pq / n;
        double s = 0.0;
        for (int p = 0; p < n; ++p) s = fma(sV[a * n + p], B[pl * NN + p + n * q], s);
        C[t] = s;
      }
      __syncthreads();
      for (int t = id; t < NP; t += P) {
        const int pl = t / NN, pq = t % NN, a = pq % n, b = pq / n;
        double s = 0.0;
        for (int q = 0; q < n; ++q) s = fma(sV[b * n + q], C[pl * NN + a + n * q], s);
        S[((((size_t)e * 3 + d) * (n + 1) + pl) * NN + pq) * 4 + l] = h2 * s;
      }
    }
  __syncthreads();   // the block's own global writes are visible after the barrier
  for (int t = id; t < 3 * NP; t += P) {
    double* v = S + ((size_t)e * 3 * NP + t) * 4;
    const double A = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    const double iA = 1.0 / A;
    v[0] *= iA;
    v[1] *= iA;
    v[2] *= iA;
    v[3] = A;
  }
}

// ---------------------------------------------------------------------------
// Sub-cell means M [E][17][P]: rows 0-4 the primitives (rho, u, v, w, p) of
// the mean state; for FV elements rows 5-16 the viscous flux tensor of the
// mean state and the means of the lifted gradients (row 5 + l*4 + c: component
// c = momentum x, y, z, energy of the flux in direction x_l).  FV elements and
// their face neighbours only (the rest return at once); a DG neighbour needs
// the primitives alone (the slopes of the FV sub-cells next to it).
template <int N, int NF>
__device__ __forceinline__ void means_of_fields(const double* __restrict__ U, const double* __restrict__ grad, int e,
                                                int id, double Je, double iJbe, const double* sV, double* A,
                                                double* B, double cm[17]) {
  using F = FvShape<N>;
  constexpr int n = F::n, P = F::P, NN = F::NN;
  // fields per pass of the three sweeps: two buffers of FCH * P doubles and the
  // table within the 48 KB of static shared memory
  constexpr int FCH = (6144 - NN) / (2 * P) >= NF ? NF : (6144 - NN) / (2 * P);
  const int i = id % n, j = (id / n) % n, k = id / NN;
#pragma unroll
  for (int r0 = 0; r0 < NF; r0 += FCH) {
#pragma unroll
    for (int r = r0; r < r0 + FCH && r < NF; ++r)
      A[(r - r0) * P + id] = Je * (r < 5 ? U[((size_t)e * 5 + r) * P + id] : grad[((size_t)e * 12 + r - 5) * P + id]);
    __syncthreads();
#pragma unroll
    for (int r = r0; r < r0 + FCH && r < NF; ++r) B[(r - r0) * P + id] = sweep<n>(sV, A + (r - r0) * P, 0, i, j, k);
    __syncthreads();
#pragma unroll
    for (int r = r0; r < r0 + FCH && r < NF; ++r) A[(r - r0) * P + id] = sweep<n>(sV, B + (r - r0) * P, 1, i, j, k);
    __syncthreads();
#pragma unroll
    for (int r = r0; r < r0 + FCH && r < NF; ++r) cm[r] = sweep<n>(sV, A + (r - r0) * P, 2, i, j, k) * iJbe;
    __syncthreads();   // A is refilled by the next pass
  }
}

template <int N>
__global__ void __launch_bounds__(FvShape<N>::P)
k_fv_means(const double* __restrict__ U, const double* __restrict__ grad, const double* __restrict__ J,
           const double* __restrict__ iJb, const int* __restrict__ mask, const int* __restrict__ elem_nbr,
           const double* __restrict__ tab, double* __restrict__ M, int E, Gas g) {
  using F = FvShape<N>;
  constexpr int P = F::P, NN = F::NN;
  constexpr int FCH = (6144 - NN) / (2 * P) >= 17 ? 17 : (6144 - NN) / (2 * P);
  __shared__ double sV[NN], A[FCH * P], B[FCH * P];
  __shared__ int s_fv;
  const int e = blockIdx.x, id = threadIdx.x;
  int mine = 0;
  if (id < 6) {   // a mortar neighbour (negative entry) is a DG side
    const int nb = elem_nbr[e * 6 + id];
    mine = nb < 0 ? 0 : mask[dg_idx(nb >> 3, E, kSiteFvNbr)];
  }
  else if (id == 6) {
    mine = mask[e];
    s_fv = mine;
  }
  if (!__syncthreads_or(mine)) return;   // uniform for the block
  for (int t = id; t < NN; t += P) sV[t] = tab[t];
  const double Je = J[(size_t)e * P + id], iJbe = iJb[(size_t)e * P + id];
  double cm[17];
  const bool fv = s_fv != 0;
  if (fv) means_of_fields<N, 17>(U, grad, e, id, Je, iJbe, sV, A, B, cm);
  else means_of_fields<N, 5>(U, grad, e, id, Je, iJbe, sV, A, B, cm);
  const double ir = 1.0 / cm[0];
  const double u = cm[1] * ir, v = cm[2] * ir, w = cm[3] * ir;
  const double p = g.gm1 * (cm[4] - 0.5 * (cm[1] * u + cm[2] * v + cm[3] * w));
  double* o = M + (size_t)e * 17 * P + id;
  o[0] = cm[0];
  o[P] = u;
  o[2 * P] = v;
  o[3 * P] = w;
  o[4 * P] = p;
  if (fv) {
    double vt[12];
    visc_tensor(g, u, v, w, p * ir, cm + 5, vt);
#pragma unroll
    for (int r = 0; r < 12; ++r) o[(5 + r) * P] = vt[r];
  }
}

// ---------------------------------------------------------------------------
// Faces with an FV side: master-outward sub-face fluxes Fb [F][5][NN].  An FV
// side enters with its reconstructed state and the viscous flux tensor of its
// sub-cell; the DG side of a mixed face with the means over each sub-face of
// its trace (state and nodal viscous flux tensor, (V x V) of the face-node
// values) and takes the nodal form of the sub-face fluxes as its face flux.
template <int N>
__global__ void __launch_bounds__(FvShape<N>::FACE_THREADS)
k_fv_face(const FaceInfo* __restrict__ faces, const int* __restrict__ mask, const double* __restrict__ U,
          const double* __restrict__ grad, const double* __restrict__ Uf, const double* __restrict__ gf,
          const double* __restrict__ M, const double* __restrict__ S, const double* __restrict__ tab,
          double* __restrict__ Fb, double* __restrict__ fstar, int F, int E, Gas g) {
  using Fs = FvShape<N>;
  constexpr int n = Fs::n, P = Fs::P, NN = Fs::NN, FPB = Fs::FPB;
  __shared__ double sV[NN], sVi[NN];
  __shared__ double sA[FPB][17][NN];   // DG trace: face-node values, then sub-face means; F* sweep
  __shared__ double sB[FPB][17][NN];   // first sweep of the trace; then the sub-face fluxes
  const int lf = threadIdx.x / NN, ab = threadIdx.x % NN;
  const int f = blockIdx.x * FPB + lf;
  for (int t = threadIdx.x; t < NN; t += Fs::FACE_THREADS) {
    sV[t] = tab[t];
    sVi[t] = tab[NN + t];
  }
  bool act = false, mixed = false, fvM = false, fvS = false;
  int eM = 0, fM = 0, eS = 0, fS = 0, flip = 0;
  if (f < F) {
    const FaceInfo fi = faces[f];
    eM = dg_idx(fi.master >> 3, E, kSiteFvFace);
    fM = fi.master & 7;
    eS = dg_idx(fi.slave >> 3, E, kSiteFvFace);
    fS = fi.slave & 7;
    flip = fi.flip;
    fvM = mask[eM] != 0;
    fvS = mask[eS] != 0;
    act = fvM || fvS;
    mixed = fvM != fvS;
  }
  const int a = ab % n, b = ab / n;
  // the DG side's trace at its face point (a, b) of its own face-local indices:
  // the face node (LGL nodes), or the values interpolated to the face (Uf, gf:
  // Gauss nodes)
  if (mixed) {
    const int eD = fvM ? eS : eM, fD = fvM ? fS : fM;
    double q[5], gr[12], vt[12];
    if (Uf != nullptr) {
      const size_t o = (size_t)eD * 6 + fD;
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = Uf[(o * 5 + v) * NN + ab];
#pragma unroll
      for (int r = 0; r < 12; ++r) gr[r] = gf[(o * 12 + r) * NN + ab];
    } else {
      const int node = face_node<n>(fD, a, b);
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = U[((size_t)eD * 5 + v) * P + node];
#pragma unroll
      for (int r = 0; r < 12; ++r) gr[r] = grad[((size_t)eD * 12 + r) * P + node];
    }
    const double ir = 1.0 / q[0];
    const double u = q[1] * ir, v = q[2] * ir, w = q[3] * ir;
    const double p = g.gm1 * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w));
    visc_tensor(g, u, v, w, p * ir, gr, vt);
#pragma unroll
    for (int v2 = 0; v2 < 5; ++v2) sA[lf][v2][ab] = q[v2];
#pragma unroll
    for (int r = 0; r < 12; ++r) sA[lf][5 + r][ab] = vt[r];
  }
  __syncthreads();
  if (mixed) {   // means across the first face index
#pragma unroll
    for (int r = 0; r < 17; ++r) {
      double t = 0.0;
#pragma unroll
      for (int pp = 0; pp < n; ++pp) t = fma(sV[a * n + pp], sA[lf][r][pp + n * b], t);
      sB[lf][r][ab] = t;
    }
  }
  __syncthreads();
  if (mixed) {   // ... and the second: the trace's sub-face means
#pragma unroll
    for (int r = 0; r < 17; ++r) {
      double t = 0.0;
#pragma unroll
      for (int qq = 0; qq < n; ++qq) t = fma(sV[b * n + qq], sB[lf][r][a + n * qq], t);
      sA[lf][r][ab] = t;
    }
  }
  __syncthreads();
  double out[5];
  if (act) {
    int a2, b2;
    apply_flip<n>(flip, a, b, a2, b2);
    const int dM = fM >> 1, sM = fM & 1, dS = fS >> 1, sS = fS & 1;
    const int cM0 = face_node<n>(fM, a, b), cS0 = face_node<n>(fS, a2, b2);
    const double* mMp = M + (size_t)eM * 17 * P;
    const double* mSp = M + (size_t)eS * 17 * P;
    double stM[5], stS[5];
    const double* vM;
    const double* vS;
    int vsM, vsS;
    if (fvM) {
      const int cM1 = line_cell<n>(dM, sM ? N - 1 : 1, a, b);
#pragma unroll
      for (int v = 0; v < 5; ++v) {   // face value: w0 + slope/2 towards the face
        const double w0 = mMp[v * P + cM0];
        stM[v] = w0 + 0.5 * minmod(mSp[v * P + cS0] - w0, w0 - mMp[v * P + cM1]);
      }
      vM = mMp + 5 * P + cM0;
      vsM = P;
    } else {
      const double* tq = &sA[lf][0][ab];   // trace means, the master's own indices
      const double ir = 1.0 / tq[0];
      stM[0] = tq[0];
      stM[1] = tq[NN] * ir;
      stM[2] = tq[2 * NN] * ir;
      stM[3] = tq[3 * NN] * ir;
      stM[4] = g.gm1 * (tq[4 * NN] - 0.5 * (tq[NN] * stM[1] + tq[2 * NN] * stM[2] + tq[3 * NN] * stM[3]));
      vM = tq + 5 * NN;
      vsM = NN;
    }
    if (fvS) {
      const int cS1 = line_cell<n>(dS, sS ? N - 1 : 1, a2, b2);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const double w0 = mSp[v * P + cS0];
        stS[v] = w0 + 0.5 * minmod(mMp[v * P + cM0] - w0, w0 - mSp[v * P + cS1]);
      }
      vS = mSp + 5 * P + cS0;
      vsS = P;
    } else {
      const double* tq = &sA[lf][0][a2 + n * b2];   // the slave's own indices of this sub-face
      const double ir = 1.0 / tq[0];
      stS[0] = tq[0];
      stS[1] = tq[NN] * ir;
      stS[2] = tq[2 * NN] * ir;
      stS[3] = tq[3 * NN] * ir;
      stS[4] = g.gm1 * (tq[4 * NN] - 0.5 * (tq[NN] * stS[1] + tq[2 * NN] * stS[2] + tq[3 * NN] * stS[3]));
      vS = tq + 5 * NN;
      vsS = NN;
    }
    const double* Sp = S + ((((size_t)eM * 3 + dM) * (n + 1) + sM * n) * NN + ab) * 4;
    const double sg = sM ? 1.0 : -1.0;
    fv_subface_flux(stM, stS, vM, vsM, vS, vsS, sg * Sp[0], sg * Sp[1], sg * Sp[2], Sp[3], g, out);
#pragma unroll
    for (int v = 0; v < 5; ++v) Fb[((size_t)f * 5 + v) * NN + ab] = out[v];
  }
  if (mixed) {
#pragma unroll
    for (int v = 0; v < 5; ++v) sB[lf][v][ab] = out[v];
  }
  __syncthreads();
  // (V^-1 (x) V^-1) (Fb / h^2) in two sweeps: first index, then second
  if (mixed) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double t = 0.0;
#pragma unroll
      for (int aa = 0; aa < n; ++aa) t = fma(sVi[a * n + aa], sB[lf][v][aa + n * b], t);
      sA[lf][v][ab] = t;
    }
  }
  __syncthreads();
  if (mixed) {
    const double ih2 = 1.0 / (Fs::h * Fs::h);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double t = 0.0;
#pragma unroll
      for (int bb = 0; bb < n; ++bb) t = fma(sVi[b * n + bb], sA[lf][v][a + n * bb], t);
      fstar[((size_t)f * 5 + v) * NN + ab] = t * ih2;
    }
  }
}

// ---------------------------------------------------------------------------
// FV residual of each FV element, its Jacobian, source and RK update (the
// same epilogue as a DG element).  One thread per sub-cell / node.
template <int N>
constexpr size_t fv_volume_smem() {
  using F = FvShape<N>;
  return sizeof(double) * ((size_t)F::NN + 20 * (size_t)F::P + 30 * (size_t)F::NN);
}

template <int N>
__global__ void __launch_bounds__(FvShape<N>::P)
k_fv_volume(StageArgs a, const int* __restrict__ lists, const int* __restrict__ elem_face,
            const int* __restrict__ elem_nbr, const double* __restrict__ M, const double* __restrict__ S,
            const double* __restrict__ Fb, const double* __restrict__ metrics, const double* __restrict__ mms,
            const double* __restrict__ tab, int E, Gas g) {
  using F = FvShape<N>;
  constexpr int n = F::n, P = F::P, NN = F::NN;
  const int id = threadIdx.x;
  if ((int)blockIdx.x >= lists[2 * E + 1]) return;   // uniform for the block: one block per FV element
  const int e = dg_idx(lists[E + blockIdx.x], E, kSiteFvNbr);
  extern __shared__ __align__(16) double fsm[];
  double* sVi = fsm;
  double* sW = sVi + NN;      // [5][P] mean primitives
  double* sH = sW + 5 * P;    // [6][5][NN] neighbours' sub-cells across each face
  double* sFm = sH + 30 * NN; // [5][P] reconstruction at the -xi_d face / map buffer
  double* sFp = sFm + 5 * P;  // [5][P] reconstruction at the +xi_d face / map buffer
  double* sF = sFp + 5 * P;   // [5][P] flux through the +xi_d plane of each sub-cell
  __shared__ double s_tc[2];
  if (id == 0 && g.source == DG_SOURCE_MMS) sincospi(a.clock[0] + a.c_stage * a.clock[1], &s_tc[0], &s_tc[1]);
  for (int t = id; t < NN; t += P) sVi[t] = tab[NN + t];
  const double* Me = M + (size_t)e * 17 * P;
#pragma unroll
  for (int v = 0; v < 5; ++v) sW[v * P + id] = Me[v * P + id];
  for (int t = id; t < 6 * NN; t += P) {
    const int f = t / NN, ab = t % NN;
    const int code = elem_face[e * 6 + f], nb = elem_nbr[e * 6 + f];
    const int e2 = dg_idx(nb >> 3, E, kSiteFvNbr), f2 = nb & 7;
    int a2, b2;
    apply_flip<n>(code & 7, ab % n, ab / n, a2, b2);
    const int cell = face_node<n>(f2, a2, b2);
#pragma unroll
    for (int v = 0; v < 5; ++v) sH[(f * 5 + v) * NN + ab] = M[((size_t)e2 * 17 + v) * P + cell];
  }
  __syncthreads();
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  double res[5] = {0, 0, 0, 0, 0};   // outward sub-face fluxes of this sub-cell
  // unrolled up to N = 7 (ijk[d] in registers); at N = 8, 9 the 729 / 1000
  // threads leave too few registers for the unrolled body
#pragma unroll (N <= 7 ? 3 : 1)
  for (int d = 0; d < 3; ++d) {
    const int m = ijk[d];
    const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
    const int ab = (d == 0 ? j : i) + n * (d == 2 ? j : k);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double w0 = sW[v * P + id];
      const double wm = m > 0 ? sW[v * P + id - stride] : sH[((2 * d) * 5 + v) * NN + ab];
      const double wp = m < N ? sW[v * P + id + stride] : sH[((2 * d + 1) * 5 + v) * NN + ab];
      const double sl = minmod(wp - w0, w0 - wm);
      sFm[v * P + id] = w0 - 0.5 * sl;
      sFp[v * P + id] = w0 + 0.5 * sl;
    }
    __syncthreads();
    if (m < N) {
      double wl[5], wr[5], out[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        wl[v] = sFp[v * P + id];
        wr[v] = sFm[v * P + id + stride];
      }
      const double* Sp = S + ((((size_t)e * 3 + d) * (n + 1) + m + 1) * NN + ab) * 4;
      fv_subface_flux(wl, wr, Me + 5 * P + id, P, Me + 5 * P + id + stride, P, Sp[0], Sp[1], Sp[2], Sp[3], g, out);
#pragma unroll
      for (int v = 0; v < 5; ++v) sF[v * P + id] = out[v];
    }
    __syncthreads();
    // +xi_d flux through the element face 2d + s, from the face's sub-face fluxes
    auto face_flux = [&](int s, int v) {
      const int code = elem_face[e * 6 + 2 * d + s];
      const int fid = dg_idx(code >> 4, 3L * E, kSiteFvFace);
      const double sgn = s ? 1.0 : -1.0;
      if (code & 8) return sgn * Fb[((size_t)fid * 5 + v) * NN + ab];
      int am, bm;
      apply_flip<n>(code & 7, ab % n, ab / n, am, bm);
      return -sgn * Fb[((size_t)fid * 5 + v) * NN + am + n * bm];
    };
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double fp = m < N ? sF[v * P + id] : face_flux(1, v);
      const double fm = m > 0 ? sF[v * P + id - stride] : face_flux(0, v);
      res[v] += fp - fm;
    }
    __syncthreads();
  }
  // J R at the nodes: V3^-1 of the sub-cell values -(outward fluxes)/h^3
  const double ih3 = 1.0 / (F::h * F::h * F::h);
#pragma unroll
  for (int v = 0; v < 5; ++v) sFm[v * P + id] = -res[v] * ih3;
  __syncthreads();
#pragma unroll
  for (int v = 0; v < 5; ++v) sFp[v * P + id] = sweep<n>(sVi, sFm + v * P, 0, i, j, k);
  __syncthreads();
#pragma unroll
  for (int v = 0; v < 5; ++v) sFm[v * P + id] = sweep<n>(sVi, sFp + v * P, 1, i, j, k);
  __syncthreads();
  double jr[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) jr[v] = sweep<n>(sVi, sFm + v * P, 2, i, j, k);
  double src[5] = {0, 0, 0, 0, 0};
  if (g.source == DG_SOURCE_MMS) mms_source<double>(g, mms, e, P, id, s_tc[0], s_tc[1], src);
  const double iJ = metrics[((size_t)e * 10 + 9) * P + id];
  const size_t o0 = (size_t)e * 5 * P + id;
  if (a.mode == 0) {
#pragma unroll
    for (int c = 0; c < 5; ++c) a.Ut[o0 + (size_t)c * P] = fma(jr[c], iJ, src[c]);
  } else {
    const double dt = a.clock[1];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const size_t o = o0 + (size_t)c * P;
      const double gk = fma(a.A, a.Gk[o], dt * fma(jr[c], iJ, src[c]));
      a.Gk[o] = gk;
      a.Uw[o] = fma(a.B, gk, a.U[o]);
    }
  }
}

// ---------------------------------------------------------------------------
// Element lists of a mask, one block: lists[0..nDG) the DG elements,
// lists[E..E+nFV) the FV elements (both ascending), lists[2E] = nDG,
// lists[2E+1] = nFV.
constexpr int kListThreads = 1024;

__global__ void __launch_bounds__(kListThreads) k_fv_lists(const int* __restrict__ mask, int* __restrict__ lists,
                                                           int E) {
  __shared__ int warp_fv[kListThreads / 32];
  __shared__ int base_fv;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (t == 0) base_fv = 0;
  __syncthreads();
  for (int c0 = 0; c0 < E; c0 += kListThreads) {
    const int e = c0 + t;
    const int fv = e < E && mask[e] != 0 ? 1 : 0;
    // inclusive scan of the FV flags: within the warp, then over the warps
    const unsigned bal = __ballot_sync(0xffffffffu, fv);
    const int in_warp = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_fv[wid] = __popc(bal);
    __syncthreads();
    if (wid == 0) {
      int v = warp_fv[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      warp_fv[lane] = v;   // inclusive over the warps
    }
    __syncthreads();
    const int before_fv = base_fv + (wid > 0 ? warp_fv[wid - 1] : 0) + in_warp;   // FV elements before e
    if (e < E) {
      if (fv) lists[E + before_fv] = e;
      else lists[e - before_fv] = e;
    }
    __syncthreads();
    if (t == 0) base_fv += warp_fv[kListThreads / 32 - 1];
    __syncthreads();
  }
  if (t == 0) {
    lists[2 * E] = E - base_fv;
    lists[2 * E + 1] = base_fv;
  }
}

// ---------------------------------------------------------------------------
// Host side: tables, set-up and launches.

// Gauss-Legendre rule of n points (Newton on P_n from the three-term recurrence).
static void gl_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int r = 0; r < n; ++r) {
    double t = std::cos(M_PI * (r + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p1 = t, p0 = 1.0;
      dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dx = p1 / dp;
      t -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (t * p1 - p0) / (t * t - 1.0);
    x[r] = t;
    w[r] = 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

// Lagrange polynomial j of the nodes x at s.
static double lagrange_at(const std::vector<double>& x, int j, double s) {
  double v = 1.0;
  for (size_t m = 0; m < x.size(); ++m)
    if ((int)m != j) v *= (s - x[m]) / (x[j] - x[m]);
  return v;
}

void fv_tables(int N, const std::vector<double>& x, std::vector<double>& tab) {
  const int n = N + 1, NN = n * n;
  const double h = 2.0 / n;
  tab.assign(2 * NN + (n + 1) * n, 0.0);
  std::vector<double> gx, gw;
  gl_rule(n, gx, gw);   // exact for the degree-N Lagrange polynomials on each sub-interval
  for (int a = 0; a < n; ++a)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s += gw[q] * lagrange_at(x, j, -1.0 + h * (a + 0.5 * (1.0 + gx[q])));
      tab[a * n + j] = 0.5 * s;
    }
  // V^-1 by Gauss-Jordan elimination with partial pivoting
  std::vector<double> A(tab.begin(), tab.begin() + NN), I(NN, 0.0);
  for (int r = 0; r < n; ++r) I[r * n + r] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    for (int k = 0; k < n; ++k) {
      std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(I[c * n + k], I[piv * n + k]);
    }
    const double dinv = 1.0 / A[c * n + c];
    for (int k = 0; k < n; ++k) {
      A[c * n + k] *= dinv;
      I[c * n + k] *= dinv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[r * n + c];
      for (int k = 0; k < n; ++k) {
        A[r * n + k] -= f * A[c * n + k];
        I[r * n + k] -= f * I[c * n + k];
      }
    }
  }
  for (int t = 0; t < NN; ++t) tab[NN + t] = I[t];
  for (int pl = 0; pl <= n; ++pl)
    for (int m = 0; m < n; ++m) tab[2 * NN + pl * n + m] = lagrange_at(x, m, -1.0 + pl * h);
}

template <int N>
static size_t fv_geom_smem() {
  using F = FvShape<N>;
  return sizeof(double) * ((size_t)F::NN + (F::n + 1) * F::n + F::P + 2 * (size_t)F::NP);
}

template <int N>
static cudaError_t fv_setup_N(const Ctx& c, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_fv_volume<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fv_volume_smem<N>());
  if (e != cudaSuccess) return e;
  k_fv_geom<N><<<c.E, FvShape<N>::P, fv_geom_smem<N>(), s>>>(c.d_metrics, c.d_J, c.d_fv_tab, c.d_fv_iJb,
                                                                c.d_fv_S, c.E);
  return cudaGetLastError();
}

template <int N>
static cudaError_t fv_stage_N(const Ctx& c, const StageArgs& a, cudaStream_t s) {
  using F = FvShape<N>;
  k_fv_means<N><<<c.E, F::P, 0, s>>>(a.U, (const double*)c.d_grad, c.d_J, c.d_fv_iJb, c.d_fv_mask, c.d_elem_nbr,
                                      c.d_fv_tab, c.d_fv_M, c.E, c.gas);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the conforming faces: an FV element has no mortar face
  if (c.nfaces_conf > 0)
    k_fv_face<N><<<(c.nfaces_conf + F::FPB - 1) / F::FPB, F::FACE_THREADS, 0, s>>>(
        c.d_faces, c.d_fv_mask, a.U, (const double*)c.d_grad, c.prm.nodes == DG_NODES_LG ? c.d_Uf : nullptr,
        c.prm.nodes == DG_NODES_LG ? c.d_gf : nullptr, c.d_fv_M, c.d_fv_S, c.d_fv_tab, c.d_fv_Fb,
        (double*)c.d_fstar, c.nfaces_conf, c.E, c.gas);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  StageArgs b = a;
  b.list = c.d_fv_lists;
  b.list_len = c.d_fv_lists + 2 * c.E;
  if ((e = launch_volume(c, b, s, false)) != cudaSuccess) return e;
  k_fv_volume<N><<<c.E, F::P, fv_volume_smem<N>(), s>>>(a, c.d_fv_lists, c.d_elem_face, c.d_elem_nbr, c.d_fv_M,
                                                         c.d_fv_S, c.d_fv_Fb, c.d_metrics, c.d_mms, c.d_fv_tab,
                                                         c.E, c.gas);
  return cudaGetLastError();
}

#define DG_FV_DISPATCH(FN, ...)              \
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

cudaError_t fv_setup(const Ctx& c, cudaStream_t s) { DG_FV_DISPATCH(fv_setup_N, c, s) }

cudaError_t launch_fv_lists(const Ctx& c, cudaStream_t s) {
  k_fv_lists<<<1, kListThreads, 0, s>>>(c.d_fv_mask, c.d_fv_lists, c.E);
  return cudaGetLastError();
}

cudaError_t launch_fv_stage(const Ctx& c, const StageArgs& a, cudaStream_t s) { DG_FV_DISPATCH(fv_stage_N, c, a, s) }

// Host reader of this file's bounds-check error word (0 in normal builds).
DG_BOUNDS_READER(bounds_word_fv)

}  // namespace dg
