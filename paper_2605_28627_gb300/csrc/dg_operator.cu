// Stage kernels of R(U) (GALAEXI Sec. 3.1, Eqs. 2-3), FP64, one thread per
// volume or face node:
//   lift   : BR1 lifting of (u, v, w, T) -> grad          (element kernel)
//   face   : Riemann + averaged viscous flux -> fstar     (face-node kernel)
// The volume kernel (split-form volume integral, surface integral, Jacobian,
// source, LSERK update) is in dg_volume.cu.
#include "dg_physics.cuh"

namespace dg {

template <int N>
struct Shape {
  static constexpr int n = N + 1;
  static constexpr int P = n * n * n;
  static constexpr int NN = n * n;
  static constexpr int EPB = P >= 128 ? 1 : (128 + P - 1) / P;   // elements per block
  static constexpr int THREADS = EPB * P;
};

// rcp for the operator type: FP64 by hardware approximation + one cubic
// Newton-Raphson step (below 1 ulp); FP32 by the approximation alone (1 ulp).
__device__ __forceinline__ double rcp_lf(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}
__device__ __forceinline__ float rcp_lf(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// BR1 lifting (Sec. 3.1, Eq. 3), strong form with the non-conservative volume
// part: g_l = (1/J)[ sum_d Ja^d_l D_d phi + sum_faces (phi* - phi) n_l sJ / w_0 ]
// with phi* = (phi + phi_nbr)/2 and the element's own outward n sJ = (2s-1) Ja^d.
// R is the operator arithmetic; metrics and the output gradients are in R.
template <int N, typename R>
__global__ void __launch_bounds__(Shape<N>::THREADS)
k_lift(const double* __restrict__ U, const R* __restrict__ metrics, const int* __restrict__ elem_nbr,
       const int* __restrict__ elem_face, const double* __restrict__ Dg, R* __restrict__ grad, int E, Gas g,
       double inv_w0d) {
  using S = Shape<N>;
  constexpr int n = S::n, P = S::P;
  __shared__ R sD[n * n];
  __shared__ R sphi[S::EPB][4][P];
  const int le = threadIdx.x / P, id = threadIdx.x % P;
  const int e = blockIdx.x * S::EPB + le;
  const bool active = e < E;
  for (int a = threadIdx.x; a < n * n; a += blockDim.x) sD[a] = R(Dg[a]);
  const R gm1 = R(g.gm1), inv_R = R(g.inv_R), inv_w0 = R(inv_w0d);
  R phi[4] = {0, 0, 0, 0};
  if (active) {
    const double* q = U + (size_t)e * 5 * P + id;
    const R rho = R(q[0]), ir = rcp_lf(rho);
    const R m0 = R(q[P]), m1 = R(q[2 * P]), m2 = R(q[3 * P]);
    const R u = m0 * ir, v = m1 * ir, w = m2 * ir;
    const R p = gm1 * (R(q[4 * P]) - R(0.5) * (m0 * u + m1 * v + m2 * w));
    phi[0] = u; phi[1] = v; phi[2] = w; phi[3] = p * ir * inv_R;
    for (int a = 0; a < 4; ++a) sphi[le][a][id] = phi[a];
  }
  __syncthreads();
  if (!active) return;
  const int i = id % n, j = (id / n) % n, k = id / (n * n);
  const int ijk[3] = {i, j, k};
  R dd[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    R s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int m = 0; m < n; ++m) {
      s0 += sD[i * n + m] * sphi[le][a][vidx<n>(m, j, k)];
      s1 += sD[j * n + m] * sphi[le][a][vidx<n>(i, m, k)];
      s2 += sD[k * n + m] * sphi[le][a][vidx<n>(i, j, m)];
    }
    dd[a][0] = s0; dd[a][1] = s1; dd[a][2] = s2;
  }
  const R* mt = metrics + (size_t)e * 10 * P + id;
  R Ja[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) Ja[r] = mt[r * P];
  R gr[12];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int l = 0; l < 3; ++l) gr[a * 3 + l] = Ja[0 * 3 + l] * dd[a][0] + Ja[1 * 3 + l] * dd[a][1] + Ja[2 * 3 + l] * dd[a][2];
  // surface part: one term per face that contains the node
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id_d = ijk[d];
    if (id_d != 0 && id_d != N) continue;
    const int s = id_d == N ? 1 : 0;
    const int f = 2 * d + s;
    const int code = elem_face[e * 6 + f];
    const int nb = elem_nbr[e * 6 + f];
    const int e2 = nb >> 3, f2 = nb & 7;
    const int p = d == 0 ? j : i;
    const int qq = d == 2 ? j : k;
    int p2, q2;
    apply_flip<n>(code & 7, p, qq, p2, q2);
    const int id2 = face_node<n>(f2, p2, q2);
    const double* q = U + (size_t)e2 * 5 * P + id2;
    const R rho = R(q[0]), ir = rcp_lf(rho);
    const R m0 = R(q[P]), m1 = R(q[2 * P]), m2 = R(q[3 * P]);
    const R u = m0 * ir, v = m1 * ir, w = m2 * ir;
    const R pr = gm1 * (R(q[4 * P]) - R(0.5) * (m0 * u + m1 * v + m2 * w));
    const R onb[4] = {u, v, w, pr * ir * inv_R};
    const R sg = s ? inv_w0 : -inv_w0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const R jump = R(0.5) * (onb[a] - phi[a]) * sg;
#pragma unroll
      for (int l = 0; l < 3; ++l) gr[a * 3 + l] += jump * Ja[d * 3 + l];
    }
  }
  const R iJ = mt[9 * P];
  R* go = grad + (size_t)e * 12 * P + id;
#pragma unroll
  for (int r = 0; r < 12; ++r) go[r * P] = gr[r] * iJ;
}

// ---------------------------------------------------------------------------
// Surface flux on every face node, master orientation (Sec. 3.1): Riemann flux
// (LLF, or the two-point EC flux) minus the BR1 average of the viscous fluxes,
// times the surface element:  F* = (F_adv(qM, qS; n) - 1/2 (f_v,M + f_v,S) . n) sJ.
template <int N, typename R>
__global__ void __launch_bounds__(128)
k_face(const double* __restrict__ U, const R* __restrict__ grad, const FaceInfo* __restrict__ faces,
       const R* __restrict__ facegeo, R* __restrict__ fstar, int F, Gas g) {
  constexpr int n = N + 1, P = n * n * n, NN = n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)F * NN) return;
  const int f = (int)(gid / NN), pq = (int)(gid % NN);
  const int p = pq % n, q = pq / n;
  const FaceInfo fi = faces[f];
  const int eM = fi.master >> 3, fM = fi.master & 7, eS = fi.slave >> 3, fS = fi.slave & 7;
  int p2, q2;
  apply_flip<n>(fi.flip, p, q, p2, q2);
  const int idM = face_node<n>(fM, p, q), idS = face_node<n>(fS, p2, q2);
  R qL[5], qR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = R(U[((size_t)eM * 5 + v) * P + idM]);
    qR[v] = R(U[((size_t)eS * 5 + v) * P + idS]);
  }
  const R gm1 = R(g.gm1), gam = R(g.gamma);
  const R* fg = facegeo + (size_t)f * 4 * NN + pq;
  const R nx = fg[0], ny = fg[NN], nz = fg[2 * NN], sJ = fg[3 * NN];
  const R irL = rcp_lf(qL[0]), irR = rcp_lf(qR[0]);
  const R uL = qL[1] * irL, vL = qL[2] * irL, wL = qL[3] * irL;
  const R uR = qR[1] * irR, vR = qR[2] * irR, wR = qR[3] * irR;
  const R pL = gm1 * (qL[4] - R(0.5) * (qL[1] * uL + qL[2] * vL + qL[3] * wL));
  const R pR = gm1 * (qR[4] - R(0.5) * (qR[1] * uR + qR[2] * vR + qR[3] * wR));
  R fa[5];
  if (g.surf_flux == DG_FLUX_EC) {
    NodePrim<R> a{qL[0], uL, vL, wL, pL, R(0.5) * qL[0] / pL};
    NodePrim<R> b{qR[0], uR, vR, wR, pR, R(0.5) * qR[0] / pR};
    ec_flux<R>(a, b, nx, ny, nz, R(g.inv_gm1), fa);
  } else {
    R fL[5], fR[5];
    euler_flux<R>(qL, uL, vL, wL, pL, nx, ny, nz, fL);
    euler_flux<R>(qR, uR, vR, wR, pR, nx, ny, nz, fR);
    const R cL = sqrt(gam * pL * irL), cR = sqrt(gam * pR * irR);
    const R lL = fabs(uL * nx + vL * ny + wL * nz) + cL;
    const R lR = fabs(uR * nx + vR * ny + wR * nz) + cR;
    const R lmax = lR > lL ? lR : lL;
#pragma unroll
    for (int v = 0; v < 5; ++v) fa[v] = R(0.5) * (fL[v] + fR[v]) - R(0.5) * lmax * (qR[v] - qL[v]);
  }
  R gL[12], gR[12];
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    gL[r] = grad[((size_t)eM * 12 + r) * P + idM];
    gR[r] = grad[((size_t)eS * 12 + r) * P + idS];
  }
  R fvL[4], fvR[4];
  const R mu = R(g.mu), lam = R(g.mu * g.kappa);
  visc_flux<R>(gL, uL, vL, wL, mu, lam, nx, ny, nz, fvL);
  visc_flux<R>(gR, uR, vR, wR, mu, lam, nx, ny, nz, fvR);
  R* fo = fstar + (size_t)f * 5 * NN + pq;
  fo[0] = fa[0] * sJ;
#pragma unroll
  for (int v = 1; v < 5; ++v) fo[(size_t)v * NN] = (fa[v] - R(0.5) * (fvL[v - 1] + fvR[v - 1])) * sJ;
}

// ---------------------------------------------------------------------------
template <int N, typename R>
static cudaError_t lift_NR(const Ctx& c, const double* U, cudaStream_t s) {
  using S = Shape<N>;
  const int blocks = (c.E + S::EPB - 1) / S::EPB;
  const R* metrics = (const R*)(sizeof(R) == 8 ? (const void*)c.d_metrics : (const void*)c.d_metrics_f);
  k_lift<N, R><<<blocks, S::THREADS, 0, s>>>(U, metrics, c.d_elem_nbr, c.d_elem_face, c.d_D, (R*)c.d_grad, c.E,
                                             c.gas, 1.0 / c.w[0]);
  return cudaGetLastError();
}

template <int N, typename R>
static cudaError_t face_NR(const Ctx& c, const double* U, cudaStream_t s) {
  const long tot = (long)c.nfaces * (N + 1) * (N + 1);
  const int blocks = (int)((tot + 127) / 128);
  const R* fgeo = (const R*)(sizeof(R) == 8 ? (const void*)c.d_facegeo : (const void*)c.d_facegeo_f);
  k_face<N, R><<<blocks, 128, 0, s>>>(U, (const R*)c.d_grad, c.d_faces, fgeo, (R*)c.d_fstar, c.nfaces, c.gas);
  return cudaGetLastError();
}

template <int N>
static cudaError_t lift_N(const Ctx& c, const double* U, bool fp64, cudaStream_t s) {
  return fp64 ? lift_NR<N, double>(c, U, s) : lift_NR<N, float>(c, U, s);
}

template <int N>
static cudaError_t face_N(const Ctx& c, const double* U, cudaStream_t s) {
  return c.prm.precision == DG_FP32OP ? face_NR<N, float>(c, U, s) : face_NR<N, double>(c, U, s);
}

#define DG_DISPATCH(FN, ...)                 \
  switch (c.N) {                             \
    case 1: return FN<1>(__VA_ARGS__);       \
    case 2: return FN<2>(__VA_ARGS__);       \
    case 3: return FN<3>(__VA_ARGS__);       \
    case 4: return FN<4>(__VA_ARGS__);       \
    case 5: return FN<5>(__VA_ARGS__);       \
    case 6: return FN<6>(__VA_ARGS__);       \
    case 7: return FN<7>(__VA_ARGS__);       \
    default: return cudaErrorInvalidValue;   \
  }

cudaError_t launch_lift(const Ctx& c, const double* U, cudaStream_t s) {
  DG_DISPATCH(lift_N, c, U, c.prm.precision != DG_FP32OP, s)
}
cudaError_t launch_lift_fp64(const Ctx& c, const double* U, cudaStream_t s) { DG_DISPATCH(lift_N, c, U, true, s) }
cudaError_t launch_face(const Ctx& c, const double* U, cudaStream_t s) { DG_DISPATCH(face_N, c, U, s) }
cudaError_t setup_kernels(int N) { return setup_volume(N); }

}  // namespace dg
