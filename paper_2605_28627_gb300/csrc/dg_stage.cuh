// Stage-kernel bodies of R(U) (GALAEXI Sec. 3.1, Eqs. 2-3), shared by the
// single-context kernels and the persistent ensemble kernels.  Each body
// processes one tile (EPB elements, or one block of face nodes) given by an
// explicit tile index, so the same code runs with blockIdx or a tile table.
//
// Volume body -- FP64-pipe-aware design (also used in FP32):
//  * Symmetric pair reuse: F#(q_i, q_m) = F#(q_m, q_i), so each unordered
//    pair on a line is evaluated once, in rounds of a fixed cyclic shift s;
//    the partner's share goes through shared memory.  For even n the last
//    shift (s = n/2) pairs each node with the opposite one, so it holds only
//    half as many pairs as nodes: those are packed onto the first threads of
//    the sweep's exchange group (whole warps idle instead of every other
//    lane, which the narrow FP64 pipe would still charge) and both shares go
//    through shared memory.
//  * Barriers span only a sweep's exchange group where that is a whole
//    number of warps (a k-plane for the xi and eta sweeps at N = 7, an
//    element when a block holds several).
//  * The diagonal terms 2 D_ii f(q_i) . Ja_i vanish for interior LGL nodes
//    and cancel exactly against the -f . n sJ / w_0 part of the surface term
//    at the two end nodes (2 D_00 = -1/w_0, 2 D_NN = 1/w_0), so neither is
//    evaluated.
//  * Reciprocals instead of divides, logarithmic means by the Ismail-Roe
//    series with the reciprocal series for 1/F, constant factors folded into
//    scaled copies of D (FP64) or applied once to the sums (FP32), the
//    series/log switch decided in integer ALU (FP64) or by one warp vote
//    (FP32).
//  * The viscous part of the surface term rides in the diagonal of the
//    viscous line sums; the lifting's face jumps start its line sums.
#pragma once

#include "dg_bulk.cuh"
#include "dg_physics.cuh"

namespace dg {

// Element tiles: EPB elements per block, one thread per node.  The default
// packs small elements until a block has at least 128 threads.
constexpr int default_epb(int P) { return P >= 128 ? 1 : (128 + P - 1) / P; }

template <int N, int EPB_ = default_epb((N + 1) * (N + 1) * (N + 1))>
struct Shape {
  static constexpr int n = N + 1;
  static constexpr int P = n * n * n;
  static constexpr int NN = n * n;
  static constexpr int EPB = EPB_;
  static constexpr int THREADS = EPB * P;
};

template <int N, int EPB_ = default_epb((N + 1) * (N + 1) * (N + 1))>
struct VShape : Shape<N, EPB_> {
  static constexpr int ROUNDS = (N + 1) / 2;    // shifts s = 1..n/2 (s = n/2 half-used for even n)
};

// Blocks per SM the single-context volume kernel's register and shared-memory
// budget must allow.  FP32 (latency-bound): enough for about 32 warps per SM at
// N <= 5 (+8 to +16 % at N = 2, 4, 5 over two blocks; 48 warps lost 6 to 23 %
// there), 33 to 48 at N = 6..8, where a hundred-odd bytes of spilled registers
// per thread pay.  FP64 at N = 6, 7: two -- a hundred-odd bytes of spilled
// registers cost less than an SM with only 11 or 16 warps to feed its FP64
// pipe from (+2.4 % at N = 6, +0.5 % at N = 7; at N = 4, 5 a third block did
// not pay).
template <int N, typename R>
constexpr int vol_min_blocks() {
  constexpr int threads = Shape<N>::THREADS;
  if (sizeof(R) == 4) {
    if (N == 6 || N == 7) return 3;                 // 33 and 48 warps: +11 %, +1 %
    if (N == 8) return 2;                           // 46 warps: +10 %
    return threads <= 512 ? (1024 / threads > 2 ? 1024 / threads : 2) : 1;
  }
  return (N == 6 || N == 7) ? 2 : 1;
}

// Exchange buffers of the pair loop: one per round when they fit the shared
// memory of vol_min_blocks blocks per SM (all rounds of a direction then share
// one barrier), else one (a barrier per round).  The choice fixes the order in
// which a node sums its pair terms, so every kernel that runs the volume body
// for this (N, R) -- the single-context tile and both ensemble tiles -- takes
// the same value and gives bit-identical results.
template <int N, typename R>
struct VXbuf {
  static constexpr int P = (N + 1) * (N + 1) * (N + 1), ROUNDS = (N + 1) / 2, EPB = Shape<N>::EPB,
                       MINB = vol_min_blocks<N, R>();
  static constexpr size_t base_words = 3 * (N + 1) * (N + 1) + (((N + 1) * (N + 1) + 3) & ~3) +
                                       (size_t)EPB * (21 + (sizeof(R) == 4 ? 1 : 0)) * P;
  static constexpr size_t budget = MINB == 1 ? 200 * 1024 : (226 * 1024) / MINB - 1024;
  static constexpr int value = sizeof(R) * (base_words + (size_t)EPB * 5 * P * ROUNDS) <= budget ? ROUNDS : 1;
  static constexpr int PER_ELEM = (21 + 5 * value) * P;   // operator words of smem per element
};

template <int N, typename R, int EPB>
constexpr size_t volume_smem_bytes() {
  // the FP32 operator keeps one more word per node (the offset pressure term)
  return sizeof(R) * (3 * (N + 1) * (N + 1) + (((N + 1) * (N + 1) + 3) & ~3) + EPB * VXbuf<N, R>::PER_ELEM +
                      (sizeof(R) == 4 ? EPB * (N + 1) * (N + 1) * (N + 1) : 0));
}

// 1/x: hardware reciprocal approximation refined by one cubic Newton-Raphson
// step y <- y (1 + e + e^2), e = 1 - x y, which cubes the relative error
// (2^-20 -> below 1 ulp).  In FP32 the approximation alone is within 1 ulp.
// The .ftz forms flush subnormals: valid for positive normal x whose
// reciprocal is normal (a subnormal 1/x becomes 0, a zero or subnormal x
// gives a non-finite result), which covers the operators' densities,
// pressures and their sums.  dg_check_reciprocals tests these bounds.
__device__ __forceinline__ double rcp_op(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  const double t = fma(e, e, e);
  return fma(y, t, y);
}
// 1/x with one quadratic Newton-Raphson step y <- y + y e (relative error
// ~2^-40), for reciprocals whose error is damped by the use
__device__ __forceinline__ double rcp_op_q(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  return fma(y, fma(-x, y, 1.0), y);
}
__device__ __forceinline__ float rcp_op_q(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_op(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---------------------------------------------------------------------------
// BR1 lifting (Sec. 3.1, Eq. 3), strong form with the non-conservative volume
// part: g_l = (1/J)[ sum_d Ja^d_l D_d phi + sum_faces (phi* - phi) n_l sJ / w_0 ]
// with phi* = (phi + phi_nbr)/2 and the element's own outward n sJ = (2s-1) Ja^d.
// R is the operator arithmetic; metrics and the output gradients are in R.
//
// The face jumps (phi* - phi)(+-1/w_0) are computed once per face point by
// threads packed over the element's 6 (N+1)^2 face points (the neighbour
// primitives and the differences would otherwise run on every node thread of
// a warp that holds one face node: on the narrow FP64 pipe masked lanes cost
// as much as active ones) and kept in shared memory; a node thread starts its
// line sums of direction d from the jump of its d-face, so the surface term
// costs it no arithmetic.
template <int N, typename R, int EPB>
constexpr size_t lift_smem_bytes() {
  // [EPB][4][P] primitives phi, [EPB][6][4][n^2] face jumps
  return sizeof(R) * (size_t)EPB * (4 * (N + 1) * (N + 1) * (N + 1) + 24 * (N + 1) * (N + 1));
}

// MORTAR: a face whose neighbour entry is negative is a mortar side, whose
// neighbour state (the big face's interpolated state on a quadrant, or the
// state that gives the projected face average on a big face) is read from
// mvirt[-1 - entry][5][NN] (entry -1 - (5 m + side), m < n_mortar) in the
// side's own face-node order.
template <int N, typename R, int EPB, bool MORTAR = false>
__device__ __forceinline__ void lift_body(const double* __restrict__ U, const R* __restrict__ metrics,
                                          const int* __restrict__ elem_nbr, const int* __restrict__ elem_face,
                                          const double* __restrict__ Dg, R* __restrict__ grad, int E, const Gas& g,
                                          double inv_w0d, int blk, const double* __restrict__ mvirt = nullptr,
                                          int n_mortar = 0) {
  using S = Shape<N, EPB>;
  constexpr int n = S::n, P = S::P, NN = S::NN, NF = 6 * NN;
  constexpr int NI = (EPB * NF + S::THREADS - 1) / S::THREADS;   // face points per thread
  __shared__ R sD[n * n];
  extern __shared__ __align__(16) unsigned char lift_raw[];
  R* sphi = reinterpret_cast<R*>(lift_raw);   // [EPB][4][P]
  R* sjmp = sphi + EPB * 4 * P;               // [EPB][6][4][NN]
  const int le = threadIdx.x / P, id = threadIdx.x % P;
  const int e = blk * S::EPB + le;
  const bool active = e < E;
  // neighbour state at face point t (element le2, face f, point pq)
  auto load_nbr = [&](int t, double qv[5]) {
    const int le2 = t / NF, r2 = t - le2 * NF;
    const int e2 = blk * EPB + le2;
    if (t < EPB * NF && e2 < E) {
      const int f = r2 / NN, pq = r2 - f * NN;
      const int code = elem_face[e2 * 6 + f], nb = elem_nbr[e2 * 6 + f];
      if constexpr (MORTAR) {
        if (nb < 0) {
          const double* q = mvirt + (size_t)dg_idx(-1 - nb, 5L * n_mortar, kSiteMortar) * 5 * NN + pq;
#pragma unroll
          for (int v = 0; v < 5; ++v) qv[v] = q[v * NN];
          return;
        }
      }
      int p2, q2;
      apply_flip<n>(code & 7, pq % n, pq / n, p2, q2);
      const int enb = dg_idx(nb >> 3, E, kSiteLiftNbr);
      const double* q = U + (size_t)enb * 5 * P + face_node<n>(nb & 7, p2, q2);
#pragma unroll
      for (int v = 0; v < 5; ++v) qv[v] = q[v * P];
    }
  };
  // with one face point per thread its neighbour state is loaded before the
  // first barrier (latency hidden behind the primitives), else in the pass
  double qn[5];
  if constexpr (NI == 1) load_nbr(threadIdx.x, qn);
  for (int a = threadIdx.x; a < n * n; a += blockDim.x) sD[a] = to_op<R>(Dg[a]);
  const R gm1 = gsel<R>(g.gm1, g.f_gm1), inv_R = gsel<R>(g.inv_R, g.f_inv_R), inv_w0 = to_op<R>(inv_w0d);
  if (active) {
    const double* q = U + (size_t)e * 5 * P + id;
    const R rho = to_op<R>(q[0]), ir = rcp_op(rho);
    const R m0 = to_op<R>(q[P]), m1 = to_op<R>(q[2 * P]), m2 = to_op<R>(q[3 * P]);
    const R u = m0 * ir, v = m1 * ir, w = m2 * ir;
    const R p = gm1 * (to_op<R>(q[4 * P]) - R(0.5) * (m0 * u + m1 * v + m2 * w));
    const R phi[4] = {u, v, w, p * ir * inv_R};
#pragma unroll
    for (int a = 0; a < 4; ++a) sphi[(le * 4 + a) * P + id] = phi[a];
  }
  __syncthreads();
  // face jumps (phi_nbr - phi)/2 (+-1/w_0), whole warps over the face points
#pragma unroll 1
  for (int it = 0; it < NI; ++it) {
    const int t = threadIdx.x + it * S::THREADS;
    const int le2 = t / NF, r2 = t - le2 * NF;
    if constexpr (NI > 1) load_nbr(t, qn);
    if (t < EPB * NF && blk * EPB + le2 < E) {
      const int f = r2 / NN, pq = r2 - f * NN;
      const int node = face_node<n>(f, pq % n, pq / n);
      const R rho = to_op<R>(qn[0]), ir = rcp_op(rho);
      const R m0 = to_op<R>(qn[1]), m1 = to_op<R>(qn[2]), m2 = to_op<R>(qn[3]);
      const R u = m0 * ir, v = m1 * ir, w = m2 * ir;
      const R pr = gm1 * (to_op<R>(qn[4]) - R(0.5) * (m0 * u + m1 * v + m2 * w));
      const R onb[4] = {u, v, w, pr * ir * inv_R};
      const R hs = (f & 1) ? R(0.5) * inv_w0 : R(-0.5) * inv_w0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
        sjmp[((le2 * 6 + f) * 4 + a) * NN + pq] = (onb[a] - sphi[(le2 * 4 + a) * P + node]) * hs;
    }
  }
  __syncthreads();
  if (!active) return;
  // g_l = (1/J) sum_d Ja^d_l (D_d phi + jump_d): the surface term of a face in
  // direction d multiplies the same metric term as that direction's volume
  // term, so the jump (zero off the face) starts the line sum
  const int i = id % n, j = (id / n) % n, k = id / (n * n);
  const int ijk[3] = {i, j, k};
  const R* jm[3] = {nullptr, nullptr, nullptr};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id_d = ijk[d];
    if (id_d == 0 || id_d == N)
      jm[d] = sjmp + (le * 6 + 2 * d + (id_d == N ? 1 : 0)) * 4 * NN + (d == 0 ? j : i) + n * (d == 2 ? j : k);
  }
  const R* ph = sphi + le * 4 * P;
  R dd[4][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    R s0 = jm[0] ? jm[0][a * NN] : R(0), s1 = jm[1] ? jm[1][a * NN] : R(0), s2 = jm[2] ? jm[2][a * NN] : R(0);
#pragma unroll
    for (int m = 0; m < n; ++m) {
      s0 += sD[i * n + m] * ph[a * P + vidx<n>(m, j, k)];
      s1 += sD[j * n + m] * ph[a * P + vidx<n>(i, m, k)];
      s2 += sD[k * n + m] * ph[a * P + vidx<n>(i, j, m)];
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
    for (int l = 0; l < 3; ++l)
      gr[a * 3 + l] = Ja[0 * 3 + l] * dd[a][0] + Ja[1 * 3 + l] * dd[a][1] + Ja[2 * 3 + l] * dd[a][2];
  const R iJ = mt[9 * P];
  R* go = grad + (size_t)e * 12 * P + id;
#pragma unroll
  for (int r = 0; r < 12; ++r) go[r * P] = gr[r] * iJ;
}

// ---------------------------------------------------------------------------
// Surface flux on every face node, master orientation (Sec. 3.1): Riemann flux
// (LLF, or the two-point EC flux) minus the BR1 average of the viscous fluxes,
// times the surface element:  F* = (F_adv(qM, qS; n) - 1/2 (f_v,M + f_v,S) . n) sJ.
// Numerical flux at one face point from the two sides' FP64 states (dL, dR)
// and lifted gradients (gL, gR), unit normal n of the master side and surface
// element sJ: writes F* (5 values, `stride` apart) to fo.
template <typename R>
__device__ __forceinline__ void face_flux_core(const double dL[5], const double dR[5], const R gL[12],
                                               const R gR[12], R nx, R ny, R nz, R sJ, const Gas& g, R* fo,
                                               size_t stride) {
  R qL[5], qR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = to_op<R>(dL[v]);
    qR[v] = to_op<R>(dR[v]);
  }
  const R gm1 = gsel<R>(g.gm1, g.f_gm1), gam = gsel<R>(g.gamma, g.f_gamma);
  const R irL = rcp_op(qL[0]), irR = rcp_op(qR[0]);
  const R uL = qL[1] * irL, vL = qL[2] * irL, wL = qL[3] * irL;
  const R uR = qR[1] * irR, vR = qR[2] * irR, wR = qR[3] * irR;
  const R pL = gm1 * (qL[4] - R(0.5) * (qL[1] * uL + qL[2] * vL + qL[3] * wL));
  const R pR = gm1 * (qR[4] - R(0.5) * (qR[1] * uR + qR[2] * vR + qR[3] * wR));
  // Pressure in the momentum flux.  The FP32 operator uses p - p_ref with the
  // energy difference E - p_ref/(gamma-1) taken in FP64 (one add per node):
  // a constant pressure has no discrete divergence (metric identities), so R
  // is unchanged, while the FP32 rounding of a large background pressure
  // (low Mach numbers) no longer enters the momentum equations.
  R pmL = pL, pmR = pR;
  if constexpr (sizeof(R) == 4) {
    pmL = gm1 * (to_op<R>(dL[4] - g.E_ref) - R(0.5) * (qL[1] * uL + qL[2] * vL + qL[3] * wL));
    pmR = gm1 * (to_op<R>(dR[4] - g.E_ref) - R(0.5) * (qR[1] * uR + qR[2] * vR + qR[3] * wR));
  }
  // State jumps for the dissipation terms: in FP32 mode taken from the FP64
  // states before rounding, so that a small jump of a large quantity (the
  // energy at low Mach numbers) keeps its digits.
  R dq[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    if constexpr (sizeof(R) == 4) dq[v] = to_op<R>(dR[v] - dL[v]);
    else dq[v] = qR[v] - qL[v];
  }
  R fa[5];
  if (g.surf_flux == DG_FLUX_EC) {
    NodePrim<R> a{qL[0], uL, vL, wL, pL, R(0.5) * qL[0] / pL};
    NodePrim<R> b{qR[0], uR, vR, wR, pR, R(0.5) * qR[0] / pR};
    if constexpr (sizeof(R) == 4)
      ec_flux_off<R>(a, b, qL[0] * pmL / pL, qR[0] * pmR / pR, gsel<R>(g.p_ref, g.f_p_ref), nx, ny, nz,
                     gsel<R>(g.inv_gm1, g.f_inv_gm1), fa);
    else
      ec_flux<R>(a, b, nx, ny, nz, gsel<R>(g.inv_gm1, g.f_inv_gm1), fa);
  } else if (g.surf_flux == DG_FLUX_ROE) {
    roe_flux<R>(qL, uL, vL, wL, pL, qR, uR, vR, wR, pR, nx, ny, nz, gam, gm1, fa, pmL, pmR, dq[0]);
  } else {
    R fL[5], fR[5];
    euler_flux_pm<R>(qL, uL, vL, wL, pL, pmL, nx, ny, nz, fL);
    euler_flux_pm<R>(qR, uR, vR, wR, pR, pmR, nx, ny, nz, fR);
    const R cL = sqrt(gam * pL * irL), cR = sqrt(gam * pR * irR);
    const R lL = fabs(uL * nx + vL * ny + wL * nz) + cL;
    const R lR = fabs(uR * nx + vR * ny + wR * nz) + cR;
    const R lmax = lR > lL ? lR : lL;
#pragma unroll
    for (int v = 0; v < 5; ++v) fa[v] = R(0.5) * (fL[v] + fR[v]) - R(0.5) * lmax * dq[v];
  }
  R fvL[4], fvR[4];
  const R mu = gsel<R>(g.mu, g.f_mu), lam = gsel<R>(g.mu * g.kappa, g.f_lam);
  R sfL = R(1), sfR = R(1);
  if (g.visc_law == DG_VISC_SUTHERLAND) {
    const R inv_R = gsel<R>(g.inv_R, g.f_inv_R);
    sfL = visc_factor<R>(g, pL * irL * inv_R);
    sfR = visc_factor<R>(g, pR * irR * inv_R);
  }
  visc_flux<R>(gL, uL, vL, wL, mu * sfL, lam * sfL, nx, ny, nz, fvL);
  visc_flux<R>(gR, uR, vR, wR, mu * sfR, lam * sfR, nx, ny, nz, fvR);
  fo[0] = fa[0] * sJ;
#pragma unroll
  for (int v = 1; v < 5; ++v) fo[(size_t)v * stride] = (fa[v] - R(0.5) * (fvL[v - 1] + fvR[v - 1])) * sJ;
}

template <int N, typename R>
__device__ __forceinline__ void face_body(const double* __restrict__ U, const R* __restrict__ grad,
                                          const FaceInfo* __restrict__ faces, const R* __restrict__ facegeo,
                                          R* __restrict__ fstar, int F, int E, const Gas& g, long gid) {
  constexpr int n = N + 1, P = n * n * n, NN = n * n;
  if (gid >= (long)F * NN) return;
  const int f = (int)(gid / NN), pq = (int)(gid % NN);
  const int p = pq % n, q = pq / n;
  const FaceInfo fi = faces[f];
  // every local face of a periodic mesh has a neighbour: F = 3 E
  const int eM = dg_idx(fi.master >> 3, E, kSiteFaceElems), fM = fi.master & 7;
  const int eS = dg_idx(fi.slave >> 3, E, kSiteFaceElems), fS = fi.slave & 7;
  int p2, q2;
  apply_flip<n>(fi.flip, p, q, p2, q2);
  const int idM = face_node<n>(fM, p, q), idS = face_node<n>(fS, p2, q2);
  double dL[5], dR[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    dL[v] = U[((size_t)eM * 5 + v) * P + idM];
    dR[v] = U[((size_t)eS * 5 + v) * P + idS];
  }
  R gL[12], gR[12];
#pragma unroll
  for (int r = 0; r < 12; ++r) {
    gL[r] = grad[((size_t)eM * 12 + r) * P + idM];
    gR[r] = grad[((size_t)eS * 12 + r) * P + idS];
  }
  const R* fg = facegeo + (size_t)f * 4 * NN + pq;
  face_flux_core<R>(dL, dR, gL, gR, fg[0], fg[NN], fg[2 * NN], fg[3 * NN], g, fstar + (size_t)f * 5 * NN + pq, NN);
}

// Switch of the logarithmic mean between the series and the logarithm.  In
// FP64 below u = 1e-4 (four series terms are exact to rounding; decided on the
// high word in integer ALU), in FP32 below u = 1e-2 (truncation < 1e-9).
__device__ __forceinline__ bool small_u(double u) { return __double2hiint(u) < 0x3F1A36E2; }
__device__ __forceinline__ bool small_u(float u) { return u < 1e-2f; }

// 1/F(u) = u^(1/2) / atanh(u^(1/2)) = 1 - u/3 - 4u^2/45 - 44u^3/945 - ...
template <typename R>
__device__ __forceinline__ R inv_atanh_ratio(R u) {
  return fma(u, fma(u, fma(u, R(-44.0 / 945.0), R(-4.0 / 45.0)), R(-1.0 / 3.0)), R(1));
}
// F(u) = atanh(u^(1/2)) / u^(1/2) = 1 + u/3 + u^2/5 + u^3/7 + ...
template <typename R>
__device__ __forceinline__ R atanh_ratio(R u) {
  return fma(u, fma(u, fma(u, R(1.0 / 7.0), R(1.0 / 5.0)), R(1.0 / 3.0)), R(1));
}
// F for the logarithmic branch, in the ratio form of Ismail & Roe.
template <typename R>
__device__ __noinline__ R atanh_ratio_log(R a, R b) {
  const R z = a / b;
  return log(z) / (R(2) * ((z - R(1)) / (z + R(1))));
}

// Named barrier: the `count` threads (whole warps) of group `id` (1..15), the
// number taken from a register.  ptxas then reserves all 16 hardware barriers
// for the kernel, which limits it to four blocks per SM: for kernels that run
// fewer blocks anyway (one 512-thread element per block).
__device__ __forceinline__ void bar_sync_reg(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// The same with the barrier number an immediate in every branch of a switch,
// so that ptxas reserves only MAXID + 1 barriers (1 <= id <= MAXID <= 15): for
// kernels of small blocks that need more than four per SM.
template <int MAXID>
__device__ __forceinline__ void bar_sync(int id, int count) {
  static_assert(MAXID >= 1 && MAXID <= 15, "named barriers 1..15");
#define DG_BAR_CASE(k) \
  case k:              \
    if constexpr (k <= MAXID) asm volatile("bar.sync %0, %1;" ::"n"(k), "r"(count) : "memory"); \
    break;
  switch (id) {
    DG_BAR_CASE(1) DG_BAR_CASE(2) DG_BAR_CASE(3) DG_BAR_CASE(4) DG_BAR_CASE(5)
    DG_BAR_CASE(6) DG_BAR_CASE(7) DG_BAR_CASE(8) DG_BAR_CASE(9) DG_BAR_CASE(10)
    DG_BAR_CASE(11) DG_BAR_CASE(12) DG_BAR_CASE(13) DG_BAR_CASE(14) DG_BAR_CASE(15)
    default: break;
  }
#undef DG_BAR_CASE
}

// Bulk prefetch of [p, p + bytes) into L2, trimmed inward to 16-byte
// boundaries (the instruction's alignment rule); a hint, no data is returned.
__device__ __forceinline__ void l2_prefetch(const void* p, size_t bytes) {
  const size_t a = reinterpret_cast<size_t>(p);
  const size_t lo = (a + 15) & ~size_t(15), hi = (a + bytes) & ~size_t(15);
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

// Chandrashekar's two-point flux of one node pair (a, b) in one direction,
// scaled for the scaled copies of D: F = (8 f_rho, 16 f_m, 32 f_E).  Taken as
// densities and b = beta/4 = rho/(8p) of both nodes and the pair sums of
// velocity su = u_a + u_b, |u|^2 (sk), metric term sn = Ja^d_a + Ja^d_b and,
// for the FP32 operator, rho (p - p_ref)/p (sdl; unused in FP64).  The factor
// 1/4 on beta (exact) folds the 4 of 16 p_hat into the reciprocal.
template <typename R>
__device__ __forceinline__ void ec_pair(R ra, R rb, R ba, R bb, R su0, R su1, R su2, R sk, R sdl, R sn0, R sn1,
                                        R sn2, R inv_gm1, const Gas& g, R F[5]) {
  const R sr = ra + rb, sb = ba + bb;
  // 1/(rho_a + rho_b) enters only through u_rho = fr^2 < 1e-4 on the series
  // branch, so one quadratic Newton step (relative error ~1e-12) suffices
  const R rr = rcp_op_q(sr), rbt = rcp_op(sb);   // rbt = 4/(beta_a + beta_b)
  const R fr = (ra - rb) * rr, fb = (ba - bb) * rbt;
  const R ur = fr * fr, ubt = fb * fb;
  R rln2, hib;                    // 2 rho_ln and 2/beta_ln
  bool all_series = false;
  // FP32 operator: one warp vote instead of two divergent branches per pair
  // (the issue slots, not the FP32 pipe, bound that kernel); a smooth field
  // takes the series for every pair
  if constexpr (sizeof(R) == 4) all_series = __all_sync(__activemask(), small_u(ur) && small_u(ubt));
  if (all_series) {
    rln2 = sr * inv_atanh_ratio(ur);
    hib = atanh_ratio(ubt) * rbt;
  } else {
    if (small_u(ur)) rln2 = sr * inv_atanh_ratio(ur);
    else rln2 = sr / atanh_ratio_log(ra, rb);
    if (small_u(ubt)) hib = atanh_ratio(ubt) * rbt;
    else hib = atanh_ratio_log(ba, bb) * rbt;
  }
  const R un4 = fma(su0, sn0, fma(su1, sn1, su2 * sn2));
  const R Xf = rln2 * un4;                      // 8 f_rho
  // 16 p_hat n_avg = Y4 (n_a + n_b); the FP32 operator uses p_hat - p_ref
  R Y4 = sr * rbt;
  if constexpr (sizeof(R) == 4) Y4 = sdl * rbt;
  const R M0 = fma(Xf, su0, Y4 * sn0);          // 16 f_m
  const R M1 = fma(Xf, su1, Y4 * sn1);
  const R M2 = fma(Xf, su2, Y4 * sn2);
  const R Z = fma(hib, inv_gm1, -sk);
  R E32 = fma(Xf, Z, fma(su0, M0, fma(su1, M1, su2 * M2)));   // 32 f_E
  if constexpr (sizeof(R) == 4) E32 = fma(R(8) * g.f_p_ref, un4, E32);     // p_ref {u}.n back
  F[0] = Xf; F[1] = M0; F[2] = M1; F[3] = M2; F[4] = E32;
}

// R is the operator arithmetic: double (FP64 path) or float (FP32-operator
// path, state and RK update stay FP64).  metrics, grad and fstar are stored in R.
// Manufactured source, density wave rho = 2 + A sin(phi), phi = pi (x+y+z-t),
// u = (1,1,1), p = 1: residual of Eq. 1 = [2r', 2r', 2r', 2r', 3r' - lambda Lap T],
// r' = pi A cos(phi).  sin/cos of phi from those of pi (x+y+z) (per node, set
// up once: mms [E][2][P]) and of pi t (st, ct; once per block) by the
// angle-difference identities.  Evaluated in the operator type.
template <typename R>
__device__ __forceinline__ void mms_source(const Gas& g, const double* __restrict__ mms, int e, int P, int id,
                                           double st_d, double ct_d, R src[5]) {
  const R sa = to_op<R>(mms[((size_t)e * 2) * P + id]), ca = to_op<R>(mms[((size_t)e * 2 + 1) * P + id]);
  const R st = to_op<R>(st_d), ct = to_op<R>(ct_d);
  const R sphi = fma(sa, ct, -ca * st);
  const R cphi = fma(ca, ct, sa * st);
  const R A = gsel<R>(g.mms_amp, g.f_mms_amp);
  const R rw = R(2) + A * sphi;
  const R irw = rcp_op(rw);
  const R rp = R(M_PI) * A * cphi;
  const R lapT = R(3) * gsel<R>(g.inv_R, g.f_inv_R) * fma(R(M_PI) * R(M_PI) * A, sphi, R(2) * rp * rp * irw) *
                 (irw * irw);
  src[0] = src[1] = src[2] = src[3] = R(2) * rp;
  src[4] = fma(-gsel<R>(g.mu * g.kappa, g.f_lam), lapT, R(3) * rp);
}

// LIST: the element slots come from a.list (the DG elements when FV sub-cell
// elements exist); without it slot = element, as in every other launch.
template <int N, typename R, int EPB_, bool LIST = false>
__device__ __forceinline__ void volume_body(const StageArgs& a, const R* __restrict__ metrics,
                                            const double* __restrict__ iJ64, const R* __restrict__ grad,
                                            const R* __restrict__ fstar, const int* __restrict__ elem_face,
                                            const double* __restrict__ mms, const double* __restrict__ Dg, int E,
                                            const Gas& g, double inv_w0d, int blk) {
  using S = VShape<N, EPB_>;
  constexpr int n = S::n, P = S::P, NN = S::NN, EPB = S::EPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* smem = reinterpret_cast<R*>(smem_raw);
  R* sD = smem;                       // D
  R* sT0 = sD + n * n;                // D/4   (mass: X = 8 f_rho)
  R* sT1 = sT0 + n * n;               // D/8   (momentum: M = 16 f_m)
  R* sT2 = sT1 + n * n;               // D/16  (energy: 32 f_E)
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  constexpr int XB = VXbuf<N, R>::value;
  constexpr int PER_ELEM = VXbuf<N, R>::PER_ELEM;
  R* const tile0 = sT2 + ((n * n + 3) & ~3);   // element tiles, PER_ELEM words each
  R* base = tile0 + le * PER_ELEM;
  R* sR = base;                       // rho
  R* sU = sR + P;                     // u, v, w
  R* sB = sU + 3 * P;                 // beta / 4 = rho / (8 p)
  R* sK = sB + P;                     // |u|^2
  R* sJd = sK + P;                    // [3][P]  Ja^d of the direction being swept
  R* sFv = sJd + 3 * P;               // [3][4][P] (f_v . Ja^d), momentum + energy
  R* sX = sFv + 12 * P;               // [XB][5][P] exchange of partner shares (one per round if XB > 1)
  R* sDl = tile0 + EPB * PER_ELEM + le * P;   // FP32 only: rho (p - p_ref) / p
  // element slot -> element (with LIST, idle slots past the list's end)
  int nslot = E, e = blk * EPB + le;
  if constexpr (LIST) {
    nslot = *a.list_len;
    e = e < nslot ? a.list[e] : E;
    if constexpr (EPB == 1) {
      if (e >= E) return;   // the whole block, before any barrier
    }
  }
  const bool active = e < E;
  __shared__ double s_tc[3];          // sin, cos of pi t (manufactured source); B_s dt (FP32 operator)
  if (threadIdx.x == 0) {
    if (g.source == DG_SOURCE_MMS) sincospi(a.clock[0] + a.c_stage * a.clock[1], &s_tc[0], &s_tc[1]);
    if constexpr (sizeof(R) == 4) s_tc[2] = a.B * a.clock[1];
  }
  // The epilogue's operands (LSERK register, 1/J, source phases) and the face
  // fluxes are read only after the sweeps: ask for them in L2 now, one bulk
  // prefetch per contiguous range, so that those loads do not wait on DRAM.
  if (active && id < 9) {
    if (id == 0 && a.mode == 1) l2_prefetch(a.Gk + (size_t)e * 5 * P, 5 * P * sizeof(double));
    else if (id == 1) {
      if constexpr (sizeof(R) == 8) l2_prefetch(iJ64 + (size_t)e * 10 * P + 9 * P, P * sizeof(double));
      else l2_prefetch(metrics + (size_t)e * 10 * P + 9 * P, P * sizeof(R));
    } else if (id == 2 && g.source == DG_SOURCE_MMS) l2_prefetch(mms + (size_t)e * 2 * P, 2 * P * sizeof(double));
    else if (id >= 3)
      l2_prefetch(fstar + (size_t)dg_idx(elem_face[e * 6 + id - 3] >> 4, a.nfaces > 0 ? a.nfaces : 3L * E,
                                         kSiteVolFace) * 5 * NN,
                  5 * NN * sizeof(R));
  }
  const R inv_w0 = to_op<R>(inv_w0d);
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const double d = Dg[t];
    const R dr = to_op<R>(d);       // the scalings by powers of two are exact
    // sD's diagonal is read only by the viscous line sums: at the two end
    // nodes it carries the viscous part of the surface term too,
    // D_00 + 1/w_0 and D_NN - 1/w_0 (the pair sweeps use m != r only)
    sD[t] = t == 0 ? dr + inv_w0 : (t == n * n - 1 ? dr - inv_w0 : dr);
    sT0[t] = R(0.25) * dr;
    sT1[t] = R(0.125) * dr;
    sT2[t] = R(0.0625) * dr;
  }
  // FP64: each element's state (5P contiguous doubles) comes into shared
  // memory by a bulk copy (cp.async.bulk) issued by its first thread, into the
  // region of the metric terms and viscous fluxes, which the prologue fills
  // only after every node has read its state; the metric terms are loaded
  // meanwhile.
  // FP32: per-thread loads (the bulk staging measured 2-6 % slower there: the
  // FP32 kernel is latency-bound and its two extra barriers are not hidden).
  double q[5] = {0, 0, 0, 0, 0};
  R Ja[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if constexpr (sizeof(R) == 8) {
    // one barrier per element, initialised and armed by the element's first thread
    __shared__ uint64_t s_bar[EPB];
    if (active && id == 0) {
      const double* src = a.U + (size_t)e * 5 * P;
      bulk_bar_init(&s_bar[le]);
      bulk_expect(&s_bar[le], bulk_middle_bytes(src, 5 * P));
      bulk_stage_range(bulk_stage_ptr(sJd, src), src, 5 * P, &s_bar[le]);
    }
    if (active) {
      const R* mt = metrics + (size_t)e * 10 * P + id;
#pragma unroll
      for (int r = 0; r < 9; ++r) Ja[r] = mt[r * P];
    }
    __syncthreads();   // the barriers are initialised, the head and tail doubles stored
    if (active) {
      bulk_wait(&s_bar[le], 0);
      const double* st = bulk_stage_ptr(sJd, a.U + (size_t)e * 5 * P);
#pragma unroll
      for (int r = 0; r < 5; ++r) q[r] = st[r * P + id];
    }
    __syncthreads();   // every node has its state: the region is free
    if (active && id == 0) bulk_bar_inval(&s_bar[le]);   // re-initialised by the next tile of a persistent kernel
  } else {
    if (active) {
#pragma unroll
      for (int r = 0; r < 5; ++r) q[r] = a.U[((size_t)e * 5 + r) * P + id];
      const R* mt = metrics + (size_t)e * 10 * P + id;
#pragma unroll
      for (int r = 0; r < 9; ++r) Ja[r] = mt[r * P];
    }
  }
  R rho = R(1), u = 0, v = 0, w = 0, beta = 0, kk = 0;
  if (active) {
    rho = to_op<R>(q[0]);
    const R ir = rcp_op(rho);
    u = to_op<R>(q[1]) * ir; v = to_op<R>(q[2]) * ir; w = to_op<R>(q[3]) * ir;
    kk = u * u + v * v + w * w;
    const R p = gsel<R>(g.gm1, g.f_gm1) * fma(R(-0.5) * rho, kk, to_op<R>(q[4]));
    beta = R(0.125) * rho * rcp_op(p);   // beta / 4
    sR[id] = rho; sU[id] = u; sU[P + id] = v; sU[2 * P + id] = w; sB[id] = beta; sK[id] = kk;
    if constexpr (sizeof(R) == 4) {
      // offset form of the momentum flux (see face_body): p - p_ref from the
      // FP64 energy difference, stored as rho (p - p_ref) / p
      const R pm = g.f_gm1 * fma(R(-0.5) * rho, kk, to_op<R>(q[4] - g.E_ref));
      sDl[id] = rho * pm * rcp_op(p);
    }
    R gr[12];
    const R* gg = grad + (size_t)e * 12 * P + id;
#pragma unroll
    for (int r = 0; r < 12; ++r) gr[r] = gg[r * P];
    R mu = gsel<R>(g.mu, g.f_mu), lam = gsel<R>(g.mu * g.kappa, g.f_lam);
    if (g.visc_law == DG_VISC_SUTHERLAND) {
      const R sf = visc_factor<R>(g, p * ir * gsel<R>(g.inv_R, g.f_inv_R));
      mu *= sf;
      lam *= sf;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R fv[4];
      visc_flux<R>(gr, u, v, w, mu, lam, Ja[d * 3], Ja[d * 3 + 1], Ja[d * 3 + 2], fv);
#pragma unroll
      for (int c = 0; c < 4; ++c) sFv[(d * 4 + c) * P + id] = fv[c];
    }
  }
  // the xi sweep's metric terms go out with the node data (one barrier for both)
  sJd[id] = Ja[0];
  sJd[P + id] = Ja[1];
  sJd[2 * P + id] = Ja[2];
  __syncthreads();
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  const R inv_gm1 = gsel<R>(g.inv_gm1, g.f_inv_gm1);
  R acc[5] = {0, 0, 0, 0, 0};
  constexpr int FULL = (n - 1) / 2;       // shifts with a pair for every node
  constexpr bool HALF = (n % 2) == 0;     // the shift n/2, half as many pairs
  // FP32: one D entry per pair (one shared-memory load instead of three), the
  // accumulators scaled by 1/4, 1/8, 1/16 after the sweeps (exact)
  constexpr bool ONE_D = sizeof(R) == 4;
  // Exchange groups of the sweeps: a direction's pairs, partner shares and
  // metric terms stay inside its lines, so its barriers need only span the
  // threads that hold those lines.  SCOPE 2 (n = 8, one element per block):
  // the xi- and eta-lines of a k-plane are its 64 threads (two warps), so those
  // directions synchronise per k-plane (named barriers 1..8) and only the
  // zeta sweep uses the block barrier.  SCOPE 1 (elements of whole warps,
  // several per block): one named barrier per element.  Else the block.
  constexpr int SCOPE = (n == 8 && EPB == 1) ? 2 : ((P % 32 == 0 && EPB > 1 && EPB <= 15) ? 1 : 0);
  auto dsync = [&](int dd) {
    if constexpr (SCOPE == 2) {
      if (dd < 2) bar_sync_reg(1 + (threadIdx.x >> 6), 64);
      else __syncthreads();
    } else if constexpr (SCOPE == 1) {
      bar_sync<EPB>(1 + le, P);
    } else {
      __syncthreads();
    }
  };
  static_assert(FULL + (HALF ? 1 : 0) == S::ROUNDS, "pair-loop rounds");
  // FP32 with n = 2, 4 or 8: a xi-line is n consecutive lanes of one warp, so
  // the xi sweep passes the partner's share by a warp shuffle (no exchange
  // buffer, no barrier) and does its half-used shift on the lower half of each
  // line.  (FP64 keeps the packed exchange: its pipe charges masked lanes.)
  constexpr bool SHFL_XI = sizeof(R) == 4 && (n == 2 || n == 4 || n == 8);
  if constexpr (SHFL_XI) {
    const int r = i;
    const int line0 = id - r;
    const unsigned base = (threadIdx.x & 31u) & ~unsigned(n - 1);
#pragma unroll
    for (int s = 1; s <= (HALF ? n / 2 : FULL); ++s) {
      const bool half = HALF && s == n / 2;
      const int m = (r + s) & (n - 1);
      R F[5] = {0, 0, 0, 0, 0};
      if (active && (!half || r < n / 2)) {
        const int mid = line0 + m;
        R sdl = 0;
        if constexpr (sizeof(R) == 4) sdl = sDl[id] + sDl[mid];
        ec_pair<R>(rho, sR[mid], beta, sB[mid], u + sU[mid], v + sU[P + mid], w + sU[2 * P + mid], kk + sK[mid],
                   sdl, Ja[0] + sJd[mid], Ja[1] + sJd[P + mid], Ja[2] + sJd[2 * P + mid], inv_gm1, g, F);
        const R dm = sD[r * n + m];
        acc[0] = fma(dm, F[0], acc[0]);
        acc[1] = fma(dm, F[1], acc[1]);
        acc[2] = fma(dm, F[2], acc[2]);
        acc[3] = fma(dm, F[3], acc[3]);
        acc[4] = fma(dm, F[4], acc[4]);
      }
      // the share of the pair (r - s, r), computed by the lane of node r - s
      const int src = (r - s) & (n - 1);
      R Fs[5];
#pragma unroll
      for (int c = 0; c < 5; ++c) Fs[c] = __shfl_sync(0xffffffffu, F[c], (int)(base | unsigned(src)));
      if (active && (!half || r >= n / 2)) {
        const R dm = sD[r * n + src];
        acc[0] = fma(dm, Fs[0], acc[0]);
        acc[1] = fma(dm, Fs[1], acc[1]);
        acc[2] = fma(dm, Fs[2], acc[2]);
        acc[3] = fma(dm, Fs[3], acc[3]);
        acc[4] = fma(dm, Fs[4], acc[4]);
      }
    }
    // the eta sweep overwrites this node's metric entries, which the other
    // lanes of its xi-line (this warp) have read above
    __syncwarp();
  }
#pragma unroll
  for (int d = SHFL_XI ? 1 : 0; d < 3; ++d) {
    const int r = ijk[d];
    const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
    const int line0 = id - r * stride;
    // the partners' metric terms of this direction (shared memory holds one
    // direction at a time).  Overwriting this node's entries needs no barrier
    // before: every read of them in the previous sweep (its pair rounds) came
    // before that sweep's last barrier, which this thread has passed; the
    // barrier after the writes also orders the previous sweep's share reads
    // before this sweep's exchange-buffer writes.
    if (d > 0) {
      sJd[id] = Ja[d * 3];
      sJd[P + id] = Ja[d * 3 + 1];
      sJd[2 * P + id] = Ja[d * 3 + 2];
      dsync(d);
    }
    // the partner's share of a pair, written to this node's slot of xs
    auto take_share = [&](const R* xs, int src) {
      const int rm = r * n + src;
      const R d0 = ONE_D ? sD[rm] : sT0[rm], d1 = ONE_D ? d0 : sT1[rm], d2 = ONE_D ? d0 : sT2[rm];
      acc[0] = fma(d0, xs[id], acc[0]);
      acc[1] = fma(d1, xs[P + id], acc[1]);
      acc[2] = fma(d1, xs[2 * P + id], acc[2]);
      acc[3] = fma(d1, xs[3 * P + id], acc[3]);
      acc[4] = fma(d2, xs[4 * P + id], acc[4]);
    };
#pragma unroll (sizeof(R) == 4 && FULL > 0 ? FULL : 1)
    for (int s = 1; s <= FULL; ++s) {
      const int m = r + s < n ? r + s : r + s - n;
      const int mid = line0 + m * stride;
      R* sXs = sX + (XB > 1 ? (s - 1) * 5 * P : 0);
      if (active) {
        R F[5];
        R sdl = 0;
        if constexpr (sizeof(R) == 4) sdl = sDl[id] + sDl[mid];
        ec_pair<R>(rho, sR[mid], beta, sB[mid], u + sU[mid], v + sU[P + mid], w + sU[2 * P + mid], kk + sK[mid], sdl,
                   Ja[d * 3] + sJd[mid], Ja[d * 3 + 1] + sJd[P + mid], Ja[d * 3 + 2] + sJd[2 * P + mid], inv_gm1, g, F);
        const int rm = r * n + m;
        const R d0 = ONE_D ? sD[rm] : sT0[rm], d1 = ONE_D ? d0 : sT1[rm], d2 = ONE_D ? d0 : sT2[rm];
        acc[0] = fma(d0, F[0], acc[0]);
        acc[1] = fma(d1, F[1], acc[1]);
        acc[2] = fma(d1, F[2], acc[2]);
        acc[3] = fma(d1, F[3], acc[3]);
        acc[4] = fma(d2, F[4], acc[4]);
#pragma unroll
        for (int c = 0; c < 5; ++c) sXs[c * P + mid] = F[c];
      }
      if constexpr (XB == 1) {
        dsync(d);
        if (active) take_share(sX, r - s >= 0 ? r - s : r - s + n);   // written by the pair (r - s, r)
        dsync(d);
      }
    }
    if constexpr (HALF) {
      // s = n/2: the pairs (r, r + n/2), r < n/2, P/2 per element, numbered in
      // node order, taken by the first threads of the direction's exchange
      // group (block, element, or for n = 8 the k-plane of 64 threads in the
      // directions that stay inside it); both shares go to the exchange buffer
      constexpr int H = n / 2;
      const int t = threadIdx.x;
      int le2, w2;
      bool take;
      if constexpr (SCOPE == 2) {
        if (d < 2) { le2 = 0; w2 = 32 * (t >> 6) + (t & 63); take = (t & 63) < 32; }
        else { le2 = 0; w2 = t; take = t < P / 2; }
      } else if constexpr (SCOPE == 1) {
        le2 = le; w2 = id; take = id < P / 2;
      } else {
        le2 = t / (P / 2); w2 = t - le2 * (P / 2); take = t < EPB * (P / 2);
      }
      if (take && blk * EPB + le2 < nslot) {
        const int hi = w2 / stride;
        const int ia = w2 - hi * stride + stride * (hi % H + n * (hi / H));   // node with r < n/2
        const int ib = ia + H * stride;                                          // its partner
        const R* b2 = tile0 + le2 * PER_ELEM;
        const R* r2 = b2;
        const R* u2 = r2 + P;
        const R* be2 = u2 + 3 * P;
        const R* k2 = be2 + P;
        const R* j2 = k2 + P;
        R sdl = 0;
        if constexpr (sizeof(R) == 4) {
          const R* dl2 = tile0 + EPB * PER_ELEM + le2 * P;
          sdl = dl2[ia] + dl2[ib];
        }
        R F[5];
        ec_pair<R>(r2[ia], r2[ib], be2[ia], be2[ib], u2[ia] + u2[ib], u2[P + ia] + u2[P + ib],
                   u2[2 * P + ia] + u2[2 * P + ib], k2[ia] + k2[ib], sdl, j2[ia] + j2[ib], j2[P + ia] + j2[P + ib],
                   j2[2 * P + ia] + j2[2 * P + ib], inv_gm1, g, F);
        R* xh = tile0 + le2 * PER_ELEM + 21 * P + (XB > 1 ? FULL * 5 * P : 0);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          xh[c * P + ia] = F[c];
          xh[c * P + ib] = F[c];
        }
      }
    }
    if constexpr (XB == 1) {
      if constexpr (HALF) {
        dsync(d);
        if (active) take_share(sX, r >= n / 2 ? r - n / 2 : r + n / 2);
        dsync(d);
      }
    } else {
      // every round wrote its own buffer: one barrier, then the partners' shares
      dsync(d);
      if (active) {
#pragma unroll (sizeof(R) == 4 && FULL > 0 ? FULL : 1)
        for (int s = 1; s <= FULL; ++s) take_share(sX + (s - 1) * 5 * P, r - s >= 0 ? r - s : r - s + n);
        if constexpr (HALF) take_share(sX + FULL * 5 * P, r >= n / 2 ? r - n / 2 : r + n / 2);
      }
    }
  }
  if (!active) return;
  if constexpr (ONE_D) {
    acc[0] *= R(0.25);
#pragma unroll
    for (int c = 1; c < 4; ++c) acc[c] *= R(0.125);
    acc[4] *= R(0.0625);
  }
  // viscous volume term -sum_m D_rm (f_v . Ja^d)_m and, at the end nodes, the
  // viscous part (+-f_v . Ja^d)/w_0 of the surface term (in sD's diagonal)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int r = ijk[d];
    const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
    const int line0 = id - r * stride;
    R v0 = 0, v1 = 0, v2 = 0, v3 = 0;
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const R Drm = sD[r * n + m];
      const int mid = line0 + m * stride;
      v0 = fma(Drm, sFv[(d * 4 + 0) * P + mid], v0);
      v1 = fma(Drm, sFv[(d * 4 + 1) * P + mid], v1);
      v2 = fma(Drm, sFv[(d * 4 + 2) * P + mid], v2);
      v3 = fma(Drm, sFv[(d * 4 + 3) * P + mid], v3);
    }
    acc[1] -= v0; acc[2] -= v1; acc[3] -= v2; acc[4] -= v3;
  }
  // surface integral: F*_out / w_0 at each face containing the node (the
  // -f . n sJ part has cancelled against the diagonal volume term, the
  // viscous part is in the line sums above)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id_d = ijk[d];
    if (id_d != 0 && id_d != N) continue;
    const int sgn = id_d == N ? 1 : 0;
    const int code = elem_face[e * 6 + 2 * d + sgn];
    const int fid = dg_idx(code >> 4, a.nfaces > 0 ? a.nfaces : 3L * E, kSiteVolFace);   // F = 3 E if conforming
    const int pp = d == 0 ? j : i;
    const int qq = d == 2 ? j : k;
    const R* fsr;
    R fs_sign;
    if (code & 8) {
      fsr = fstar + (size_t)fid * 5 * NN + pp + n * qq;
      fs_sign = inv_w0;
    } else {
      int p2, q2;
      apply_flip<n>(code & 7, pp, qq, p2, q2);
      fsr = fstar + (size_t)fid * 5 * NN + p2 + n * q2;
      fs_sign = -inv_w0;
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) acc[c] = fma(fs_sign, fsr[c * NN], acc[c]);
  }
  R src[5] = {0, 0, 0, 0, 0};
  if (g.source == DG_SOURCE_MMS) mms_source<R>(g, mms, e, P, id, s_tc[0], s_tc[1], src);
  const size_t o0 = (size_t)e * 5 * P + id;
  if (a.mode == 0) {
    // R(U) itself, scaled by 1/J in FP64
    const double iJ = iJ64[(size_t)e * 10 * P + 9 * P + id];
#pragma unroll
    for (int c = 0; c < 5; ++c) a.Ut[o0 + (size_t)c * P] = fma(-to_f64(acc[c]), iJ, to_f64(src[c]));
  } else if constexpr (sizeof(R) == 8) {
    // Jacobian, source and the LSERK register update in FP64
    const double iJ = iJ64[(size_t)e * 10 * P + 9 * P + id];
    const double dt = a.clock[1];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const size_t o = o0 + (size_t)c * P;
      const double gk = fma(a.A, a.Gk[o], dt * fma(-acc[c], iJ, src[c]));
      a.Gk[o] = gk;
      a.Uw[o] = fma(a.B, gk, q[c]);
    }
  } else {
    // FP32 operator: R (sums, 1/J and source in FP32) is widened exactly and
    // the 2N-storage update runs in FP64.  The register holds G/dt, so that
    // both FP64 operations are fused multiply-adds:
    //   G' <- A_s G' + R,  U <- U + (B_s dt) G'   (G' = G/dt; zero at a step's start).
    const R iJ = metrics[(size_t)e * 10 * P + 9 * P + id];
    const double bdt = s_tc[2];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const size_t o = o0 + (size_t)c * P;
      const double gk = fma(a.A, a.Gk[o], to_f64(fma(-acc[c], iJ, src[c])));
      a.Gk[o] = gk;
      a.Uw[o] = fma(bdt, gk, q[c]);
    }
  }
}

}  // namespace dg
