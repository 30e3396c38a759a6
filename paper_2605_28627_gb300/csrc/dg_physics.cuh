// Device-side flux functions of the compressible Navier-Stokes-Fourier system
// (GALAEXI Sec. 3.1, Eq. 1), templated on the operator arithmetic type.
#pragma once

#include "dg_check.cuh"
#include "dg_internal.h"

namespace dg {

// Constant of the operator type: the FP64 value or its FP32 copy in Gas.
template <typename R>
__device__ __forceinline__ R gsel(double d, float f) {
  if constexpr (sizeof(R) == 4) return f;
  else return d;
}

// FP64 -> operator type.  For FP32 the conversion works on the bit pattern
// with integer instructions: rebias the exponent (1023 -> 127), keep the top
// 23 mantissa bits, round half away from zero on the dropped 29 bits (a carry
// moves into the exponent as it should) and flush values below the smallest
// normal float, zero included, to +-0.  On this GPU the FP64 -> FP32 convert
// instruction issues on the FP64 pipe, which the FP32 operator keeps for its
// FP64 state update; the integer form costs a few ALU slots instead.  It
// differs from round-to-nearest-even only on exact ties; |x| must stay below
// 2^128 (no overflow to infinity), which holds for every state of the solver.
template <typename R>
__device__ __forceinline__ R to_op(double x) {
  if constexpr (sizeof(R) == 4) {
    const unsigned lo = (unsigned)__double2loint(x), hi = (unsigned)__double2hiint(x);
    const unsigned h = hi & 0x7fffffffu;
    unsigned f = __funnelshift_l(lo, h - (896u << 20), 3) + ((lo >> 28) & 1u);
    f = h < (897u << 20) ? 0u : f;
    return __uint_as_float(f | (hi & 0x80000000u));
  } else {
    return x;
  }
}

// FP32 value -> operator type (identity for FP32; exact widening for FP64).
template <typename R>
__device__ __forceinline__ R to_op(float x) {
  return static_cast<R>(x);
}

// Operator type -> FP64, exact for normal floats (zero and subnormals give
// +-0); integer instructions only, as in to_op.
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) {
  const unsigned f = __float_as_uint(x);
  const unsigned a = f & 0x7fffffffu;
  const bool z = a < 0x00800000u;
  const unsigned hi = z ? 0u : (a >> 3) + (896u << 20);
  const unsigned lo = z ? 0u : a << 29;
  return __hiloint2double((int)(hi | (f & 0x80000000u)), (int)lo);
}

// Index of volume node (i, j, k), i fastest.
template <int n>
__device__ __forceinline__ int vidx(int i, int j, int k) { return i + n * (j + n * k); }

// Volume node of face node (p, q) on local face f = 2d + s; (p, q) run along
// the two other reference directions in increasing order.
template <int n>
__device__ __forceinline__ int face_node(int f, int p, int q) {
  const int d = f >> 1, e = (f & 1) * (n - 1);
  return d == 0 ? vidx<n>(e, p, q) : (d == 1 ? vidx<n>(p, e, q) : vidx<n>(p, q, e));
}

// Orientation code of the mesh format: face node (p, q) -> (p2, q2).
template <int n>
__device__ __forceinline__ void apply_flip(int flip, int p, int q, int& p2, int& q2) {
  const int a = (flip & 1) ? q : p;
  const int b = (flip & 1) ? p : q;
  p2 = (flip & 2) ? (n - 1 - a) : a;
  q2 = (flip & 4) ? (n - 1 - b) : b;
}

// Logarithmic mean (a - b)/(ln a - ln b) after Ismail & Roe (2009): with
// f = (a - b)/(a + b) and u = f^2 the mean is (a + b) / (2 F(u)),
// F = atanh(f)/f = 1 + u/3 + u^2/5 + u^3/7 + ... (series below u = 1e-4,
// where four terms are exact to rounding), else F = ln(a/b) / (2 f).
template <typename R>
__device__ __forceinline__ R log_mean(R a, R b) {
  const R s = a + b;
  const R f = (a - b) / s;
  const R u = f * f;
  R F;
  if (u < R(1e-4)) {
    F = R(1) + u * (R(1) / R(3) + u * (R(1) / R(5) + u * (R(1) / R(7))));
  } else {
    // ratio form: ln(zeta) and (zeta - 1)/(zeta + 1) see the same rounded zeta,
    // so its rounding error cancels in the quotient
    const R z = a / b;
    F = log(z) / (R(2) * ((z - R(1)) / (z + R(1))));
  }
  return s / (R(2) * F);
}

// Primitive quantities of a node used by the two-point flux.
template <typename R>
struct NodePrim {
  R rho, u, v, w, p, beta;   // beta = rho / (2 p)
};

template <typename R>
__device__ __forceinline__ NodePrim<R> make_prim(const double q[5], const Gas& g) {
  NodePrim<R> a;
  const R rho = R(q[0]);
  const R ir = R(1) / rho;
  a.rho = rho;
  a.u = R(q[1]) * ir;
  a.v = R(q[2]) * ir;
  a.w = R(q[3]) * ir;
  a.p = R(g.gm1) * (R(q[4]) - R(0.5) * (R(q[1]) * a.u + R(q[2]) * a.v + R(q[3]) * a.w));
  a.beta = R(0.5) * rho / a.p;
  return a;
}

// Entropy-conserving, kinetic-energy-preserving two-point flux of
// Chandrashekar (2013) in the direction of the (unnormalised) vector n:
//   f_rho = rho_ln {u}.n,  f_m = f_rho {u} + p_hat n,  p_hat = {rho}/(2{beta}),
//   f_E = f_rho (1/(2(gamma-1) beta_ln) - 1/2 {|u|^2}) + {u} . f_m.
template <typename R>
__device__ __forceinline__ void ec_flux(const NodePrim<R>& a, const NodePrim<R>& b, R nx, R ny, R nz,
                                        R inv_gm1, R f[5]) {
  const R rho_ln = log_mean(a.rho, b.rho);
  const R beta_ln = log_mean(a.beta, b.beta);
  const R ua = R(0.5) * (a.u + b.u), va = R(0.5) * (a.v + b.v), wa = R(0.5) * (a.w + b.w);
  const R p_hat = R(0.5) * (a.rho + b.rho) / (a.beta + b.beta);
  const R ke = R(0.25) * (a.u * a.u + a.v * a.v + a.w * a.w + b.u * b.u + b.v * b.v + b.w * b.w);
  const R un = ua * nx + va * ny + wa * nz;
  const R fr = rho_ln * un;
  f[0] = fr;
  f[1] = fr * ua + p_hat * nx;
  f[2] = fr * va + p_hat * ny;
  f[3] = fr * wa + p_hat * nz;
  f[4] = fr * (R(0.5) * inv_gm1 / beta_ln - ke) + ua * f[1] + va * f[2] + wa * f[3];
}

// Euler flux f(q) . n with separate pressures in the momentum (pm) and energy
// (p) components: pm = p - p_ref for the FP32 operator's offset form (see
// face_body), pm = p otherwise.
template <typename R>
__device__ __forceinline__ void euler_flux_pm(const R q[5], R u, R v, R w, R p, R pm, R nx, R ny, R nz, R f[5]) {
  const R un = u * nx + v * ny + w * nz;
  f[0] = q[0] * un;
  f[1] = q[1] * un + pm * nx;
  f[2] = q[2] * un + pm * ny;
  f[3] = q[3] * un + pm * nz;
  f[4] = (q[4] + p) * un;
}

// Two-point flux of ec_flux in the offset form: the momentum flux carries
// p_hat - p_ref, computed as (dl_a + dl_b) / (2 (beta_a + beta_b)) from the
// per-node dl = rho (p - p_ref) / p (= rho - 2 p_ref beta), and the energy flux
// adds p_ref {u}.n back, so the result equals ec_flux minus p_ref n in the
// momentum components.
template <typename R>
__device__ __forceinline__ void ec_flux_off(const NodePrim<R>& a, const NodePrim<R>& b, R dla, R dlb, R p_ref, R nx,
                                            R ny, R nz, R inv_gm1, R f[5]) {
  const R rho_ln = log_mean(a.rho, b.rho);
  const R beta_ln = log_mean(a.beta, b.beta);
  const R ua = R(0.5) * (a.u + b.u), va = R(0.5) * (a.v + b.v), wa = R(0.5) * (a.w + b.w);
  const R p_off = R(0.5) * (dla + dlb) / (a.beta + b.beta);
  const R ke = R(0.25) * (a.u * a.u + a.v * a.v + a.w * a.w + b.u * b.u + b.v * b.v + b.w * b.w);
  const R un = ua * nx + va * ny + wa * nz;
  const R fr = rho_ln * un;
  f[0] = fr;
  f[1] = fr * ua + p_off * nx;
  f[2] = fr * va + p_off * ny;
  f[3] = fr * wa + p_off * nz;
  f[4] = fr * (R(0.5) * inv_gm1 / beta_ln - ke) + ua * f[1] + va * f[2] + wa * f[3] + p_ref * un;
}

// Euler flux f(q) . n for an arbitrary vector n.
template <typename R>
__device__ __forceinline__ void euler_flux(const R q[5], R u, R v, R w, R p, R nx, R ny, R nz, R f[5]) {
  const R un = u * nx + v * ny + w * nz;
  f[0] = q[0] * un;
  f[1] = q[1] * un + p * nx;
  f[2] = q[2] * un + p * ny;
  f[3] = q[3] * un + p * nz;
  f[4] = (q[4] + p) * un;
}

// Roe's approximate Riemann solver with the Harten-Hyman (1983) entropy fix
// on the acoustic waves, unit direction n (the surface flux of Sec. 3.1):
// F = (f(qL) + f(qR)).n/2 - sum_k |lambda_k| alpha_k r_k / 2, Roe averages with
// sqrt(rho) weights; |lambda| -> delta = max(0, lambda - lambda(qL),
// lambda(qR) - lambda) where |lambda| < delta.
template <typename R>
__device__ __forceinline__ void roe_flux(const R qL[5], R uL, R vL, R wL, R pL, const R qR[5], R uR, R vR, R wR,
                                         R pR, R nx, R ny, R nz, R gamma, R gm1, R F[5], R pmL, R pmR, R dr) {
  R fL[5], fR[5];
  euler_flux_pm<R>(qL, uL, vL, wL, pL, pmL, nx, ny, nz, fL);
  euler_flux_pm<R>(qR, uR, vR, wR, pR, pmR, nx, ny, nz, fR);
  const R sL = sqrt(qL[0]), sR = sqrt(qR[0]);
  const R is = R(1) / (sL + sR);
  const R wl = sL * is, wr = sR * is;
  const R HL = (qL[4] + pL) / qL[0], HR = (qR[4] + pR) / qR[0];
  const R u = wl * uL + wr * uR, v = wl * vL + wr * vR, w = wl * wL + wr * wR;
  const R H = wl * HL + wr * HR;
  const R q2 = u * u + v * v + w * w;
  const R c = sqrt(gm1 * (H - R(0.5) * q2));
  const R rho = sL * sR;
  const R un = u * nx + v * ny + w * nz;
  const R dp = pmR - pmL;   // = pR - pL; the jumps dr, dp come from the caller (FP64 differences in FP32 mode)
  const R du = uR - uL, dv = vR - vL, dw = wR - wL;
  const R dun = du * nx + dv * ny + dw * nz;
  const R ic2 = R(1) / (c * c);
  const R a1 = (dp - rho * c * dun) * R(0.5) * ic2;
  const R a2 = dr - dp * ic2;
  const R a5 = (dp + rho * c * dun) * R(0.5) * ic2;
  R l1 = fabs(un - c);
  const R l2 = fabs(un);
  R l5 = fabs(un + c);
  const R unL = uL * nx + vL * ny + wL * nz, unR = uR * nx + vR * ny + wR * nz;
  const R cL = sqrt(gamma * pL / qL[0]), cR = sqrt(gamma * pR / qR[0]);
  const R d1 = fmax(fmax(R(0), (un - c) - (unL - cL)), (unR - cR) - (un - c));
  const R d5 = fmax(fmax(R(0), (un + c) - (unL + cL)), (unR + cR) - (un + c));
  if (l1 < d1) l1 = d1;
  if (l5 < d5) l5 = d5;
  const R A1 = l1 * a1, A5 = l5 * a5;
  const R udu = u * du + v * dv + w * dw;
  const R D0 = A1 + l2 * a2 + A5;
  const R D1 = A1 * (u - c * nx) + l2 * (a2 * u + rho * (du - dun * nx)) + A5 * (u + c * nx);
  const R D2 = A1 * (v - c * ny) + l2 * (a2 * v + rho * (dv - dun * ny)) + A5 * (v + c * ny);
  const R D3 = A1 * (w - c * nz) + l2 * (a2 * w + rho * (dw - dun * nz)) + A5 * (w + c * nz);
  const R D4 = A1 * (H - un * c) + l2 * (a2 * R(0.5) * q2 + rho * (udu - un * dun)) + A5 * (H + un * c);
  F[0] = R(0.5) * (fL[0] + fR[0] - D0);
  F[1] = R(0.5) * (fL[1] + fR[1] - D1);
  F[2] = R(0.5) * (fL[2] + fR[2] - D2);
  F[3] = R(0.5) * (fL[3] + fR[3] - D3);
  F[4] = R(0.5) * (fL[4] + fR[4] - D4);
}

// Factor mu(T)/mu_ref of the viscosity law: 1, or Sutherland's (1893)
// (T/T_ref)^(3/2) (T_ref + S)/(T + S); the heat conductivity scales with it.
template <typename R>
__device__ __forceinline__ R visc_factor(const Gas& g, R T) {
  if (g.visc_law != DG_VISC_SUTHERLAND) return R(1);
  const R x = T * gsel<R>(g.inv_T_ref, g.f_inv_T_ref);
  return x * sqrt(x) * (gsel<R>(g.suth_c, g.f_suth_c) / (T + gsel<R>(g.S_suth, g.f_S_suth)));
}

// Viscous flux (Newtonian stress with Stokes' hypothesis, Fourier heat flux)
// dotted with n: returns the momentum and energy components fv[0..3].
// g[phi*3 + l] = d phi / d x_l, phi = (u, v, w, T).
template <typename R>
__device__ __forceinline__ void visc_flux(const R g[12], R u, R v, R w, R mu, R kappa_mu, R nx, R ny,
                                          R nz, R fv[4]) {
  const R div = g[0] + g[4] + g[8];
  const R t00 = mu * (R(2) * g[0] - R(2.0 / 3.0) * div);
  const R t11 = mu * (R(2) * g[4] - R(2.0 / 3.0) * div);
  const R t22 = mu * (R(2) * g[8] - R(2.0 / 3.0) * div);
  const R t01 = mu * (g[1] + g[3]);
  const R t02 = mu * (g[2] + g[6]);
  const R t12 = mu * (g[5] + g[7]);
  // tau . n
  fv[0] = t00 * nx + t01 * ny + t02 * nz;
  fv[1] = t01 * nx + t11 * ny + t12 * nz;
  fv[2] = t02 * nx + t12 * ny + t22 * nz;
  // (tau . u + lambda grad T) . n
  fv[3] = fv[0] * u + fv[1] * v + fv[2] * w + kappa_mu * (g[9] * nx + g[10] * ny + g[11] * nz);
}

}  // namespace dg
