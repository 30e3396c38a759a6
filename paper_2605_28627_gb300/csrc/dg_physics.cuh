// Device-side flux functions of the compressible Navier-Stokes-Fourier system
// (GALAEXI Sec. 3.1, Eq. 1), templated on the operator arithmetic type.
#pragma once

#include "dg_internal.h"

namespace dg {

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
