// Reverse-mode (vector-Jacobian) derivatives of the pointwise pieces of the
// DGSEM operator (GALAEXI Sec. 3.1, Eqs. 1-3), written by hand from the
// forward formulas in dg_physics.cuh / dg_stage.cuh.  FP64.  Branches follow
// the primal values (the log-mean series/log switch as in the forward); at the
// kinks of the LLF speed max(|u.n| + c) -- a tie, or u.n = 0, to within 1e-12
// of the local scale -- the derivative is the mean of the one-sided ones.
#pragma once

#include "dg_physics.cuh"

namespace dg {

// Primitive adjoints (rho, u, v, w, p) -> conserved adjoints.
// rho = q0, u_a = q_{1+a}/rho, p = (gamma-1)(q4 - |q_{1:3}|^2 / (2 rho)).
__device__ __forceinline__ void prim_vjp(const double q[5], double rb, const double ub[3], double pb, double gm1,
                                         double qb[5]) {
  const double ir = 1.0 / q[0];
  const double u0 = q[1] * ir, u1 = q[2] * ir, u2 = q[3] * ir;
  const double k = 0.5 * (u0 * u0 + u1 * u1 + u2 * u2);
  const double gp = gm1 * pb;
  qb[0] += rb - (ub[0] * u0 + ub[1] * u1 + ub[2] * u2) * ir + gp * k;
  qb[1] += ub[0] * ir - gp * u0;
  qb[2] += ub[1] * ir - gp * u1;
  qb[3] += ub[2] * ir - gp * u2;
  qb[4] += gp;
}

// 1/x for the adjoint's positive operands (densities, pressures, beta sums,
// log means): hardware approximation and one cubic Newton-Raphson step
// (below 1 ulp), a fraction of an IEEE division on GB300's narrow FP64 pipe.
__device__ __forceinline__ double adj_rcp(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// Logarithmic mean and its partial derivatives, consistent with log_mean():
// series branch L = s G(u), G = 1/F2, F2 = 2 (1 + u/3 + u^2/5 + u^3/7),
// u = f^2, f = (a-b)/s; with du/da = 4 f b / s^2 and du/db = -4 f a / s^2,
// dL/da = G + c b and dL/db = G - c a, c = 4 G'(u) f / s = -4 F2'(u) G^2 f / s;
// logarithmic branch L = (a - b) / ln(a/b) with dL/da = (1 - L/a)/ln(a/b),
// dL/db = (L/b - 1)/ln(a/b).
__device__ __forceinline__ double log_mean_d(double a, double b, double& La, double& Lb) {
  const double s = a + b;
  const double is = adj_rcp(s);
  const double f = (a - b) * is;
  const double u = f * f;
  if (u < 1e-4) {
    const double F2 = fma(u, fma(u, fma(u, 2.0 / 7.0, 2.0 / 5.0), 2.0 / 3.0), 2.0);
    const double F2p_m4 = fma(u, fma(u, -24.0 / 7.0, -16.0 / 5.0), -8.0 / 3.0);   // -4 F2'(u)
    const double G = adj_rcp(F2);
    const double c = F2p_m4 * (G * G) * (f * is);
    La = fma(c, b, G);
    Lb = fma(-c, a, G);
    return s * G;
  }
  const double z = a / b;
  const double F = log(z) / (2.0 * ((z - 1.0) / (z + 1.0)));
  const double L = s / (2.0 * F);
  const double ell = log(z);
  La = (1.0 - L / a) / ell;
  Lb = (L / b - 1.0) / ell;
  return L;
}

// Adjoint of the Chandrashekar two-point flux f(a, b; n) (ec_flux): given
// fb = df-bar (5), adds to the primitive adjoints (rho, u, v, w, p) of a and b.
// hipA, hipB are 1/(2p), bipA, bipB are beta/p and kA, kB are |u|^2 of the two
// states (per node, so the volume kernel computes them once per node, not once
// per pair; the p members of A and B are not read).
__device__ __forceinline__ void ec_flux_vjp(const NodePrim<double>& A, const NodePrim<double>& B, double nx,
                                            double ny, double nz, double inv_gm1, const double fb[5], double pa[5],
                                            double pbv[5], double hipA, double hipB, double bipA, double bipB,
                                            double kA, double kB) {
  double Lra, Lrb, Lba, Lbb;
  const double rho_ln = log_mean_d(A.rho, B.rho, Lra, Lrb);
  const double beta_ln = log_mean_d(A.beta, B.beta, Lba, Lbb);
  const double ua = 0.5 * (A.u + B.u), va = 0.5 * (A.v + B.v), wa = 0.5 * (A.w + B.w);
  const double sr = A.rho + B.rho, sb = A.beta + B.beta;
  const double isb = adj_rcp(sb), ibl = adj_rcp(beta_ln);
  const double p_hat = 0.5 * sr * isb;
  const double K = 0.25 * (kA + kB);
  const double un = ua * nx + va * ny + wa * nz;
  const double f0 = rho_ln * un;
  const double fm0 = f0 * ua + p_hat * nx, fm1 = f0 * va + p_hat * ny, fm2 = f0 * wa + p_hat * nz;
  const double H = 0.5 * inv_gm1 * ibl - K;
  // f4 = f0 H + ubar . fm
  const double fmb0 = fb[1] + fb[4] * ua, fmb1 = fb[2] + fb[4] * va, fmb2 = fb[3] + fb[4] * wa;
  double ubb0 = fb[4] * fm0 + f0 * fmb0;
  double ubb1 = fb[4] * fm1 + f0 * fmb1;
  double ubb2 = fb[4] * fm2 + f0 * fmb2;
  const double f0b = fb[0] + fb[4] * H + fmb0 * ua + fmb1 * va + fmb2 * wa;
  const double Hb = fb[4] * f0;
  const double phb = fmb0 * nx + fmb1 * ny + fmb2 * nz;
  const double rlb = f0b * un;
  const double unb = f0b * rho_ln;
  ubb0 += unb * nx; ubb1 += unb * ny; ubb2 += unb * nz;
  const double blb = -Hb * 0.5 * inv_gm1 * (ibl * ibl);
  const double Kb = -Hb;
  // ubar = (u_a + u_b)/2, K = (|u_a|^2 + |u_b|^2)/4
  pa[1] += 0.5 * ubb0 + 0.5 * Kb * A.u;  pbv[1] += 0.5 * ubb0 + 0.5 * Kb * B.u;
  pa[2] += 0.5 * ubb1 + 0.5 * Kb * A.v;  pbv[2] += 0.5 * ubb1 + 0.5 * Kb * B.v;
  pa[3] += 0.5 * ubb2 + 0.5 * Kb * A.w;  pbv[3] += 0.5 * ubb2 + 0.5 * Kb * B.w;
  // p_hat = sr / (2 sb)
  const double srb = phb * 0.5 * isb;
  const double sbb = -phb * p_hat * isb;
  double rab = srb + rlb * Lra, rbb = srb + rlb * Lrb;
  const double bab = sbb + blb * Lba, bbb = sbb + blb * Lbb;
  // beta = rho / (2 p): d beta / d rho = 1/(2p), d beta / d p = -beta/p
  rab = fma(bab, hipA, rab);  pa[4] = fma(-bab, bipA, pa[4]);
  rbb = fma(bbb, hipB, rbb);  pbv[4] = fma(-bbb, bipB, pbv[4]);
  pa[0] += rab;
  pbv[0] += rbb;
}

__device__ __forceinline__ void ec_flux_vjp(const NodePrim<double>& A, const NodePrim<double>& B, double nx,
                                            double ny, double nz, double inv_gm1, const double fb[5], double pa[5],
                                            double pbv[5]) {
  const double ipA = adj_rcp(A.p), ipB = adj_rcp(B.p);
  ec_flux_vjp(A, B, nx, ny, nz, inv_gm1, fb, pa, pbv, 0.5 * ipA, 0.5 * ipB, A.beta * ipA, B.beta * ipB,
              A.u * A.u + A.v * A.v + A.w * A.w, B.u * B.u + B.v * B.v + B.w * B.w);
}

// Adjoint of the Euler flux f(q) . n (q conserved, n any vector): adds to qb.
__device__ __forceinline__ void euler_flux_vjp(const double q[5], double u, double v, double w, double p, double nx,
                                               double ny, double nz, const double fb[5], double gm1, double qb[5]) {
  const double un = u * nx + v * ny + w * nz;
  double mb0 = fb[0] * nx + fb[1] * un, mb1 = fb[0] * ny + fb[2] * un, mb2 = fb[0] * nz + fb[3] * un;
  const double unb = fb[1] * q[1] + fb[2] * q[2] + fb[3] * q[3] + fb[4] * (q[4] + p);
  const double pbar = fb[1] * nx + fb[2] * ny + fb[3] * nz + fb[4] * un;
  const double Eb = fb[4] * un;
  // direct dependence on m (f0 = m . n, f_m = m un) is in mb; un and p via primitives
  qb[1] += mb0; qb[2] += mb1; qb[3] += mb2;
  qb[4] += Eb;
  const double ub[3] = {unb * nx, unb * ny, unb * nz};
  prim_vjp(q, 0.0, ub, pbar, gm1, qb);
}

// Adjoint of the local Lax-Friedrichs flux (llf in k_face): adds to qbL, qbR.
__device__ __forceinline__ void llf_vjp(const double qL[5], const double qR[5], double nx, double ny, double nz,
                                        double gamma, double gm1, const double fb[5], double qbL[5], double qbR[5]) {
  const double irL = 1.0 / qL[0], irR = 1.0 / qR[0];
  const double uL = qL[1] * irL, vL = qL[2] * irL, wL = qL[3] * irL;
  const double uR = qR[1] * irR, vR = qR[2] * irR, wR = qR[3] * irR;
  const double pL = gm1 * (qL[4] - 0.5 * (qL[1] * uL + qL[2] * vL + qL[3] * wL));
  const double pR = gm1 * (qR[4] - 0.5 * (qR[1] * uR + qR[2] * vR + qR[3] * wR));
  const double cL = sqrt(gamma * pL * irL), cR = sqrt(gamma * pR * irR);
  const double unL = uL * nx + vL * ny + wL * nz, unR = uR * nx + vR * ny + wR * nz;
  const double lL = fabs(unL) + cL, lR = fabs(unR) + cR;
  const bool right = lR > lL;
  const double lmax = right ? lR : lL;
  double half[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) half[c] = 0.5 * fb[c];
  euler_flux_vjp(qL, uL, vL, wL, pL, nx, ny, nz, half, gm1, qbL);
  euler_flux_vjp(qR, uR, vR, wR, pR, nx, ny, nz, half, gm1, qbR);
  double lb = 0.0;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    qbR[c] -= 0.5 * lmax * fb[c];
    qbL[c] += 0.5 * lmax * fb[c];
    lb -= 0.5 * fb[c] * (qR[c] - qL[c]);
  }
  // lambda = |u . n| + c of the chosen side; c = sqrt(gamma p / rho):
  // dc = c/2 (dp/p - drho/rho).  At the kinks (a tie of the two speeds, or
  // u . n = 0, to within 1e-12 of the local scale, as on symmetry planes) the
  // derivative is the mean of the one-sided derivatives.
  const bool tie = fabs(lR - lL) <= 1e-12 * fmax(lL, lR);
  const double sideL = tie ? 0.5 : (right ? 0.0 : 1.0), sideR = tie ? 0.5 : (right ? 1.0 : 0.0);
  {
    const double lbw = lb * sideL;
    const double sg = fabs(unL) <= 1e-12 * cL ? 0.0 : (unL < 0.0 ? -1.0 : 1.0);
    const double ub[3] = {lbw * sg * nx, lbw * sg * ny, lbw * sg * nz};
    prim_vjp(qL, -lbw * 0.5 * cL / qL[0], ub, lbw * 0.5 * cL / pL, gm1, qbL);
  }
  {
    const double lbw = lb * sideR;
    const double sg = fabs(unR) <= 1e-12 * cR ? 0.0 : (unR < 0.0 ? -1.0 : 1.0);
    const double ub[3] = {lbw * sg * nx, lbw * sg * ny, lbw * sg * nz};
    prim_vjp(qR, -lbw * 0.5 * cR / qR[0], ub, lbw * 0.5 * cR / pR, gm1, qbR);
  }
}

// Forward-mode dual number (value, one directional derivative) to
// differentiate the Roe flux mechanically: the templated forward flux runs on
// it.  Kinks follow the value as in the oracle's dual numbers: |x| by the sign
// of the value (derivative +1 at 0), max ties to its first argument.  In a
// namespace of its own, found by argument-dependent lookup, so that sqrt,
// fabs and fmax of doubles keep their meaning everywhere else.
namespace ad {
struct Dual {
  double v, d;
  __device__ Dual() : v(0.0), d(0.0) {}
  __device__ Dual(double x) : v(x), d(0.0) {}
  __device__ Dual(double x, double dx) : v(x), d(dx) {}
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, fma(a.d, b.v, a.v * b.d)); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ bool operator<(Dual a, Dual b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(Dual a, Dual b) { return a.v > b.v; }
__device__ __forceinline__ Dual sqrt(Dual a) {
  const double s = ::sqrt(a.v);
  return Dual(s, a.d / (2.0 * s));
}
__device__ __forceinline__ Dual fabs(Dual a) { return a.v < 0.0 ? -a : a; }
__device__ __forceinline__ Dual fmax(Dual a, Dual b) { return b.v > a.v ? b : a; }
}  // namespace ad

// Adjoint of the Roe flux with the Harten-Hyman entropy fix (roe_flux, FP64,
// no pressure offset) w.r.t. both conserved states: ten forward passes on
// dual numbers, one per input component, each contracted with fb.
static __device__ __noinline__ void roe_vjp(const double qL[5], const double qR[5], double nx, double ny, double nz,
                                     double gamma, double gm1, const double fb[5], double qbL[5], double qbR[5]) {
  using ad::Dual;
#pragma unroll 1
  for (int k = 0; k < 10; ++k) {
    Dual a[5], b[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      a[v] = Dual(qL[v], k == v ? 1.0 : 0.0);
      b[v] = Dual(qR[v], k == 5 + v ? 1.0 : 0.0);
    }
    const Dual irL = Dual(1.0) / a[0], irR = Dual(1.0) / b[0];
    const Dual uL = a[1] * irL, vL = a[2] * irL, wL = a[3] * irL;
    const Dual uR = b[1] * irR, vR = b[2] * irR, wR = b[3] * irR;
    const Dual pL = Dual(gm1) * (a[4] - Dual(0.5) * (a[1] * uL + a[2] * vL + a[3] * wL));
    const Dual pR = Dual(gm1) * (b[4] - Dual(0.5) * (b[1] * uR + b[2] * vR + b[3] * wR));
    Dual F[5];
    roe_flux<Dual>(a, uL, vL, wL, pL, b, uR, vR, wR, pR, Dual(nx), Dual(ny), Dual(nz), Dual(gamma), Dual(gm1), F, pL,
                   pR, b[0] - a[0]);
    double s = 0.0;
#pragma unroll
    for (int v = 0; v < 5; ++v) s = fma(fb[v], F[v].d, s);
    if (k < 5) qbL[k] += s;
    else qbR[k - 5] += s;
  }
}

// Viscosity factor s(T) = mu(T)/mu_ref and ds/dT: Sutherland's law
// s = x^(3/2) (T_ref + S)/(T + S), x = T/T_ref, so ds/dT = s (3/(2T) - 1/(T + S));
// s = 1, ds = 0 for constant viscosity.
__device__ __forceinline__ void visc_factor_d(const Gas& g, double T, double& s, double& ds) {
  if (g.visc_law != DG_VISC_SUTHERLAND) {
    s = 1.0;
    ds = 0.0;
    return;
  }
  const double x = T * g.inv_T_ref, den = 1.0 / (T + g.S_suth);
  s = x * sqrt(x) * g.suth_c * den;
  ds = s * (1.5 / T - den);
}

// Adjoint of visc_flux (f_v . n, 4 components) w.r.t. the gradients g (12)
// and the velocity (3); returns fb . f_v1, f_v1 the flux with unit viscosity
// (f_v = mu f_v1 is linear in mu: the return value is d(fb . f_v)/d mu, and
// with Sutherland's law the caller scales it by s(T) and, for the T-derivative,
// by mu_ref ds/dT).
__device__ __forceinline__ double visc_flux_vjp(const double g[12], double u, double v, double w, double mu,
                                                double kappa, double nx, double ny, double nz, const double fb[4],
                                                double gb[12], double ub[3]) {
  // forward with mu = 1 for the mu-derivative
  double fv1[4];
  visc_flux<double>(g, u, v, w, 1.0, kappa, nx, ny, nz, fv1);
  const double mub = fb[0] * fv1[0] + fb[1] * fv1[1] + fb[2] * fv1[2] + fb[3] * fv1[3];
  // fv_a = mu * fv1_a (a < 3), fv3 = sum_a fv_a u_a + kappa mu grad T . n
  ub[0] += fb[3] * mu * fv1[0];
  ub[1] += fb[3] * mu * fv1[1];
  ub[2] += fb[3] * mu * fv1[2];
  const double a0 = fb[0] + fb[3] * u, a1 = fb[1] + fb[3] * v, a2 = fb[2] + fb[3] * w;
  const double km = kappa * mu * fb[3];
  gb[9] += km * nx; gb[10] += km * ny; gb[11] += km * nz;
  // fv_a = sum_l n_l tau_la, tau symmetric: tau-bar of the symmetric components
  const double t00 = nx * a0, t11 = ny * a1, t22 = nz * a2;
  const double t01 = nx * a1 + ny * a0, t02 = nx * a2 + nz * a0, t12 = ny * a2 + nz * a1;
  // tau_aa = mu (2 g_aa - 2/3 div), tau_ab = mu (g_ab + g_ba)
  const double divb = -(2.0 / 3.0) * mu * (t00 + t11 + t22);
  gb[0] += 2.0 * mu * t00 + divb;
  gb[4] += 2.0 * mu * t11 + divb;
  gb[8] += 2.0 * mu * t22 + divb;
  gb[1] += mu * t01; gb[3] += mu * t01;
  gb[2] += mu * t02; gb[6] += mu * t02;
  gb[5] += mu * t12; gb[7] += mu * t12;
  return mub;
}

}  // namespace dg
