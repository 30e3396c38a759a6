// Volume kernel of R(U) (GALAEXI Sec. 3.1): split-form flux differencing with
// the entropy-conserving, kinetic-energy-preserving two-point flux of
// Chandrashekar (2013), the viscous volume term, the surface integral, the
// Jacobian, the source and the LSERK4-5 stage update, one element per block
// (several for small N), one thread per node.
//
// The kernel is bound by the FP64 pipe, so the design minimises FP64
// instructions:
//  * Symmetric pair reuse: F#(q_i, q_m) = F#(q_m, q_i), so each unordered
//    pair on a line is evaluated once, in rounds of a fixed cyclic shift s;
//    the partner's share goes through shared memory.
//  * The diagonal terms 2 D_ii f(q_i) . Ja_i vanish for interior LGL nodes
//    and cancel exactly against the -f . n sJ / w_0 part of the surface term
//    at the two end nodes (2 D_00 = -1/w_0, 2 D_NN = 1/w_0), so neither is
//    evaluated.
//  * Reciprocals instead of divides (hardware approximation + one cubic
//    Newton-Raphson step), logarithmic means by the Ismail-Roe series with
//    the reciprocal series for 1/F, constant factors folded into scaled copies
//    of D, the series/log switch decided on the exponent word in integer ALU.
#include "dg_physics.cuh"

namespace dg {

template <int N>
struct VShape {
  static constexpr int n = N + 1;
  static constexpr int P = n * n * n;
  static constexpr int NN = n * n;
  static constexpr int EPB = P >= 128 ? 1 : (128 + P - 1) / P;
  static constexpr int THREADS = EPB * P;
  static constexpr int ROUNDS = n / 2;          // shifts s = 1..n/2 (s = n/2 half-used for even n)
  static constexpr int PER_ELEM = 32 * P;       // doubles of shared memory per element
};

// 1/x: hardware reciprocal approximation refined by one cubic Newton-Raphson
// step y <- y (1 + e + e^2), e = 1 - x y, which cubes the relative error
// (2^-20 -> below 1 ulp).  In FP32 the approximation alone is within 1 ulp.
__device__ __forceinline__ double rcp_op(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  const double t = fma(e, e, e);
  return fma(y, t, y);
}
__device__ __forceinline__ float rcp_op(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
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

// R is the operator arithmetic: double (FP64 path) or float (FP32-operator
// path, state and RK update stay FP64).  metrics, grad and fstar are stored in R.
template <int N, typename R>
__global__ void __launch_bounds__(VShape<N>::THREADS)
k_volume2(StageArgs a, const R* __restrict__ metrics, const double* __restrict__ iJ64,
          const R* __restrict__ grad, const R* __restrict__ fstar, const int* __restrict__ elem_face,
          const double* __restrict__ X, const double* __restrict__ Dg, int E, Gas g, double inv_w0d) {
  using S = VShape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN, EPB = S::EPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* smem = reinterpret_cast<R*>(smem_raw);
  R* sD = smem;                       // D
  R* sT0 = sD + n * n;                // D/4   (mass: X = 8 f_rho)
  R* sT1 = sT0 + n * n;               // D/8   (momentum: M = 16 f_m)
  R* sT2 = sT1 + n * n;               // D/16  (energy: 32 f_E)
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  R* base = sT2 + ((n * n + 3) & ~3) + le * S::PER_ELEM;
  R* sR = base;                       // rho
  R* sU = sR + P;                     // u, v, w
  R* sB = sU + 3 * P;                 // beta = rho / (2 p)
  R* sK = sB + P;                     // |u|^2
  R* sJa = sK + P;                    // [9][P]  Ja^d_l at row d*3+l
  R* sFv = sJa + 9 * P;               // [3][4][P] (f_v . Ja^d), momentum + energy
  R* sX = sFv + 12 * P;               // [5][P] exchange of partner shares
  const int e = blockIdx.x * EPB + le;
  const bool active = e < E;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const double d = Dg[t];
    sD[t] = R(d);
    sT0[t] = R(0.25 * d);
    sT1[t] = R(0.125 * d);
    sT2[t] = R(0.0625 * d);
  }
  const R inv_w0 = R(inv_w0d);
  double q[5] = {0, 0, 0, 0, 0};
  R Ja[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  R rho = R(1), u = 0, v = 0, w = 0, beta = 0, kk = 0;
  if (active) {
#pragma unroll
    for (int r = 0; r < 5; ++r) q[r] = a.U[((size_t)e * 5 + r) * P + id];
    const R* mt = metrics + (size_t)e * 10 * P + id;
#pragma unroll
    for (int r = 0; r < 9; ++r) { Ja[r] = mt[r * P]; sJa[r * P + id] = Ja[r]; }
    rho = R(q[0]);
    const R ir = rcp_op(rho);
    u = R(q[1]) * ir; v = R(q[2]) * ir; w = R(q[3]) * ir;
    kk = u * u + v * v + w * w;
    const R p = R(g.gm1) * fma(R(-0.5) * rho, kk, R(q[4]));
    beta = R(0.5) * rho * rcp_op(p);
    sR[id] = rho; sU[id] = u; sU[P + id] = v; sU[2 * P + id] = w; sB[id] = beta; sK[id] = kk;
    R gr[12];
    const R* gg = grad + (size_t)e * 12 * P + id;
#pragma unroll
    for (int r = 0; r < 12; ++r) gr[r] = gg[r * P];
    const R mu = R(g.mu), lam = R(g.mu * g.kappa);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      R fv[4];
      visc_flux<R>(gr, u, v, w, mu, lam, Ja[d * 3], Ja[d * 3 + 1], Ja[d * 3 + 2], fv);
#pragma unroll
      for (int c = 0; c < 4; ++c) sFv[(d * 4 + c) * P + id] = fv[c];
    }
  }
  __syncthreads();
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  const R inv4 = R(4.0 * g.inv_gm1);
  R acc[5] = {0, 0, 0, 0, 0};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int r = ijk[d];
    const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
    const int line0 = id - r * stride;
#pragma unroll 1
    for (int s = 1; s <= S::ROUNDS; ++s) {
      const bool half = (2 * s == n);
      const int m = r + s < n ? r + s : r + s - n;
      const int mid = line0 + m * stride;
      if (active && !(half && r >= s)) {
        const R rb = sR[mid], bb = sB[mid];
        const R sr = rho + rb, sb = beta + bb;
        const R rr = rcp_op(sr), rbt = rcp_op(sb);
        const R fr = (rho - rb) * rr, fb = (beta - bb) * rbt;
        const R ur = fr * fr, ub = fb * fb;
        R rln2, hib;                    // 2 rho_ln and 1/(2 beta_ln)
        if (small_u(ur)) rln2 = sr * inv_atanh_ratio(ur);
        else rln2 = sr / atanh_ratio_log(rho, rb);
        if (small_u(ub)) hib = atanh_ratio(ub) * rbt;
        else hib = atanh_ratio_log(beta, bb) * rbt;
        const R su0 = u + sU[mid], su1 = v + sU[P + mid], su2 = w + sU[2 * P + mid];
        const R sn0 = Ja[d * 3] + sJa[(d * 3) * P + mid];
        const R sn1 = Ja[d * 3 + 1] + sJa[(d * 3 + 1) * P + mid];
        const R sn2 = Ja[d * 3 + 2] + sJa[(d * 3 + 2) * P + mid];
        const R un4 = fma(su0, sn0, fma(su1, sn1, su2 * sn2));
        const R Xf = rln2 * un4;                      // 8 f_rho
        const R Y4 = R(4) * sr * rbt;                  // 16 p_hat / |n_avg| scale
        const R M0 = fma(Xf, su0, Y4 * sn0);          // 16 f_m
        const R M1 = fma(Xf, su1, Y4 * sn1);
        const R M2 = fma(Xf, su2, Y4 * sn2);
        const R Z = fma(hib, inv4, -(kk + sK[mid]));
        const R E32 = fma(Xf, Z, fma(su0, M0, fma(su1, M1, su2 * M2)));   // 32 f_E
        const int rm = r * n + m;
        acc[0] = fma(sT0[rm], Xf, acc[0]);
        acc[1] = fma(sT1[rm], M0, acc[1]);
        acc[2] = fma(sT1[rm], M1, acc[2]);
        acc[3] = fma(sT1[rm], M2, acc[3]);
        acc[4] = fma(sT2[rm], E32, acc[4]);
        sX[mid] = Xf; sX[P + mid] = M0; sX[2 * P + mid] = M1; sX[3 * P + mid] = M2; sX[4 * P + mid] = E32;
      }
      __syncthreads();
      const int src = r - s >= 0 ? r - s : r - s + n;   // the node whose pair (src, r) wrote here
      if (active && !(half && src >= s)) {
        const int rm = r * n + src;
        acc[0] = fma(sT0[rm], sX[id], acc[0]);
        acc[1] = fma(sT1[rm], sX[P + id], acc[1]);
        acc[2] = fma(sT1[rm], sX[2 * P + id], acc[2]);
        acc[3] = fma(sT1[rm], sX[3 * P + id], acc[3]);
        acc[4] = fma(sT2[rm], sX[4 * P + id], acc[4]);
      }
      __syncthreads();
    }
  }
  if (!active) return;
  // viscous volume term: -sum_m D_rm (f_v . Ja^d)_m
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
  // surface integral: (F*_out + f_v . n sJ) / w_0 at each face containing the
  // node (the -f . n sJ part has cancelled against the diagonal volume term)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id_d = ijk[d];
    if (id_d != 0 && id_d != N) continue;
    const int sgn = id_d == N ? 1 : 0;
    const int code = elem_face[e * 6 + 2 * d + sgn];
    const int fid = code >> 4;
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
    const R vs = sgn ? inv_w0 : -inv_w0;
    acc[0] = fma(fs_sign, fsr[0], acc[0]);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      acc[1 + c] = fma(fs_sign, fsr[(c + 1) * NN], fma(vs, sFv[(d * 4 + c) * P + id], acc[1 + c]));
  }
  const double t = a.clock[0] + a.c_stage * a.clock[1];
  double src[5] = {0, 0, 0, 0, 0};
  if (g.source == DG_SOURCE_MMS) {
    const double x = X[((size_t)e * 3 + 0) * P + id], y = X[((size_t)e * 3 + 1) * P + id],
                 z = X[((size_t)e * 3 + 2) * P + id];
    // density wave rho = 2 + A sin(pi (x+y+z-t)), u = (1,1,1), p = 1:
    // residual of Eq. 1 = [2r', 2r', 2r', 2r', 3r' - lambda Lap T], r' = pi A cos(phi)
    double sphi, cphi;
    sincospi(x + y + z - t, &sphi, &cphi);
    const double A = g.mms_amp;
    const double rw = 2.0 + A * sphi;
    const double rp = M_PI * A * cphi;
    const double lapT = 3.0 * g.inv_R * (M_PI * M_PI * A * sphi + 2.0 * rp * rp / rw) / (rw * rw);
    src[0] = src[1] = src[2] = src[3] = 2.0 * rp;
    src[4] = 3.0 * rp - g.mu * g.kappa * lapT;
  }
  // Jacobian, source and RK update in FP64
  const double iJ = iJ64[(size_t)e * 10 * P + 9 * P + id];
  if (a.mode == 0) {
#pragma unroll
    for (int c = 0; c < 5; ++c) a.Ut[((size_t)e * 5 + c) * P + id] = fma(-(double)acc[c], iJ, src[c]);
  } else {
    const double dt = a.clock[1];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const size_t o = ((size_t)e * 5 + c) * P + id;
      const double gk = fma(a.A, a.Gk[o], dt * fma(-(double)acc[c], iJ, src[c]));
      a.Gk[o] = gk;
      a.Uw[o] = fma(a.B, gk, q[c]);
    }
  }
}

template <int N, typename R>
static size_t volume2_smem() {
  using S = VShape<N>;
  return sizeof(R) * (3 * S::n * S::n + ((S::n * S::n + 3) & ~3) + S::EPB * S::PER_ELEM);
}

template <int N, typename R>
cudaError_t volume2_setup() {
  return cudaFuncSetAttribute(k_volume2<N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)volume2_smem<N, R>());
}

template <int N, typename R>
cudaError_t volume2_launch(const Ctx& c, const StageArgs& a, cudaStream_t s) {
  using S = VShape<N>;
  const int blocks = (c.E + S::EPB - 1) / S::EPB;
  const R* metrics = (const R*)(sizeof(R) == 8 ? (const void*)c.d_metrics : (const void*)c.d_metrics_f);
  k_volume2<N, R><<<blocks, S::THREADS, volume2_smem<N, R>(), s>>>(
      a, metrics, c.d_metrics, (const R*)c.d_grad, (const R*)c.d_fstar, c.d_elem_face, c.d_X, c.d_D, c.E, c.gas,
      1.0 / c.w[0]);
  return cudaGetLastError();
}

template <int N>
static cudaError_t volume_any(const Ctx& c, const StageArgs& a, cudaStream_t s) {
  return c.prm.precision == DG_FP32OP ? volume2_launch<N, float>(c, a, s) : volume2_launch<N, double>(c, a, s);
}

template <int N>
static cudaError_t setup_any() {
  cudaError_t e = volume2_setup<N, double>();
  return e != cudaSuccess ? e : volume2_setup<N, float>();
}

cudaError_t launch_volume(const Ctx& c, const StageArgs& a, cudaStream_t s) {
  switch (c.N) {
    case 1: return volume_any<1>(c, a, s);
    case 2: return volume_any<2>(c, a, s);
    case 3: return volume_any<3>(c, a, s);
    case 4: return volume_any<4>(c, a, s);
    case 5: return volume_any<5>(c, a, s);
    case 6: return volume_any<6>(c, a, s);
    case 7: return volume_any<7>(c, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t setup_volume(int N) {
  switch (N) {
    case 1: return setup_any<1>();
    case 2: return setup_any<2>();
    case 3: return setup_any<3>();
    case 4: return setup_any<4>();
    case 5: return setup_any<5>();
    case 6: return setup_any<6>();
    case 7: return setup_any<7>();
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dg
