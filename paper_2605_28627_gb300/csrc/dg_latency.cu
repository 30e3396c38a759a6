// Latency variants of the FP64 lifting, face-flux and volume kernels for
// meshes too small to fill the GPU (GALAEXI Sec. 3.1, Eqs. 2-3; the method's steps are
// those of dg_stage.cuh).
//
// With few elements (the 4^3 Taylor-Green case has 128 warps for the GPU's
// 608 SM sub-partitions) every warp runs alone on its sub-partition, and the
// FP64 pipe, which takes a warp instruction in about 76 cycles, makes a
// kernel last as long as its longest warp's FP64 instruction stream.  These
// kernels spread a node's work over three threads, one per reference
// direction d: the d-thread evaluates the split-form pairs, the viscous flux,
// the viscous line sum and the surface terms of its direction (volume), or
// the line derivatives of its direction and one component of every lifted
// gradient (lifting); the three directions' partial sums are added in a
// fixed order.  The face flux (LLF) takes two threads per face node, one per
// side.  One element per block of 3 (N+1)^3 threads, N <= 3.  The
// sums are grouped differently from the one-thread-per-node kernels, so
// results agree with them to rounding, not bit for bit.
#include "dg_stage.cuh"

namespace dg {

template <int N>
struct LatShape {
  static constexpr int n = N + 1, P = n * n * n, NN = n * n, THREADS = 3 * P;
};

// ---------------------------------------------------------------------------
// Lifting: thread (d, node) forms D_d phi + jump_d for the four lifted
// variables, then the d-th component of their gradients
// g_{a,d} = (1/J) sum_d' Ja^{d'}_d (D_d' phi_a + jump_d').
template <int N>
constexpr size_t lift_lat_smem_bytes() {
  constexpr int P = LatShape<N>::P, NN = LatShape<N>::NN;
  return sizeof(double) * ((size_t)4 * P + 24 * NN + 12 * P);
}

template <int N>
__global__ void __launch_bounds__(LatShape<N>::THREADS)
k_lift_lat(const double* __restrict__ U, const double* __restrict__ metrics, const int* __restrict__ elem_nbr,
           const int* __restrict__ elem_face, const double* __restrict__ Dg, double* __restrict__ grad, int E,
           Gas g, double inv_w0) {
  using S = LatShape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN, NF = 6 * NN;
  __shared__ double sD[n * n];
  extern __shared__ __align__(16) unsigned char lat_raw[];
  double* sphi = reinterpret_cast<double*>(lat_raw);   // [4][P]
  double* sjmp = sphi + 4 * P;                         // [6][4][NN]
  double* sdd = sjmp + 24 * NN;                        // [4][3][P]: D_d phi_a + jump_d
  const int d = threadIdx.x / P, id = threadIdx.x - d * P;
  const int e = blockIdx.x;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sD[t] = Dg[t];
  if (d == 0) {
    const double* q = U + (size_t)e * 5 * P + id;
    const double rho = q[0], ir = rcp_op(rho);
    const double m0 = q[P], m1 = q[2 * P], m2 = q[3 * P];
    const double u = m0 * ir, v = m1 * ir, w = m2 * ir;
    const double p = g.gm1 * (q[4 * P] - 0.5 * (m0 * u + m1 * v + m2 * w));
    sphi[id] = u; sphi[P + id] = v; sphi[2 * P + id] = w; sphi[3 * P + id] = p * ir * g.inv_R;
  }
  __syncthreads();
  // face jumps (phi_nbr - phi)/2 (+-1/w_0), threads over the 6 (N+1)^2 face points
  for (int t = threadIdx.x; t < NF; t += blockDim.x) {
    const int f = t / NN, pq = t - f * NN;
    const int code = elem_face[e * 6 + f], nb = elem_nbr[e * 6 + f];
    int p2, q2;
    apply_flip<n>(code & 7, pq % n, pq / n, p2, q2);
    const int enb = dg_idx(nb >> 3, E, kSiteLiftNbr);
    const double* qn = U + (size_t)enb * 5 * P + face_node<n>(nb & 7, p2, q2);
    const double rho = qn[0], ir = rcp_op(rho);
    const double m0 = qn[P], m1 = qn[2 * P], m2 = qn[3 * P];
    const double u = m0 * ir, v = m1 * ir, w = m2 * ir;
    const double pr = g.gm1 * (qn[4 * P] - 0.5 * (m0 * u + m1 * v + m2 * w));
    const double onb[4] = {u, v, w, pr * ir * g.inv_R};
    const int node = face_node<n>(f, pq % n, pq / n);
    const double hs = (f & 1) ? 0.5 * inv_w0 : -0.5 * inv_w0;
#pragma unroll
    for (int a = 0; a < 4; ++a) sjmp[(f * 4 + a) * NN + pq] = (onb[a] - sphi[a * P + node]) * hs;
  }
  __syncthreads();
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  const int r = ijk[d];
  const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
  const int line0 = id - r * stride;
  const double* jm = nullptr;
  if (r == 0 || r == N)
    jm = sjmp + (2 * d + (r == N ? 1 : 0)) * 4 * NN + (d == 0 ? j : i) + n * (d == 2 ? j : k);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    double s = jm ? jm[a * NN] : 0.0;
#pragma unroll
    for (int m = 0; m < n; ++m) s += sD[r * n + m] * sphi[a * P + line0 + m * stride];
    sdd[(a * 3 + d) * P + id] = s;
  }
  __syncthreads();
  // component l = d of the four gradients
  const double* mt = metrics + (size_t)e * 10 * P + id;
  const double J0 = mt[(0 * 3 + d) * P], J1 = mt[(1 * 3 + d) * P], J2 = mt[(2 * 3 + d) * P];
  const double iJ = mt[9 * P];
  double* go = grad + (size_t)e * 12 * P + id;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const double gr = J0 * sdd[(a * 3) * P + id] + J1 * sdd[(a * 3 + 1) * P + id] + J2 * sdd[(a * 3 + 2) * P + id];
    go[(a * 3 + d) * P] = gr * iJ;
  }
}

// ---------------------------------------------------------------------------
// Volume: thread (d, node) takes direction d's pairs, viscous line sum and
// surface terms; the three partial sums meet in shared memory, and thread
// (d, node) finishes the variables c = d and c = d + 3.
template <int N>
constexpr size_t volume_lat_smem_bytes() {
  constexpr int n = N + 1, P = n * n * n;
  // D and its three scalings, rho, u (3), beta/4, |u|^2, J a (9), f_v . J a (12),
  // the three directions' exchange buffers (15), which also hold the partial sums
  return sizeof(double) * ((size_t)4 * n * n + 6 * P + 9 * P + 12 * P + 15 * P);
}

template <int N>
__global__ void __launch_bounds__(LatShape<N>::THREADS)
k_volume_lat(StageArgs a, const double* __restrict__ metrics, const double* __restrict__ grad,
             const double* __restrict__ fstar, const int* __restrict__ elem_face, const double* __restrict__ mms,
             const double* __restrict__ Dg, int E, Gas g, double inv_w0) {
  using S = LatShape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN;
  extern __shared__ __align__(16) unsigned char lat_raw[];
  double* sD = reinterpret_cast<double*>(lat_raw);   // D, viscous surface part in the end diagonals
  double* sT0 = sD + n * n;                          // D/4, D/8, D/16 (scaled two-point fluxes)
  double* sT1 = sT0 + n * n;
  double* sT2 = sT1 + n * n;
  double* sR = sT2 + n * n;                          // rho
  double* sU = sR + P;                               // u, v, w
  double* sB = sU + 3 * P;                           // beta / 4
  double* sK = sB + P;                               // |u|^2
  double* sJ = sK + P;                               // [9][P] J a^d_l, row 3 d + l
  double* sFv = sJ + 9 * P;                          // [3][4][P] (f_v . J a^d)
  double* sX = sFv + 12 * P;                         // [3][5][P] exchange per direction, then partial sums
  __shared__ double s_tc[2];
  const int d = threadIdx.x / P, id = threadIdx.x - d * P;
  const int e = blockIdx.x;
  if (threadIdx.x == 0 && g.source == DG_SOURCE_MMS)
    sincospi(a.clock[0] + a.c_stage * a.clock[1], &s_tc[0], &s_tc[1]);
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const double dr = Dg[t];
    sD[t] = t == 0 ? dr + inv_w0 : (t == n * n - 1 ? dr - inv_w0 : dr);
    sT0[t] = 0.25 * dr;
    sT1[t] = 0.125 * dr;
    sT2[t] = 0.0625 * dr;
  }
  const double* mt = metrics + (size_t)e * 10 * P + id;
  const double Ja0 = mt[(d * 3) * P], Ja1 = mt[(d * 3 + 1) * P], Ja2 = mt[(d * 3 + 2) * P];
  sJ[(d * 3) * P + id] = Ja0;
  sJ[(d * 3 + 1) * P + id] = Ja1;
  sJ[(d * 3 + 2) * P + id] = Ja2;
  if (d == 0) {
    const double* q = a.U + (size_t)e * 5 * P + id;
    const double rho = q[0], ir = rcp_op(rho);
    const double u = q[P] * ir, v = q[2 * P] * ir, w = q[3 * P] * ir;
    const double kk = u * u + v * v + w * w;
    const double p = g.gm1 * fma(-0.5 * rho, kk, q[4 * P]);
    sR[id] = rho; sU[id] = u; sU[P + id] = v; sU[2 * P + id] = w; sK[id] = kk;
    sB[id] = 0.125 * rho * rcp_op(p);
  }
  __syncthreads();
  const double rho = sR[id], u = sU[id], v = sU[P + id], w = sU[2 * P + id], beta = sB[id], kk = sK[id];
  {
    // viscous flux of this direction from the lifted gradients
    double gr[12];
    const double* gg = grad + (size_t)e * 12 * P + id;
#pragma unroll
    for (int r2 = 0; r2 < 12; ++r2) gr[r2] = gg[r2 * P];
    double mu = g.mu, lam = g.mu * g.kappa;
    if (g.visc_law == DG_VISC_SUTHERLAND) {
      // T = p / (rho R) with p from beta/4 = rho / (8 p)
      const double sf = visc_factor<double>(g, 0.125 * rcp_op(beta) * g.inv_R);
      mu *= sf;
      lam *= sf;
    }
    double fv[4];
    visc_flux<double>(gr, u, v, w, mu, lam, Ja0, Ja1, Ja2, fv);
#pragma unroll
    for (int c = 0; c < 4; ++c) sFv[(d * 4 + c) * P + id] = fv[c];
  }
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  const int r = ijk[d];
  const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
  const int line0 = id - r * stride;
  const double* sJd = sJ + d * 3 * P;
  double* sXd = sX + d * 5 * P;
  double acc[5] = {0, 0, 0, 0, 0};
  constexpr int FULL = (n - 1) / 2;
  constexpr bool HALF = (n % 2) == 0;
  __syncthreads();
  auto take_share = [&](int src) {
    const int rm = r * n + src;
    acc[0] = fma(sT0[rm], sXd[id], acc[0]);
    acc[1] = fma(sT1[rm], sXd[P + id], acc[1]);
    acc[2] = fma(sT1[rm], sXd[2 * P + id], acc[2]);
    acc[3] = fma(sT1[rm], sXd[3 * P + id], acc[3]);
    acc[4] = fma(sT2[rm], sXd[4 * P + id], acc[4]);
  };
#pragma unroll 1
  for (int s = 1; s <= FULL; ++s) {
    const int m = r + s < n ? r + s : r + s - n;
    const int mid = line0 + m * stride;
    double F[5];
    ec_pair<double>(rho, sR[mid], beta, sB[mid], u + sU[mid], v + sU[P + mid], w + sU[2 * P + mid], kk + sK[mid],
                    0.0, Ja0 + sJd[mid], Ja1 + sJd[P + mid], Ja2 + sJd[2 * P + mid], g.inv_gm1, g, F);
    const int rm = r * n + m;
    acc[0] = fma(sT0[rm], F[0], acc[0]);
    acc[1] = fma(sT1[rm], F[1], acc[1]);
    acc[2] = fma(sT1[rm], F[2], acc[2]);
    acc[3] = fma(sT1[rm], F[3], acc[3]);
    acc[4] = fma(sT2[rm], F[4], acc[4]);
#pragma unroll
    for (int c = 0; c < 5; ++c) sXd[c * P + mid] = F[c];
    __syncthreads();
    take_share(r - s >= 0 ? r - s : r - s + n);
    __syncthreads();
  }
  if constexpr (HALF) {
    // s = n/2: the pairs (r, r + n/2), r < n/2, on the direction's first P/2 threads
    constexpr int H = n / 2;
    if (id < P / 2) {
      const int hi = id / stride;
      const int ia = id - hi * stride + stride * (hi % H + n * (hi / H));
      const int ib = ia + H * stride;
      double F[5];
      ec_pair<double>(sR[ia], sR[ib], sB[ia], sB[ib], sU[ia] + sU[ib], sU[P + ia] + sU[P + ib],
                      sU[2 * P + ia] + sU[2 * P + ib], sK[ia] + sK[ib], 0.0, sJd[ia] + sJd[ib],
                      sJd[P + ia] + sJd[P + ib], sJd[2 * P + ia] + sJd[2 * P + ib], g.inv_gm1, g, F);
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        sXd[c * P + ia] = F[c];
        sXd[c * P + ib] = F[c];
      }
    }
    __syncthreads();
    take_share(r >= n / 2 ? r - n / 2 : r + n / 2);
  }
  // viscous line sum of direction d, with the viscous surface part in the end diagonals
  {
    double v0 = 0, v1 = 0, v2 = 0, v3 = 0;
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const double Drm = sD[r * n + m];
      const int mid = line0 + m * stride;
      v0 = fma(Drm, sFv[(d * 4 + 0) * P + mid], v0);
      v1 = fma(Drm, sFv[(d * 4 + 1) * P + mid], v1);
      v2 = fma(Drm, sFv[(d * 4 + 2) * P + mid], v2);
      v3 = fma(Drm, sFv[(d * 4 + 3) * P + mid], v3);
    }
    acc[1] -= v0; acc[2] -= v1; acc[3] -= v2; acc[4] -= v3;
  }
  // surface integral on the face of direction d through the node
  if (r == 0 || r == N) {
    const int code = elem_face[e * 6 + 2 * d + (r == N ? 1 : 0)];
    const int fid = dg_idx(code >> 4, 3L * E, kSiteVolFace);   // F = 3 E
    const int pp = d == 0 ? j : i;
    const int qq = d == 2 ? j : k;
    const double* fsr;
    double fs_sign;
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
  // the three directions' sums, in the order d = 0, 1, 2
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 5; ++c) sXd[c * P + id] = acc[c];
  __syncthreads();
  const double iJ = mt[9 * P];
  double sa = 0.0, ca = 0.0;
  if (g.source == DG_SOURCE_MMS) {
    sa = mms[((size_t)e * 2) * P + id];
    ca = mms[((size_t)e * 2 + 1) * P + id];
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = d + 3 * h;
    if (c >= 5) break;
    const double tot = (sX[c * P + id] + sX[(5 + c) * P + id]) + sX[(10 + c) * P + id];
    // manufactured source (density wave, see volume_body)
    double src = 0.0;
    if (g.source == DG_SOURCE_MMS) {
      const double st = s_tc[0], ct = s_tc[1];
      const double sphi = fma(sa, ct, -ca * st);
      const double cphi = fma(ca, ct, sa * st);
      const double A = g.mms_amp;
      const double rp = M_PI * A * cphi;
      if (c < 4) {
        src = 2.0 * rp;
      } else {
        const double rw = 2.0 + A * sphi;
        const double irw = rcp_op(rw);
        const double lapT = 3.0 * g.inv_R * fma(M_PI * M_PI * A, sphi, 2.0 * rp * rp * irw) * (irw * irw);
        src = fma(-(g.mu * g.kappa), lapT, 3.0 * rp);
      }
    }
    const size_t o = ((size_t)e * 5 + c) * P + id;
    if (a.mode == 0) {
      a.Ut[o] = fma(-tot, iJ, src);
    } else {
      const double gk = fma(a.A, a.Gk[o], a.clock[1] * fma(-tot, iJ, src));
      a.Gk[o] = gk;
      a.Uw[o] = fma(a.B, gk, a.U[o]);
    }
  }
}

// ---------------------------------------------------------------------------
// Face flux with the LLF Riemann flux: two threads per face node, one per
// side (even lane: master, odd lane: slave), each forming its side's
// primitives, Euler flux, wave speed and viscous flux; the partner's values
// come by warp shuffle, and the even lane writes the mass and momentum
// components of F*, the odd lane the energy component:
//   F* = (1/2 (f_L + f_R) . n - 1/2 lambda_max (q_R - q_L) - 1/2 (f_v,L + f_v,R) . n) sJ.
template <int N>
__global__ void __launch_bounds__(64)
k_face_lat(const double* __restrict__ U, const double* __restrict__ grad, const FaceInfo* __restrict__ faces,
           const double* __restrict__ facegeo, double* __restrict__ fstar, int F, Gas g) {
  constexpr int n = N + 1, P = n * n * n, NN = n * n;
  const long gid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 1;
  const int side = threadIdx.x & 1;
  const bool live = gid < (long)F * NN;
  const long gsafe = live ? gid : 0;
  const int f = (int)(gsafe / NN), pq = (int)(gsafe % NN);
  const int p = pq % n, q = pq / n;
  const FaceInfo fi = faces[f];
  int e, lf, pp = p, qq = q;
  if (side == 0) {
    e = dg_idx(fi.master >> 3, F / 3, kSiteFaceElems);   // F = 3 E
    lf = fi.master & 7;
  } else {
    e = dg_idx(fi.slave >> 3, F / 3, kSiteFaceElems);
    lf = fi.slave & 7;
    apply_flip<n>(fi.flip, p, q, pp, qq);
  }
  const int node = face_node<n>(lf, pp, qq);
  double qs[5], gs[12];
#pragma unroll
  for (int v = 0; v < 5; ++v) qs[v] = U[((size_t)e * 5 + v) * P + node];
#pragma unroll
  for (int r = 0; r < 12; ++r) gs[r] = grad[((size_t)e * 12 + r) * P + node];
  const double* fg = facegeo + (size_t)f * 4 * NN + pq;
  const double nx = fg[0], ny = fg[NN], nz = fg[2 * NN], sJ = fg[3 * NN];
  const double ir = rcp_op(qs[0]);
  const double u = qs[1] * ir, v = qs[2] * ir, w = qs[3] * ir;
  const double pr = g.gm1 * (qs[4] - 0.5 * (qs[1] * u + qs[2] * v + qs[3] * w));
  double fa[5];
  euler_flux_pm<double>(qs, u, v, w, pr, pr, nx, ny, nz, fa);
  const double lam = fabs(u * nx + v * ny + w * nz) + sqrt(g.gamma * pr * ir);
  double mu = g.mu, lk = g.mu * g.kappa;
  if (g.visc_law == DG_VISC_SUTHERLAND) {
    const double sf = visc_factor<double>(g, pr * ir * g.inv_R);
    mu *= sf;
    lk *= sf;
  }
  double fv[4];
  visc_flux<double>(gs, u, v, w, mu, lk, nx, ny, nz, fv);
  // the partner side's values
  double qo[5], fo[5], fvo[4];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    qo[c] = __shfl_xor_sync(0xffffffffu, qs[c], 1);
    fo[c] = __shfl_xor_sync(0xffffffffu, fa[c], 1);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) fvo[c] = __shfl_xor_sync(0xffffffffu, fv[c], 1);
  const double lamo = __shfl_xor_sync(0xffffffffu, lam, 1);
  if (!live) return;
  // left = master (even lane), right = slave (odd lane)
  const double lL = side ? lamo : lam, lR = side ? lam : lamo;
  const double lmax = lR > lL ? lR : lL;
  double* out = fstar + (size_t)f * 5 * NN + pq;
  if (side == 0) {
    out[0] = (0.5 * (fa[0] + fo[0]) - 0.5 * lmax * (qo[0] - qs[0])) * sJ;
#pragma unroll
    for (int c = 1; c < 4; ++c)
      out[(size_t)c * NN] = (0.5 * (fa[c] + fo[c]) - 0.5 * lmax * (qo[c] - qs[c]) - 0.5 * (fv[c - 1] + fvo[c - 1])) * sJ;
  } else {
    out[(size_t)4 * NN] = (0.5 * (fo[4] + fa[4]) - 0.5 * lmax * (qs[4] - qo[4]) - 0.5 * (fvo[3] + fv[3])) * sJ;
  }
}

// ---------------------------------------------------------------------------
template <int N>
static cudaError_t lat_setup() {
  cudaError_t e = cudaFuncSetAttribute(k_lift_lat<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)lift_lat_smem_bytes<N>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_volume_lat<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)volume_lat_smem_bytes<N>());
  return e;
}

cudaError_t setup_latency(int N) {
  switch (N) {
    case 1: return lat_setup<1>();
    case 2: return lat_setup<2>();
    case 3: return lat_setup<3>();
    default: return cudaSuccess;
  }
}

// Whether the context takes the latency kernels: FP64, LGL nodes, N <= 3 and
// at most kLatencyNodes nodes.  They pay where the one-thread-per-node kernels
// leave sub-partitions idle -- elements of at most two warps, few of them --
// and lose where an element already spans an SM's four sub-partitions or the
// mesh fills the GPU (Taylor-Green, CUDA events per stage: 4^3 N = 3
// 39.1 -> 25.2 us, 6^3 N = 3 40.0 -> 35.5 us; but 8^3 N = 3 59.3 -> 64.1 us
// and 4^3 N = 5 61.4 -> 66.0 us).
bool use_latency_kernels(const Ctx& c) {
  return c.prm.precision == DG_FP64 && c.prm.nodes == DG_NODES_LGL && c.N <= 3 && c.M == 0 &&
         (long)c.E * c.P <= kLatencyNodes;
}

template <int N>
static cudaError_t lift_lat_N(const Ctx& c, const double* U, cudaStream_t s) {
  k_lift_lat<N><<<c.E, LatShape<N>::THREADS, lift_lat_smem_bytes<N>(), s>>>(
      U, c.d_metrics, c.d_elem_nbr, c.d_elem_face, c.d_D, (double*)c.d_grad, c.E, c.gas, 1.0 / c.w[0]);
  return cudaGetLastError();
}

template <int N>
static cudaError_t volume_lat_N(const Ctx& c, const StageArgs& a, cudaStream_t s) {
  k_volume_lat<N><<<c.E, LatShape<N>::THREADS, volume_lat_smem_bytes<N>(), s>>>(
      a, c.d_metrics, (const double*)c.d_grad, (const double*)c.d_fstar, c.d_elem_face, c.d_mms, c.d_D, c.E, c.gas,
      1.0 / c.w[0]);
  return cudaGetLastError();
}

cudaError_t launch_lift_lat(const Ctx& c, const double* U, cudaStream_t s) {
  switch (c.N) {
    case 1: return lift_lat_N<1>(c, U, s);
    case 2: return lift_lat_N<2>(c, U, s);
    case 3: return lift_lat_N<3>(c, U, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int N>
static cudaError_t face_lat_N(const Ctx& c, const double* U, cudaStream_t s) {
  const long threads = 2L * c.nfaces * (N + 1) * (N + 1);
  k_face_lat<N><<<(int)((threads + 63) / 64), 64, 0, s>>>(U, (const double*)c.d_grad, c.d_faces, c.d_facegeo,
                                                         (double*)c.d_fstar, c.nfaces, c.gas);
  return cudaGetLastError();
}

cudaError_t launch_face_lat(const Ctx& c, const double* U, cudaStream_t s) {
  switch (c.N) {
    case 1: return face_lat_N<1>(c, U, s);
    case 2: return face_lat_N<2>(c, U, s);
    case 3: return face_lat_N<3>(c, U, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_volume_lat(const Ctx& c, const StageArgs& a, cudaStream_t s) {
  switch (c.N) {
    case 1: return volume_lat_N<1>(c, a, s);
    case 2: return volume_lat_N<2>(c, a, s);
    case 3: return volume_lat_N<3>(c, a, s);
    default: return cudaErrorInvalidValue;
  }
}

// Host reader of this file's bounds-check error word (0 in normal builds).
DG_BOUNDS_READER(bounds_word_latency)

}  // namespace dg
