// Discrete adjoint of R(U) and of the LSERK4-5 step (FP64).
//
// (dR/dU)^T lambda is the exact transpose of the discrete operator of
// dg_stage.cuh, evaluated by hand-written reverse-mode kernels:
//   A1 volume   : split-form pairs (two-point flux VJP, symmetric reuse with the
//                 partner's share through shared memory), viscous volume term
//                 (D^T, then the viscous-flux VJP), the surface flux seeds;
//   A2 face     : LLF / two-point flux VJP and the BR1-averaged viscous flux VJP
//                 on every face node, both sides;
//   A3 gather   : per node, the face contributions of the node's faces;
//   A4 lifting  : transpose of the BR1 lifting (D^T along lines, own and
//                 neighbour surface terms), then the primitive-variable VJP.
// Everything is gathered (no atomics); d/dmu is reduced from block partials
// in a fixed order.  The step adjoint recomputes the five stage states from
// the step's start state and runs the stages backwards; dg_adjoint_solve runs
// the whole time interval backwards with binomial checkpointing.
#include <algorithm>
#include <vector>

#include "dg_adjoint_fn.cuh"
#include "dg_gauss.cuh"
#include "dg_mortar.cuh"
#include "dg_stage.cuh"

namespace dg {

struct AdjBufs {
  double* qbar;      // [E][5][P]   conserved adjoint from the volume kernel
  double* gbar;      // [E][12][P]  gradient adjoint from the volume kernel
  double* fseed;     // [F][2][5][NN] surface-flux adjoint seeds (master, slave side)
  double* face;      // [F][2][17][NN] per side: conserved adjoint (5) + gradient adjoint (12)
  double* gtil;      // [E][12][P]  total gradient adjoint / J
  double* mupart;    // block partials of d/dmu
  int n_mu;
  double* mx;        // [M][5][4][NN] mortar sides' terms of the lifting transpose (own point order)
  int F;             // face slots (conforming faces, then the mortars' slots)
};

// ---------------------------------------------------------------------------
// Words per node of the volume adjoint's element tile: rho, u, v, w, beta,
// beta/p, 1/(2p) and |u|^2 (8), metric terms (9), lamV (5), the partner's
// adjoint (5).
constexpr int kAdjVolWords = 27;

// A1: volume adjoint.  lamV = -lambda / J.  Two blocks per SM where a block
// has at most 256 threads (one alone leaves the SM seven or eight warps).
template <int N>
__global__ void __launch_bounds__(Shape<N>::THREADS, Shape<N>::THREADS <= 256 ? 2 : 1)
k_adj_volume(const double* __restrict__ U, const double* __restrict__ lam, const double* __restrict__ metrics,
             const double* __restrict__ grad, const int* __restrict__ elem_face, const double* __restrict__ Dg,
             int E, Gas g, double inv_w0, AdjBufs b) {
  using S = Shape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN, EPB = S::EPB;
  constexpr int FULL = (n - 1) / 2;       // shifts with a pair for every node
  constexpr bool HALF = (n % 2) == 0;     // the shift n/2, half as many pairs
  extern __shared__ double adj_smem[];
  double* sD = adj_smem;                                   // [n*n]
  double* sD2 = sD + n * n;                                // [n*n] 2 D (exact)
  double* base = adj_smem + ((2 * n * n + 1) & ~1);
  __shared__ double smu[S::THREADS];
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  double* eb = base + (size_t)le * kAdjVolWords * P;
  // rho, u, v, w, beta/p, beta, 1/(2p), |u|^2 (the flux VJP reads no p)
  auto sPr = [&](int c, int node) -> double& { return eb[c * P + node]; };
  auto sJa = [&](int c, int node) -> double& { return eb[(8 + c) * P + node]; };    // [9]
  auto sL = [&](int c, int node) -> double& { return eb[(17 + c) * P + node]; };    // lamV [5]
  auto sX = [&](int c, int node) -> double& { return eb[(22 + c) * P + node]; };    // partner's adjoint [5]
  const int e = blockIdx.x * EPB + le;
  const bool active = e < E;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    sD[t] = Dg[t];
    sD2[t] = 2.0 * Dg[t];
  }
  double q[5] = {1, 0, 0, 0, 1}, Ja[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, iJ = 0.0, lv[5] = {0, 0, 0, 0, 0};
  NodePrim<double> me{1, 0, 0, 0, 1, 0.5};
  double hip_me = 0.5, bip_me = 0.5, k_me = 0.0;
  if (active) {
#pragma unroll
    for (int c = 0; c < 5; ++c) q[c] = U[((size_t)e * 5 + c) * P + id];
    const double* mt = metrics + (size_t)e * 10 * P + id;
#pragma unroll
    for (int r = 0; r < 9; ++r) { Ja[r] = mt[r * P]; sJa(r, id) = Ja[r]; }
    iJ = mt[9 * P];
#pragma unroll
    for (int c = 0; c < 5; ++c) { lv[c] = -lam[((size_t)e * 5 + c) * P + id] * iJ; sL(c, id) = lv[c]; }
    const double ir = 1.0 / q[0];
    me.rho = q[0]; me.u = q[1] * ir; me.v = q[2] * ir; me.w = q[3] * ir;
    me.p = g.gm1 * (q[4] - 0.5 * (q[1] * me.u + q[2] * me.v + q[3] * me.w));
    me.beta = 0.5 * q[0] / me.p;
    sPr(0, id) = me.rho; sPr(1, id) = me.u; sPr(2, id) = me.v; sPr(3, id) = me.w;
    const double ip = adj_rcp(me.p);
    hip_me = 0.5 * ip;
    bip_me = me.beta * ip;
    sPr(4, id) = bip_me; sPr(5, id) = me.beta;
    k_me = me.u * me.u + me.v * me.v + me.w * me.w;
    sPr(6, id) = hip_me; sPr(7, id) = k_me;
  }
  __syncthreads();
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  double pr[5] = {0, 0, 0, 0, 0};   // own primitive adjoint (rho, u, v, w, p)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int r = ijk[d];
    const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
    const int line0 = id - r * stride;
#pragma unroll 1
    for (int s = 1; s <= FULL; ++s) {
      const int m = r + s < n ? r + s : r + s - n;
      const int mid = line0 + m * stride;
      double pm[5] = {0, 0, 0, 0, 0};
      if (active) {
        NodePrim<double> ot{sPr(0, mid), sPr(1, mid), sPr(2, mid), sPr(3, mid), sPr(4, mid), sPr(5, mid)};
        const double nx = 0.5 * (Ja[d * 3] + sJa(d * 3, mid));
        const double ny = 0.5 * (Ja[d * 3 + 1] + sJa(d * 3 + 1, mid));
        const double nz = 0.5 * (Ja[d * 3 + 2] + sJa(d * 3 + 2, mid));
        const double Drm2 = sD2[r * n + m], Dmr2 = sD2[m * n + r];
        double wb[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) wb[c] = fma(Drm2, lv[c], Dmr2 * sL(c, mid));
        ec_flux_vjp(me, ot, nx, ny, nz, g.inv_gm1, wb, pr, pm, hip_me, sPr(6, mid), bip_me, sPr(4, mid), k_me,
                    sPr(7, mid));
#pragma unroll
        for (int c = 0; c < 5; ++c) sX(c, mid) = pm[c];
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int c = 0; c < 5; ++c) pr[c] += sX(c, id);
      }
      __syncthreads();
    }
    if constexpr (HALF) {
      // s = n/2: the pairs (r, r + n/2), r < n/2, P/2 per element, taken by
      // the first EPB P/2 threads of the block (whole warps instead of every
      // other lane); both adjoint shares go through shared memory
      constexpr int H = n / 2;
      const int t = threadIdx.x;
      const int le2 = t / (P / 2), w2 = t - le2 * (P / 2);
      if (t < EPB * (P / 2) && blockIdx.x * EPB + le2 < E) {
        const int hi = w2 / stride;
        const int ra = hi % H, rb = ra + H;
        const int ia = w2 - hi * stride + stride * (ra + n * (hi / H));   // node with r < n/2
        const int ib = ia + H * stride;                                     // its partner
        double* e2 = base + (size_t)le2 * kAdjVolWords * P;
        NodePrim<double> A{e2[ia], e2[P + ia], e2[2 * P + ia], e2[3 * P + ia], e2[4 * P + ia], e2[5 * P + ia]};
        NodePrim<double> B{e2[ib], e2[P + ib], e2[2 * P + ib], e2[3 * P + ib], e2[4 * P + ib], e2[5 * P + ib]};
        const double* ja = e2 + (8 + d * 3) * P;
        const double nx = 0.5 * (ja[ia] + ja[ib]);
        const double ny = 0.5 * (ja[P + ia] + ja[P + ib]);
        const double nz = 0.5 * (ja[2 * P + ia] + ja[2 * P + ib]);
        const double Drm2 = sD2[ra * n + rb], Dmr2 = sD2[rb * n + ra];
        const double* l2 = e2 + 17 * P;
        double wb[5], pa[5] = {0, 0, 0, 0, 0}, pb[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int c = 0; c < 5; ++c) wb[c] = fma(Drm2, l2[c * P + ia], Dmr2 * l2[c * P + ib]);
        ec_flux_vjp(A, B, nx, ny, nz, g.inv_gm1, wb, pa, pb, e2[6 * P + ia], e2[6 * P + ib], e2[4 * P + ia],
                    e2[4 * P + ib], e2[7 * P + ia], e2[7 * P + ib]);
        double* x2 = e2 + 22 * P;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          x2[c * P + ia] = pa[c];
          x2[c * P + ib] = pb[c];
        }
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int c = 0; c < 5; ++c) pr[c] += sX(c, id);
      }
      __syncthreads();
    }
  }
  double mub = 0.0;
  if (active) {
    // viscous volume term: Fv_bar^d(m) = -sum_i D_im lamV_i, plus the surface term sg lamV / w_0
    double gr[12];
    const double* gg = grad + (size_t)e * 12 * P + id;
#pragma unroll
    for (int r2 = 0; r2 < 12; ++r2) gr[r2] = gg[r2 * P];
    double gb[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    double ub[3] = {0, 0, 0};
    // viscosity law: mu = mu_ref s(T), T = p / (rho R)
    const double Tn = me.p / me.rho * g.inv_R;
    double sv, dsv, vr = 0.0;
    visc_factor_d(g, Tn, sv, dsv);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int r = ijk[d];
      const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
      const int line0 = id - r * stride;
      double fb[4] = {0, 0, 0, 0};
#pragma unroll
      for (int i2 = 0; i2 < n; ++i2) {
        const double Dir = sD[i2 * n + r];
        const int nid = line0 + i2 * stride;
#pragma unroll
        for (int c = 0; c < 4; ++c) fb[c] -= Dir * sL(1 + c, nid);
      }
      if (r == 0 || r == N) {
        const double vs = r == N ? inv_w0 : -inv_w0;
#pragma unroll
        for (int c = 0; c < 4; ++c) fb[c] += vs * lv[1 + c];
      }
      vr += visc_flux_vjp(gr, me.u, me.v, me.w, g.mu * sv, g.kappa, Ja[d * 3], Ja[d * 3 + 1], Ja[d * 3 + 2], fb,
                          gb, ub);
    }
    mub += sv * vr;
    pr[1] += ub[0]; pr[2] += ub[1]; pr[3] += ub[2];
    if (dsv != 0.0) {   // through T = p / (rho R)
      const double Tb = g.mu * dsv * vr;
      pr[4] += Tb * g.inv_R / me.rho;
      pr[0] -= Tb * Tn / me.rho;
    }
    double qb[5] = {0, 0, 0, 0, 0};
    const double uu[3] = {pr[1], pr[2], pr[3]};
    prim_vjp(q, pr[0], uu, pr[4], g.gm1, qb);
#pragma unroll
    for (int c = 0; c < 5; ++c) b.qbar[((size_t)e * 5 + c) * P + id] = qb[c];
#pragma unroll
    for (int r2 = 0; r2 < 12; ++r2) b.gbar[((size_t)e * 12 + r2) * P + id] = gb[r2];
    // surface-flux seeds: F*_out enters with +1/w_0 (master) or -1/w_0 (slave, mapped)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int id_d = ijk[d];
      if (id_d != 0 && id_d != N) continue;
      const int code = elem_face[e * 6 + 2 * d + (id_d == N ? 1 : 0)];
      const int fid = dg_idx(code >> 4, b.F, kSiteAdjFace);
      const int pp = d == 0 ? j : i;
      const int qq = d == 2 ? j : k;
      if (code & 8) {
        double* fs = b.fseed + ((size_t)fid * 2 + 0) * 5 * NN + pp + n * qq;
#pragma unroll
        for (int c = 0; c < 5; ++c) fs[c * NN] = lv[c] * inv_w0;
      } else {
        int p2, q2;
        apply_flip<n>(code & 7, pp, qq, p2, q2);
        double* fs = b.fseed + ((size_t)fid * 2 + 1) * 5 * NN + p2 + n * q2;
#pragma unroll
        for (int c = 0; c < 5; ++c) fs[c * NN] = -lv[c] * inv_w0;
      }
    }
  }
  // block partial of d/dmu (the block need not be a whole number of warps,
  // so the partials go through shared memory, summed by one thread in order)
  smu[threadIdx.x] = mub;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int t = 0; t < S::THREADS; ++t) s += smu[t];
    b.mupart[blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Face VJP at one face point: from the adjoint Fb of F* (F* = (f* - f_v avg) sJ)
// to the conserved (5) and gradient (12) adjoints of the two sides, added to
// qbL, gbL (side L, whose outward normal (nx, ny, nz) is) and qbR, gbR; returns
// the d/dmu contribution.
__device__ __forceinline__ double face_vjp_point(const double qL[5], const double qR[5], const double gL[12],
                                                 const double gR[12], double nx, double ny, double nz, double sJ,
                                                 const double Fb[5], const Gas& g, double qbL[5], double qbR[5],
                                                 double gbL[12], double gbR[12]) {
  double fa_b[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) fa_b[c] = Fb[c] * sJ;
  if (g.surf_flux == DG_FLUX_EC) {
    const double irL = 1.0 / qL[0], irR = 1.0 / qR[0];
    NodePrim<double> A{qL[0], qL[1] * irL, qL[2] * irL, qL[3] * irL, 0, 0};
    A.p = g.gm1 * (qL[4] - 0.5 * (qL[1] * A.u + qL[2] * A.v + qL[3] * A.w));
    A.beta = 0.5 * qL[0] / A.p;
    NodePrim<double> B{qR[0], qR[1] * irR, qR[2] * irR, qR[3] * irR, 0, 0};
    B.p = g.gm1 * (qR[4] - 0.5 * (qR[1] * B.u + qR[2] * B.v + qR[3] * B.w));
    B.beta = 0.5 * qR[0] / B.p;
    double pa[5] = {0, 0, 0, 0, 0}, pb[5] = {0, 0, 0, 0, 0};
    ec_flux_vjp(A, B, nx, ny, nz, g.inv_gm1, fa_b, pa, pb);
    const double ua[3] = {pa[1], pa[2], pa[3]}, ubv[3] = {pb[1], pb[2], pb[3]};
    prim_vjp(qL, pa[0], ua, pa[4], g.gm1, qbL);
    prim_vjp(qR, pb[0], ubv, pb[4], g.gm1, qbR);
  } else if (g.surf_flux == DG_FLUX_ROE) {
    roe_vjp(qL, qR, nx, ny, nz, g.gamma, g.gm1, fa_b, qbL, qbR);
  } else {
    llf_vjp(qL, qR, nx, ny, nz, g.gamma, g.gm1, fa_b, qbL, qbR);
  }
  // viscous part: F* includes -1/2 (f_v(L) + f_v(R)) . n sJ
  double fvb[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) fvb[c] = -0.5 * Fb[1 + c] * sJ;
  double ubL[3] = {0, 0, 0}, ubR[3] = {0, 0, 0};
  const double irL = 1.0 / qL[0], irR = 1.0 / qR[0];
  // viscosity law on each side: mu = mu_ref s(T), T = p / (rho R)
  const double uL = qL[1] * irL, vL = qL[2] * irL, wL = qL[3] * irL;
  const double uR = qR[1] * irR, vR = qR[2] * irR, wR = qR[3] * irR;
  const double TL = g.gm1 * (qL[4] - 0.5 * (qL[1] * uL + qL[2] * vL + qL[3] * wL)) * irL * g.inv_R;
  const double TR = g.gm1 * (qR[4] - 0.5 * (qR[1] * uR + qR[2] * vR + qR[3] * wR)) * irR * g.inv_R;
  double sL, dsL, sR, dsR;
  visc_factor_d(g, TL, sL, dsL);
  visc_factor_d(g, TR, sR, dsR);
  const double vrL = visc_flux_vjp(gL, uL, vL, wL, g.mu * sL, g.kappa, nx, ny, nz, fvb, gbL, ubL);
  const double vrR = visc_flux_vjp(gR, uR, vR, wR, g.mu * sR, g.kappa, nx, ny, nz, fvb, gbR, ubR);
  const double TbL = g.mu * dsL * vrL, TbR = g.mu * dsR * vrR;   // through T = p / (rho R)
  prim_vjp(qL, -TbL * TL * irL, ubL, TbL * g.inv_R * irL, g.gm1, qbL);
  prim_vjp(qR, -TbR * TR * irR, ubR, TbR * g.inv_R * irR, g.gm1, qbR);
  return sL * vrL + sR * vrR;
}

// A2: face adjoint, one thread per face node of the conforming faces (master
// orientation); the mortars' slots follow them (k_adj_mortar_face).  FACE:
// Gauss nodes, where U and grad are the face values [E][6][5|12][NN].
template <int N, bool FACE = false>
__global__ void __launch_bounds__(128)
k_adj_face(const double* __restrict__ U, const double* __restrict__ grad, const FaceInfo* __restrict__ faces,
           const double* __restrict__ facegeo, int F, int E, Gas g, AdjBufs b, int mu_offset) {
  constexpr int n = N + 1, NN = n * n;
  __shared__ double smu[4];
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double mub = 0.0;
  if (gid < (long)F * NN) {
    const int f = (int)(gid / NN), pq = (int)(gid % NN);
    const int p = pq % n, q = pq / n;
    const FaceInfo fi = faces[f];
    const int eM = dg_idx(fi.master >> 3, E, kSiteAdjFace), fM = fi.master & 7;
    const int eS = dg_idx(fi.slave >> 3, E, kSiteAdjFace), fS = fi.slave & 7;
    int p2, q2;
    apply_flip<n>(fi.flip, p, q, p2, q2);
    int su, sg;
    const double* uM = side_ptr<n, FACE, 5>(U, eM, fM, p, q, su);
    const double* uS = side_ptr<n, FACE, 5>(U, eS, fS, p2, q2, su);
    const double* gM = side_ptr<n, FACE, 12>(grad, eM, fM, p, q, sg);
    const double* gS = side_ptr<n, FACE, 12>(grad, eS, fS, p2, q2, sg);
    double qL[5], qR[5], Fb[5];
    const double* s0 = b.fseed + ((size_t)f * 2 + 0) * 5 * NN + pq;
    const double* s1 = b.fseed + ((size_t)f * 2 + 1) * 5 * NN + pq;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      qL[c] = uM[c * su];
      qR[c] = uS[c * su];
      Fb[c] = s0[c * NN] + s1[c * NN];
    }
    const double* fg = facegeo + (size_t)f * 4 * NN + pq;
    double gL[12], gR[12], gbL[12], gbR[12];
#pragma unroll
    for (int r = 0; r < 12; ++r) {
      gL[r] = gM[r * sg];
      gR[r] = gS[r * sg];
      gbL[r] = 0.0;
      gbR[r] = 0.0;
    }
    double qbL[5] = {0, 0, 0, 0, 0}, qbR[5] = {0, 0, 0, 0, 0};
    mub = face_vjp_point(qL, qR, gL, gR, fg[0], fg[NN], fg[2 * NN], fg[3 * NN], Fb, g, qbL, qbR, gbL, gbR);
    double* oL = b.face + ((size_t)f * 2 + 0) * 17 * NN + pq;
    double* oR = b.face + ((size_t)f * 2 + 1) * 17 * NN + pq;
#pragma unroll
    for (int c = 0; c < 5; ++c) { oL[c * NN] = qbL[c]; oR[c * NN] = qbR[c]; }
#pragma unroll
    for (int r = 0; r < 12; ++r) { oL[(5 + r) * NN] = gbL[r]; oR[(5 + r) * NN] = gbR[r]; }
  }
  for (int o = 16; o > 0; o >>= 1) mub += __shfl_down_sync(0xffffffffu, mub, o);
  if ((threadIdx.x & 31) == 0) smu[threadIdx.x >> 5] = mub;
  __syncthreads();
  if (threadIdx.x == 0) b.mupart[mu_offset + blockIdx.x] = smu[0] + smu[1] + smu[2] + smu[3];
}

// A2': mortar faces (Sec. 3.2.2, Algorithm 1), one block per mortar, a thread
// per quadrant node.  Forward: on quadrant k the flux of the small side's
// state and gradients and the big side's interpolated ones, F_k; on the big
// face F_B = -P1(F_k), P1 the projection with the quadrature (scale 1).  So
// the quadrant flux's adjoint is its own slot's seed minus P1^T of the big
// slot's seed; the face VJP at each quadrant point gives the small side's
// adjoints (its slot, own point order) and those of the interpolated big-side
// values, which go back to the big face's nodes by the transposed
// interpolation (the big slot).
template <int N>
static size_t adj_mortar_face_smem() {
  constexpr int n = N + 1, NN = n * n;
  return sizeof(double) * ((size_t)8 * NN + n + 17 * NN + 34 * NN + 5 * NN + 10 * NN + 68 * NN + 68 * NN);
}

// FACE: Gauss nodes, U and grad the face values [E][6][5|12][NN].
template <int N, bool FACE = false>
__global__ void __launch_bounds__(MortarShape<N>::THREADS)
k_adj_mortar_face(const double* __restrict__ U, const double* __restrict__ grad, const double* __restrict__ facegeo,
                  const int* __restrict__ mortars, const double* __restrict__ tab, int E, Gas g, AdjBufs b,
                  int mu_offset) {
  using S = MortarShape<N>;
  constexpr int n = S::n, NN = S::NN, T = S::THREADS;
  extern __shared__ double am[];
  double* sI = am;                  // [2][n][n] I_h[x][j]
  double* sIT = sI + 2 * NN;        // [2][j][x]
  double* sW = sIT + 2 * NN;        // [2][x][j] w_x I_h[x][j]
  double* sWT = sW + 2 * NN;        // [2][j][x] w_x I_h[x][j]
  double* sw = sWT + 2 * NN;        // [n]
  double* sB = sw + n;              // [17][NN] big face: state, gradients
  double* sT = sB + 17 * NN;        // [2][17][NN]
  double* sY = sT + 34 * NN;        // [5][NN] big slot seed / (w_i w_j)
  double* sT2 = sY + 5 * NN;        // [2][5][NN]
  double* sX = sT2 + 10 * NN;       // [4][17][NN] adjoints of the interpolated big-side values
  double* sS = sX + 68 * NN;        // [4][17][NN]
  const int m = blockIdx.x, t = threadIdx.x;
  const int* r = mortars + (size_t)m * 20;
  const int eB = dg_idx(r[0], E, kSiteMortar), fB = r[1], slotB = dg_idx(r[2], b.F, kSiteMortar);
  mortar_tables<n>(tab, sI, sIT, sW, sw, t, T);
  for (int x = t; x < 2 * NN; x += T) {   // sWT[h][j][a] = w_a I_h[a][j]
    const int h = x / NN, rr = x - h * NN, a = rr / n, j = rr - a * n;
    sWT[h * NN + j * n + a] = tab[2 * NN + a] * tab[x];
  }
  if (t < NN) {
    const int i = t % n, j = t / n;
    int su, sg;
    const double* qb = side_ptr<n, FACE, 5>(U, eB, fB, i, j, su);
    const double* gb = side_ptr<n, FACE, 12>(grad, eB, fB, i, j, sg);
#pragma unroll
    for (int v = 0; v < 5; ++v) sB[v * NN + t] = qb[v * su];
#pragma unroll
    for (int x = 0; x < 12; ++x) sB[(5 + x) * NN + t] = gb[x * sg];
    const double iww = 1.0 / (tab[2 * NN + i] * tab[2 * NN + j]);
#pragma unroll
    for (int v = 0; v < 5; ++v) sY[v * NN + t] = b.fseed[((size_t)slotB * 2 * 5 + v) * NN + t] * iww;
  }
  __syncthreads();
  mortar_sweep1<n, 17>(sIT, sB, sT, t, T);
  mortar_sweep1<n, 5>(sWT, sY, sT2, t, T);
  __syncthreads();
  const int k = t / NN, pq = t % NN, pp = pq % n, qq = pq / n;
  double qR[17], z[5];
  mortar_sweep2<n, 17>(sI, sT, k, pp, qq, qR);
  mortar_sweep2<n, 5>(sW, sT2, k, pp, qq, z);   // P1^T of the big slot's seed at this quadrant point
  const int es = dg_idx(r[3 + 4 * k], E, kSiteMortar), fs = r[4 + 4 * k], fl = r[5 + 4 * k];
  const int slot = dg_idx(r[6 + 4 * k], b.F, kSiteMortar);
  int p2, q2;
  apply_flip<n>(fl, pp, qq, p2, q2);
  const int o = p2 + n * q2;
  int su, sg;
  const double* qs = side_ptr<n, FACE, 5>(U, es, fs, p2, q2, su);
  const double* gs = side_ptr<n, FACE, 12>(grad, es, fs, p2, q2, sg);
  double qL[5], gL[12], Fb[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = qs[v * su];
    Fb[v] = b.fseed[((size_t)slot * 2 * 5 + v) * NN + o] - z[v];
  }
#pragma unroll
  for (int x = 0; x < 12; ++x) gL[x] = gs[x * sg];
  const double* fg = facegeo + (size_t)slot * 4 * NN + o;
  double qbL[5] = {0, 0, 0, 0, 0}, qbR[5] = {0, 0, 0, 0, 0}, gbL[12], gbR[12];
#pragma unroll
  for (int x = 0; x < 12; ++x) { gbL[x] = 0.0; gbR[x] = 0.0; }
  double mub = face_vjp_point(qL, qR, gL, qR + 5, fg[0], fg[NN], fg[2 * NN], fg[3 * NN], Fb, g, qbL, qbR, gbL, gbR);
  double* os = b.face + ((size_t)slot * 2 + 0) * 17 * NN + o;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    os[v * NN] = qbL[v];
    sX[(k * 17 + v) * NN + pq] = qbR[v];
  }
#pragma unroll
  for (int x = 0; x < 12; ++x) {
    os[(5 + x) * NN] = gbL[x];
    sX[(k * 17 + 5 + x) * NN + pq] = gbR[x];
  }
  __syncthreads();
  mortar_proj1<n, 17>(sI, sX, sS, t, T);   // transposed interpolation, first direction
  __syncthreads();
  for (int ox = t; ox < 17 * NN; ox += T) {
    const int f = ox / NN, ij = ox - f * NN;
    b.face[((size_t)slotB * 2 + 0) * 17 * NN + (size_t)f * NN + ij] = mortar_proj2<n, 17>(sI, sS, f, ij % n, ij / n);
  }
  // d/dmu: the block's partial, summed in a fixed order
  __shared__ double smu[MortarShape<N>::THREADS];
  smu[t] = mub;
  __syncthreads();
  if (t == 0) {
    double acc = 0.0;
    for (int x = 0; x < T; ++x) acc += smu[x];
    b.mupart[mu_offset + m] = acc;
  }
}

// A3': the mortar sides' terms of the lifting transpose.  Forward: the face
// average of quadrant k is star_k = (phi_s + I_k phi_B)/2, that of the big face
// star_B = P(star_k) (point-value projection, scale 1/4).  With Y = the
// lifting's own surface weight at a face point (Y = gtil . n sJ / w_0), the
// derivative w.r.t. phi at each side's points, beside the own -Y/2:
//   small side k: + (P^T Y_B)_k / 2,
//   big side    : - Y_B / 2 + sum_k I_k^T ((P^T Y_B)_k + Y_k) / 2.
// FACE: Gauss nodes, where Y is the weak lifting's surface sum S of the face
// point (lgf, own point order) and the own term is +Y/2 (no -phi term).
template <int N, bool FACE = false>
__global__ void __launch_bounds__(MortarShape<N>::THREADS)
k_adj_mortar_lift(const double* __restrict__ metrics, const int* __restrict__ mortars, const double* __restrict__ tab,
                  int E, double inv_w0, AdjBufs b, const double* __restrict__ lgf) {
  using S = MortarShape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN, T = S::THREADS;
  __shared__ double sI[2 * NN], sIT[2 * NN], sW[2 * NN], sWT[2 * NN], sw[n];
  __shared__ double sYB[4 * NN], sYs[4 * NN];    // Y_B / (w_i w_j); Y_B
  __shared__ double sT[8 * NN], sV[16 * NN], sS[16 * NN];
  const int m = blockIdx.x, t = threadIdx.x;
  const int* r = mortars + (size_t)m * 20;
  const int eB = dg_idx(r[0], E, kSiteMortar), fB = r[1];
  mortar_tables<n>(tab, sI, sIT, sW, sw, t, T);
  for (int x = t; x < 2 * NN; x += T) {
    const int h = x / NN, rr = x - h * NN, a = rr / n, j = rr - a * n;
    sWT[h * NN + j * n + a] = tab[2 * NN + a] * tab[x];
  }
  // Y at a face point of (e, f): inv_w0 (2s-1) sum_l gtil_{phi,l} Ja^d_l
  auto Yat = [&](int e, int f, int p, int q, double y[4]) {
    if constexpr (FACE) {
      const double* sf = lgf + ((size_t)e * 6 + f) * 9 * NN + p + n * q;
#pragma unroll
      for (int ph = 0; ph < 4; ++ph) y[ph] = sf[ph * NN];
      return;
    }
    const int node = face_node<n>(f, p, q), d = f >> 1;
    const double sg = (f & 1) ? inv_w0 : -inv_w0;
    const double* mt = metrics + (size_t)e * 10 * P + node;
    const double a0 = mt[(d * 3) * P], a1 = mt[(d * 3 + 1) * P], a2 = mt[(d * 3 + 2) * P];
    const double* gt = b.gtil + (size_t)e * 12 * P + node;
#pragma unroll
    for (int ph = 0; ph < 4; ++ph) y[ph] = sg * (gt[(ph * 3) * P] * a0 + gt[(ph * 3 + 1) * P] * a1 + gt[(ph * 3 + 2) * P] * a2);
  };
  if (t < NN) {
    const int i = t % n, j = t / n;
    double y[4];
    Yat(eB, fB, i, j, y);
    const double iww = 1.0 / (tab[2 * NN + i] * tab[2 * NN + j]);
#pragma unroll
    for (int ph = 0; ph < 4; ++ph) {
      sYs[ph * NN + t] = y[ph];
      sYB[ph * NN + t] = 0.25 * y[ph] * iww;
    }
  }
  __syncthreads();
  mortar_sweep1<n, 4>(sWT, sYB, sT, t, T);
  __syncthreads();
  const int k = t / NN, pq = t % NN, pp = pq % n, qq = pq / n;
  double z[4];
  mortar_sweep2<n, 4>(sW, sT, k, pp, qq, z);   // (P^T Y_B)_k at this quadrant point
  const int es = dg_idx(r[3 + 4 * k], E, kSiteMortar), fs = r[4 + 4 * k], fl = r[5 + 4 * k];
  int p2, q2;
  apply_flip<n>(fl, pp, qq, p2, q2);
  double ys[4];
  Yat(es, fs, p2, q2, ys);
  double* xs = b.mx + (size_t)(5 * m + k) * 4 * NN + p2 + n * q2;
#pragma unroll
  for (int ph = 0; ph < 4; ++ph) {
    xs[ph * NN] = 0.5 * z[ph];
    sV[(k * 4 + ph) * NN + pq] = z[ph] + ys[ph];
  }
  __syncthreads();
  mortar_proj1<n, 4>(sI, sV, sS, t, T);   // transposed interpolation
  __syncthreads();
  if (t < NN) {
    const int i = t % n, j = t / n;
    double* xb = b.mx + (size_t)(5 * m + 4) * 4 * NN + t;
#pragma unroll
    for (int ph = 0; ph < 4; ++ph) xb[ph * NN] = -0.5 * sYs[ph * NN + t] + 0.5 * mortar_proj2<n, 4>(sI, sS, ph, i, j);
  }
}

// A3: per node, add the face contributions of the node's faces; store the
// total gradient adjoint divided by J, and the conserved adjoint so far.
template <int N>
__global__ void __launch_bounds__(128)
k_adj_gather(const double* __restrict__ metrics, const int* __restrict__ elem_face, int E, AdjBufs b) {
  constexpr int n = N + 1, P = n * n * n, NN = n * n;
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long)E * P) return;
  const int e = (int)(t / P), id = (int)(t % P);
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  double gb[12], qb[5];
#pragma unroll
  for (int r = 0; r < 12; ++r) gb[r] = b.gbar[((size_t)e * 12 + r) * P + id];
#pragma unroll
  for (int c = 0; c < 5; ++c) qb[c] = b.qbar[((size_t)e * 5 + c) * P + id];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id_d = ijk[d];
    if (id_d != 0 && id_d != N) continue;
    const int code = elem_face[e * 6 + 2 * d + (id_d == N ? 1 : 0)];
    const int fid = dg_idx(code >> 4, b.F, kSiteAdjFace);
    const int pp = d == 0 ? j : i;
    const int qq = d == 2 ? j : k;
    int pm = pp, qm = qq, side = 0;
    if (!(code & 8)) { apply_flip<n>(code & 7, pp, qq, pm, qm); side = 1; }
    const double* src = b.face + ((size_t)fid * 2 + side) * 17 * NN + pm + n * qm;
#pragma unroll
    for (int c = 0; c < 5; ++c) qb[c] += src[c * NN];
#pragma unroll
    for (int r = 0; r < 12; ++r) gb[r] += src[(5 + r) * NN];
  }
  const double iJ = metrics[(size_t)e * 10 * P + 9 * P + id];
#pragma unroll
  for (int r = 0; r < 12; ++r) b.gtil[((size_t)e * 12 + r) * P + id] = gb[r] * iJ;
#pragma unroll
  for (int c = 0; c < 5; ++c) b.qbar[((size_t)e * 5 + c) * P + id] = qb[c];
}

// ---------------------------------------------------------------------------
// A4: transpose of the lifting, then the primitive VJP; out = total adjoint.
// MORTAR: a face whose neighbour entry is negative is a mortar side, whose
// partner term comes from b.mx (k_adj_mortar_lift).
template <int N, bool MORTAR = false>
__global__ void __launch_bounds__(Shape<N>::THREADS)
k_adj_lift(const double* __restrict__ U, const double* __restrict__ metrics, const int* __restrict__ elem_nbr,
           const int* __restrict__ elem_face, const double* __restrict__ Dg, int E, Gas g, double inv_w0, AdjBufs b,
           double* __restrict__ out, int n_mortar) {
  using S = Shape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN, EPB = S::EPB;
  extern __shared__ double adj_smem[];
  double* sD = adj_smem;                                   // [n*n]
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  double* sY = adj_smem + ((n * n + 1) & ~1) + (size_t)le * 12 * P;   // Y^d_phi = sum_l Ja^d_l gtil_{phi,l}, row phi*3+d
  const int e = blockIdx.x * EPB + le;
  const bool active = e < E;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sD[t] = Dg[t];
  double Ja[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gt[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (active) {
    const double* mt = metrics + (size_t)e * 10 * P + id;
#pragma unroll
    for (int r = 0; r < 9; ++r) Ja[r] = mt[r * P];
#pragma unroll
    for (int r = 0; r < 12; ++r) gt[r] = b.gtil[((size_t)e * 12 + r) * P + id];
#pragma unroll
    for (int ph = 0; ph < 4; ++ph)
#pragma unroll
      for (int d = 0; d < 3; ++d)
        sY[(ph * 3 + d) * P + id] = Ja[d * 3] * gt[ph * 3] + Ja[d * 3 + 1] * gt[ph * 3 + 1] + Ja[d * 3 + 2] * gt[ph * 3 + 2];
  }
  __syncthreads();
  if (!active) return;
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  double phib[4] = {0, 0, 0, 0};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int r = ijk[d];
    const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
    const int line0 = id - r * stride;
#pragma unroll
    for (int i2 = 0; i2 < n; ++i2) {
      const double Dir = sD[i2 * n + r];
      const int nid = line0 + i2 * stride;
#pragma unroll
      for (int ph = 0; ph < 4; ++ph) phib[ph] += Dir * sY[(ph * 3 + d) * P + nid];
    }
  }
  // surface terms: own -1/2 gtil . nsJ / w0, neighbour partner +1/2 gtil' . nsJ' / w0
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int id_d = ijk[d];
    if (id_d != 0 && id_d != N) continue;
    const int s = id_d == N ? 1 : 0;
    const double sg = s ? 1.0 : -1.0;
#pragma unroll
    for (int ph = 0; ph < 4; ++ph)
      phib[ph] -= 0.5 * inv_w0 * sg * (gt[ph * 3] * Ja[d * 3] + gt[ph * 3 + 1] * Ja[d * 3 + 1] + gt[ph * 3 + 2] * Ja[d * 3 + 2]);
    const int f = 2 * d + s;
    const int code = elem_face[e * 6 + f];
    const int nb = elem_nbr[e * 6 + f];
    const int pp = d == 0 ? j : i;
    const int qq = d == 2 ? j : k;
    if constexpr (MORTAR) {
      if (nb < 0) {
        const double* xm = b.mx + (size_t)dg_idx(-1 - nb, 5L * n_mortar, kSiteMortar) * 4 * NN + pp + n * qq;
#pragma unroll
        for (int ph = 0; ph < 4; ++ph) phib[ph] += xm[ph * NN];
        continue;
      }
    }
    const int e2 = dg_idx(nb >> 3, E, kSiteAdjFace), f2 = nb & 7;
    int p2, q2;
    apply_flip<n>(code & 7, pp, qq, p2, q2);
    const int id2 = face_node<n>(f2, p2, q2);
    const int d2 = f2 >> 1;
    const double sg2 = (f2 & 1) ? 1.0 : -1.0;
    const double* mt2 = metrics + (size_t)e2 * 10 * P + id2;
    const double n0 = sg2 * mt2[(d2 * 3) * P], n1 = sg2 * mt2[(d2 * 3 + 1) * P], n2 = sg2 * mt2[(d2 * 3 + 2) * P];
    const double* g2 = b.gtil + (size_t)e2 * 12 * P + id2;
#pragma unroll
    for (int ph = 0; ph < 4; ++ph)
      phib[ph] += 0.5 * inv_w0 * (g2[(ph * 3) * P] * n0 + g2[(ph * 3 + 1) * P] * n1 + g2[(ph * 3 + 2) * P] * n2);
  }
  // phi = (u, v, w, T), T = p / (rho R)
  double q[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) q[c] = U[((size_t)e * 5 + c) * P + id];
  const double ir = 1.0 / q[0];
  const double u = q[1] * ir, v = q[2] * ir, w = q[3] * ir;
  const double p = g.gm1 * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w));
  const double T = p * ir * g.inv_R;
  const double ub[3] = {phib[0], phib[1], phib[2]};
  double qb[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) qb[c] = b.qbar[((size_t)e * 5 + c) * P + id];
  prim_vjp(q, -phib[3] * T * ir, ub, phib[3] * ir * g.inv_R, g.gm1, qb);
#pragma unroll
  for (int c = 0; c < 5; ++c) out[((size_t)e * 5 + c) * P + id] = qb[c];
}

// ---------------------------------------------------------------------------
// Legendre-Gauss nodes (the weak form of Eqs. 2 and 3, kernels of dg_gauss.cu).
// Forward, at node i with index r along direction d (face point pq of its line):
//   R_i = (1/J_i) [ sum_d sum_m Dw[r][m] Ft^d_m - sum_{d,s} l_s(r)/w_r Fout_{2d+s}(pq) ] + Q,
//   Ft^d = (f - f_v)(q, g) . Ja^d, Fout the outward surface flux (master F*,
//   slave -F* at the mapped point), Dw[r][m] = (w_m / w_r) D_{m r};
//   J g_i = - sum_d sum_m Dw[r][m] (phi Ja^d)_m + sum_{d,s} l_s(r)/w_r phi*_{2d+s}(pq) n sJ,
//   phi* = (phi(Uf own) + phi(Uf nbr)) / 2 at the face points;
//   Uf_f(pq) = sum_m l_s(m) U(line m), gf likewise from g.
// Five kernels: B1 volume and surface seeds, A2 (FACE) the face VJP on the
// face values, B3 the gradients' adjoint per node and the lifting's surface
// sums per face point, B4 the face values' adjoint, B5 the lifting's volume
// transpose and the transposed prolongation.  lamV = lambda / J.
// Per element face, lgf [E][6][9][NN]: the surface sums S (4) and the adjoint
// of the face values Uf (5), own point order.

// B1: Ft-bar^d_m = sum_r Dw[r][m] lamV_r along the line through m, then the
// Euler and viscous flux VJPs (qbar, gbar, d/dmu); the surface seeds
// Fout-bar_f(pq) = - sum_r l_s(r)/w_r lamV_r, stored as the adjoint of F*
// (master: as is; slave: negated, at the master's point).
template <int N>
__global__ void __launch_bounds__(Shape<N>::THREADS)
k_adjlg_volume(const double* __restrict__ U, const double* __restrict__ lam, const double* __restrict__ metrics,
               const double* __restrict__ grad, const int* __restrict__ elem_face, const double* __restrict__ tab,
               int E, Gas g, AdjBufs b) {
  using S = Shape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN;
  extern __shared__ double adjlg_smem[];
  __shared__ double sDw[n * n], sT[2 * n];
  __shared__ double smu[S::THREADS];
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  const int e = blockIdx.x * S::EPB + le;
  const bool active = e < E;
  double* sL = adjlg_smem + (size_t)le * 5 * P;   // lamV [5][P]
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sDw[t] = tab[GaussTab::Dw(n) + t];
  for (int t = threadIdx.x; t < 2 * n; t += blockDim.x) sT[t] = tab[GaussTab::lmw(n) + t];
  if (active) {
    const double iJ = metrics[((size_t)e * 10 + 9) * P + id];
#pragma unroll
    for (int c = 0; c < 5; ++c) sL[c * P + id] = lam[((size_t)e * 5 + c) * P + id] * iJ;
  }
  __syncthreads();
  double mub = 0.0;
  if (active) {
    const int i = id % n, j = (id / n) % n, k = id / NN;
    const int ijk[3] = {i, j, k};
    double q[5], gr[12], Ja[9];
#pragma unroll
    for (int c = 0; c < 5; ++c) q[c] = U[((size_t)e * 5 + c) * P + id];
#pragma unroll
    for (int r = 0; r < 12; ++r) gr[r] = grad[((size_t)e * 12 + r) * P + id];
#pragma unroll
    for (int r = 0; r < 9; ++r) Ja[r] = metrics[((size_t)e * 10 + r) * P + id];
    const double ir = 1.0 / q[0];
    const double u = q[1] * ir, v = q[2] * ir, w = q[3] * ir;
    const double p = g.gm1 * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w));
    const double Tn = p * ir * g.inv_R;
    double sv, dsv;
    visc_factor_d(g, Tn, sv, dsv);
    double qb[5] = {0, 0, 0, 0, 0}, gb[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, ub[3] = {0, 0, 0}, vr = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int r = ijk[d];
      const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
      const int line0 = id - r * stride;
      double fb[5] = {0, 0, 0, 0, 0};
      for (int r2 = 0; r2 < n; ++r2) {
        const double c = sDw[r2 * n + r];
        const int nid = line0 + r2 * stride;
#pragma unroll
        for (int x = 0; x < 5; ++x) fb[x] = fma(c, sL[x * P + nid], fb[x]);
      }
      euler_flux_vjp(q, u, v, w, p, Ja[d * 3], Ja[d * 3 + 1], Ja[d * 3 + 2], fb, g.gm1, qb);
      const double fvb[4] = {-fb[1], -fb[2], -fb[3], -fb[4]};
      vr += visc_flux_vjp(gr, u, v, w, g.mu * sv, g.kappa, Ja[d * 3], Ja[d * 3 + 1], Ja[d * 3 + 2], fvb, gb, ub);
    }
    mub = sv * vr;
    const double Tb = g.mu * dsv * vr;   // through T = p / (rho R)
    prim_vjp(q, -Tb * Tn * ir, ub, Tb * g.inv_R * ir, g.gm1, qb);
#pragma unroll
    for (int c = 0; c < 5; ++c) b.qbar[((size_t)e * 5 + c) * P + id] = qb[c];
#pragma unroll
    for (int r = 0; r < 12; ++r) b.gbar[((size_t)e * 12 + r) * P + id] = gb[r];
    for (int o = id; o < 30 * NN; o += P) {
      const int f = o / (5 * NN), rr = o - f * 5 * NN, x = rr / NN, pq = rr - x * NN;
      const int pp = pq % n, qq = pq / n, d = f >> 1;
      const double* lw = sT + (f & 1) * n;
      double s = 0.0;
      for (int r2 = 0; r2 < n; ++r2) s = fma(lw[r2], sL[x * P + line_node<n>(d, r2, pp, qq)], s);
      const int code = elem_face[e * 6 + f];
      const int fid = dg_idx(code >> 4, b.F, kSiteAdjFace);
      if (code & 8) {
        b.fseed[((size_t)fid * 2 * 5 + x) * NN + pq] = -s;
      } else {
        int p2, q2;
        apply_flip<n>(code & 7, pp, qq, p2, q2);
        b.fseed[(((size_t)fid * 2 + 1) * 5 + x) * NN + p2 + n * q2] = s;
      }
    }
  }
  smu[threadIdx.x] = mub;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int t = 0; t < S::THREADS; ++t) acc += smu[t];
    b.mupart[blockIdx.x] = acc;
  }
}

// B3: per node, the gradients' adjoint (the volume's, plus the transposed
// prolongation of the face VJP's gf-adjoints, l_s(r) each), divided by J ->
// gtil; then per face point of the element's faces the lifting's surface sum
// S_f(pq) = sum_r l_s(r)/w_r (n sJ) . gtil(line r), per lifting variable.
template <int N>
__global__ void __launch_bounds__(Shape<N>::THREADS)
k_adjlg_gather(const double* __restrict__ metrics, const double* __restrict__ facegeo,
               const int* __restrict__ elem_face, const double* __restrict__ tab, int E, AdjBufs b,
               double* __restrict__ lgf) {
  using S = Shape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN;
  extern __shared__ double adjlg_smem[];
  __shared__ double sT[4 * n];   // l(-1)/w, l(+1)/w, l(-1), l(+1)
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  const int e = blockIdx.x * S::EPB + le;
  const bool active = e < E;
  double* sG = adjlg_smem + (size_t)le * 12 * P;   // gtil [12][P]
  for (int t = threadIdx.x; t < 4 * n; t += blockDim.x) sT[t] = tab[GaussTab::lmw(n) + t];
  __syncthreads();
  if (active) {
    const int i = id % n, j = (id / n) % n, k = id / NN;
    const int ijk[3] = {i, j, k};
    double gb[12];
#pragma unroll
    for (int r = 0; r < 12; ++r) gb[r] = b.gbar[((size_t)e * 12 + r) * P + id];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int pp = d == 0 ? j : i, qq = d == 2 ? j : k;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int code = elem_face[e * 6 + 2 * d + s];
        const int fid = dg_idx(code >> 4, b.F, kSiteAdjFace);
        int pm = pp, qm = qq, side = 0;
        if (!(code & 8)) { apply_flip<n>(code & 7, pp, qq, pm, qm); side = 1; }
        const double c = sT[(2 + s) * n + ijk[d]];
        const double* src = b.face + (((size_t)fid * 2 + side) * 17 + 5) * NN + pm + n * qm;
#pragma unroll
        for (int r = 0; r < 12; ++r) gb[r] = fma(c, src[r * NN], gb[r]);
      }
    }
    const double iJ = metrics[((size_t)e * 10 + 9) * P + id];
#pragma unroll
    for (int r = 0; r < 12; ++r) {
      const double gt = gb[r] * iJ;
      b.gtil[((size_t)e * 12 + r) * P + id] = gt;
      sG[r * P + id] = gt;
    }
  }
  __syncthreads();
  if (!active) return;
  for (int o = id; o < 24 * NN; o += P) {
    const int f = o / (4 * NN), rr = o - f * 4 * NN, ph = rr / NN, pq = rr - ph * NN;
    const int pp = pq % n, qq = pq / n, d = f >> 1;
    const int code = elem_face[e * 6 + f];
    const int fid = dg_idx(code >> 4, b.F, kSiteAdjFace);
    const bool master = code & 8;
    int p2 = pp, q2 = qq;
    if (!master) apply_flip<n>(code & 7, pp, qq, p2, q2);
    const double* fg = facegeo + (size_t)fid * 4 * NN + p2 + n * q2;
    const double sJ = master ? fg[3 * NN] : -fg[3 * NN];
    const double n0 = sJ * fg[0], n1 = sJ * fg[NN], n2 = sJ * fg[2 * NN];
    const double* lw = sT + (f & 1) * n;
    double s = 0.0;
    for (int r2 = 0; r2 < n; ++r2) {
      const int node = line_node<n>(d, r2, pp, qq);
      s = fma(lw[r2], n0 * sG[(ph * 3) * P + node] + n1 * sG[(ph * 3 + 1) * P + node] + n2 * sG[(ph * 3 + 2) * P + node], s);
    }
    lgf[(((size_t)e * 6 + f) * 9 + ph) * NN + pq] = s;
  }
}

// B4: per element face point, the adjoint of the face values Uf: the face
// VJP's share plus that of the face average phi* in the own and the
// neighbour's lifting, (S_own + S_nbr)/2, through the lifting variables.
// A mortar side (negative neighbour entry) takes, in place of the neighbour's
// half, its term from b.mx (k_adj_mortar_lift in FACE mode).
template <int N>
__global__ void __launch_bounds__(128)
k_adjlg_facephi(const double* __restrict__ Uf, const int* __restrict__ elem_face, const int* __restrict__ elem_nbr,
                int E, Gas g, AdjBufs b, double* __restrict__ lgf, int n_mortar) {
  constexpr int n = N + 1, NN = n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)E * 6 * NN) return;
  const int ef = (int)(gid / NN), pq = (int)(gid % NN);
  const int e = ef / 6, f = ef - 6 * e, pp = pq % n, qq = pq / n;
  const int code = elem_face[e * 6 + f], nb = elem_nbr[e * 6 + f];
  const int fid = dg_idx(code >> 4, b.F, kSiteAdjFace);
  int p2, q2;
  apply_flip<n>(code & 7, pp, qq, p2, q2);
  const double* So = lgf + (size_t)ef * 9 * NN + pq;
  double phb[4];
  if (nb < 0) {
    const double* xm = b.mx + (size_t)dg_idx(-1 - nb, 5L * n_mortar, kSiteMortar) * 4 * NN + pq;
#pragma unroll
    for (int ph = 0; ph < 4; ++ph) phb[ph] = 0.5 * So[ph * NN] + xm[ph * NN];
  } else {
    const int e2 = dg_idx(nb >> 3, E, kSiteAdjFace), f2 = nb & 7;
    const double* Sn = lgf + ((size_t)e2 * 6 + f2) * 9 * NN + p2 + n * q2;
#pragma unroll
    for (int ph = 0; ph < 4; ++ph) phb[ph] = 0.5 * (So[ph * NN] + Sn[ph * NN]);
  }
  const bool master = code & 8;
  const double* fa = b.face + ((size_t)fid * 2 + (master ? 0 : 1)) * 17 * NN + (master ? pq : p2 + n * q2);
  double q[5], qb[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    q[v] = Uf[(size_t)ef * 5 * NN + (size_t)v * NN + pq];
    qb[v] = fa[v * NN];
  }
  const double ir = 1.0 / q[0];
  const double u = q[1] * ir, v = q[2] * ir, w = q[3] * ir;
  const double T = g.gm1 * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w)) * ir * g.inv_R;
  const double ub[3] = {phb[0], phb[1], phb[2]};
  prim_vjp(q, -phb[3] * T * ir, ub, phb[3] * ir * g.inv_R, g.gm1, qb);
  double* out = lgf + ((size_t)ef * 9 + 4) * NN + pq;
#pragma unroll
  for (int x = 0; x < 5; ++x) out[x * NN] = qb[x];
}

// B5: per node, the lifting's volume transpose
//   phi-bar_a(m) = - sum_d sum_l Ja^d_l(m) sum_r Dw[r][m] gtil_{a,l}(line r),
// through the lifting variables to the state, plus the transposed
// prolongation of the face values' adjoint (l_s(r) each) and the volume's qbar.
template <int N>
__global__ void __launch_bounds__(Shape<N>::THREADS)
k_adjlg_lift(const double* __restrict__ U, const double* __restrict__ metrics, const double* __restrict__ tab,
             int E, Gas g, AdjBufs b, const double* __restrict__ lgf, double* __restrict__ out) {
  using S = Shape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN;
  extern __shared__ double adjlg_smem[];
  __shared__ double sDw[n * n], sL[2 * n];   // weak D; l(-1), l(+1)
  const int le = threadIdx.x / P, id = threadIdx.x - le * P;
  const int e = blockIdx.x * S::EPB + le;
  const bool active = e < E;
  double* sG = adjlg_smem + (size_t)le * 12 * P;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sDw[t] = tab[GaussTab::Dw(n) + t];
  for (int t = threadIdx.x; t < 2 * n; t += blockDim.x) sL[t] = tab[GaussTab::lm(n) + t];
  if (active)
#pragma unroll
    for (int r = 0; r < 12; ++r) sG[r * P + id] = b.gtil[((size_t)e * 12 + r) * P + id];
  __syncthreads();
  if (!active) return;
  const int i = id % n, j = (id / n) % n, k = id / NN;
  const int ijk[3] = {i, j, k};
  double Ja[9];
#pragma unroll
  for (int r = 0; r < 9; ++r) Ja[r] = metrics[((size_t)e * 10 + r) * P + id];
  double phib[4] = {0, 0, 0, 0};
  double qb[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) qb[c] = b.qbar[((size_t)e * 5 + c) * P + id];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int r = ijk[d];
    const int stride = d == 0 ? 1 : (d == 1 ? n : NN);
    const int line0 = id - r * stride;
    double W[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int r2 = 0; r2 < n; ++r2) {
      const double c = sDw[r2 * n + r];
      const int nid = line0 + r2 * stride;
#pragma unroll
      for (int x = 0; x < 12; ++x) W[x] = fma(c, sG[x * P + nid], W[x]);
    }
#pragma unroll
    for (int ph = 0; ph < 4; ++ph)
      phib[ph] -= Ja[d * 3] * W[ph * 3] + Ja[d * 3 + 1] * W[ph * 3 + 1] + Ja[d * 3 + 2] * W[ph * 3 + 2];
    const int pq = d == 0 ? j + n * k : (d == 1 ? i + n * k : i + n * j);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const double c = sL[s * n + r];
      const double* src = lgf + (((size_t)e * 6 + 2 * d + s) * 9 + 4) * NN + pq;
#pragma unroll
      for (int x = 0; x < 5; ++x) qb[x] = fma(c, src[x * NN], qb[x]);
    }
  }
  double q[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) q[c] = U[((size_t)e * 5 + c) * P + id];
  const double ir = 1.0 / q[0];
  const double u = q[1] * ir, v = q[2] * ir, w = q[3] * ir;
  const double T = g.gm1 * (q[4] - 0.5 * (q[1] * u + q[2] * v + q[3] * w)) * ir * g.inv_R;
  const double ub[3] = {phib[0], phib[1], phib[2]};
  prim_vjp(q, -phib[3] * T * ir, ub, phib[3] * ir * g.inv_R, g.gm1, qb);
#pragma unroll
  for (int c = 0; c < 5; ++c) out[((size_t)e * 5 + c) * P + id] = qb[c];
}

// d/dmu: fold the block partials in a fixed order and add to *acc.
__global__ void k_adj_mu_fold(const double* __restrict__ part, int n, double scale, double* __restrict__ acc) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += 256) s += part[t];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) acc[0] += scale * sh[0];
}

// Elementwise: y = a*y + b*x  (a, b host scalars)
__global__ void k_axpby(double* y, const double* x, double a, double b, size_t len) {
  // a == 0 overwrites y (whatever it held, including NaN)
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (size_t)gridDim.x * blockDim.x)
    y[t] = (a == 0.0 ? 0.0 : a * y[t]) + b * x[t];
}

template <int N>
static size_t adj_volume_smem() {
  using S = Shape<N>;
  return sizeof(double) * (((2 * S::n * S::n + 1) & ~1) + (size_t)S::EPB * kAdjVolWords * S::P);
}

template <int N>
static size_t adj_lift_smem() {
  using S = Shape<N>;
  return sizeof(double) * (((S::n * S::n + 1) & ~1) + (size_t)S::EPB * 12 * S::P);
}

template <int N>
static cudaError_t adj_setup_N() {
  cudaError_t e = cudaFuncSetAttribute(k_adj_volume<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)adj_volume_smem<N>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_lift<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adj_lift_smem<N>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_lift<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)adj_lift_smem<N>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_mortar_face<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)adj_mortar_face_smem<N>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_mortar_face<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)adj_mortar_face_smem<N>());
  using S = Shape<N>;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adjlg_volume<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * S::EPB * 5 * S::P));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adjlg_gather<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * S::EPB * 12 * S::P));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adjlg_lift<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * S::EPB * 12 * S::P));
  return e;
}

cudaError_t setup_adjoint(int N) {
  switch (N) {
    case 1: return adj_setup_N<1>();
    case 2: return adj_setup_N<2>();
    case 3: return adj_setup_N<3>();
    case 4: return adj_setup_N<4>();
    case 5: return adj_setup_N<5>();
    case 6: return adj_setup_N<6>();
    case 7: return adj_setup_N<7>();
    case 8: return adj_setup_N<8>();
    case 9: return adj_setup_N<9>();
    default: return cudaErrorInvalidValue;
  }
}

// number of d/dmu partials one VJP writes
int adjoint_mu_partials(const Ctx& c) {
  const int epb = default_epb(c.P);
  return (c.E + epb - 1) / epb + (int)(((long)c.nfaces_conf * c.NN + 127) / 128) + c.M;
}

template <int N>
static cudaError_t vjp_N(const Ctx& c, const double* U, const double* lam, double* out, const AdjBufs& b,
                         double* dJdmu, double mu_scale, cudaStream_t s) {
  using S = Shape<N>;
  constexpr int NN = (N + 1) * (N + 1);
  const int blocks = (c.E + S::EPB - 1) / S::EPB;
  const double inv_w0 = 1.0 / c.w[0];
  const double* grad = (const double*)c.d_grad;
  k_adj_volume<N><<<blocks, S::THREADS, adj_volume_smem<N>(), s>>>(U, lam, c.d_metrics, grad, c.d_elem_face, c.d_D,
                                                                   c.E, c.gas, inv_w0, b);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const long tot = (long)c.nfaces_conf * NN;   // the conforming faces; the mortars' slots follow
  const int fblocks = (int)((tot + 127) / 128);
  if (fblocks > 0)
    k_adj_face<N><<<fblocks, 128, 0, s>>>(U, grad, c.d_faces, c.d_facegeo, c.nfaces_conf, c.E, c.gas, b, blocks);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (c.M > 0) {
    k_adj_mortar_face<N><<<c.M, MortarShape<N>::THREADS, adj_mortar_face_smem<N>(), s>>>(
        U, grad, c.d_facegeo, c.d_mortars, c.d_mortar_tab, c.E, c.gas, b, blocks + fblocks);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const long nodes = (long)c.E * c.P;
  k_adj_gather<N><<<(int)((nodes + 127) / 128), 128, 0, s>>>(c.d_metrics, c.d_elem_face, c.E, b);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (c.M > 0) {
    k_adj_mortar_lift<N><<<c.M, MortarShape<N>::THREADS, 0, s>>>(c.d_metrics, c.d_mortars, c.d_mortar_tab, c.E,
                                                                 inv_w0, b, nullptr);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    k_adj_lift<N, true><<<blocks, S::THREADS, adj_lift_smem<N>(), s>>>(U, c.d_metrics, c.d_elem_nbr, c.d_elem_face,
                                                                       c.d_D, c.E, c.gas, inv_w0, b, out, c.M);
  } else {
    k_adj_lift<N><<<blocks, S::THREADS, adj_lift_smem<N>(), s>>>(U, c.d_metrics, c.d_elem_nbr, c.d_elem_face, c.d_D,
                                                                 c.E, c.gas, inv_w0, b, out, 0);
  }
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (dJdmu) {
    k_adj_mu_fold<<<1, 256, 0, s>>>(b.mupart, blocks + fblocks + c.M, mu_scale, dJdmu);
    err = cudaGetLastError();
  }
  return err;
}

// Gauss nodes (conforming meshes): B1, A2 on the face values, B3, B4, B5.
template <int N>
static cudaError_t vjp_lg_N(const Ctx& c, const double* U, const double* lam, double* out, const AdjBufs& b,
                            double* dJdmu, double mu_scale, cudaStream_t s) {
  using S = Shape<N>;
  constexpr int NN = (N + 1) * (N + 1);
  const int blocks = (c.E + S::EPB - 1) / S::EPB;
  const size_t sm5 = sizeof(double) * S::EPB * 5 * S::P, sm12 = sizeof(double) * S::EPB * 12 * S::P;
  k_adjlg_volume<N><<<blocks, S::THREADS, sm5, s>>>(U, lam, c.d_metrics, (const double*)c.d_grad, c.d_elem_face,
                                                    c.d_lgb, c.E, c.gas, b);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int fblocks = (int)(((long)c.nfaces_conf * NN + 127) / 128);
  if (fblocks > 0)
    k_adj_face<N, true><<<fblocks, 128, 0, s>>>(c.d_Uf, (const double*)c.d_gf, c.d_faces, c.d_facegeo,
                                                c.nfaces_conf, c.E, c.gas, b, blocks);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (c.M > 0) {
    k_adj_mortar_face<N, true><<<c.M, MortarShape<N>::THREADS, adj_mortar_face_smem<N>(), s>>>(
        c.d_Uf, (const double*)c.d_gf, c.d_facegeo, c.d_mortars, c.d_mortar_tab, c.E, c.gas, b, blocks + fblocks);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  k_adjlg_gather<N><<<blocks, S::THREADS, sm12, s>>>(c.d_metrics, c.d_facegeo, c.d_elem_face, c.d_lgb, c.E, b,
                                                     c.d_adj_lgf);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (c.M > 0) {
    k_adj_mortar_lift<N, true><<<c.M, MortarShape<N>::THREADS, 0, s>>>(c.d_metrics, c.d_mortars, c.d_mortar_tab,
                                                                       c.E, 0.0, b, c.d_adj_lgf);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const long fp = (long)c.E * 6 * NN;
  k_adjlg_facephi<N><<<(int)((fp + 127) / 128), 128, 0, s>>>(c.d_Uf, c.d_elem_face, c.d_elem_nbr, c.E, c.gas, b,
                                                             c.d_adj_lgf, c.M);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  k_adjlg_lift<N><<<blocks, S::THREADS, sm12, s>>>(U, c.d_metrics, c.d_lgb, c.E, c.gas, b, c.d_adj_lgf, out);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  if (dJdmu) {
    k_adj_mu_fold<<<1, 256, 0, s>>>(b.mupart, blocks + fblocks + c.M, mu_scale, dJdmu);
    err = cudaGetLastError();
  }
  return err;
}

cudaError_t launch_vjp(const Ctx& c, const double* U, const double* lam, double* out, double* dJdmu,
                       double mu_scale, cudaStream_t s) {
  // forward recomputation of the FP64 lifted gradients at U
  cudaError_t err = launch_lift_fp64(c, U, s);
  if (err != cudaSuccess) return err;
  AdjBufs b{c.d_adj_qbar, c.d_adj_gbar, c.d_adj_fseed, c.d_adj_face, c.d_adj_gtil, c.d_adj_mu, 0, c.d_adj_mx,
            c.nfaces};
  if (c.prm.nodes == DG_NODES_LG) {
    switch (c.N) {
      case 1: return vjp_lg_N<1>(c, U, lam, out, b, dJdmu, mu_scale, s);
      case 2: return vjp_lg_N<2>(c, U, lam, out, b, dJdmu, mu_scale, s);
      case 3: return vjp_lg_N<3>(c, U, lam, out, b, dJdmu, mu_scale, s);
      case 4: return vjp_lg_N<4>(c, U, lam, out, b, dJdmu, mu_scale, s);
      case 5: return vjp_lg_N<5>(c, U, lam, out, b, dJdmu, mu_scale, s);
      case 6: return vjp_lg_N<6>(c, U, lam, out, b, dJdmu, mu_scale, s);
      case 7: return vjp_lg_N<7>(c, U, lam, out, b, dJdmu, mu_scale, s);
      case 8: return vjp_lg_N<8>(c, U, lam, out, b, dJdmu, mu_scale, s);
      case 9: return vjp_lg_N<9>(c, U, lam, out, b, dJdmu, mu_scale, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (c.N) {
    case 1: return vjp_N<1>(c, U, lam, out, b, dJdmu, mu_scale, s);
    case 2: return vjp_N<2>(c, U, lam, out, b, dJdmu, mu_scale, s);
    case 3: return vjp_N<3>(c, U, lam, out, b, dJdmu, mu_scale, s);
    case 4: return vjp_N<4>(c, U, lam, out, b, dJdmu, mu_scale, s);
    case 5: return vjp_N<5>(c, U, lam, out, b, dJdmu, mu_scale, s);
    case 6: return vjp_N<6>(c, U, lam, out, b, dJdmu, mu_scale, s);
    case 7: return vjp_N<7>(c, U, lam, out, b, dJdmu, mu_scale, s);
    case 8: return vjp_N<8>(c, U, lam, out, b, dJdmu, mu_scale, s);
    case 9: return vjp_N<9>(c, U, lam, out, b, dJdmu, mu_scale, s);
    default: return cudaErrorInvalidValue;
  }
}

// Objective J = sum_nodes w_i w_j w_k J 1/2 rho |u|^2 (volume-integrated kinetic
// energy) and, optionally, dJ/dU.  Block partials into part[], folded later.
template <int N>
__global__ void __launch_bounds__(256)
k_kinetic(const double* __restrict__ U, const double* __restrict__ Jac, const double* __restrict__ w,
          double* __restrict__ grad, double* __restrict__ part, int E) {
  constexpr int n = N + 1, P = n * n * n;
  __shared__ double sh[8];
  double acc = 0.0;
  const long total = (long)E * P;
  for (long t = (long)blockIdx.x * 256 + threadIdx.x; t < total; t += (long)gridDim.x * 256) {
    const int e = (int)(t / P), id = (int)(t % P);
    const int i = id % n, j = (id / n) % n, k = id / (n * n);
    const double wq = w[i] * w[j] * w[k] * Jac[t];
    const double* q = U + (size_t)e * 5 * P + id;
    const double ir = 1.0 / q[0];
    const double u = q[P] * ir, v = q[2 * P] * ir, ww = q[3 * P] * ir;
    const double k2 = 0.5 * (u * u + v * v + ww * ww);
    acc += wq * q[0] * k2;
    if (grad) {
      double* gp = grad + (size_t)e * 5 * P + id;
      gp[0] = -wq * k2;
      gp[P] = wq * u;
      gp[2 * P] = wq * v;
      gp[3 * P] = wq * ww;
      gp[4 * P] = 0.0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int a = 0; a < 8; ++a) s2 += sh[a];
    part[blockIdx.x] = s2;
  }
}

cudaError_t launch_kinetic(const Ctx& c, const double* U, double* grad, double* d_out, cudaStream_t s) {
  const long total = (long)c.E * c.P;
  const int blocks = (int)std::min<long>((total + 255) / 256, c.red_len);
  cudaError_t err;
  switch (c.N) {
    case 1: k_kinetic<1><<<blocks, 256, 0, s>>>(U, c.d_J, c.d_w, grad, c.d_red, c.E); break;
    case 2: k_kinetic<2><<<blocks, 256, 0, s>>>(U, c.d_J, c.d_w, grad, c.d_red, c.E); break;
    case 3: k_kinetic<3><<<blocks, 256, 0, s>>>(U, c.d_J, c.d_w, grad, c.d_red, c.E); break;
    case 4: k_kinetic<4><<<blocks, 256, 0, s>>>(U, c.d_J, c.d_w, grad, c.d_red, c.E); break;
    case 5: k_kinetic<5><<<blocks, 256, 0, s>>>(U, c.d_J, c.d_w, grad, c.d_red, c.E); break;
    case 6: k_kinetic<6><<<blocks, 256, 0, s>>>(U, c.d_J, c.d_w, grad, c.d_red, c.E); break;
    case 7: k_kinetic<7><<<blocks, 256, 0, s>>>(U, c.d_J, c.d_w, grad, c.d_red, c.E); break;
    case 8: k_kinetic<8><<<blocks, 256, 0, s>>>(U, c.d_J, c.d_w, grad, c.d_red, c.E); break;
    case 9: k_kinetic<9><<<blocks, 256, 0, s>>>(U, c.d_J, c.d_w, grad, c.d_red, c.E); break;
    default: return cudaErrorInvalidValue;
  }
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  cudaMemsetAsync(d_out, 0, sizeof(double), s);
  k_adj_mu_fold<<<1, 256, 0, s>>>(c.d_red, blocks, 1.0, d_out);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double* y, const double* x, double a, double b, size_t len, cudaStream_t s) {
  const size_t blocks = std::min<size_t>((len + 255) / 256, 152 * 16);
  k_axpby<<<(unsigned)blocks, 256, 0, s>>>(y, x, a, b, len);
  return cudaGetLastError();
}

// Host reader of this file's bounds-check error word (0 in normal builds).
DG_BOUNDS_READER(bounds_word_adjoint)

}  // namespace dg
