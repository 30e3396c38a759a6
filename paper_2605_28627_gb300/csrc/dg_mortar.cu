// Mortars (GALAEXI Sec. 3.2.2, Algorithm 1; Kopriva 1996): a big face split
// into four quadrants k = a + 2 b that are faces of four small elements.
//
// Data of the big face go to the nodes of each quadrant (numbered (pp, qq)
// along the big face's directions) by interpolation,
//   v_k(pp, qq) = sum_ij I_a[pp][i] I_b[qq][j] v(i, j),  I_h[x][j] = l_j((x_x + 2h - 1)/2),
// and quadrant data come back onto the big face by the projection with the
// LGL quadrature, which keeps face integrals:
//   v(i, j) = scale / (w_i w_j) sum_k sum_{pp,qq} w_pp w_qq I_a[pp][i] I_b[qq][j] v_k(pp, qq),
// scale = 1/4 for point values, 1 for fluxes times sJ.
//
// k_mortar_lift (before the lifting kernel): the lifting's neighbour state of
//   every mortar side, stored as a conservative state in the side's own
//   face-node order: on a quadrant, the big face's interpolated lifting
//   variables (u, v, w, T); on the big face, the one whose average with the
//   big side's values is the projection of the quadrants' averages.
// k_mortar_flux (after the lifting): the Riemann and viscous fluxes on the
//   quadrants from the small side's state and gradients and the big side's
//   interpolated ones, with the small face's geometry, and on the big face
//   their projection, pointing out of the big element.
// On Legendre-Gauss nodes (FACE) the same maps act on the face values of the
// state and of the lifted gradients at the Gauss face points (Uf, gf), and the
// projection with the Gauss weights is the L2 projection.
// One block per mortar, a thread per quadrant node.  With the FP32 operator
// (R = float) the gradients, face geometry and fluxes are FP32 as in the
// conforming face kernel; the states stay FP64 and the maps run in FP64.
#include "dg_mortar.cuh"

namespace dg {

// Q: the type of the state or face values read (FP32 face values with the FP32
// operator on Gauss nodes).
template <int N, bool FACE, typename Q = double>
__global__ void __launch_bounds__(MortarShape<N>::THREADS)
k_mortar_lift(const Q* __restrict__ U, const int* __restrict__ mortars, const double* __restrict__ tab,
              double* __restrict__ virt, int E, Gas g) {
  using S = MortarShape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN, T = S::THREADS;
  __shared__ double sI[2 * NN], sIT[2 * NN], sW[2 * NN], sw[n];
  __shared__ double buf[44 * NN];
  double* sB = buf;                 // [4][NN]  lifting variables at the big face's nodes
  double* sT = buf + 4 * NN;        // [2][4][NN] first interpolation sweep
  double* sS = buf + 12 * NN;       // [4][4][NN] face averages on the quadrants, big-face order
  double* sP = buf + 28 * NN;       // [4][4][NN] first projection sweep
  const int m = blockIdx.x, t = threadIdx.x;
  const int* r = mortars + (size_t)m * 20;
  const int eB = dg_idx(r[0], E, kSiteMortar), fB = r[1];
  mortar_tables<n>(tab, sI, sIT, sW, sw, t, T);
  if (t < NN) {
    double ph[4];
    int st;
    const Q* q = side_ptr<n, FACE, 5>(U, eB, fB, t % n, t / n, st);
    lift_vars(q, st, g, ph, sizeof(Q) == 4 ? g.E_ref : 0.0);
#pragma unroll
    for (int a = 0; a < 4; ++a) sB[a * NN + t] = ph[a];
  }
  __syncthreads();
  mortar_sweep1<n, 4>(sIT, sB, sT, t, T);
  __syncthreads();
  const int k = t / NN, pq = t % NN, pp = pq % n, qq = pq / n;
  {
    double ib[4];
    mortar_sweep2<n, 4>(sI, sT, k, pp, qq, ib);
    const int es = dg_idx(r[3 + 4 * k], E, kSiteMortar), fs = r[4 + 4 * k], fl = r[5 + 4 * k];
    int p2, q2;
    apply_flip<n>(fl, pp, qq, p2, q2);
    double ps[4];
    int st;
    const Q* q = side_ptr<n, FACE, 5>(U, es, fs, p2, q2, st);
    lift_vars(q, st, g, ps, sizeof(Q) == 4 ? g.E_ref : 0.0);
#pragma unroll
    for (int a = 0; a < 4; ++a) sS[(k * 4 + a) * NN + pq] = 0.5 * (ps[a] + ib[a]);
    encode_vars(ib, g, virt + (size_t)(5 * m + k) * 5 * NN + p2 + n * q2, NN);
  }
  __syncthreads();
  mortar_proj1<n, 4>(sW, sS, sP, t, T);
  __syncthreads();
  if (t < NN) {
    const int i = t % n, j = t / n;
    const double sc = 0.25 / (sw[i] * sw[j]);
    double ph[4];
#pragma unroll
    for (int x = 0; x < 4; ++x)   // average with the big side's values = the projection
      ph[x] = 2.0 * (mortar_proj2<n, 4>(sW, sP, x, i, j) * sc) - sB[x * NN + t];
    encode_vars(ph, g, virt + (size_t)(5 * m + 4) * 5 * NN + t, NN);
  }
}

template <int N, typename R, bool FACE, typename Q = double>
__global__ void __launch_bounds__(MortarShape<N>::THREADS)
k_mortar_flux(const Q* __restrict__ U, const R* __restrict__ grad, const R* __restrict__ facegeo,
              const int* __restrict__ mortars, const double* __restrict__ tab, R* __restrict__ fstar, int E, int F,
              Gas g) {
  using S = MortarShape<N>;
  constexpr int n = S::n, P = S::P, NN = S::NN, T = S::THREADS;
  __shared__ double sI[2 * NN], sIT[2 * NN], sW[2 * NN], sw[n];
  __shared__ double buf[51 * NN];
  double* sB = buf;                 // [17][NN] the big face's state and gradients
  double* sT = buf + 17 * NN;       // [2][17][NN] first interpolation sweep
  double* sF = buf;                 // [4][5][NN] quadrant fluxes, big-face order (after the sweeps)
  double* sP = buf + 20 * NN;       // [4][5][NN] first projection sweep
  const int m = blockIdx.x, t = threadIdx.x;
  const int* r = mortars + (size_t)m * 20;
  const int eB = dg_idx(r[0], E, kSiteMortar), fB = r[1], slotB = dg_idx(r[2], F, kSiteMortar);
  mortar_tables<n>(tab, sI, sIT, sW, sw, t, T);
  if (t < NN) {
    int su, sg;
    const Q* qb = side_ptr<n, FACE, 5>(U, eB, fB, t % n, t / n, su);
    const R* gb = side_ptr<n, FACE, 12>(grad, eB, fB, t % n, t / n, sg);
#pragma unroll
    for (int v = 0; v < 5; ++v) sB[v * NN + t] = (double)qb[v * su];
    if (sizeof(Q) == 4) sB[4 * NN + t] += g.E_ref;   // FP32 face values carry E - E_ref
#pragma unroll
    for (int x = 0; x < 12; ++x) sB[(5 + x) * NN + t] = (double)gb[x * sg];
  }
  __syncthreads();
  mortar_sweep1<n, 17>(sIT, sB, sT, t, T);
  __syncthreads();
  const int k = t / NN, pq = t % NN, pp = pq % n, qq = pq / n;
  double qR[17];
  mortar_sweep2<n, 17>(sI, sT, k, pp, qq, qR);
  __syncthreads();   // sT is read; its space takes the fluxes
  {
    const int es = dg_idx(r[3 + 4 * k], E, kSiteMortar), fs = r[4 + 4 * k], fl = r[5 + 4 * k];
    const int slot = dg_idx(r[6 + 4 * k], F, kSiteMortar);
    int p2, q2;
    apply_flip<n>(fl, pp, qq, p2, q2);
    const int o = p2 + n * q2;
    int su, sg;
    const Q* qs = side_ptr<n, FACE, 5>(U, es, fs, p2, q2, su);
    const R* gs = side_ptr<n, FACE, 12>(grad, es, fs, p2, q2, sg);
    double dL[5];
    R gL[12], gR[12];
#pragma unroll
    for (int v = 0; v < 5; ++v) dL[v] = (double)qs[v * su];
    if (sizeof(Q) == 4) dL[4] += g.E_ref;
#pragma unroll
    for (int x = 0; x < 12; ++x) {
      gL[x] = gs[x * sg];
      gR[x] = (R)qR[5 + x];
    }
    const R* fg = facegeo + (size_t)slot * 4 * NN + o;
    R Fq[5];
    face_flux_core<R>(dL, qR, gL, gR, fg[0], fg[NN], fg[2 * NN], fg[3 * NN], g, Fq, 1);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      sF[(k * 5 + v) * NN + pq] = (double)Fq[v];
      fstar[((size_t)slot * 5 + v) * NN + o] = Fq[v];
    }
  }
  __syncthreads();
  mortar_proj1<n, 5>(sW, sF, sP, t, T);
  __syncthreads();
  for (int o = t; o < 5 * NN; o += T) {   // out of the big element
    const int v = o / NN, ij = o - v * NN, i = ij % n, j = ij / n;
    fstar[((size_t)slotB * 5 + v) * NN + ij] = (R)(mortar_proj2<n, 5>(sW, sP, v, i, j) * (-1.0 / (sw[i] * sw[j])));
  }
}

template <int N>
static cudaError_t mortar_lift_N(const Ctx& c, const double* U, cudaStream_t s) {
  if (c.prm.nodes == DG_NODES_LG && c.prm.precision == DG_FP32OP)
    k_mortar_lift<N, true, float><<<c.M, MortarShape<N>::THREADS, 0, s>>>(
        reinterpret_cast<const float*>(c.d_Uf), c.d_mortars, c.d_mortar_tab, c.d_mortar_virt, c.E, c.gas);
  else if (c.prm.nodes == DG_NODES_LG)
    k_mortar_lift<N, true><<<c.M, MortarShape<N>::THREADS, 0, s>>>(c.d_Uf, c.d_mortars, c.d_mortar_tab,
                                                                   c.d_mortar_virt, c.E, c.gas);
  else
    k_mortar_lift<N, false><<<c.M, MortarShape<N>::THREADS, 0, s>>>(U, c.d_mortars, c.d_mortar_tab,
                                                                    c.d_mortar_virt, c.E, c.gas);
  return cudaGetLastError();
}

template <int N>
static cudaError_t mortar_flux_N(const Ctx& c, const double* U, cudaStream_t s) {
  constexpr int T = MortarShape<N>::THREADS;
  if (c.prm.nodes == DG_NODES_LG && c.prm.precision == DG_FP32OP)   // FP32 face values
    k_mortar_flux<N, float, true, float><<<c.M, T, 0, s>>>(
        reinterpret_cast<const float*>(c.d_Uf), reinterpret_cast<const float*>(c.d_gf), c.d_facegeo_f, c.d_mortars,
        c.d_mortar_tab, (float*)c.d_fstar, c.E, c.nfaces, c.gas);
  else if (c.prm.nodes == DG_NODES_LG)   // the face values of the state and gradients
    k_mortar_flux<N, double, true><<<c.M, T, 0, s>>>(c.d_Uf, c.d_gf, c.d_facegeo, c.d_mortars, c.d_mortar_tab,
                                                     (double*)c.d_fstar, c.E, c.nfaces, c.gas);
  else if (c.prm.precision == DG_FP32OP)
    k_mortar_flux<N, float, false><<<c.M, T, 0, s>>>(U, (const float*)c.d_grad, c.d_facegeo_f, c.d_mortars,
                                                     c.d_mortar_tab, (float*)c.d_fstar, c.E, c.nfaces, c.gas);
  else
    k_mortar_flux<N, double, false><<<c.M, T, 0, s>>>(U, (const double*)c.d_grad, c.d_facegeo, c.d_mortars,
                                                      c.d_mortar_tab, (double*)c.d_fstar, c.E, c.nfaces, c.gas);
  return cudaGetLastError();
}

#define DG_MORTAR_DISPATCH(FN, ...)          \
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

cudaError_t launch_mortar_lift(const Ctx& c, const double* U, cudaStream_t s) {
  if (c.M == 0) return cudaSuccess;
  DG_MORTAR_DISPATCH(mortar_lift_N, c, U, s)
}

cudaError_t launch_mortar_flux(const Ctx& c, const double* U, cudaStream_t s) {
  if (c.M == 0) return cudaSuccess;
  DG_MORTAR_DISPATCH(mortar_flux_N, c, U, s)
}

// Host reader of this file's bounds-check error word (0 in normal builds).
DG_BOUNDS_READER(bounds_word_mortar)

}  // namespace dg
