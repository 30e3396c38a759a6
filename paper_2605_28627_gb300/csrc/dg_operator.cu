// Single-context launchers of the lifting and face-flux kernels (bodies in
// dg_stage.cuh): one thread per volume node (lifting) or face node (face flux).
#include "dg_stage.cuh"

namespace dg {

// The FP32 lifting is latency-bound: its register allocation must leave room
// for 48 warps per SM (three 512-thread blocks at N = 7, twelve at N = 3).
// MORTAR: mortar sides read their neighbour state from mvirt.
template <int N, typename R, bool MORTAR = false>
__global__ void __launch_bounds__(Shape<N>::THREADS,
                                  sizeof(R) == 4 && Shape<N>::THREADS < 1536 ? 1536 / Shape<N>::THREADS : 1)
k_lift(const double* __restrict__ U, const R* __restrict__ metrics, const int* __restrict__ elem_nbr,
       const int* __restrict__ elem_face, const double* __restrict__ Dg, R* __restrict__ grad, int E, Gas g,
       double inv_w0, const double* __restrict__ mvirt, int n_mortar) {
  lift_body<N, R, Shape<N>::EPB, MORTAR>(U, metrics, elem_nbr, elem_face, Dg, grad, E, g, inv_w0, blockIdx.x,
                                         mvirt, n_mortar);
}

// FVSKIP: faces with an FV sub-cell element on either side are left to the FV
// face kernel (fv_mask: [E], 1 for an FV element).
template <int N, typename R, bool FVSKIP>
__global__ void __launch_bounds__(128)
k_face(const double* __restrict__ U, const R* __restrict__ grad, const FaceInfo* __restrict__ faces,
       const R* __restrict__ facegeo, R* __restrict__ fstar, int F, int E, Gas g, const int* __restrict__ fv_mask) {
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (FVSKIP) {
    constexpr int NN = (N + 1) * (N + 1);
    if (gid >= (long)F * NN) return;
    const FaceInfo fi = faces[gid / NN];
    if (fv_mask[dg_idx(fi.master >> 3, E, kSiteFaceElems)] || fv_mask[dg_idx(fi.slave >> 3, E, kSiteFaceElems)])
      return;
  }
  face_body<N, R>(U, grad, faces, facegeo, fstar, F, E, g, gid);
}

// ---------------------------------------------------------------------------
template <int N, typename R>
static cudaError_t lift_NR(const Ctx& c, const double* U, cudaStream_t s) {
  using S = Shape<N>;
  const int blocks = (c.E + S::EPB - 1) / S::EPB;
  const R* metrics = (const R*)(sizeof(R) == 8 ? (const void*)c.d_metrics : (const void*)c.d_metrics_f);
  if (c.M > 0) {   // the mortar sides' neighbour states first
    cudaError_t e = launch_mortar_lift(c, U, s);
    if (e != cudaSuccess) return e;
    k_lift<N, R, true><<<blocks, S::THREADS, lift_smem_bytes<N, R, S::EPB>(), s>>>(
        U, metrics, c.d_elem_nbr, c.d_elem_face, c.d_D, (R*)c.d_grad, c.E, c.gas, 1.0 / c.w[0], c.d_mortar_virt, c.M);
    return cudaGetLastError();
  }
  k_lift<N, R><<<blocks, S::THREADS, lift_smem_bytes<N, R, S::EPB>(), s>>>(
      U, metrics, c.d_elem_nbr, c.d_elem_face, c.d_D, (R*)c.d_grad, c.E, c.gas, 1.0 / c.w[0], nullptr, 0);
  return cudaGetLastError();
}

template <int N, typename R, bool FVSKIP>
static cudaError_t face_NR(const Ctx& c, const double* U, cudaStream_t s) {
  // the conforming faces (the mortars' slots follow them)
  const long tot = (long)c.nfaces_conf * (N + 1) * (N + 1);
  const int blocks = (int)((tot + 127) / 128);
  const R* fgeo = (const R*)(sizeof(R) == 8 ? (const void*)c.d_facegeo : (const void*)c.d_facegeo_f);
  if (blocks > 0)
    k_face<N, R, FVSKIP><<<blocks, 128, 0, s>>>(U, (const R*)c.d_grad, c.d_faces, fgeo, (R*)c.d_fstar, c.nfaces_conf,
                                                 c.E, c.gas, c.d_fv_mask);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && c.M > 0) e = launch_mortar_flux(c, U, s);
  return e;
}

template <int N>
static cudaError_t lift_N(const Ctx& c, const double* U, bool fp64, cudaStream_t s) {
  return fp64 ? lift_NR<N, double>(c, U, s) : lift_NR<N, float>(c, U, s);
}

template <int N>
static cudaError_t face_N(const Ctx& c, const double* U, cudaStream_t s) {
  if (c.prm.precision == DG_FP32OP) return face_NR<N, float, false>(c, U, s);
  return c.fv_on ? face_NR<N, double, true>(c, U, s) : face_NR<N, double, false>(c, U, s);
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
    case 8: return FN<8>(__VA_ARGS__);       \
    case 9: return FN<9>(__VA_ARGS__);       \
    default: return cudaErrorInvalidValue;   \
  }

// On Gauss nodes the lifting launcher also computes the face values of U
// first (k_prolong_lg), and the face kernel works on face values.
cudaError_t launch_lift(const Ctx& c, const double* U, cudaStream_t s, bool latency_ok) {
  if (c.prm.nodes == DG_NODES_LG) return launch_lift_lg(c, U, s);
  if (latency_ok && use_latency_kernels(c)) return launch_lift_lat(c, U, s);
  DG_DISPATCH(lift_N, c, U, c.prm.precision != DG_FP32OP, s)
}
cudaError_t launch_lift_fp64(const Ctx& c, const double* U, cudaStream_t s) {
  if (c.prm.nodes == DG_NODES_LG) return launch_lift_lg(c, U, s, true);
  if (use_latency_kernels(c)) return launch_lift_lat(c, U, s);
  DG_DISPATCH(lift_N, c, U, true, s)
}
cudaError_t launch_face(const Ctx& c, const double* U, cudaStream_t s, bool latency_ok) {
  if (c.prm.nodes == DG_NODES_LG) return launch_face_lg(c, s);
  if (latency_ok && use_latency_kernels(c) && c.prm.surf_flux == DG_FLUX_LLF) return launch_face_lat(c, U, s);
  DG_DISPATCH(face_N, c, U, s)
}
template <int N>
static cudaError_t setup_lift_N() {
  cudaError_t e = cudaFuncSetAttribute(k_lift<N, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)lift_smem_bytes<N, double, Shape<N>::EPB>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lift<N, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lift_smem_bytes<N, double, Shape<N>::EPB>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lift<N, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lift_smem_bytes<N, float, Shape<N>::EPB>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_lift<N, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lift_smem_bytes<N, float, Shape<N>::EPB>());
  return e;
}

cudaError_t setup_kernels(int N) {
  cudaError_t e;
  switch (N) {
    case 1: e = setup_lift_N<1>(); break;
    case 2: e = setup_lift_N<2>(); break;
    case 3: e = setup_lift_N<3>(); break;
    case 4: e = setup_lift_N<4>(); break;
    case 5: e = setup_lift_N<5>(); break;
    case 6: e = setup_lift_N<6>(); break;
    case 7: e = setup_lift_N<7>(); break;
    case 8: e = setup_lift_N<8>(); break;
    case 9: e = setup_lift_N<9>(); break;
    default: return cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) e = setup_volume(N);
  if (e == cudaSuccess) e = setup_latency(N);
  return e == cudaSuccess ? setup_gauss(N) : e;
}

// Host reader of this file's bounds-check error word (0 in normal builds).
DG_BOUNDS_READER(bounds_word_operator)

}  // namespace dg
