// Single-context launcher of the volume kernel (body in dg_stage.cuh): split-form
// flux differencing, viscous volume term, surface integral, Jacobian, source
// and LSERK stage update, one element per block (several for small N).
#include "dg_stage.cuh"

namespace dg {

// LIST: the DG elements of a context with FV sub-cell elements (FP64 only).
template <int N, typename R, bool LIST>
__global__ void __launch_bounds__(VShape<N>::THREADS, vol_min_blocks<N, R>())
k_volume2(StageArgs a, const R* __restrict__ metrics, const double* __restrict__ iJ64,
          const R* __restrict__ grad, const R* __restrict__ fstar, const int* __restrict__ elem_face,
          const double* __restrict__ mms, const double* __restrict__ Dg, int E, Gas g, double inv_w0) {
  volume_body<N, R, VShape<N>::EPB, LIST>(a, metrics, iJ64, grad, fstar, elem_face, mms, Dg, E, g, inv_w0,
                                          blockIdx.x);
}

template <int N, typename R>
static size_t volume2_smem() {
  return volume_smem_bytes<N, R, VShape<N>::EPB>();
}

template <int N, typename R, bool LIST>
cudaError_t volume2_setup() {
  return cudaFuncSetAttribute(k_volume2<N, R, LIST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)volume2_smem<N, R>());
}

template <int N, typename R, bool LIST>
cudaError_t volume2_launch(const Ctx& c, const StageArgs& a0, cudaStream_t s) {
  using S = VShape<N>;
  const int blocks = (c.E + S::EPB - 1) / S::EPB;
  const R* metrics = (const R*)(sizeof(R) == 8 ? (const void*)c.d_metrics : (const void*)c.d_metrics_f);
  StageArgs a = a0;
  a.nfaces = c.nfaces;
  k_volume2<N, R, LIST><<<blocks, S::THREADS, volume2_smem<N, R>(), s>>>(
      a, metrics, c.d_metrics, (const R*)c.d_grad, (const R*)c.d_fstar, c.d_elem_face, c.d_mms, c.d_D, c.E, c.gas,
      1.0 / c.w[0]);
  return cudaGetLastError();
}

template <int N>
static cudaError_t volume_any(const Ctx& c, const StageArgs& a, cudaStream_t s) {
  if (c.prm.precision == DG_FP32OP) return volume2_launch<N, float, false>(c, a, s);
  return a.list != nullptr ? volume2_launch<N, double, true>(c, a, s) : volume2_launch<N, double, false>(c, a, s);
}

template <int N>
static cudaError_t setup_any() {
  cudaError_t e = volume2_setup<N, double, false>();
  if (e == cudaSuccess) e = volume2_setup<N, double, true>();
  return e != cudaSuccess ? e : volume2_setup<N, float, false>();
}

cudaError_t launch_volume(const Ctx& c, const StageArgs& a, cudaStream_t s, bool latency_ok) {
  // with FV sub-cell elements: the FV stage, which calls back here with the
  // list of the DG elements
  if (c.fv_on && a.list == nullptr) return launch_fv_stage(c, a, s);
  if (c.prm.nodes == DG_NODES_LG) return launch_volume_lg(c, a, s);
  if (latency_ok && use_latency_kernels(c)) return launch_volume_lat(c, a, s);
  switch (c.N) {
    case 1: return volume_any<1>(c, a, s);
    case 2: return volume_any<2>(c, a, s);
    case 3: return volume_any<3>(c, a, s);
    case 4: return volume_any<4>(c, a, s);
    case 5: return volume_any<5>(c, a, s);
    case 6: return volume_any<6>(c, a, s);
    case 7: return volume_any<7>(c, a, s);
    case 8: return volume_any<8>(c, a, s);
    case 9: return volume_any<9>(c, a, s);
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
    case 8: return setup_any<8>();
    case 9: return setup_any<9>();
    default: return cudaErrorInvalidValue;
  }
}

// Host reader of this file's bounds-check error word (0 in normal builds).
DG_BOUNDS_READER(bounds_word_volume)
DG_BULK_READER(bulk_word_volume)

}  // namespace dg
