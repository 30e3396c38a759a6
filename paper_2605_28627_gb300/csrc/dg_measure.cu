// Measurement helpers: per-kernel event timing of an LSERK stage and an
// arithmetic-throughput probe (FP64 DFMA and FP32 FFMA chains); checks of the
// operator kernels' conversions and reciprocals against the hardware and IEEE
// division.
#include "dg_adjoint_fn.cuh"
#include "dg_stage.cuh"

namespace dg {

// Eight independent FMA chains per thread; the loop is long enough that the
// launch is dominated by the arithmetic pipe.
template <typename T>
__global__ void k_fma_chain(T* out, T a, T b, int iters) {
  T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
  T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  }
  const T s = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (s == T(-1.2345)) out[0] = s;   // keeps the chains alive, never true in practice
}

template <typename T>
static double fma_tflops(int sms, int iters, void* buf) {
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_fma_chain<T><<<blocks, threads>>>((T*)buf, T(0.999999), T(1e-7), iters);   // warm-up
  cudaEventRecord(e0);
  k_fma_chain<T><<<blocks, threads>>>((T*)buf, T(0.999999), T(1e-7), iters);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
  return flops / (ms * 1e-3) / 1e12;
}

// Both conversions of the FP32 operator next to the hardware ones.
__global__ void k_convert_check(const double* __restrict__ x, int n, float* __restrict__ f,
                                double* __restrict__ d) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const float fb = to_op<float>(x[t]);
    f[t] = fb;
    f[n + t] = __double2float_rn(x[t]);
    d[t] = to_f64(fb);
    d[n + t] = (double)fb;
  }
}

// The reciprocals of the operator kernels next to each other: the FP64
// operators' cubic and quadratic refinements, the adjoint's, and the FP32
// operators' approximation (of x rounded to FP32).
__global__ void k_rcp_check(const double* __restrict__ x, int n, double* __restrict__ d, float* __restrict__ f) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const double v = x[t];
    d[t] = rcp_op(v);
    d[n + t] = rcp_op_q(v);
    d[2 * n + t] = adj_rcp(v);
    const float vf = __double2float_rn(v);
    f[t] = rcp_op(vf);
    f[n + t] = rcp_op_q(vf);
  }
}

}  // namespace dg

using namespace dg;

extern "C" dg_status dg_check_reciprocals(const double* d_x, int32_t n, double* d_d, float* d_f, dg_stream stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_d || !d_f))) return DG_EINVAL;
  if (n == 0) return DG_OK;
  const int blocks = (n + 255) / 256;
  k_rcp_check<<<blocks < 152 * 8 ? blocks : 152 * 8, 256, 0, (cudaStream_t)stream>>>(d_x, n, d_d, d_f);
  if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;
  return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? DG_OK : DG_ECUDA;
}

extern "C" dg_status dg_check_conversions(const double* d_x, int32_t n, float* d_f, double* d_d, dg_stream stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_f || !d_d))) return DG_EINVAL;
  if (n == 0) return DG_OK;
  const int blocks = (n + 255) / 256;
  k_convert_check<<<blocks < 152 * 8 ? blocks : 152 * 8, 256, 0, (cudaStream_t)stream>>>(d_x, n, d_f, d_d);
  if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;
  return cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? DG_OK : DG_ECUDA;
}

extern "C" dg_status dg_probe_peaks(int device, double* out) {
  if (!out) return DG_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return DG_ECUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return DG_ECUDA;
  void* buf = nullptr;
  if (cudaMalloc(&buf, 16) != cudaSuccess) return DG_ENOMEM;
  out[0] = fma_tflops<double>(prop.multiProcessorCount, 96, buf);
  out[1] = fma_tflops<float>(prop.multiProcessorCount, 4096, buf);
  cudaError_t err = cudaGetLastError();
  cudaFree(buf);
  return err == cudaSuccess ? DG_OK : DG_ECUDA;
}
