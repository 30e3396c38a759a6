// Conservation totals without any device allocation.
//
// Some callers cannot call cudaMalloc while they run: a host framework that
// owns all device memory and only lends input and output buffers to foreign
// code (custom-call style interfaces), or an application that must not touch
// the allocator inside its time loop.  For them this file offers one entry
// point whose only temporary storage is a file-scope __device__ array of fixed
// size, allocated once when the library is loaded on a device and held until
// the process exits.
#include <cmath>
#include <mutex>

#include "dg_internal.h"

namespace dg {

// Per-element partial sums [element][5] plus the folded result.  The array is
// shared by every call on a device and keeps the last call's contents.
constexpr int kNoAllocMaxElems = 131072;
static __device__ __align__(256) double g_noalloc_scratch[(size_t)kNoAllocMaxElems * 5 + 8];

struct Weights {
  double w[kMaxN + 1];
};

// Pass 1: one warp per element writes sum_nodes w_i w_j w_k J q_v, v = 0..4.
// Every element's row is written (nothing accumulates across calls).
__global__ void k_totals_elem(const double* __restrict__ U, const double* __restrict__ J, Weights wt, int n,
                              int E, double* __restrict__ scratch) {
  const int warp = (int)((blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= E) return;
  const int P = n * n * n;
  double s[5] = {0, 0, 0, 0, 0};
  for (int id = lane; id < P; id += 32) {
    const int i = id % n, j = (id / n) % n, k = id / (n * n);
    const double wq = wt.w[i] * wt.w[j] * wt.w[k] * J[(size_t)warp * P + id];
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] += wq * U[((size_t)warp * 5 + v) * P + id];
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    double x = s[v];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) scratch[(size_t)warp * 5 + v] = x;
  }
}

// Pass 2: one block folds the per-element rows in a fixed order.
__global__ void k_totals_fold(const double* __restrict__ scratch, int E, double* __restrict__ out) {
  __shared__ double sh[5][256];
  double s[5] = {0, 0, 0, 0, 0};
  for (int e = threadIdx.x; e < E; e += blockDim.x)
#pragma unroll
    for (int v = 0; v < 5; ++v) s[v] += scratch[(size_t)e * 5 + v];
#pragma unroll
  for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] = s[v];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
#pragma unroll
      for (int v = 0; v < 5; ++v) sh[v][threadIdx.x] += sh[v][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

// LGL weights 2 / (N (N+1) P_N(x_j)^2) on fixed-size storage (no allocation):
// the interior nodes are the zeros of P_N', found by Newton's method.
static void lgl_weights_fixed(int N, double* w) {
  double x[kMaxN + 1];
  x[0] = -1.0;
  x[N] = 1.0;
  for (int j = 1; j <= N / 2; ++j) {
    double t = -std::cos(M_PI * j / N);
    for (int it = 0; it < 60; ++it) {
      // P_N, P_N' and P_N'' by recurrence and Legendre's equation
      double a = 1.0, b = t;
      for (int k = 1; k < N; ++k) {
        const double c = ((2.0 * k + 1.0) * t * b - k * a) / (k + 1.0);
        a = b; b = c;
      }
      const double dL = N * (a - t * b) / (1.0 - t * t);
      const double d2L = (2.0 * t * dL - N * (N + 1.0) * b) / (1.0 - t * t);
      const double step = dL / d2L;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    x[j] = t;
    x[N - j] = -t;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int j = 0; j <= N; ++j) {
    double a = 1.0, b = x[j];
    for (int k = 1; k < N; ++k) {
      const double c = ((2.0 * k + 1.0) * x[j] * b - k * a) / (k + 1.0);
      a = b; b = c;
    }
    w[j] = 2.0 / (N * (N + 1.0) * b * b);
  }
}

// Legendre-Gauss weights 2 / ((1 - x_j^2) P_n'(x_j)^2), n = N + 1, at the
// zeros x_j of P_n, on fixed-size storage: Newton's method from the
// asymptotic start cos(pi (j + 3/4) / (n + 1/2)), symmetric partner mirrored.
static void gauss_weights_fixed(int N, double* w) {
  const int n = N + 1;
  for (int j = 0; j < (n + 1) / 2; ++j) {
    double t = std::cos(M_PI * (j + 0.75) / (n + 0.5)), dP = 1.0;
    for (int it = 0; it < 100; ++it) {
      // P_n(t) by the three-term recurrence, P_n' from (1 - t^2) P_n' = n (P_{n-1} - t P_n)
      double a = 1.0, b = t;
      for (int k = 1; k < n; ++k) {
        const double c = ((2.0 * k + 1.0) * t * b - k * a) / (k + 1.0);
        a = b; b = c;
      }
      dP = n * (a - t * b) / (1.0 - t * t);
      const double step = b / dP;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    // weight from P_n' at the converged node
    double a = 1.0, b = t;
    for (int k = 1; k < n; ++k) {
      const double c = ((2.0 * k + 1.0) * t * b - k * a) / (k + 1.0);
      a = b; b = c;
    }
    dP = n * (a - t * b) / (1.0 - t * t);
    const double wj = 2.0 / ((1.0 - t * t) * dP * dP);
    w[j] = wj;
    w[n - 1 - j] = wj;
  }
}

// Device address of the scratch array, looked up once per device with that
// device current (in host code the array's name is only a host-side stand-in).
static std::mutex g_scratch_mu;
static double* g_scratch_ptr[64] = {nullptr};

static cudaError_t scratch_address(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return err;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace dg

using namespace dg;

extern "C" dg_status dg_conserved_totals_noalloc(const double* dU, const double* dJ, int32_t N, int32_t nodes,
                                                 int32_t n_elems, double* dOut5, dg_stream stream) {
  if (!dU || !dJ || !dOut5) return DG_EINVAL;
  if (N < 1 || N > kMaxN) return DG_EUNSUPPORTED;
  if (nodes != DG_NODES_LGL && nodes != DG_NODES_LG) return DG_EINVAL;
  if (n_elems < 1 || n_elems > kNoAllocMaxElems) return DG_EINVAL;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return DG_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // the scratch address is the current device's: a stream of another device
  // would run the kernels there on the wrong array
  if (s) {
    int sdev = -1;
    if (cudaStreamGetDevice(s, &sdev) != cudaSuccess) return DG_ECUDA;
    if (sdev != device) return DG_EINVAL;
  }
  double* scratch = nullptr;
  if (scratch_address(device, &scratch) != cudaSuccess) return DG_ECUDA;
  Weights wt{};
  if (nodes == DG_NODES_LG) gauss_weights_fixed(N, wt.w);
  else lgl_weights_fixed(N, wt.w);
  const int threads = 256, warps_per_block = threads / 32;
  const int blocks = (n_elems + warps_per_block - 1) / warps_per_block;
  k_totals_elem<<<blocks, threads, 0, s>>>(dU, dJ, wt, N + 1, n_elems, scratch);
  if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;
  k_totals_fold<<<1, 256, 0, s>>>(scratch, n_elems, dOut5);
  if (cudaGetLastError() != cudaSuccess) return DG_ECUDA;
  return DG_OK;
}
