// Geometry of the curvilinear elements on the GPU (GALAEXI Sec. 3.1: mapping
// chi: E -> Omega, its Jacobian matrix and determinant, contravariant metric
// terms; face normals and surface elements).  FP64, run once at set-up.
//
// Node positions are the degree-N interpolant of the mesh's equispaced
// samples evaluated at the LGL nodes.  The metric terms use Kopriva's (2006)
// conservative curl form
//   J a^d_c = -[curl_xi (X_l grad_xi X_m)]_d,   (c, m, l) cyclic,
// which satisfies the discrete metric identities sum_d D_d (J a^d) = 0 and so
// keeps a uniform flow exactly uniform on curved meshes.
#include "dg_physics.cuh"

namespace dg {

template <int N>
__global__ void __launch_bounds__((N + 1) * (N + 1) * (N + 1)) k_geometry(const double* __restrict__ xgeo, int ngeo, const double* __restrict__ Vg,
                           const double* __restrict__ Dg, double* __restrict__ metrics, double* __restrict__ Jout,
                           double* __restrict__ Xout, int* __restrict__ bad, int E) {
  constexpr int n = N + 1, P = n * n * n;
  extern __shared__ double sm[];
  const int m = ngeo + 1, m3 = m * m * m;
  double* sx = sm;                 // [3][m3]
  double* sV = sx + 3 * m3;        // [n][m]
  double* sD = sV + n * m;         // [n][n]
  double* sX = sD + n * n;         // [3][P]
  double* sdX = sX + 3 * P;        // [3 c][3 d][P]
  double* sv = sdX + 9 * P;        // [3][P]
  const int e = blockIdx.x;
  const int id = threadIdx.x;
  // Coordinates relative to the element's corner sample (also its first LGL
  // node): interpolation and the discrete curl form are translation
  // invariant, and working with small relative coordinates avoids the
  // cancellation that large absolute coordinates cause.
  const double* xe = xgeo + (size_t)e * 3 * m3;
  const double g0[3] = {xe[0], xe[m3], xe[2 * m3]};
  for (int t = id; t < 3 * m3; t += blockDim.x) sx[t] = xe[t] - g0[t / m3];
  for (int t = id; t < n * m; t += blockDim.x) sV[t] = Vg[t];
  for (int t = id; t < n * n; t += blockDim.x) sD[t] = Dg[t];
  __syncthreads();
  const int i = id % n, j = (id / n) % n, k = id / (n * n);
  // interpolation of the equispaced samples
  for (int c = 0; c < 3; ++c) {
    double s = 0.0;
    for (int c3 = 0; c3 < m; ++c3) {
      double sj = 0.0;
      for (int b3 = 0; b3 < m; ++b3) {
        double si = 0.0;
        for (int a3 = 0; a3 < m; ++a3) si += sV[i * m + a3] * sx[c * m3 + a3 + m * (b3 + m * c3)];
        sj += sV[j * m + b3] * si;
      }
      s += sV[k * m + c3] * sj;
    }
    sX[c * P + id] = s;
  }
  __syncthreads();
  for (int c = 0; c < 3; ++c) {
    double d0 = 0, d1 = 0, d2 = 0;
    for (int q = 0; q < n; ++q) {
      d0 += sD[i * n + q] * sX[c * P + vidx<n>(q, j, k)];
      d1 += sD[j * n + q] * sX[c * P + vidx<n>(i, q, k)];
      d2 += sD[k * n + q] * sX[c * P + vidx<n>(i, j, q)];
    }
    sdX[(c * 3 + 0) * P + id] = d0;
    sdX[(c * 3 + 1) * P + id] = d1;
    sdX[(c * 3 + 2) * P + id] = d2;
  }
  __syncthreads();
  double A[3][3];
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) A[c][d] = sdX[(c * 3 + d) * P + id];
  const double Jv = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                    A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                    A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (!(Jv > 0.0)) atomicExch(bad, 1);
  double Ja[3][3];   // [d][c]
  for (int c = 0; c < 3; ++c) {
    const int mm = (c + 1) % 3, ll = (c + 2) % 3;
    for (int r = 0; r < 3; ++r) sv[r * P + id] = sX[ll * P + id] * sdX[(mm * 3 + r) * P + id];
    __syncthreads();
    double D0v1 = 0, D0v2 = 0, D1v0 = 0, D1v2 = 0, D2v0 = 0, D2v1 = 0;
    for (int q = 0; q < n; ++q) {
      const double a0 = sD[i * n + q], a1 = sD[j * n + q], a2 = sD[k * n + q];
      D0v1 += a0 * sv[1 * P + vidx<n>(q, j, k)];
      D0v2 += a0 * sv[2 * P + vidx<n>(q, j, k)];
      D1v0 += a1 * sv[0 * P + vidx<n>(i, q, k)];
      D1v2 += a1 * sv[2 * P + vidx<n>(i, q, k)];
      D2v0 += a2 * sv[0 * P + vidx<n>(i, j, q)];
      D2v1 += a2 * sv[1 * P + vidx<n>(i, j, q)];
    }
    Ja[0][c] = -(D1v2 - D2v1);
    Ja[1][c] = -(D2v0 - D0v2);
    Ja[2][c] = -(D0v1 - D1v0);
    __syncthreads();
  }
  double* mt = metrics + (size_t)e * 10 * P + id;
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c) mt[(d * 3 + c) * P] = Ja[d][c];
  mt[9 * P] = 1.0 / Jv;
  Jout[(size_t)e * P + id] = Jv;
  for (int c = 0; c < 3; ++c) Xout[((size_t)e * 3 + c) * P + id] = sX[c * P + id] + g0[c];
}

// Face normal and surface element of the master side: n sJ = (2s-1) J a^d.
template <int N>
__global__ void k_face_geometry(const FaceInfo* __restrict__ faces, const double* __restrict__ metrics,
                                double* __restrict__ facegeo, int F) {
  constexpr int n = N + 1, P = n * n * n, NN = n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)F * NN) return;
  const int f = (int)(gid / NN), pq = (int)(gid % NN);
  const int p = pq % n, q = pq / n;
  const FaceInfo fi = faces[f];
  const int e = dg_idx(fi.master >> 3, F / 3, kSiteGeomFace), lf = fi.master & 7;   // F = 3 E
  const int d = lf >> 1;
  const double sg = (lf & 1) ? 1.0 : -1.0;
  const int node = face_node<n>(lf, p, q);
  const double* mt = metrics + (size_t)e * 10 * P + node;
  const double nx = sg * mt[(d * 3 + 0) * P], ny = sg * mt[(d * 3 + 1) * P], nz = sg * mt[(d * 3 + 2) * P];
  const double sJ = sqrt(nx * nx + ny * ny + nz * nz);
  double* fg = facegeo + (size_t)f * 4 * NN + pq;
  fg[0] = nx / sJ;
  fg[NN] = ny / sJ;
  fg[2 * NN] = nz / sJ;
  fg[3 * NN] = sJ;
}

template <int N>
static cudaError_t geometry_N(Ctx& c, const double* d_xgeo, int ngeo, const double* d_V, int* d_bad,
                              cudaStream_t s) {
  constexpr int n = N + 1, P = n * n * n;
  const int m = ngeo + 1;
  const size_t smem = sizeof(double) * (3 * m * m * m + n * m + n * n + 15 * P);
  cudaError_t err = cudaFuncSetAttribute(k_geometry<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  k_geometry<N><<<c.E, P, smem, s>>>(d_xgeo, ngeo, d_V, c.d_D, c.d_metrics, c.d_J, c.d_X, d_bad, c.E);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  const long tot = (long)c.nfaces * n * n;
  k_face_geometry<N><<<(int)((tot + 127) / 128), 128, 0, s>>>(c.d_faces, c.d_metrics, c.d_facegeo, c.nfaces);
  return cudaGetLastError();
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, size_t n) {
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x)
    b[t] = (float)a[t];
}

// FP32 copy of FP64 geometry for the FP32-operator path.
cudaError_t launch_to_float(const double* a, float* b, size_t n, cudaStream_t s) {
  const size_t blocks = (n + 255) / 256;
  k_to_float<<<(unsigned)(blocks < 152 * 32 ? blocks : 152 * 32), 256, 0, s>>>(a, b, n);
  return cudaGetLastError();
}

cudaError_t build_geometry(Ctx& c, const double* d_xgeo, int ngeo, int* d_bad, cudaStream_t s) {
  // Lagrange interpolation matrix from ngeo+1 equispaced points to the LGL nodes.
  const int m = ngeo + 1;
  std::vector<double> V((size_t)c.n * m);
  for (int i = 0; i < c.n; ++i)
    for (int a = 0; a < m; ++a) {
      const double ea = -1.0 + 2.0 * a / ngeo;
      double l = 1.0;
      for (int b = 0; b < m; ++b) {
        if (b == a) continue;
        const double eb = -1.0 + 2.0 * b / ngeo;
        l *= (c.x[i] - eb) / (ea - eb);
      }
      V[(size_t)i * m + a] = l;
    }
  double* d_V = nullptr;
  cudaError_t err = cudaMalloc(&d_V, sizeof(double) * V.size());
  if (err != cudaSuccess) return err;
  err = cudaMemcpyAsync(d_V, V.data(), sizeof(double) * V.size(), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) {
    switch (c.N) {
      case 1: err = geometry_N<1>(c, d_xgeo, ngeo, d_V, d_bad, s); break;
      case 2: err = geometry_N<2>(c, d_xgeo, ngeo, d_V, d_bad, s); break;
      case 3: err = geometry_N<3>(c, d_xgeo, ngeo, d_V, d_bad, s); break;
      case 4: err = geometry_N<4>(c, d_xgeo, ngeo, d_V, d_bad, s); break;
      case 5: err = geometry_N<5>(c, d_xgeo, ngeo, d_V, d_bad, s); break;
      case 6: err = geometry_N<6>(c, d_xgeo, ngeo, d_V, d_bad, s); break;
      case 7: err = geometry_N<7>(c, d_xgeo, ngeo, d_V, d_bad, s); break;
      case 8: err = geometry_N<8>(c, d_xgeo, ngeo, d_V, d_bad, s); break;
      case 9: err = geometry_N<9>(c, d_xgeo, ngeo, d_V, d_bad, s); break;
      default: err = cudaErrorInvalidValue;
    }
  }
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(d_V);
  return err != cudaSuccess ? err : e2;
}

// Host reader of this file's bounds-check error word (0 in normal builds).
DG_BOUNDS_READER(bounds_word_geometry)

}  // namespace dg
