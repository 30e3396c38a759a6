// C ABI of the DGSEM hot path: context set-up (mesh checks, LGL basis, face
// maps, GPU geometry), stage sequencing of R(U) and of LSERK4-5 (captured in a
// CUDA graph), host-buffer end-to-end entry, diagnostics.
#include <cstdio>
#include <cstring>
#include <cmath>
#include <new>

#include "dg_internal.h"

namespace dg {

static thread_local std::string g_init_error = "no error";

// Legendre polynomial P_N and its first two derivatives at x (three-term
// recurrence; second derivative from Legendre's equation).
static void legendre(int N, double x, double& L, double& dL, double& d2L) {
  double a = 1.0, b = x;
  if (N == 0) { L = 1.0; dL = 0.0; d2L = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    const double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
    a = b; b = c;
  }
  L = b;
  // (1 - x^2) P_N' = N (P_{N-1} - x P_N)
  dL = N * (a - x * b) / (1.0 - x * x);
  d2L = (2.0 * x * dL - N * (N + 1.0) * L) / (1.0 - x * x);
}

// LGL nodes (+-1 and the zeros of P_N'), weights 2/(N(N+1) P_N^2) and the
// collocation derivative matrix D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)),
// with the diagonal set so that every row sums to zero (D 1 = 0 exactly).
static void lgl_basis(int N, std::vector<double>& x, std::vector<double>& w, std::vector<double>& D) {
  const int n = N + 1;
  x.assign(n, 0.0); w.assign(n, 0.0); D.assign((size_t)n * n, 0.0);
  x[0] = -1.0; x[N] = 1.0;
  for (int j = 1; j <= N / 2; ++j) {
    // Newton on P_N' from a Chebyshev-Lobatto start; symmetric partner mirrored
    double t = -std::cos(M_PI * j / N);
    for (int it = 0; it < 60; ++it) {
      double L, dL, d2L;
      legendre(N, t, L, dL, d2L);
      const double step = dL / d2L;
      t -= step;
      if (std::fabs(step) < 1e-17) break;
    }
    x[j] = t;
    x[N - j] = -t;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  std::vector<double> LN(n);
  for (int j = 0; j < n; ++j) {
    double L = 1.0, a = 1.0, b = x[j];
    for (int k = 1; k < N; ++k) {
      const double c = ((2.0 * k + 1.0) * x[j] * b - k * a) / (k + 1.0);
      a = b; b = c;
    }
    L = N == 0 ? 1.0 : b;
    LN[j] = L;
    w[j] = 2.0 / (N * (N + 1.0) * L * L);
  }
  for (int i = 0; i < n; ++i) {
    double row = 0.0;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      const double dij = LN[i] / (LN[j] * (x[i] - x[j]));
      D[(size_t)i * n + j] = dij;
      row += dij;
    }
    D[(size_t)i * n + i] = -row;
  }
}

bool bounds_failed(cudaStream_t s, char* msg, size_t len) {
#ifdef DG_BOUNDS_CHECK
  cudaStreamSynchronize(s);
  const unsigned long long words[9] = {bounds_word_operator(), bounds_word_volume(), bounds_word_gauss(),
                                       bounds_word_geometry(), bounds_word_adjoint(), bounds_word_ensemble(),
                                       bounds_word_latency(), bounds_word_fv(), bounds_word_mortar()};
  if (bulk_word_volume() || bulk_word_ensemble()) {
    std::snprintf(msg, len, "a bulk copy into shared memory did not complete within its wait limit");
    return true;
  }
  for (unsigned long long w : words)
    if (w) {
      long long idx = (long long)(w & 0xffffffffffffull);
      if (idx & (1ll << 47)) idx -= (1ll << 48);   // sign of the recorded index
      std::snprintf(msg, len, "bounds check: gather site %d read index %lld out of range",
                    (int)((w >> 48) & 0x7fff), idx);
      return true;
    }
#else
  (void)s; (void)msg; (void)len;
#endif
  return false;
}

static dg_status fail(Ctx* c, dg_status st, const char* what, cudaError_t e = cudaSuccess) {
  char buf[512];
  if (e != cudaSuccess) std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  else std::snprintf(buf, sizeof buf, "%s", what);
  if (c) c->err = buf; else g_init_error = buf;
  return st;
}

// Checked builds: report a recorded out-of-range gather index after the
// call's launches (synchronises the stream); normal builds: DG_OK at once.
static dg_status checked(Ctx* c, cudaStream_t s) {
  char msg[160];
  if (bounds_failed(s, msg, sizeof msg)) return fail(c, DG_ECUDA, msg);
  return DG_OK;
}

#define DG_CUDA(call, ctx, what)                                   \
  do {                                                             \
    cudaError_t _e = (call);                                       \
    if (_e != cudaSuccess)                                         \
      return fail(ctx, _e == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA, what, _e); \
  } while (0)

static void release(Ctx* c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  void* bufs[] = {c->d_modal, c->d_D, c->d_metrics, c->d_J, c->d_X, c->d_mms, c->d_Uf, c->d_gf, c->d_lgb, c->d_facegeo, c->d_metrics_f, c->d_facegeo_f,
                  c->d_grad, c->d_fstar, c->d_red, c->d_w, c->d_clock, c->d_U, c->d_G,
                  c->d_adj_qbar, c->d_adj_gbar, c->d_adj_gtil, c->d_adj_fseed, c->d_adj_face, c->d_adj_mu,
                  c->d_adj_stage, c->d_adj_work, c->d_adj_mx, c->d_adj_lgf, c->d_fv_pin, c->d_fv_tab, c->d_fv_iJb, c->d_fv_S, c->d_fv_M, c->d_fv_Fb};
  for (void* p : bufs) if (p) cudaFree(p);
  if (c->d_faces) cudaFree(c->d_faces);
  if (c->d_elem_face) cudaFree(c->d_elem_face);
  if (c->d_elem_nbr) cudaFree(c->d_elem_nbr);
  if (c->d_minmask) cudaFree(c->d_minmask);
  if (c->d_fv_mask) cudaFree(c->d_fv_mask);
  if (c->d_fv_lists) cudaFree(c->d_fv_lists);
  if (c->d_mortars) cudaFree(c->d_mortars);
  if (c->d_mortar_tab) cudaFree(c->d_mortar_tab);
  if (c->d_mortar_virt) cudaFree(c->d_mortar_virt);
  if (c->h_out) cudaFreeHost(c->h_out);
  if (c->h_clock) cudaFreeHost(c->h_clock);
}

// The RK step sequence for one call: per step, zero the register, five stages
// of (lift, face, volume+update), advance the clock.
static cudaError_t enqueue_steps(Ctx& c, double* U, double* G, int nsteps, cudaStream_t s) {
  cudaError_t err = cudaSuccess;
  const size_t bytes = sizeof(double) * (size_t)c.E * 5 * c.P;
  const RkScheme rk = rk_scheme(c.prm.rk_scheme);
  for (int st = 0; st < nsteps; ++st) {
    if ((err = cudaMemsetAsync(G, 0, bytes, s)) != cudaSuccess) return err;
    for (int k = 0; k < rk.stages; ++k) {
      if ((err = launch_fv_switch(c, U, s)) != cudaSuccess) return err;
      if ((err = launch_lift(c, U, s)) != cudaSuccess) return err;
      if ((err = launch_face(c, U, s)) != cudaSuccess) return err;
      StageArgs a{U, U, G, nullptr, c.d_clock, rk.C[k], rk.A[k], rk.B[k], 1};
      if ((err = launch_volume(c, a, s)) != cudaSuccess) return err;
    }
    if ((err = launch_clock_advance(c.d_clock, s)) != cudaSuccess) return err;
  }
  return err;
}

}  // namespace dg

using namespace dg;

struct dg_ctx : public dg::Ctx {};

// Set-up temporaries of dg_init (mesh samples on the device, the Jacobian
// flag, the set-up stream), freed on every exit, exceptions included.
struct InitScratch {
  cudaStream_t s = nullptr;
  double* d_xgeo = nullptr;
  int* d_bad = nullptr;
  ~InitScratch() {
    if (d_xgeo) cudaFree(d_xgeo);
    if (d_bad) cudaFree(d_bad);
    if (s) cudaStreamDestroy(s);
  }
};

// `c` holds the context under construction, so that the caller can free it
// if a host allocation throws half-way.
static dg_status init_impl(const dg_mesh* mesh, const dg_params* prm, int device, dg_ctx** out, dg_ctx*& c) {
  if (out) *out = nullptr;
  if (!mesh || !prm || !out) return fail(nullptr, DG_EINVAL, "dg_init: null argument");
  if (prm->N < 1 || prm->N > kMaxN) return fail(nullptr, DG_EUNSUPPORTED, "dg_init: N must be in 1..9");
  if (prm->precision != DG_FP64 && prm->precision != DG_FP32OP)
    return fail(nullptr, DG_EINVAL, "dg_init: unknown precision");
  if (prm->surf_flux != DG_FLUX_LLF && prm->surf_flux != DG_FLUX_EC && prm->surf_flux != DG_FLUX_ROE)
    return fail(nullptr, DG_EINVAL, "dg_init: unknown surface flux");
  if (prm->source != DG_SOURCE_NONE && prm->source != DG_SOURCE_MMS)
    return fail(nullptr, DG_EINVAL, "dg_init: unknown source");
  if (!(prm->gamma > 1.0) || !(prm->R > 0.0) || !(prm->Pr > 0.0) || !(prm->mu >= 0.0))
    return fail(nullptr, DG_EINVAL, "dg_init: gas constants out of range");
  if (prm->rk_scheme != DG_RK45 && prm->rk_scheme != DG_RK414)
    return fail(nullptr, DG_EINVAL, "dg_init: unknown Runge-Kutta scheme");
  if (prm->nodes != DG_NODES_LGL && prm->nodes != DG_NODES_LG)
    return fail(nullptr, DG_EINVAL, "dg_init: unknown node set");
  if (prm->visc_law != DG_VISC_CONSTANT && prm->visc_law != DG_VISC_SUTHERLAND)
    return fail(nullptr, DG_EINVAL, "dg_init: unknown viscosity law");
  if (prm->visc_law == DG_VISC_SUTHERLAND && (!(prm->T_ref > 0.0) || !(prm->S_suth >= 0.0)))
    return fail(nullptr, DG_EINVAL, "dg_init: Sutherland constants out of range");
  if (mesh->n_elems < 1 || mesh->ngeo < 1 || mesh->ngeo > 12 || !mesh->xgeo || !mesh->face_nbr ||
      mesh->n_mortars < 0 || (mesh->n_mortars > 0 && !mesh->mortars))
    return fail(nullptr, DG_EINVAL, "dg_init: bad mesh sizes or null arrays");
  const int E = mesh->n_elems, M = mesh->n_mortars;
  // mortar table: every side names its mortar back
  for (int m = 0; m < M; ++m) {
    const int* r = mesh->mortars + (size_t)m * 14;
    bool ok = r[0] >= 0 && r[0] < E && r[1] >= 0 && r[1] < 6 &&
              mesh->face_nbr[(size_t)(r[0] * 6 + r[1]) * 3] == -1 - m &&
              mesh->face_nbr[(size_t)(r[0] * 6 + r[1]) * 3 + 1] == 0;
    for (int k = 0; k < 4 && ok; ++k) {
      const int es = r[2 + 3 * k], fs = r[3 + 3 * k], fl = r[4 + 3 * k];
      ok = es >= 0 && es < E && fs >= 0 && fs < 6 && fl >= 0 && fl < 8 &&
           mesh->face_nbr[(size_t)(es * 6 + fs) * 3] == -1 - m && mesh->face_nbr[(size_t)(es * 6 + fs) * 3 + 1] == k;
    }
    if (!ok) return fail(nullptr, DG_EMESH, "dg_init: mortar table does not match the face connectivity");
  }
  // connectivity checks: range and reciprocity
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      const int* r = mesh->face_nbr + (size_t)(e * 6 + f) * 3;
      if (r[0] < 0) {   // a side of mortar -1 - r[0]
        const int m = -1 - r[0];
        if (m >= M || r[1] < 0 || r[1] > 3) return fail(nullptr, DG_EMESH, "dg_init: face connectivity out of range");
        const int* mr = mesh->mortars + (size_t)m * 14;
        if (!(mr[0] == e && mr[1] == f) && !(mr[2 + 3 * r[1]] == e && mr[3 + 3 * r[1]] == f))
          return fail(nullptr, DG_EMESH, "dg_init: face connectivity not reciprocal");
        continue;
      }
      if (r[0] >= E || r[1] < 0 || r[1] > 5 || r[2] < 0 || r[2] > 7)
        return fail(nullptr, DG_EMESH, "dg_init: face connectivity out of range");
      const int* b = mesh->face_nbr + (size_t)(r[0] * 6 + r[1]) * 3;
      if (b[0] != e || b[1] != f) return fail(nullptr, DG_EMESH, "dg_init: face connectivity not reciprocal");
      if (r[0] == e && r[1] == f) return fail(nullptr, DG_EMESH, "dg_init: face is its own neighbour");
    }
  c = new (std::nothrow) dg_ctx();
  if (!c) return fail(nullptr, DG_ENOMEM, "dg_init: host allocation failed");
  auto bail = [&](dg_status st) {
    g_init_error = c->err;
    release(c);
    delete c;
    c = nullptr;
    return st;
  };
  c->device = device;
  c->N = prm->N; c->n = prm->N + 1; c->P = c->n * c->n * c->n; c->NN = c->n * c->n; c->E = E;
  c->prm = *prm;
  Gas& g = c->gas;
  g.gamma = prm->gamma; g.R = prm->R; g.Pr = prm->Pr; g.mu = prm->mu;
  g.gm1 = prm->gamma - 1.0; g.inv_gm1 = 1.0 / g.gm1;
  g.kappa = prm->gamma * prm->R / (prm->gamma - 1.0) / prm->Pr;
  g.inv_R = 1.0 / prm->R;
  g.mms_amp = prm->mms_amp; g.surf_flux = prm->surf_flux; g.source = prm->source;
  g.p_ref = prm->p_ref; g.E_ref = prm->p_ref / (prm->gamma - 1.0);
  g.visc_law = prm->visc_law;
  g.inv_T_ref = prm->visc_law == DG_VISC_SUTHERLAND ? 1.0 / prm->T_ref : 1.0;
  g.S_suth = prm->visc_law == DG_VISC_SUTHERLAND ? prm->S_suth : 0.0;
  g.suth_c = prm->visc_law == DG_VISC_SUTHERLAND ? prm->T_ref + prm->S_suth : 1.0;
  set_float_copies(g);
  lgl_basis(c->N, c->x, c->w, c->D);
  // faces: the side with the smaller (e*6 + f) is the master
  std::vector<FaceInfo> faces;
  std::vector<int> elem_face((size_t)E * 6), elem_nbr((size_t)E * 6);
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      const int* r = mesh->face_nbr + (size_t)(e * 6 + f) * 3;
      if (r[0] < 0) continue;   // mortar sides: below
      elem_nbr[e * 6 + f] = r[0] * 8 + r[1];
      if (e * 6 + f < r[0] * 6 + r[1]) {
        elem_face[e * 6 + f] = (int)faces.size() * 16 + 8 + r[2];
        faces.push_back(FaceInfo{e * 8 + f, r[0] * 8 + r[1], r[2], 0});
      }
    }
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      const int* r = mesh->face_nbr + (size_t)(e * 6 + f) * 3;
      if (r[0] >= 0 && e * 6 + f > r[0] * 6 + r[1])
        elem_face[e * 6 + f] = (elem_face[r[0] * 6 + r[1]] >> 4) * 16 + r[2];
    }
  c->nfaces_conf = (int)faces.size();
  // mortars: a face slot of its own for each small side and the big side, each
  // the master of its slot; the lifting reads the side's neighbour state from
  // the mortar array (elem_nbr = -1 - (5 m + side), side 4 = big)
  c->M = M;
  std::vector<int> mtab((size_t)M * 20, 0);
  for (int m = 0; m < M; ++m) {
    const int* r = mesh->mortars + (size_t)m * 14;
    int* t = &mtab[(size_t)m * 20];
    t[0] = r[0];
    t[1] = r[1];
    for (int k = 0; k < 4; ++k) {
      const int es = r[2 + 3 * k], fs = r[3 + 3 * k];
      t[3 + 4 * k] = es;
      t[4 + 4 * k] = fs;
      t[5 + 4 * k] = r[4 + 3 * k];
      t[6 + 4 * k] = (int)faces.size();
      elem_face[es * 6 + fs] = (int)faces.size() * 16 + 8;
      elem_nbr[es * 6 + fs] = -1 - (5 * m + k);
      faces.push_back(FaceInfo{es * 8 + fs, r[0] * 8 + r[1], r[4 + 3 * k], m});
    }
    t[2] = (int)faces.size();
    elem_face[r[0] * 6 + r[1]] = (int)faces.size() * 16 + 8;
    elem_nbr[r[0] * 6 + r[1]] = -1 - (5 * m + 4);
    faces.push_back(FaceInfo{r[0] * 8 + r[1], r[0] * 8 + r[1], 0, m});
  }
  c->nfaces = (int)faces.size();
  if (cudaSetDevice(device) != cudaSuccess) { fail(c, DG_ECUDA, "dg_init: cudaSetDevice"); return bail(DG_ECUDA); }
  const size_t P = c->P, NN = c->NN;
  auto alloc = [&](void** p, size_t bytes, const char* what) -> bool {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) { fail(c, e == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA, what, e); return false; }
    return true;
  };
  const int red_rows = 152 * 8;
  c->red_len = red_rows;
  if (!alloc((void**)&c->d_D, sizeof(double) * NN, "alloc D") ||
      !alloc((void**)&c->d_metrics, sizeof(double) * E * 10 * P, "alloc metrics") ||
      !alloc((void**)&c->d_J, sizeof(double) * E * P, "alloc J") ||
      !alloc((void**)&c->d_X, sizeof(double) * E * 3 * P, "alloc X") ||
      !alloc((void**)&c->d_facegeo, sizeof(double) * c->nfaces * 4 * NN, "alloc facegeo") ||
      !alloc((void**)&c->d_faces, sizeof(FaceInfo) * c->nfaces, "alloc faces") ||
      !alloc((void**)&c->d_elem_face, sizeof(int) * E * 6, "alloc elem_face") ||
      !alloc((void**)&c->d_elem_nbr, sizeof(int) * E * 6, "alloc elem_nbr") ||
      !alloc((void**)&c->d_grad, sizeof(double) * E * 12 * P, "alloc grad") ||
      !alloc((void**)&c->d_fstar, sizeof(double) * c->nfaces * 5 * NN, "alloc fstar") ||
      !alloc((void**)&c->d_red, sizeof(double) * (red_rows + 1) * kRedValues, "alloc reduction") ||
      !alloc((void**)&c->d_w, sizeof(double) * c->n, "alloc w") ||
      !alloc((void**)&c->d_modal, sizeof(double) * NN, "alloc modal table") ||
      !alloc((void**)&c->d_minmask, sizeof(int), "alloc mask") ||
      !alloc((void**)&c->d_clock, sizeof(double) * 2, "alloc clock") ||
      (M > 0 && (!alloc((void**)&c->d_mortars, sizeof(int) * M * 20, "alloc mortar table") ||
                 !alloc((void**)&c->d_mortar_tab, sizeof(double) * (2 * NN + c->n), "alloc mortar interpolation") ||
                 !alloc((void**)&c->d_mortar_virt, sizeof(double) * M * 25 * NN, "alloc mortar states"))) ||
      (prm->source == DG_SOURCE_MMS && !alloc((void**)&c->d_mms, sizeof(double) * E * 2 * P, "alloc source phases")) ||
      (prm->nodes == DG_NODES_LG &&
       (!alloc((void**)&c->d_Uf, sizeof(double) * E * 6 * 5 * NN, "alloc face states") ||
        !alloc((void**)&c->d_gf, sizeof(double) * E * 6 * 12 * NN, "alloc face gradients") ||
        !alloc((void**)&c->d_lgb, sizeof(double) * (2 * NN + 5 * c->n), "alloc Gauss basis"))) ||
      (prm->precision == DG_FP32OP &&
       (!alloc((void**)&c->d_metrics_f, sizeof(float) * E * 10 * P, "alloc metrics (fp32)") ||
        !alloc((void**)&c->d_facegeo_f, sizeof(float) * c->nfaces * 4 * NN, "alloc facegeo (fp32)"))))
    return bail(c->err.find("out of memory") != std::string::npos ? DG_ENOMEM : DG_ECUDA);
  if (cudaMallocHost((void**)&c->h_out, sizeof(double) * 16) != cudaSuccess ||
      cudaMallocHost((void**)&c->h_clock, sizeof(double) * 2) != cudaSuccess) {
    fail(c, DG_ENOMEM, "dg_init: pinned host allocation failed");
    return bail(DG_ENOMEM);
  }
  std::vector<double> gtab, modal;
  if (prm->nodes == DG_NODES_LG) {
    std::vector<double> gx;
    gauss_table(c->N, c->x, gtab, &gx);
    c->dt_factor = gauss_dt_factor(c->N, c->x, c->w, c->D, gtab);
    const std::vector<double> gw(gtab.begin() + 2 * NN + 4 * c->n, gtab.begin() + 2 * NN + 5 * c->n);
    modal_table(c->N, gx, gw, false, modal);
  } else {
    modal_table(c->N, c->x, c->w, true, modal);
  }
  InitScratch tmp;
  if (cudaStreamCreateWithFlags(&tmp.s, cudaStreamNonBlocking) != cudaSuccess) {
    tmp.s = nullptr;
    fail(c, DG_ECUDA, "dg_init: stream");
    return bail(DG_ECUDA);
  }
  cudaStream_t s = tmp.s;
  const int minmask = 1 << 8;
  const size_t m3 = (size_t)(mesh->ngeo + 1) * (mesh->ngeo + 1) * (mesh->ngeo + 1);
  cudaError_t err = cudaMalloc(&tmp.d_xgeo, sizeof(double) * E * 3 * m3);
  if (err == cudaSuccess) err = cudaMalloc(&tmp.d_bad, sizeof(int));
  double* d_xgeo = tmp.d_xgeo;
  int* d_bad = tmp.d_bad;
  if (err == cudaSuccess) err = cudaMemcpyAsync(d_xgeo, mesh->xgeo, sizeof(double) * E * 3 * m3, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemsetAsync(d_bad, 0, sizeof(int), s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->d_D, c->D.data(), sizeof(double) * NN, cudaMemcpyHostToDevice, s);
  if (prm->nodes == DG_NODES_LG) {
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(c->d_lgb, gtab.data(), sizeof(double) * gtab.size(), cudaMemcpyHostToDevice, s);
    // quadrature weights of the Gauss nodes for the integrals
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(c->d_w, gtab.data() + 2 * NN + 4 * c->n, sizeof(double) * c->n, cudaMemcpyHostToDevice, s);
  } else if (err == cudaSuccess) {
    err = cudaMemcpyAsync(c->d_w, c->w.data(), sizeof(double) * c->n, cudaMemcpyHostToDevice, s);
  }
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->d_minmask, &minmask, sizeof(int), cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(c->d_modal, modal.data(), sizeof(double) * NN, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->d_faces, faces.data(), sizeof(FaceInfo) * c->nfaces, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->d_elem_face, elem_face.data(), sizeof(int) * E * 6, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess) err = cudaMemcpyAsync(c->d_elem_nbr, elem_nbr.data(), sizeof(int) * E * 6, cudaMemcpyHostToDevice, s);
  // mortars: the table and the interpolation of the node set's Lagrange
  // basis to its nodes on each half of [-1, 1], I[k][a][j] = l_j((x_a + 2k - 1)/2),
  // with the node set's weights w (LGL, or Legendre-Gauss)
  std::vector<double> mI(M > 0 ? 2 * NN + c->n : 0);
  if (M > 0) {
    const int n = c->n;
    std::vector<double> xs_set = c->x, ws_set = c->w;
    if (prm->nodes == DG_NODES_LG) {
      std::vector<double> gtab;
      gauss_table(c->N, c->x, gtab, &xs_set, &ws_set);
    }
    for (int k = 0; k < 2; ++k)
      for (int a = 0; a < n; ++a)
        for (int j = 0; j < n; ++j) {
          const double xs = 0.5 * (xs_set[a] + 2.0 * k - 1.0);
          double l = 1.0;
          for (int m = 0; m < n; ++m)
            if (m != j) l *= (xs - xs_set[m]) / (xs_set[j] - xs_set[m]);
          mI[(size_t)(k * n + a) * n + j] = l;
        }
    for (int a = 0; a < n; ++a) mI[2 * NN + a] = ws_set[a];
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(c->d_mortars, mtab.data(), sizeof(int) * mtab.size(), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(c->d_mortar_tab, mI.data(), sizeof(double) * mI.size(), cudaMemcpyHostToDevice, s);
  }
  if (err == cudaSuccess) err = setup_kernels(c->N);
  if (err == cudaSuccess) err = build_geometry(*c, d_xgeo, mesh->ngeo, d_bad, s);
  if (err == cudaSuccess && prm->nodes == DG_NODES_LG) err = gauss_geometry(*c, d_bad, s);
  if (err == cudaSuccess && prm->source == DG_SOURCE_MMS) err = launch_mms_phase(*c, s);
  if (err == cudaSuccess && prm->precision == DG_FP32OP) {
    err = launch_to_float(c->d_metrics, c->d_metrics_f, (size_t)E * 10 * P, s);
    if (err == cudaSuccess) err = launch_to_float(c->d_facegeo, c->d_facegeo_f, (size_t)c->nfaces * 4 * NN, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  }
  int bad = 0;
  if (err == cudaSuccess) err = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) {
    fail(c, err == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA, "dg_init: geometry", err);
    return bail(err == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA);
  }
  if (bad) {
    fail(c, DG_EMESH, "dg_init: non-positive Jacobian at a node");
    return bail(DG_EMESH);
  }
  {
    char msg[160];
    if (bounds_failed(s, msg, sizeof msg)) {
      fail(c, DG_ECUDA, msg);
      return bail(DG_ECUDA);
    }
  }
  c->err = "no error";
  *out = c;
  return DG_OK;
}

extern "C" {

// Host containers (face lists, tables) may throw on a mesh too large for host
// memory; no exception leaves the C ABI.
dg_status dg_init(const dg_mesh* mesh, const dg_params* prm, int device, dg_ctx** out) {
  dg_ctx* c = nullptr;
  try {
    return init_impl(mesh, prm, device, out, c);
  } catch (const std::bad_alloc&) {
    if (c) {                // the half-built context and its device buffers
      release(c);
      delete c;
    }
    if (out) *out = nullptr;
    g_init_error = "dg_init: host memory exhausted";
    return DG_ENOMEM;
  }
}

dg_status dg_destroy(dg_ctx* c) {
  if (!c) return DG_EINVAL;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  release(c);
  delete c;
  return DG_OK;
}

size_t dg_state_len(const dg_ctx* c) { return c ? (size_t)c->E * 5 * c->P : 0; }

const char* dg_last_error(const dg_ctx* c) { return c ? c->err.c_str() : g_init_error.c_str(); }

dg_status dg_time_derivative(dg_ctx* c, const double* dU, double* dUt, double t, dg_stream stream) {
  if (!c || !dU || !dUt) return fail(c, DG_EINVAL, "dg_time_derivative: null argument");
  if (dU == dUt) return fail(c, DG_EINVAL, "dg_time_derivative: dU and dUt alias");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  DG_CUDA(launch_set_clock(c->d_clock, t, 0.0, s), c, "clock");
  DG_CUDA(launch_fv_switch(*c, dU, s), c, "FV switch kernels");
  DG_CUDA(launch_lift(*c, dU, s), c, "lift kernel");
  DG_CUDA(launch_face(*c, dU, s), c, "face kernel");
  StageArgs a{dU, nullptr, nullptr, dUt, c->d_clock, 0.0, 0.0, 0.0, 0};
  DG_CUDA(launch_volume(*c, a, s), c, "volume kernel");
  return checked(c, s);
}

dg_status dg_rk_step(dg_ctx* c, double* dU, double* dG, double t, double dt, int32_t nsteps, dg_stream stream) {
  if (!c || !dU || !dG) return fail(c, DG_EINVAL, "dg_rk_step: null argument");
  if (nsteps < 0) return fail(c, DG_EINVAL, "dg_rk_step: nsteps < 0");
  if (dU == dG) return fail(c, DG_EINVAL, "dg_rk_step: dU and dG alias");
  if (nsteps == 0) return DG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  DG_CUDA(launch_set_clock(c->d_clock, t, dt, s), c, "clock");
  if (!c->graph || c->graph_U != dU || c->graph_G != dG || c->graph_nsteps != nsteps) {
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    cudaStream_t cs;
    DG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), c, "capture stream");
    cudaGraph_t gr = nullptr;
    cudaError_t err = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
      cudaError_t e1 = enqueue_steps(*c, dU, dG, nsteps, cs);
      err = cudaStreamEndCapture(cs, &gr);
      if (e1 != cudaSuccess) err = e1;
    }
    if (err == cudaSuccess) err = cudaGraphInstantiate(&c->graph, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    cudaStreamDestroy(cs);
    if (err != cudaSuccess) { c->graph = nullptr; return fail(c, DG_ECUDA, "dg_rk_step: graph capture", err); }
    c->graph_U = dU; c->graph_G = dG; c->graph_nsteps = nsteps;
  }
  DG_CUDA(cudaGraphLaunch(c->graph, s), c, "dg_rk_step: graph launch");
  return checked(c, s);
}

dg_status dg_advance_host(dg_ctx* c, double* hU, double t, double dt, int32_t nsteps, dg_stream stream) {
  if (!c || !hU) return fail(c, DG_EINVAL, "dg_advance_host: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * dg_state_len(c);
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  if (!c->d_U) DG_CUDA(cudaMalloc(&c->d_U, bytes), c, "dg_advance_host: state allocation");
  if (!c->d_G) DG_CUDA(cudaMalloc(&c->d_G, bytes), c, "dg_advance_host: register allocation");
  DG_CUDA(cudaMemcpyAsync(c->d_U, hU, bytes, cudaMemcpyHostToDevice, s), c, "dg_advance_host: H2D");
  dg_status st = dg_rk_step(c, c->d_U, c->d_G, t, dt, nsteps, stream);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemcpyAsync(hU, c->d_U, bytes, cudaMemcpyDeviceToHost, s), c, "dg_advance_host: D2H");
  DG_CUDA(cudaStreamSynchronize(s), c, "dg_advance_host: sync");
  return DG_OK;
}

dg_status dg_integrals(dg_ctx* c, const double* dU, double* out, dg_stream stream) {
  if (!c || !dU || !out) return fail(c, DG_EINVAL, "dg_integrals: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  DG_CUDA(launch_integrals(*c, dU, s), c, "integrals kernel");
  const int rows = reduction_rows(*c);
  DG_CUDA(cudaMemcpyAsync(c->h_out, c->d_red + (size_t)rows * kRedValues, sizeof(double) * kRedValues,
                          cudaMemcpyDeviceToHost, s), c, "integrals copy");
  DG_CUDA(cudaStreamSynchronize(s), c, "integrals sync");
  if (checked(c, s) != DG_OK) return DG_ECUDA;
  const double* h = c->h_out;
  for (int a = 0; a < 5; ++a) out[a] = h[a];
  const double vol = h[5];
  out[5] = 0.5 * h[6] / vol;
  out[6] = c->prm.mu * h[7] / vol;
  out[7] = h[8];
  for (int a = 0; a < 8; ++a)
    if (!std::isfinite(out[a])) return fail(c, DG_ENONFINITE, "dg_integrals: non-finite value");
  return DG_OK;
}

dg_status dg_max_dt(dg_ctx* c, const double* dU, double cfl, double dfl, double* host_dt, dg_stream stream) {
  if (!c || !dU || !host_dt) return fail(c, DG_EINVAL, "dg_max_dt: null argument");
  if (!(cfl > 0.0) || !(dfl > 0.0)) return fail(c, DG_EINVAL, "dg_max_dt: cfl and dfl must be > 0");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  DG_CUDA(launch_max_dt(*c, dU, cfl, dfl, s), c, "dt kernel");
  const int rows = reduction_rows(*c);
  DG_CUDA(cudaMemcpyAsync(c->h_out, c->d_red + (size_t)rows * 2, sizeof(double) * 2, cudaMemcpyDeviceToHost, s),
          c, "dt copy");
  DG_CUDA(cudaStreamSynchronize(s), c, "dt sync");
  const double lc = c->h_out[0], lv = c->h_out[1];
  if (!std::isfinite(lc) || !std::isfinite(lv)) return fail(c, DG_ENONFINITE, "dg_max_dt: non-finite value");
  const double h = 2.0 / (2.0 * c->N + 1.0);
  // node-set factor on the convective bound, its square on the viscous one
  // (the second-derivative operator's spectral radius scales as the square)
  const double fa = c->dt_factor;
  double dt = lc > 0.0 ? fa * cfl * h / lc : HUGE_VAL;
  if (lv > 0.0) dt = std::fmin(dt, fa * fa * dfl * h * h / lv);
  *host_dt = dt;
  return DG_OK;
}

dg_status dg_indicator(dg_ctx* c, const double* dU, int32_t var, double log10_threshold, double* dEta,
                       int32_t* dFlag, dg_stream stream) {
  if (!c || !dU || !dEta) return fail(c, DG_EINVAL, "dg_indicator: null argument");
  if (var < DG_IND_RHO || var > DG_IND_RHOP) return fail(c, DG_EINVAL, "dg_indicator: unknown indicator quantity");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  DG_CUDA(launch_indicator(*c, dU, var, log10_threshold, dEta, dFlag, s), c, "indicator kernel");
  return checked(c, s);
}

}  // extern "C"

// The FV sub-cell buffers and tables, set up once per context.
static dg_status fv_alloc_impl(dg_ctx* c, cudaStream_t s) {
  if (c->d_fv_mask) return DG_OK;
  const size_t E = c->E, P = c->P, NN = c->NN, n = c->n;
  std::vector<double> tab, nodes = c->x;   // the context's node set: LGL, or Gauss below
  if (c->prm.nodes == DG_NODES_LG) {
    std::vector<double> gtab;
    gauss_table(c->N, c->x, gtab, &nodes);
  }
  fv_tables(c->N, nodes, tab);
  DG_CUDA(cudaMalloc(&c->d_fv_tab, sizeof(double) * tab.size()), c, "FV tables");
  DG_CUDA(cudaMalloc(&c->d_fv_iJb, sizeof(double) * E * P), c, "FV sub-cell Jacobians");
  DG_CUDA(cudaMalloc(&c->d_fv_S, sizeof(double) * E * 3 * (n + 1) * NN * 4), c, "FV area vectors");
  DG_CUDA(cudaMalloc(&c->d_fv_M, sizeof(double) * E * 17 * P), c, "FV sub-cell means");
  DG_CUDA(cudaMalloc(&c->d_fv_Fb, sizeof(double) * (size_t)c->nfaces * 5 * NN), c, "FV sub-face fluxes");
  DG_CUDA(cudaMemcpyAsync(c->d_fv_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, s), c,
          "FV tables copy");
  DG_CUDA(fv_setup(*c, s), c, "FV geometry kernel");
  // the host table must outlive the copy
  DG_CUDA(cudaStreamSynchronize(s), c, "FV set-up");
  DG_CUDA(cudaMalloc(&c->d_fv_lists, sizeof(int) * (2 * E + 2)), c, "FV element lists");
  if (c->M > 0) {   // the elements with a mortar face, which stay DG (the mortar maps act on DG traces)
    std::vector<int> nbr(E * 6), pin(E, 0);
    DG_CUDA(cudaMemcpyAsync(nbr.data(), c->d_elem_nbr, sizeof(int) * E * 6, cudaMemcpyDeviceToHost, s), c,
            "neighbour table copy");
    DG_CUDA(cudaStreamSynchronize(s), c, "FV set-up");
    c->fv_pin.assign(E, 0);
    for (size_t e = 0; e < E; ++e)
      for (int f = 0; f < 6; ++f)
        if (nbr[e * 6 + f] < 0) pin[e] = c->fv_pin[e] = 1;
    DG_CUDA(cudaMalloc(&c->d_fv_pin, sizeof(int) * E), c, "FV pins");
    DG_CUDA(cudaMemcpyAsync(c->d_fv_pin, pin.data(), sizeof(int) * E, cudaMemcpyHostToDevice, s), c, "pin copy");
    DG_CUDA(cudaStreamSynchronize(s), c, "FV set-up");   // the host table must outlive the copy
  }
  DG_CUDA(cudaMalloc(&c->d_fv_mask, sizeof(int) * E), c, "FV mask");
  return DG_OK;
}

// fv_alloc_impl with host-memory exhaustion turned into DG_ENOMEM (no C++
// exception leaves the C entry points); buffers already made stay with the
// context and are freed with it.
static dg_status fv_alloc(dg_ctx* c, cudaStream_t s) {
  try {
    return fv_alloc_impl(c, s);
  } catch (const std::bad_alloc&) {
    return fail(c, DG_ENOMEM, "FV set-up: host memory exhausted");
  }
}

// Whether the stages run the FV kernels; a captured RK graph has the other
// launch sequence after a change.
static void set_fv_on(dg_ctx* c, bool on) {
  if (on != c->fv_on && c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->fv_on = on;
}

extern "C" {

dg_status dg_set_fv_mask(dg_ctx* c, const int32_t* dMask, dg_stream stream) {
  if (!c) return fail(c, DG_EINVAL, "dg_set_fv_mask: null context");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  const bool on = dMask != nullptr;
  if (on && c->prm.precision != DG_FP64)
    return fail(c, DG_EUNSUPPORTED, "dg_set_fv_mask: the FV sub-cell operator is built for the FP64 operator");
  if (on) {
    const dg_status st = fv_alloc(c, s);
    if (st != DG_OK) return st;
    if (c->M > 0) {   // no element with a mortar face may be an FV element
      std::vector<int32_t> h;
      try {
        h.resize(c->E);
      } catch (const std::bad_alloc&) {
        return fail(c, DG_ENOMEM, "dg_set_fv_mask: host memory exhausted");
      }
      DG_CUDA(cudaMemcpyAsync(h.data(), dMask, sizeof(int32_t) * c->E, cudaMemcpyDeviceToHost, s), c, "mask copy");
      DG_CUDA(cudaStreamSynchronize(s), c, "mask check");
      for (int e = 0; e < c->E; ++e)
        if (h[e] && c->fv_pin[e])
          return fail(c, DG_EUNSUPPORTED, "dg_set_fv_mask: an element with a mortar face stays a DG element");
    }
    DG_CUDA(cudaMemcpyAsync(c->d_fv_mask, dMask, sizeof(int) * c->E, cudaMemcpyDeviceToDevice, s), c,
            "FV mask copy");
    DG_CUDA(launch_fv_lists(*c, s), c, "FV element lists kernel");
  } else if (c->fv_switch) {   // all DG until the switch marks elements again
    DG_CUDA(cudaMemsetAsync(c->d_fv_mask, 0, sizeof(int) * c->E, s), c, "FV mask clear");
    DG_CUDA(launch_fv_lists(*c, s), c, "FV element lists kernel");
  }
  set_fv_on(c, on || c->fv_switch);
  return checked(c, s);
}

// Automatic DG/FV switching before every evaluation of R(U).
dg_status dg_set_fv_switch(dg_ctx* c, int32_t var, double log10_upper, double log10_lower, dg_stream stream) {
  if (!c) return fail(c, DG_EINVAL, "dg_set_fv_switch: null context");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  if (var < 0) {   // off; the mask in effect stays
    if (c->fv_switch && c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    c->fv_switch = false;
    return DG_OK;
  }
  if (var > DG_IND_RHOP) return fail(c, DG_EINVAL, "dg_set_fv_switch: unknown indicator quantity");
  if (!(log10_upper >= log10_lower) || !std::isfinite(log10_upper) || !std::isfinite(log10_lower))
    return fail(c, DG_EINVAL, "dg_set_fv_switch: thresholds must be finite with upper >= lower");
  if (c->prm.precision != DG_FP64)
    return fail(c, DG_EUNSUPPORTED, "dg_set_fv_switch: the FV sub-cell operator is built for the FP64 operator");
  const bool fresh = !c->d_fv_mask;
  const dg_status st = fv_alloc(c, s);
  if (st != DG_OK) return st;
  if (fresh || !c->fv_on) {   // start from the all-DG mask
    DG_CUDA(cudaMemsetAsync(c->d_fv_mask, 0, sizeof(int) * c->E, s), c, "FV mask clear");
    DG_CUDA(launch_fv_lists(*c, s), c, "FV element lists kernel");
  }
  if (!c->fv_switch && c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  c->fv_switch = true;
  c->fv_sw_var = var;
  c->fv_sw_up = log10_upper;
  c->fv_sw_low = log10_lower;
  set_fv_on(c, true);
  return checked(c, s);
}

// The FV mask in effect (all zero without FV elements).
dg_status dg_get_fv_mask(dg_ctx* c, int32_t* dMask, dg_stream stream) {
  if (!c || !dMask) return fail(c, DG_EINVAL, "dg_get_fv_mask: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  if (c->fv_on)
    DG_CUDA(cudaMemcpyAsync(dMask, c->d_fv_mask, sizeof(int) * c->E, cudaMemcpyDeviceToDevice, s), c, "mask copy");
  else
    DG_CUDA(cudaMemsetAsync(dMask, 0, sizeof(int) * c->E, s), c, "mask clear");
  return DG_OK;
}

dg_status dg_initial_state(dg_ctx* c, int32_t kind, double prm0, double* dU, dg_stream stream) {
  if (!c || !dU) return fail(c, DG_EINVAL, "dg_initial_state: null argument");
  if (kind != DG_IC_TGV && kind != DG_IC_MMS) return fail(c, DG_EINVAL, "dg_initial_state: unknown kind");
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  DG_CUDA(launch_initial_state(*c, kind, prm0, dU, (cudaStream_t)stream), c, "initial state kernel");
  return DG_OK;
}

dg_status dg_node_coords(dg_ctx* c, double* dX, dg_stream stream) {
  if (!c || !dX) return fail(c, DG_EINVAL, "dg_node_coords: null argument");
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  DG_CUDA(cudaMemcpyAsync(dX, c->d_X, sizeof(double) * (size_t)c->E * 3 * c->P, cudaMemcpyDeviceToDevice,
                          (cudaStream_t)stream), c, "node coords copy");
  return DG_OK;
}

dg_status dg_geometry(dg_ctx* c, double* dJa, double* dJ, dg_stream stream) {
  if (!c) return fail(c, DG_EINVAL, "dg_geometry: null context");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  const size_t P = c->P;
  if (dJa)
    DG_CUDA(cudaMemcpy2DAsync(dJa, sizeof(double) * 9 * P, c->d_metrics, sizeof(double) * 10 * P,
                              sizeof(double) * 9 * P, c->E, cudaMemcpyDeviceToDevice, s), c, "geometry copy");
  if (dJ) DG_CUDA(cudaMemcpyAsync(dJ, c->d_J, sizeof(double) * c->E * P, cudaMemcpyDeviceToDevice, s), c, "J copy");
  return DG_OK;
}

dg_status dg_profile_stages(dg_ctx* c, double* dU, double* dG, double dt, int32_t reps, float* ms3,
                            dg_stream stream) {
  if (!c || !dU || !dG || !ms3 || reps < 1) return fail(c, DG_EINVAL, "dg_profile_stages: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  cudaEvent_t ev[4];
  for (int a = 0; a < 4; ++a) DG_CUDA(cudaEventCreate(&ev[a]), c, "event");
  double tot[3] = {0, 0, 0};
  DG_CUDA(launch_set_clock(c->d_clock, 0.0, dt, s), c, "clock");
  DG_CUDA(cudaMemsetAsync(dG, 0, sizeof(double) * dg_state_len(c), s), c, "memset");
  cudaError_t err = cudaSuccess;
  const RkScheme rk = rk_scheme(c->prm.rk_scheme);
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    const int k = r % rk.stages;
    StageArgs a{dU, dU, dG, nullptr, c->d_clock, rk.C[k], rk.A[k], rk.B[k], 1};
    cudaEventRecord(ev[0], s);
    err = launch_fv_switch(*c, dU, s);   // counted with the lifting
    if (err == cudaSuccess) err = launch_lift(*c, dU, s);
    cudaEventRecord(ev[1], s);
    if (err == cudaSuccess) err = launch_face(*c, dU, s);
    cudaEventRecord(ev[2], s);
    if (err == cudaSuccess) err = launch_volume(*c, a, s);
    cudaEventRecord(ev[3], s);
    if (err == cudaSuccess) err = cudaEventSynchronize(ev[3]);
    for (int q = 0; q < 3 && err == cudaSuccess; ++q) {
      float ms = 0.f;
      err = cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
      tot[q] += ms;
    }
  }
  for (int a = 0; a < 4; ++a) cudaEventDestroy(ev[a]);
  if (err != cudaSuccess) return fail(c, DG_ECUDA, "dg_profile_stages", err);
  for (int q = 0; q < 3; ++q) ms3[q] = (float)(tot[q] / reps);
  return DG_OK;
}

}  // extern "C"
