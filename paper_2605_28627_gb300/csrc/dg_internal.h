// Internal declarations of the DGSEM runtime (context, launch plans).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dgsem.h"

namespace dg {

constexpr int kMaxN = 9;

// LSERK4-5 of Carpenter & Kennedy (1994), five stages, 2N storage (GALAEXI
// Sec. 3.1, RK4-5): G <- A_s G + dt R(U, t + c_s dt);  U <- U + B_s G.
inline constexpr double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                                   -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
inline constexpr double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                                   1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                                   2277821191437.0 / 14882151754819.0};
inline constexpr double kRkC[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                                   2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

// RK4-14 of Niegemann, Diehl & Busch (2012), fourteen stages, 2N storage (the
// paper's alternative scheme, Sec. 3.1), to the published sixteen digits.
inline constexpr double kRk14A[14] = {0.0, -0.7188012108672410, -0.7785331173421570, -0.0053282796654044,
                                      -0.8552979934029281, -3.9564138245774565, -1.5780575380587385,
                                      -2.0837094552574054, -0.7483334182761610, -0.7032861106563359,
                                      0.0013917096117681, -0.0932075369637460, -0.9514200470875948,
                                      -7.1151571693922548};
inline constexpr double kRk14B[14] = {0.0367762454319673, 0.3136296607553959, 0.1531848691869027,
                                      0.0030097086818182, 0.3326293790646110, 0.2440251405350864,
                                      0.3718879239592277, 0.6204126221582444, 0.1524043173028741,
                                      0.0760894927419266, 0.0077604214040978, 0.0024647284755382,
                                      0.0780348340049386, 5.5059777270269628};
inline constexpr double kRk14C[14] = {0.0, 0.0367762454319673, 0.1249685262725025, 0.2446177702277698,
                                      0.2476149531070420, 0.2969311120382472, 0.3978149645802642,
                                      0.5270854589440328, 0.6981269994175695, 0.8190890835352128,
                                      0.8527059887098624, 0.8604711817462826, 0.8627060376969976,
                                      0.8734213127600976};

// A 2N-storage scheme: number of stages and coefficient tables.
struct RkScheme {
  int stages;
  const double* A;
  const double* B;
  const double* C;
};
inline RkScheme rk_scheme(int which) {
  return which == DG_RK414 ? RkScheme{14, kRk14A, kRk14B, kRk14C} : RkScheme{5, kRkA, kRkB, kRkC};
}

// Gas constants and derived coefficients, passed by value to kernels.
struct Gas {
  double gamma, R, Pr, mu;
  double gm1;        // gamma - 1
  double inv_gm1;    // 1 / (gamma - 1)
  double kappa;      // lambda / mu = c_p / Pr
  double inv_R;
  double mms_amp;
  double p_ref;      // reference pressure of the FP32 operator's momentum flux
  double E_ref;      // p_ref / (gamma - 1)
  int surf_flux;
  int source;
  int visc_law;      // DG_VISC_CONSTANT or DG_VISC_SUTHERLAND
  double inv_T_ref;  // Sutherland: 1 / T_ref
  double S_suth;     // Sutherland constant S
  double suth_c;     // T_ref + S
  // FP32 copies of the constants the FP32 operator uses, rounded once on the
  // host (set by set_float_copies)
  float f_gamma, f_gm1, f_inv_gm1, f_inv_R, f_mu, f_lam, f_p_ref, f_inv_T_ref, f_S_suth, f_suth_c, f_mms_amp;
};

inline void set_float_copies(Gas& g) {
  g.f_gamma = (float)g.gamma; g.f_gm1 = (float)g.gm1; g.f_inv_gm1 = (float)g.inv_gm1;
  g.f_inv_R = (float)g.inv_R; g.f_mu = (float)g.mu; g.f_lam = (float)(g.mu * g.kappa);
  g.f_p_ref = (float)g.p_ref;
  g.f_inv_T_ref = (float)g.inv_T_ref; g.f_S_suth = (float)g.S_suth; g.f_suth_c = (float)g.suth_c;
  g.f_mms_amp = (float)g.mms_amp;
}

// Face descriptor (master orientation): elements and local faces of both sides
// packed as e*8 + f, and the orientation code taking a master face node to the
// slave's node.
struct FaceInfo {
  int master;   // eM * 8 + fM
  int slave;    // eS * 8 + fS
  int flip;
  int pad;
};

// Operands of one stage launch.
struct StageArgs {
  const double* U;       // state (read)
  double* Uw;            // state written by the RK epilogue (== U in place) or NULL
  double* Gk;            // LSERK register or NULL
  double* Ut;            // time-derivative output (mode 0) or NULL
  const double* clock;   // device {t, dt}
  double c_stage, A, B;  // stage time fraction and LSERK coefficients
  int mode;              // 0: write Ut; 1: LSERK update
  // Element slots of the DG volume kernel: NULL, every element; else slot s <
  // *list_len is element list[s] (the DG elements when FV sub-cell elements
  // exist; both device memory, read at run time) and the other slots are idle
  const int* list = nullptr;
  const int* list_len = nullptr;
  int nfaces = 0;              // face slots (bound of the face ids; 0: 3 E, a conforming periodic mesh)
};

struct Ctx {
  int device = 0;
  int N = 0, n = 0, P = 0, NN = 0;
  int E = 0, nfaces = 0;
  dg_params prm{};
  Gas gas{};
  std::vector<double> x, w, D;   // host LGL basis
  double dt_factor = 1.0;        // time-step factor of the node set (Gauss: < 1)
  // device geometry
  double* d_D = nullptr;         // [n][n]
  double* d_metrics = nullptr;   // [E][10][P]: J a^d_l at row d*3+l, row 9 = 1/J
  double* d_J = nullptr;         // [E][P]
  double* d_X = nullptr;         // [E][3][P]
  double* d_mms = nullptr;       // [E][2][P] sin, cos of pi (x + y + z); manufactured source only
  double* d_facegeo = nullptr;   // [F][4][NN]: unit normal (3), surface element
  float* d_metrics_f = nullptr;  // FP32 copies for the FP32-operator path
  float* d_facegeo_f = nullptr;
  FaceInfo* d_faces = nullptr;   // [F]: the conforming faces, then the mortars' small and big sides
  int nfaces_conf = 0;           // conforming faces (the face kernel's range)
  // mortars (non-conforming faces, 2:1)
  int M = 0;
  int* d_mortars = nullptr;      // [M][20]: eB, fB, slot of the big side, then per quadrant eS, fS, flip, slot
  double* d_mortar_tab = nullptr;   // [2][n][n] interpolation to each half, [n] LGL weights
  double* d_mortar_virt = nullptr;  // [M][5][5][NN]: the lifting's neighbour state of each mortar side
  int* d_elem_face = nullptr;    // [E][6]: face_id * 16 + master * 8 + flip (own -> neighbour)
  int* d_elem_nbr = nullptr;     // [E][6]: e2 * 8 + f2
  // work buffers
  void* d_grad = nullptr;        // [E][12][P]: d phi / d x_l, phi = (u, v, w, T), row phi*3+l (operator type)
  void* d_fstar = nullptr;       // [F][5][NN]: surface flux times sJ, master orientation (operator type)
  // Gauss nodes only
  double* d_Uf = nullptr;        // [E][6][5][NN]: face values of U from each element
  double* d_gf = nullptr;        // [E][6][12][NN]: face values of the lifted gradients
  double* d_lgb = nullptr;       // Gauss basis table (layout GaussTab in dg_gauss.cu)
  double* d_red = nullptr;       // reduction partials [red_len + 1][9]; the last row holds the fold
  int red_len = 0;               // maximum number of partial rows
  double* d_w = nullptr;         // [n] quadrature weights of the node set
  double* d_modal = nullptr;     // [n][n] nodal -> orthonormal Legendre modes of the node set (indicator)
  // FV sub-cell elements (dg_fv.cu), allocated by the first dg_set_fv_mask
  bool fv_on = false;            // a mask is set: every stage runs the FV kernels
  bool fv_switch = false;        // the indicator sets the mask before every evaluation of R(U)
  int fv_sw_var = 2;             // its quantity (DG_IND_*) and log10 thresholds
  double fv_sw_up = 0.0, fv_sw_low = 0.0;
  int* d_fv_mask = nullptr;      // [E] 1: FV element
  int* d_fv_pin = nullptr;       // [E] 1: element with a mortar face, which stays DG (mortar meshes only)
  std::vector<char> fv_pin;      // the same on the host
  int* d_fv_lists = nullptr;     // [2E + 2]: DG elements, FV elements (ascending), their counts
  double* d_fv_tab = nullptr;    // V [n][n], V^-1 [n][n], L [n+1][n]
  double* d_fv_iJb = nullptr;     // [E][P] 1 / (sub-cell means of J)
  double* d_fv_S = nullptr;      // [E][3][n+1][NN][4] sub-face unit normals and areas
  double* d_fv_M = nullptr;      // [E][17][P] mean primitives and viscous flux tensors
  double* d_fv_Fb = nullptr;     // [F][5][NN] master-outward sub-face fluxes of faces with an FV side
  int* d_minmask = nullptr;      // bit a set: value a of the integrals is a minimum
  double* d_clock = nullptr;     // {t, dt}
  double* h_clock = nullptr;     // pinned staging for the clock
  double* h_out = nullptr;       // pinned staging for reductions
  // adjoint work buffers (allocated on first use)
  double* d_adj_qbar = nullptr;  // [E][5][P]
  double* d_adj_gbar = nullptr;  // [E][12][P]
  double* d_adj_gtil = nullptr;  // [E][12][P]
  double* d_adj_fseed = nullptr; // [F][2][5][NN]
  double* d_adj_face = nullptr;  // [F][2][17][NN]
  double* d_adj_mu = nullptr;    // block partials of d/dmu
  double* d_adj_stage = nullptr; // [5][E][5][P] stage states of one step
  double* d_adj_mx = nullptr;    // [M][5][4][NN] mortar sides' lifting-transpose terms
  double* d_adj_lgf = nullptr;   // [E][6][9][NN] Gauss nodes: lifting surface sums, face-value adjoints
  double* d_adj_work = nullptr;  // [4][E][5][P]: work state, G, G-bar, VJP scratch
  // host-buffer path
  double* d_U = nullptr;
  double* d_G = nullptr;
  // captured RK graph
  cudaGraphExec_t graph = nullptr;
  const double* graph_U = nullptr;
  const double* graph_G = nullptr;
  int graph_nsteps = 0;
  std::string err;
};

// Launchers implemented per polynomial degree (dg_operator.cu).  With
// latency_ok the FP64 lifting and volume launchers take the latency kernels
// (dg_latency.cu) for meshes too small to fill the GPU; the ensemble passes
// false, so its results do not depend on its tuned plan.
cudaError_t launch_lift(const Ctx& c, const double* U, cudaStream_t s, bool latency_ok = true);
cudaError_t launch_lift_fp64(const Ctx& c, const double* U, cudaStream_t s);   // diagnostics: always FP64
cudaError_t launch_face(const Ctx& c, const double* U, cudaStream_t s, bool latency_ok = true);
cudaError_t launch_volume(const Ctx& c, const StageArgs& a, cudaStream_t s, bool latency_ok = true);
// Latency kernels (dg_latency.cu): FP64, LGL, N <= 3, E (N+1)^3 <= kLatencyNodes.
constexpr long kLatencyNodes = 16384;
bool use_latency_kernels(const Ctx& c);
cudaError_t setup_latency(int N);
cudaError_t launch_lift_lat(const Ctx& c, const double* U, cudaStream_t s);
cudaError_t launch_volume_lat(const Ctx& c, const StageArgs& a, cudaStream_t s);
cudaError_t launch_face_lat(const Ctx& c, const double* U, cudaStream_t s);   // LLF surface flux only
cudaError_t setup_kernels(int N);
// Gauss-node operator (dg_gauss.cu); gx (may be NULL) receives the Gauss nodes
void gauss_table(int N, const std::vector<double>& xl, std::vector<double>& tab, std::vector<double>* gx = nullptr,
                 std::vector<double>* gw = nullptr);
double gauss_dt_factor(int N, const std::vector<double>& xl, const std::vector<double>& wl,
                       const std::vector<double>& Dl, const std::vector<double>& tab);
cudaError_t setup_gauss(int N);
cudaError_t gauss_geometry(Ctx& c, int* d_bad, cudaStream_t s);
// fp64: the FP64 lifting whatever the operator type (diagnostics)
cudaError_t launch_lift_lg(const Ctx& c, const double* U, cudaStream_t s, bool fp64 = false);
cudaError_t launch_face_lg(const Ctx& c, cudaStream_t s);
cudaError_t launch_volume_lg(const Ctx& c, const StageArgs& a, cudaStream_t s);
cudaError_t setup_volume(int N);

// FV sub-cell operator (dg_fv.cu): tables of the node set, the once-per-context
// geometry (Jb, area vectors) and one stage (means, sub-face fluxes, the DG
// volume kernel with the FV elements skipped, the FV residual and update).
void fv_tables(int N, const std::vector<double>& x, std::vector<double>& tab);
cudaError_t fv_setup(const Ctx& c, cudaStream_t s);
cudaError_t launch_fv_lists(const Ctx& c, cudaStream_t s);
cudaError_t launch_fv_stage(const Ctx& c, const StageArgs& a, cudaStream_t s);

// Mortars (dg_mortar.cu): the lifting's neighbour states of the mortar sides
// (before the lifting kernel) and the mortar fluxes (after the lifting).
cudaError_t launch_mortar_lift(const Ctx& c, const double* U, cudaStream_t s);
cudaError_t launch_mortar_flux(const Ctx& c, const double* U, cudaStream_t s);

// Modal troubled-cell indicator (dg_indicator.cu).
void modal_table(int N, const std::vector<double>& x, const std::vector<double>& w, bool lobatto,
                 std::vector<double>& T);
// switch_mask: flag is the FV mask, updated with hysteresis (log_thresh the
// upper, log_low the lower threshold) and the admissibility rule.
cudaError_t launch_indicator(const Ctx& c, const double* U, int var, double log_thresh, double* eta, int* flag,
                             cudaStream_t s, bool switch_mask = false, double log_low = 0.0);
// Before an evaluation of R(U) with automatic switching: the mask from the
// indicator of U, then the element lists (nothing without switching).
cudaError_t launch_fv_switch(const Ctx& c, const double* U, cudaStream_t s);

// Geometry kernels (dg_geometry.cu).
cudaError_t build_geometry(Ctx& c, const double* d_xgeo, int ngeo, int* d_bad, cudaStream_t s);
cudaError_t launch_to_float(const double* a, float* b, size_t n, cudaStream_t s);

// Diagnostics kernels (dg_diag.cu).
cudaError_t launch_integrals(Ctx& c, const double* U, cudaStream_t s);
cudaError_t launch_max_dt(Ctx& c, const double* U, double cfl, double dfl, cudaStream_t s);
cudaError_t launch_initial_state(Ctx& c, int kind, double prm0, double* U, cudaStream_t s);
cudaError_t launch_mms_phase(Ctx& c, cudaStream_t s);
cudaError_t launch_set_clock(double* clock, double t, double dt, cudaStream_t s);
cudaError_t launch_clock_advance(double* clock, cudaStream_t s);
int reduction_rows(const Ctx& c);   // partial rows used by the last reduction

// Adjoint kernels (dg_adjoint.cu).
cudaError_t setup_adjoint(int N);
int adjoint_mu_partials(const Ctx& c);
cudaError_t launch_vjp(const Ctx& c, const double* U, const double* lam, double* out, double* dJdmu, double mu_scale,
                       cudaStream_t s);
cudaError_t launch_axpby(double* y, const double* x, double a, double b, size_t len, cudaStream_t s);
cudaError_t launch_kinetic(const Ctx& c, const double* U, double* grad, double* d_out, cudaStream_t s);
constexpr int kRedValues = 9;

// Bounds checks of the indirect gathers (dg_check.cuh): each file with such
// gathers keeps its own error word; the readers return it and clear it (0 in
// normal builds).
unsigned long long bounds_word_adjoint();
unsigned long long bounds_word_ensemble();
unsigned long long bounds_word_gauss();
unsigned long long bounds_word_geometry();
unsigned long long bounds_word_latency();
unsigned long long bounds_word_fv();
unsigned long long bounds_word_mortar();
unsigned bulk_word_volume();     // bulk-copy waits that gave up (volume kernels)
unsigned bulk_word_ensemble();
unsigned long long bounds_word_operator();
unsigned long long bounds_word_volume();
// Checked builds: wait for the work on stream s and describe the first
// recorded out-of-range index in msg; returns true if there was one.  Normal
// builds: returns false at once.
bool bounds_failed(cudaStream_t s, char* msg, size_t len);

}  // namespace dg
