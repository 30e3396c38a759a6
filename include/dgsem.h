/*
 * dgsem.h -- C ABI of the GB300 (sm_103a) split-form DGSEM hot path.
 *
 * The operator is the semi-discrete DG time derivative U_t = R(U) of the 3-D
 * compressible Navier-Stokes-Fourier equations (GALAEXI, Sec. 3.1, Eq. 1) on
 * curvilinear, unstructured hexahedral meshes, discretised by the DGSEM on
 * Legendre-Gauss-Lobatto nodes (Sec. 3.1, Eq. 2) with
 *   - BR1 lifting of the primitive gradients (Sec. 3.1, Eq. 3),
 *   - a Riemann flux plus the averaged viscous flux on faces (Sec. 3.1),
 *   - the entropy-stable split-form volume integral with the two-point flux of
 *     Chandrashekar (2013) and curvilinear metric terms (Sec. 3.1),
 *   - the surface integral and the Jacobian scaling,
 * advanced by the five-stage low-storage RK4-5 of Carpenter & Kennedy (1994)
 * (Sec. 3.1, "RK4-5").
 *
 * Conventions for every entry point:
 *   - State arrays are caller-owned DEVICE buffers of float64, element-blocked
 *     and contiguous: U[e][v][k][j][i], v = (rho, rho u, rho v, rho w, rho E),
 *     i fastest, (N+1) nodes per direction; dg_state_len() doubles in total.
 *     They must be 16-byte aligned.
 *   - Calls are stream-ordered on the given CUDA stream (a cudaStream_t;
 *     NULL = legacy default stream) and return without synchronising, unless
 *     documented otherwise.
 *   - Every call returns a dg_status; on failure dg_last_error() describes it.
 *     The library never aborts the process and never falls back to the CPU.
 *   - A context owns the work buffers (lifted gradients, face fluxes, clock)
 *     of the calls made on it, so those calls must not overlap on the GPU:
 *     issue them on one stream, or order them with events.  Different
 *     contexts are independent.  A context is not thread-safe.
 */
#ifndef DGSEM_H
#define DGSEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx;           /* opaque: geometry, face maps, work buffers */
typedef struct CUstream_st* dg_stream;  /* identical to cudaStream_t */

typedef enum {
  DG_OK = 0,
  DG_EINVAL = 1,        /* bad argument (null pointer, size, range) */
  DG_ENOMEM = 2,        /* device allocation failed */
  DG_ECUDA = 3,         /* a CUDA runtime call failed */
  DG_EMESH = 4,         /* mesh rejected: connectivity or a non-positive Jacobian */
  DG_ENONFINITE = 5,    /* a reduction met NaN or Inf */
  DG_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
  DG_EUNSUPPORTED = 7   /* polynomial degree or option not built */
} dg_status;

enum { DG_FLUX_LLF = 0, DG_FLUX_EC = 1, DG_FLUX_ROE = 2 };   /* surface Riemann flux: local Lax-Friedrichs,
                                                              entropy-conservative two-point flux, Roe with
                                                              the Harten-Hyman entropy fix (Sec. 3.1) */
enum { DG_FP64 = 0, DG_FP32OP = 1 };              /* operator arithmetic */
enum { DG_SOURCE_NONE = 0, DG_SOURCE_MMS = 1 };   /* volume source term */
enum { DG_NODES_LGL = 0, DG_NODES_LG = 1 };   /* collocation nodes (Sec. 3.1): Legendre-Gauss-Lobatto with the
                                                  entropy-stable split form, or Legendre-Gauss with the standard
                                                  weak form (Eqs. 2-3); LG is FP64 only */
enum { DG_RK45 = 0, DG_RK414 = 1 };   /* 2N-storage time schemes of Sec. 3.1: LSERK4-5 (Carpenter & Kennedy
                                         1994) or RK4-14 (Niegemann, Diehl & Busch 2012); the stage update
                                         is the same, the stage count 5 or 14 */
enum { DG_VISC_CONSTANT = 0, DG_VISC_SUTHERLAND = 1 };   /* viscosity law: constant mu, or Sutherland's law
                                                           mu (T/T_ref)^(3/2) (T_ref + S)/(T + S) at each
                                                           node's temperature (the law of the dissipation
                                                           diagnostic, Sec. 4.2) */
enum { DG_IC_TGV = 0, DG_IC_MMS = 1 };            /* built-in initial states */
enum { DG_IND_RHO = 0, DG_IND_P = 1, DG_IND_RHOP = 2 };   /* quantity of the troubled-cell indicator */

/*
 * Mesh (Sec. 3.1: non-overlapping hexahedra, each the image of E = [-1,1]^3
 * under a mapping chi).  Host arrays, read only during dg_init.
 *   xgeo[e][c][k][j][i]: coordinate c of element e at the equispaced reference
 *       point (-1 + 2i/ngeo, -1 + 2j/ngeo, -1 + 2k/ngeo) of its local frame.
 *   face_nbr[e][f][0..2] = (e2, f2, flip): local face f = 2d + s (d: reference
 *       direction, s = 0 at -1, 1 at +1) of e touches local face f2 of e2.  A
 *       face node is (p, q) along the two other directions in increasing
 *       order; flip maps (p, q) on (e, f) to (p2, q2) on (e2, f2):
 *       (a, b) = flip & 1 ? (q, p) : (p, q);  p2 = flip & 2 ? N - a : a;
 *       q2 = flip & 4 ? N - b : b.  Every face must have a neighbour
 *       (periodic meshes); the relation must be reciprocal.
 *   Mortars (Sec. 3.2.2, Algorithm 1: non-conforming faces, 2:1): n_mortars
 *       records mortars[m][0..13] = (eB, fB, eS0, fS0, flip0, ..., eS3,
 *       fS3, flip3): big face fB of element eB is split into quadrants
 *       k = a + 2b (a, b: the halves along its face-local p, q directions),
 *       quadrant k being local face fS_k of element eS_k; flip_k maps a node
 *       (p, q) of the quadrant, numbered along the big face's directions, to
 *       the small face's own node.  face_nbr[eB][fB] = (-1 - m, 0, 0) and
 *       face_nbr[eS_k][fS_k] = (-1 - m, k, 0).  The quadrants must be the
 *       exact quarters of the big face (affine faces).  n_mortars = 0 and
 *       mortars = NULL for a conforming mesh.  Either node set (the maps use
 *       its basis and quadrature); the FV sub-cell operator needs a
 *       conforming mesh.
 */
typedef struct {
  int32_t n_elems;
  int32_t ngeo;               /* >= 1 */
  const double* xgeo;
  const int32_t* face_nbr;
  int32_t n_mortars;          /* >= 0 */
  const int32_t* mortars;     /* [n_mortars][14] or NULL */
} dg_mesh;

/* Gas and discretisation (Sec. 3.1, Eq. 1: perfect gas p = (gamma-1) rho eps,
 * p = rho R T, Newtonian stress with constant mu, Fourier heat flux with
 * lambda = mu c_p / Pr). */
typedef struct {
  int32_t N;                  /* polynomial degree, 1..9 */
  double gamma, R, Pr, mu;
  int32_t surf_flux;          /* DG_FLUX_LLF, DG_FLUX_EC or DG_FLUX_ROE */
  int32_t precision;          /* DG_FP64 or DG_FP32OP */
  int32_t source;             /* DG_SOURCE_NONE or DG_SOURCE_MMS */
  double mms_amp;             /* amplitude A of rho = 2 + A sin(pi(x+y+z-t)) */
  double p_ref;               /* DG_FP32OP: constant pressure taken out of the momentum flux (it has no
                                 discrete divergence); the background pressure of a low-Mach flow keeps
                                 its FP32 rounding out of the momentum equations.  Ignored in FP64. */
  int32_t visc_law;           /* DG_VISC_CONSTANT (mu above) or DG_VISC_SUTHERLAND (mu = mu(T_ref)) */
  double T_ref, S_suth;       /* Sutherland reference temperature (> 0) and constant (>= 0) */
  int32_t nodes;              /* DG_NODES_LGL or DG_NODES_LG */
  int32_t rk_scheme;          /* DG_RK45 or DG_RK414 (dg_rk_step, dg_advance_host) */
} dg_params;

/* Build a context on CUDA device `device`: basis of the node set, geometry
 * (node positions, curl-form metric terms, Jacobian, face normals) computed on
 * the GPU from the mesh, face maps and work buffers.  On Gauss nodes the
 * metric terms are those of the LGL construction evaluated at the Gauss nodes
 * and face points (Sec. 3.1 leaves this open).  Synchronous.
 * Errors: DG_EINVAL (null/size, unknown option, constants out of range),
 * DG_EUNSUPPORTED (N outside 1..9), DG_EMESH
 * (connectivity out of range or not reciprocal, Jacobian <= 0 at a node),
 * DG_ENOMEM, DG_ECUDA.  On failure *out is NULL. */
dg_status dg_init(const dg_mesh* mesh, const dg_params* prm, int device, dg_ctx** out);

/* Free everything the context owns.  Synchronises the device. */
dg_status dg_destroy(dg_ctx* ctx);

/* Number of doubles in one state array: n_elems * 5 * (N+1)^3. */
size_t dg_state_len(const dg_ctx* ctx);

/* Ut = R(U, t) (Sec. 3.1, Eqs. 2-3 in strong form).  dU, dUt: device, may not
 * alias. */
dg_status dg_time_derivative(dg_ctx* ctx, const double* dU, double* dUt, double t, dg_stream stream);

/* nsteps steps of the context's 2N-storage scheme (LSERK4-5 or RK4-14,
 * Sec. 3.1) in place: per stage s,
 *   G <- A_s G + dt R(U, t + c_s dt);  U <- U + B_s G,
 * with G (device, dg_state_len doubles, caller-owned scratch) zeroed at the
 * start of every step.  Both operations run in FP64 in either precision; with
 * DG_FP32OP the register holds G/dt (G/dt <- A_s G/dt + R; U <- U + (B_s dt)
 * G/dt), which makes both of them fused multiply-adds.  The sequence of
 * launches is captured once per (dU, dG, nsteps) into a CUDA graph and
 * replayed. */
dg_status dg_rk_step(dg_ctx* ctx, double* dU, double* dG, double t, double dt, int32_t nsteps,
                     dg_stream stream);

/* End-to-end variant with HOST buffers: copies hU (host, dg_state_len doubles)
 * to the device, advances nsteps steps, and copies the result back into hU.
 * Device state and register live in the context.  Synchronises the stream. */
dg_status dg_advance_host(dg_ctx* ctx, double* hU, double t, double dt, int32_t nsteps, dg_stream stream);

/* Volume integrals with the LGL quadrature (Sec. 4.2 diagnostics), host_out8 =
 * { int rho, int rho u, int rho v, int rho w, int rho E,
 *   E_k = 1/(2|Omega|) int rho |u|^2, eps = 1/|Omega| int mu(T) |omega|^2 (vorticity
 *   from the BR1-lifted velocity gradient; with Sutherland's law a node with
 *   T <= 0, possible only inside an FV element, adds nothing), min p }, in
 *   units rho0 = U0 = L = 1.
 * Synchronises the stream.  DG_ENONFINITE if any value is NaN/Inf. */
dg_status dg_integrals(dg_ctx* ctx, const double* dU, double* host_out8, dg_stream stream);

/* Time step of Sec. 3.1 (CFL number 0.9 for the convective and for the
 * viscous limit there):
 * dt = min(cfl * 2/((2N+1) max_nodes sum_d lambda_d),
 *          dfl * (2/(2N+1))^2 / max_nodes (mu_eff sum_d |Ja^d|^2 / J^2)),
 * lambda_d = (|u . Ja^d| + c |Ja^d|) / J, mu_eff = max(4/3, gamma/Pr) mu / rho.
 * Nodes of FV sub-cell elements whose density or pressure is not positive
 * (the nodal polynomial of admissible sub-cell means can have them) do not
 * enter.  Synchronises the stream.  DG_ENONFINITE if a node's state gives a
 * NaN or infinite speed (NaN/Inf in the state, non-positive density or
 * pressure outside FV elements). */
dg_status dg_max_dt(dg_ctx* ctx, const double* dU, double cfl, double dfl, double* host_dt, dg_stream stream);

/* Built-in initial states at the LGL nodes: DG_IC_TGV (Sec. 4.2, Eq. 6) with
 * rho0 = U0 = L = R = 1 and p0 = prm0; DG_IC_MMS at time prm0. */
dg_status dg_initial_state(dg_ctx* ctx, int32_t kind, double prm0, double* dU, dg_stream stream);

/* Modal troubled-cell indicator of Persson & Peraire (2006), the detector of
 * the FV sub-cell shock capturing (Sec. 3.1): per element, the quantity q
 * (var: DG_IND_RHO, DG_IND_P or DG_IND_RHOP = rho p) at the context's nodes is
 * expanded in the orthonormal Legendre basis sqrt((2m+1)/2) P_m per
 * direction, and
 *   dEta[e] = sum_{max(a,b,c) = N} qh_abc^2 / sum_abc qh_abc^2
 * (the energy share of the modes that truncation to degree N-1 in every
 * direction removes; 0 for a field of degree < N in each direction, 1 for a
 * pure top mode; 0 where q vanishes).  dFlag (may be NULL) receives 1 where
 * eta > 0 and log10(eta) > log10_threshold, else 0 (FP64 decision); it can
 * be passed to dg_set_fv_mask as it is.  dU: device state; dEta: device,
 * n_elems doubles; dFlag: device, n_elems int32.  DG_EINVAL for a null
 * argument or an unknown var.  Does not synchronise. */
dg_status dg_indicator(dg_ctx* ctx, const double* dU, int32_t var, double log10_threshold, double* dEta,
                       int32_t* dFlag, dg_stream stream);

/* FV sub-cell elements of the shock capturing (Sec. 3.1: a second-order
 * finite-volume scheme on (N+1)^3 integral means per element for the
 * elements the troubled-cell indicator selects).  dMask: device, n_elems
 * int32; element e is advanced by the FV operator where dMask[e] != 0, by the
 * DG operator elsewhere, in every later dg_time_derivative and dg_rk_step
 * (also in an RK graph captured before: the kernels read the mask at run
 * time).  The mask is copied on `stream` (the caller may reuse dMask after
 * the stream has passed this call).  dMask = NULL switches the FV operator
 * off (the pure DG operator, bit for bit).
 * The FV scheme: J-weighted sub-cell means of the nodal interpolant on the
 * (N+1)^3 equal sub-cubes of the reference element, sub-face area vectors
 * integrated exactly from the metric terms, minmod-limited linear
 * reconstruction of (rho, u, v, w, p), local Lax-Friedrichs sub-face fluxes
 * minus the central viscous flux of the sub-cell means (mean BR1 gradients);
 * a face between a DG and an FV element is evaluated on sub-faces, the DG side
 * entering with the means of its trace over each sub-face (its face nodes, or
 * on Gauss nodes its values interpolated to the face) and taking the sub-face
 * fluxes in nodal form, with the same face integral.  The first call allocates
 * about 18 + 12 (N+2)/(N+1) doubles per node plus 5 per face node and sets
 * up the sub-cell geometry.  FP64 operator (either node set): DG_EUNSUPPORTED
 * otherwise.  On a mesh with mortars an element with a mortar face stays a DG
 * element (the mortar maps act on DG traces): a mask that flags one gets
 * DG_EUNSUPPORTED, and the call then synchronises the stream to check the
 * mask on the host.  The adjoint entry points return DG_EUNSUPPORTED while a
 * mask is set.  dg_max_dt keeps the DG time-step restriction.  Does not
 * synchronise on conforming meshes. */
dg_status dg_set_fv_mask(dg_ctx* ctx, const int32_t* dMask, dg_stream stream);

/* Automatic switching of troubled cells between the DG and the FV sub-cell
 * operator (Sec. 3.1: the modal indicator selects the elements the FV scheme
 * takes over; Sec. 3.2.2 lists the switch as a kernel step of its own).
 * Before every later evaluation of R(U) (dg_time_derivative, each stage of
 * dg_rk_step, also inside its captured graph) the indicator of dg_indicator
 * (quantity var) of the evaluated state sets the FV mask in place: element e
 * becomes an FV element where log10(eta_e) > log10_upper or where its nodal
 * state is not admissible (density or pressure not positive at a node), a DG
 * element where log10(eta_e) < log10_lower and every node is admissible, and
 * keeps its representation in between (hysteresis; FP64 decisions); an
 * element with a mortar face stays DG.  The
 * state stays nodal in both representations, so a switch moves no data.  The
 * mask starts from the one set by dg_set_fv_mask, else all DG; dg_set_fv_mask
 * (NULL) clears it while switching is on.  var < 0 turns switching off and
 * keeps the mask in effect.  DG_EINVAL for an unknown var or thresholds that
 * are not finite with upper >= lower; DG_EUNSUPPORTED with the FP32
 * operator.  Allocates as dg_set_fv_mask does.  Does not synchronise. */
dg_status dg_set_fv_switch(dg_ctx* ctx, int32_t var, double log10_upper, double log10_lower, dg_stream stream);

/* The FV mask in effect (1: FV element), into dMask (device, n_elems int32);
 * all zero when no FV elements are set.  Stream-ordered after the launches
 * before it, so after an RK call it holds the mask of its last stage. */
dg_status dg_get_fv_mask(dg_ctx* ctx, int32_t* dMask, dg_stream stream);

/* Physical node positions X[e][c][k][j][i] (device, n_elems*3*(N+1)^3). */
dg_status dg_node_coords(dg_ctx* ctx, double* dX, dg_stream stream);

/* Geometry as used by the kernels: Ja[e][d][l][P] (J a^d, component l) and
 * J[e][P]; either pointer may be NULL.  Device buffers. */
dg_status dg_geometry(dg_ctx* ctx, double* dJa, double* dJ, dg_stream stream);

/* ---- Discrete adjoint (FP64 contexts) -------------------------------------
 * Hand-written reverse-mode kernels of the discrete operator: the exact
 * transpose of the FP64 R(U) of dg_time_derivative (branches of |.| and the
 * log-mean switch follow the primal state; at a kink of the LLF speed maximum
 * the mean of the one-sided derivatives is taken).  The paper has no
 * adjoint; these entries exist for gradient-based use of the solver.  Built
 * for both node sets (on Gauss nodes the transposes of the weak form and of
 * the face prolongations), all three surface fluxes (the Roe flux
 * differentiated on dual numbers, its kinks by the value) and constant or
 * Sutherland viscosity (the derivative of mu(T) enters through the state) on
 * conforming or 2:1 mortar meshes (the transposes of the mortars'
 * interpolation and projection) without FV sub-cell elements, for both time
 * schemes; other contexts (the FP32 operator, FV elements) get
 * DG_EUNSUPPORTED.
 * dJdmu, where present, is a device double that is ACCUMULATED (+=) with
 * lambda . dR/dmu, mu the constant viscosity or Sutherland's reference
 * viscosity (R is linear in it); NULL skips it. */

/* dout = (dR/dU)^T dv at dU (all device [state_len]); dout may alias dv. */
dg_status dg_time_derivative_vjp(dg_ctx* ctx, const double* dU, const double* dv, double* dout, double* dJdmu,
                                 double t, dg_stream stream);

/* Adjoint of one step (the context's scheme) from dU_n (state at the step's start, time t):
 * dlam_n = (dU_{n+1}/dU_n)^T dlam_np1 (may alias), dJdmu += the step's
 * lambda . dU_{n+1}/dmu.  The stage states are recomputed from dU_n.
 * DG_EINVAL if either adjoint array is dU_n. */
dg_status dg_adjoint_step(dg_ctx* ctx, const double* dU_n, const double* dlam_np1, double* dlam_n, double* dJdmu,
                          double t, double dt, dg_stream stream);

/* Adjoint of nsteps steps (the context's scheme) from dU0 at t0: dlam0 = (dU_T/dU_0)^T dlamT
 * (may alias), dJdmu += lambda . dU_T/dmu, with binomial checkpointing
 * (Griewank 1992): at most max_snapshots stored states (>= 1, the initial
 * state included; min(max_snapshots, nsteps) device buffers of one state
 * each are allocated for the call), forward recomputation in between, the
 * least number of recomputed forward steps for that many states.
 * host_counts2 (may be NULL) receives {recomputed forward steps, adjoint
 * steps}.  DG_EINVAL if either adjoint array is dU0.  Synchronises the
 * stream. */
dg_status dg_adjoint_solve(dg_ctx* ctx, const double* dU0, const double* dlamT, double* dlam0, double* dJdmu,
                           double t0, double dt, int32_t nsteps, int32_t max_snapshots, int64_t* host_counts2,
                           dg_stream stream);

/* The counts dg_adjoint_solve reports for (nsteps, max_snapshots), from its
 * schedule run without a device: host_counts2 (host, 2 values) receives
 * {recomputed forward steps, adjoint steps}.  With s = min(max_snapshots,
 * nsteps) states the first is t(nsteps, s) = r nsteps - C(s + r, s + 1), r the
 * least integer with C(s + r, s) >= nsteps (t = n (n - 1) / 2 for s = 1); the
 * second is nsteps.  DG_EINVAL for nsteps < 0, max_snapshots < 1 or a NULL
 * pointer; DG_ENOMEM if the host cannot hold the schedule's interval stack
 * (up to min(max_snapshots, nsteps) entries of 12 bytes).  Needs no GPU and
 * no context. */
dg_status dg_checkpoint_schedule(int32_t nsteps, int32_t max_snapshots, int64_t* host_counts2);

/* Objective J = sum_nodes w_i w_j w_k J 1/2 rho |u|^2 (the node set's
 * quadrature of the volume-integrated kinetic energy) into *host_J; dgrad (device, may be NULL)
 * receives dJ/dU.  Synchronises the stream. */
dg_status dg_kinetic_energy(dg_ctx* ctx, const double* dU, double* dgrad, double* host_J, dg_stream stream);

/* Change the viscosity mu of a context (the constant one, or Sutherland's
 * reference value; e.g. for derivative checks). */
dg_status dg_set_viscosity(dg_ctx* ctx, double mu);

/* ---- Batched ensemble (independent runs advanced together) ----------------
 * An ensemble groups existing contexts on one device (each with its own mesh,
 * N, gas constants; all with the same precision).  Members of equal N are
 * advanced by persistent kernels that walk a tile table over all of those
 * members; the nsteps step sequence of all members is one CUDA graph, in
 * which the independent units (a tile-table group, or one member run by the
 * single-context kernels where those won the tuning) are parallel branches.
 * Tile shape (elements per block), grid sizes and the per-member alternative
 * are chosen per N by an autotuner on the first dg_ensemble_step (timing the
 * candidates on the members' data without changing their states) and cached
 * in the text file tune_cache_path (NULL: no cache), keyed by GPU name, N and
 * precision -- not by member sizes: ensembles of very different sizes should
 * use different cache files. */
typedef struct dg_ensemble dg_ensemble;

/* The members stay owned by the caller and must outlive the ensemble.
 * DG_EINVAL if a member is NULL, appears twice (its work buffers would be
 * shared by two members) or is on another device or precision;
 * DG_EUNSUPPORTED for a member with another time scheme than the first
 * member's (the steps of all members follow one scheme, LSERK4-5 or RK4-14).
 * Members on LGL nodes with a conforming mesh and no FV elements run by the
 * tile-table kernels; members on Gauss nodes, on a mesh with mortars or with
 * FV elements (set before the ensemble is created) run as single-member
 * units of the same graph with their own stage kernels. */
dg_status dg_ensemble_create(dg_ctx* const* members, int32_t n, const char* tune_cache_path, dg_ensemble** out);
dg_status dg_ensemble_destroy(dg_ensemble* ens);

/* nsteps steps of the members' time scheme for every member r: state dU[r] with register dG[r]
 * (device arrays of the member's dg_state_len), from time t[r] with step
 * dt[r] (host arrays of n doubles).  The same steps per member as dg_rk_step
 * (the ensemble does not use the latency kernels of small meshes).
 * DG_EINVAL if a pointer is NULL or the 2n arrays are not all distinct;
 * DG_EUNSUPPORTED while a member run by the tile-table kernels has FV
 * sub-cell elements (set after the ensemble was created).
 * Waits for earlier work on `stream`, then enqueues one graph launch. */
dg_status dg_ensemble_step(dg_ensemble* ens, double* const* dU, double* const* dG, const double* t,
                           const double* dt, int32_t nsteps, dg_stream stream);

/* The tuned plan as JSON text (per N: members, elements per block, grids). */
dg_status dg_ensemble_plan(const dg_ensemble* ens, char* buf, size_t len);
const char* dg_ensemble_last_error(const dg_ensemble* ens);

/* Measurement helper: runs `reps` LSERK stages on (dU, dG) (state advanced
 * with dt) and times each stage kernel with CUDA events on `stream`;
 * host_ms3 = average milliseconds per launch of { lifting, face flux,
 * volume + update }.  Synchronises the stream. */
dg_status dg_profile_stages(dg_ctx* ctx, double* dU, double* dG, double dt, int32_t reps, float* host_ms3,
                            dg_stream stream);

/* Measurement helper: throughput of dependent-chain FP64 DFMA and FP32 FFMA
 * on `device` in TFLOP/s (FMA = 2 flop), host_out2 = {fp64, fp32}.  Used as
 * the arithmetic roof for the FP64-pipe-bound kernels.  Synchronous. */
dg_status dg_probe_peaks(int device, double* host_out2);

/* Check of the FP64 <-> FP32 conversions the FP32 operator uses (integer
 * operations on the bit patterns; no counterpart in the paper, which does not
 * describe the conversion).  For the n device values d_x: d_f[0..n) = the
 * operator's FP32 narrowing, d_f[n..2n) = the hardware round-to-nearest
 * conversion, d_d[0..n) = the operator's widening of d_f[0..n), d_d[n..2n) =
 * the hardware widening of the same.  All pointers are device memory owned
 * by the caller; d_f holds 2n floats and d_d 2n doubles.  Synchronises the
 * stream.  DG_EINVAL for n < 0 or null pointers with n > 0. */
dg_status dg_check_conversions(const double* d_x, int32_t n, float* d_f, double* d_d, dg_stream stream);

/* Check of the reciprocals the operator kernels use instead of divisions (no
 * counterpart in the paper).  For the n device values d_x:
 *   d_d[0..n)   the FP64 operator's 1/x: hardware approximation
 *               (rcp.approx.ftz.f64) refined by one cubic Newton-Raphson step,
 *               within 1 ulp of the correctly rounded 1/x;
 *   d_d[n..2n)  the same refined by one quadratic step, relative error below
 *               2^-38 (used where the error is damped, e.g. 1/(rho_a + rho_b)
 *               of the log-mean series);
 *   d_d[2n..3n) the adjoint kernels' 1/x (the cubic form);
 *   d_f[0..n), d_f[n..2n)  the FP32 operator's 1/x of x rounded to FP32 (the
 *               hardware approximation, within 1 FP32 ulp).
 * Valid for positive normal x with a normal reciprocal (the operators' densities,
 * pressures and their sums): the .ftz forms flush subnormals, so a subnormal
 * 1/x becomes 0 and a zero or subnormal x gives a non-finite result.  All
 * pointers are caller-owned device memory (d_d 3n doubles, d_f 2n floats).
 * Synchronises the stream.  DG_EINVAL for n < 0 or null pointers with n > 0. */
dg_status dg_check_reciprocals(const double* d_x, int32_t n, double* d_d, float* d_f, dg_stream stream);

/* Conservation totals sum_nodes w_i w_j w_k J q_v (v = rho, rho u, rho v,
 * rho w, rho E), the first five values of dg_integrals, for callers that may
 * not allocate device memory while they run: a host framework that owns every
 * device buffer and only lends inputs and outputs to foreign code, or an
 * application that keeps the allocator out of its time loop.  The paper has
 * no counterpart; this entry exists for such callers.
 *   dU: device state [n_elems][5][P]; dJ: device Jacobian [n_elems][P] at the
 *   context's nodes (dg_geometry); N: degree 1..9; nodes: DG_NODES_LGL or
 *   DG_NODES_LG, the node set of the context the state belongs to (its
 *   quadrature weights are used); dOut5: device, receives 5 doubles.
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its only
 * scratch is a fixed device array of n_elems <= 131072 rows of 5 doubles
 * (5 MiB) that every GPU loading the library holds until the process exits;
 * larger meshes are rejected with DG_EINVAL.  The array is shared by all
 * calls on a device and keeps the last call's contents, so calls that
 * overlap on the GPU (other streams, other threads) race.  The first call on
 * each device looks up the array's device address with that device current
 * (cudaGetSymbolAddress) and keeps it; make that first call before any stream
 * capture.  The kept address does not survive cudaDeviceReset (nor does any
 * context of this library).  Runs on the current device; `stream` must be a
 * stream of that device (DG_EINVAL otherwise).  Does not synchronise. */
dg_status dg_conserved_totals_noalloc(const double* dU, const double* dJ, int32_t N, int32_t nodes,
                                      int32_t n_elems, double* dOut5, dg_stream stream);

/* Human-readable description of the last error on ctx (or of the last failed
 * dg_init when ctx is NULL).  Never NULL. */
const char* dg_last_error(const dg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* DGSEM_H */
