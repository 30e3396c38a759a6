// C ABI of the discrete adjoint: VJP of R(U), adjoint of one LSERK4-5 step,
// the adjoint of a whole time interval with binomial checkpointing, the
// kinetic-energy objective, and the viscosity setter used for d/dmu checks.
#include <cstdio>
#include <new>
#include <vector>

#include "dg_internal.h"

namespace dg {

static dg_status afail(Ctx* c, dg_status st, const char* what, cudaError_t e = cudaSuccess) {
  char buf[512];
  if (e != cudaSuccess) std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  else std::snprintf(buf, sizeof buf, "%s", what);
  if (c) c->err = buf;
  return st;
}

#define ADJ_CUDA(call, ctx, what)                                                               \
  do {                                                                                          \
    cudaError_t _e = (call);                                                                    \
    if (_e != cudaSuccess)                                                                      \
      return afail(ctx, _e == cudaErrorMemoryAllocation ? DG_ENOMEM : DG_ECUDA, what, _e);      \
  } while (0)

// Checked builds: report a recorded out-of-range gather index (synchronises).
static dg_status adj_checked(Ctx* c, cudaStream_t s) {
  char msg[160];
  if (bounds_failed(s, msg, sizeof msg)) return afail(c, DG_ECUDA, msg);
  return DG_OK;
}

static dg_status ensure_adjoint(Ctx* c) {
  if (c->fv_on)
    return afail(c, DG_EUNSUPPORTED, "the adjoint is built for the DG operator (no FV sub-cell elements)");
  if (c->d_adj_qbar) return DG_OK;
  if (c->prm.precision != DG_FP64) return afail(c, DG_EUNSUPPORTED, "the adjoint is built for the FP64 operator");
  const size_t st = (size_t)c->E * 5 * c->P;
  const size_t nn = (size_t)c->nfaces * c->NN;
  ADJ_CUDA(setup_adjoint(c->N), c, "adjoint kernel set-up");
  ADJ_CUDA(cudaMalloc(&c->d_adj_qbar, sizeof(double) * st), c, "adjoint buffers");
  ADJ_CUDA(cudaMalloc(&c->d_adj_gbar, sizeof(double) * (size_t)c->E * 12 * c->P), c, "adjoint buffers");
  ADJ_CUDA(cudaMalloc(&c->d_adj_gtil, sizeof(double) * (size_t)c->E * 12 * c->P), c, "adjoint buffers");
  ADJ_CUDA(cudaMalloc(&c->d_adj_fseed, sizeof(double) * nn * 2 * 5), c, "adjoint buffers");
  ADJ_CUDA(cudaMalloc(&c->d_adj_face, sizeof(double) * nn * 2 * 17), c, "adjoint buffers");
  ADJ_CUDA(cudaMalloc(&c->d_adj_mu, sizeof(double) * (adjoint_mu_partials(*c) + 2)), c, "adjoint buffers");
  ADJ_CUDA(cudaMalloc(&c->d_adj_stage, sizeof(double) * st * rk_scheme(c->prm.rk_scheme).stages), c,
           "adjoint stage states");
  ADJ_CUDA(cudaMalloc(&c->d_adj_work, sizeof(double) * st * 4), c, "adjoint work");
  if (c->M > 0)
    ADJ_CUDA(cudaMalloc(&c->d_adj_mx, sizeof(double) * (size_t)c->M * 5 * 4 * c->NN), c, "adjoint mortar buffer");
  if (c->prm.nodes == DG_NODES_LG)
    ADJ_CUDA(cudaMalloc(&c->d_adj_lgf, sizeof(double) * (size_t)c->E * 6 * 9 * c->NN), c, "adjoint face buffer");
  return DG_OK;
}

// Adjoint of one step of the context's 2N-storage scheme (LSERK4-5 or
// RK4-14).  Un: state at the start of the step; lam: in = adjoint at the end
// of the step, out = adjoint at the start (in place).
static dg_status step_adjoint(Ctx* c, const double* Un, double* lam, double* dJdmu, double t, double dt,
                              cudaStream_t s) {
  const RkScheme rk = rk_scheme(c->prm.rk_scheme);
  const size_t st = (size_t)c->E * 5 * c->P, bytes = sizeof(double) * st;
  double* Ws = c->d_adj_work;           // work state
  double* G = Ws + st;                  // RK register
  double* Gb = G + st;                  // adjoint of the register
  double* tmp = Gb + st;                // dt * Gb, then VJP output
  // forward recomputation of the stage states
  ADJ_CUDA(cudaMemcpyAsync(Ws, Un, bytes, cudaMemcpyDeviceToDevice, s), c, "stage copy");
  ADJ_CUDA(cudaMemsetAsync(G, 0, bytes, s), c, "memset");
  ADJ_CUDA(launch_set_clock(c->d_clock, t, dt, s), c, "clock");
  for (int k = 0; k < rk.stages; ++k) {
    ADJ_CUDA(cudaMemcpyAsync(c->d_adj_stage + (size_t)k * st, Ws, bytes, cudaMemcpyDeviceToDevice, s), c, "stage copy");
    ADJ_CUDA(launch_lift(*c, Ws, s), c, "lift");
    ADJ_CUDA(launch_face(*c, Ws, s), c, "face");
    StageArgs a{Ws, Ws, G, nullptr, c->d_clock, rk.C[k], rk.A[k], rk.B[k], 1};
    ADJ_CUDA(launch_volume(*c, a, s), c, "volume");
  }
  // reverse sweep: Gb += B_k lam;  lam += (dR/dU)^T (dt Gb);  Gb *= A_k
  ADJ_CUDA(cudaMemsetAsync(Gb, 0, bytes, s), c, "memset");
  for (int k = rk.stages - 1; k >= 0; --k) {
    ADJ_CUDA(launch_axpby(Gb, lam, 1.0, rk.B[k], st, s), c, "axpby");
    ADJ_CUDA(launch_axpby(tmp, Gb, 0.0, dt, st, s), c, "axpby");
    ADJ_CUDA(launch_vjp(*c, c->d_adj_stage + (size_t)k * st, tmp, tmp, dJdmu, 1.0, s), c, "vjp");
    ADJ_CUDA(launch_axpby(lam, tmp, 1.0, 1.0, st, s), c, "axpby");
    ADJ_CUDA(launch_axpby(Gb, Gb, rk.A[k], 0.0, st, s), c, "axpby");
  }
  return DG_OK;
}

// forward steps from `from` (in place on U), each step zeroing the register
static dg_status advance(Ctx* c, double* U, double* G, double t, double dt, int nsteps, cudaStream_t s) {
  if (nsteps <= 0) return DG_OK;
  ADJ_CUDA(launch_set_clock(c->d_clock, t, dt, s), c, "clock");
  const size_t bytes = sizeof(double) * (size_t)c->E * 5 * c->P;
  const RkScheme rk = rk_scheme(c->prm.rk_scheme);
  for (int st = 0; st < nsteps; ++st) {
    ADJ_CUDA(cudaMemsetAsync(G, 0, bytes, s), c, "memset");
    for (int k = 0; k < rk.stages; ++k) {
      ADJ_CUDA(launch_lift(*c, U, s), c, "lift");
      ADJ_CUDA(launch_face(*c, U, s), c, "face");
      StageArgs a{U, U, G, nullptr, c->d_clock, rk.C[k], rk.A[k], rk.B[k], 1};
      ADJ_CUDA(launch_volume(*c, a, s), c, "volume");
    }
    ADJ_CUDA(launch_clock_advance(c->d_clock, s), c, "clock");
  }
  return DG_OK;
}

// Binomial checkpointing (Griewank 1992; Griewank & Walther 2000).  With s
// stored states (the one at the start of the interval included) and r forward
// sweeps, beta(s, r) = C(s + r, s) steps can be reversed; the least number of
// forward steps that reverses n steps is
//   t(n, s) = r n - beta(s + 1, r - 1),  r = rho(n, s) the least r with beta(s, r) >= n,
// and t(n, 1) = n (n - 1) / 2 (every step recomputed from the start).
static long long binom(long long s, long long r) {   // C(s + r, s)
  const long long k = s < r ? s : r, top = s < r ? r : s;
  long long v = 1;
  for (long long a = 1; a <= k; ++a) v = v * (top + a) / a;
  return v;
}

static long long rho(long long n, long long s) {
  if (s <= 1) return n > 1 ? n - 1 : 0;
  long long r = 0;
  while (binom(s, r) < n) ++r;
  return r;
}

// Where to store the next state when n > 1 steps are reversed from a stored
// state with s >= 2 states in all: the least m in [1, n-1] minimising
//   F(m) = m + t(n - m, s - 1) + t(m, s)
// (advance m steps into a new state, reverse the right part with one state
// less, then the left part).  t(., s) is convex with increments
// t(x + 1, s) - t(x, s) = rho(x + 1, s), so F(m + 1) - F(m) =
// 1 + rho(m + 1, s) - rho(n - m, s - 1) is non-decreasing and the least m where
// it is >= 0 is found by bisection.
static long long next_split(long long n, long long s) {
  long long lo = 1, hi = n - 1;
  while (lo < hi) {
    const long long mid = lo + (hi - lo) / 2;
    if (1 + rho(mid + 1, s) - rho(n - mid, s - 1) >= 0) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Runs the schedule that reverses nsteps steps with nsnap >= 1 state slots
// (slot 0 holds the initial state) on an executor X with
//   dg_status store(int from_slot, int to_slot, int i0, int m):  slot to := state at m,
//                                                                 advanced from slot from at i0;
//   dg_status adjoint(int slot, int i):                           adjoint of step i, state i in slot;
//   dg_status recompute_adjoint(int slot, int i0, int i):         the same, state i recomputed from
//                                                                 slot (state i0).
// Intervals wait on an explicit stack (right part first), so the depth of
// nesting does not grow with the number of slots.
template <class X>
static dg_status run_schedule(X& x, int nsteps, int nsnap, long long* forward, long long* adjoints) {
  struct Interval { int i0, i1, slot; };
  std::vector<Interval> pending;
  pending.push_back({0, nsteps, 0});
  *forward = 0;
  *adjoints = 0;
  while (!pending.empty()) {
    const Interval iv = pending.back();
    pending.pop_back();
    const int n = iv.i1 - iv.i0;
    const int states = nsnap - iv.slot;   // stored states usable for this interval
    dg_status st = DG_OK;
    if (n == 1) {
      st = x.adjoint(iv.slot, iv.i0);
      ++*adjoints;
    } else if (states <= 1) {
      for (int k = iv.i1 - 1; k >= iv.i0 && st == DG_OK; --k) {
        st = x.recompute_adjoint(iv.slot, iv.i0, k);
        *forward += k - iv.i0;
        ++*adjoints;
      }
    } else {
      const int m = iv.i0 + (int)next_split(n, states);
      st = x.store(iv.slot, iv.slot + 1, iv.i0, m);
      *forward += m - iv.i0;
      pending.push_back({iv.i0, m, iv.slot});
      pending.push_back({m, iv.i1, iv.slot + 1});
    }
    if (st != DG_OK) return st;
  }
  return DG_OK;
}

// The executor of dg_adjoint_solve: state slots in device memory.
struct DeviceCheckpoints {
  Ctx* c;
  std::vector<double*> snap;   // state slots
  double* lam;
  double* dJdmu;
  double t0, dt;
  cudaStream_t s;

  size_t bytes() const { return sizeof(double) * (size_t)c->E * 5 * c->P; }
  double* reg() const { return c->d_adj_work + (size_t)c->E * 5 * c->P; }   // register slot of the work area

  dg_status store(int from, int to, int i0, int m) {
    ADJ_CUDA(cudaMemcpyAsync(snap[to], snap[from], bytes(), cudaMemcpyDeviceToDevice, s), c, "copy");
    return advance(c, snap[to], reg(), t0 + i0 * dt, dt, m - i0, s);
  }
  dg_status adjoint(int slot, int i) { return step_adjoint(c, snap[slot], lam, dJdmu, t0 + i * dt, dt, s); }
  dg_status recompute_adjoint(int slot, int i0, int i) {
    double* W = c->d_adj_work;
    ADJ_CUDA(cudaMemcpyAsync(W, snap[slot], bytes(), cudaMemcpyDeviceToDevice, s), c, "copy");
    dg_status st = advance(c, W, reg(), t0 + i0 * dt, dt, i - i0, s);
    if (st != DG_OK) return st;
    // the step adjoint overwrites the work area, so it starts from a copy in
    // stage slot 4, which it reads first and rewrites only at its fifth stage
    double* keep = c->d_adj_stage + (size_t)4 * c->E * 5 * c->P;
    ADJ_CUDA(cudaMemcpyAsync(keep, W, bytes(), cudaMemcpyDeviceToDevice, s), c, "copy");
    return step_adjoint(c, keep, lam, dJdmu, t0 + i * dt, dt, s);
  }
};

// The same schedule without a device: only the counts.
struct CountOnly {
  dg_status store(int, int, int, int) { return DG_OK; }
  dg_status adjoint(int, int) { return DG_OK; }
  dg_status recompute_adjoint(int, int, int) { return DG_OK; }
};

}  // namespace dg

using namespace dg;

extern "C" {

dg_status dg_time_derivative_vjp(dg_ctx* ctx, const double* dU, const double* dv, double* dout, double* dJdmu,
                                 double t, dg_stream stream) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  (void)t;
  if (!c || !dU || !dv || !dout) return afail(c, DG_EINVAL, "dg_time_derivative_vjp: null argument");
  if (dout == dU) return afail(c, DG_EINVAL, "dg_time_derivative_vjp: dout aliases dU");
  ADJ_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  dg_status st = ensure_adjoint(c);
  if (st != DG_OK) return st;
  ADJ_CUDA(launch_vjp(*c, dU, dv, dout, dJdmu, 1.0, (cudaStream_t)stream), c, "vjp");
  return adj_checked(c, (cudaStream_t)stream);
}

dg_status dg_adjoint_step(dg_ctx* ctx, const double* dU_n, const double* dlam_np1, double* dlam_n, double* dJdmu,
                          double t, double dt, dg_stream stream) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !dU_n || !dlam_np1 || !dlam_n) return afail(c, DG_EINVAL, "dg_adjoint_step: null argument");
  if (dlam_n == dU_n || dlam_np1 == dU_n) return afail(c, DG_EINVAL, "dg_adjoint_step: an adjoint aliases the state");
  cudaStream_t s = (cudaStream_t)stream;
  ADJ_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  dg_status st = ensure_adjoint(c);
  if (st != DG_OK) return st;
  const size_t bytes = sizeof(double) * (size_t)c->E * 5 * c->P;
  if (dlam_n != dlam_np1) ADJ_CUDA(cudaMemcpyAsync(dlam_n, dlam_np1, bytes, cudaMemcpyDeviceToDevice, s), c, "copy");
  st = step_adjoint(c, dU_n, dlam_n, dJdmu, t, dt, s);
  return st != DG_OK ? st : adj_checked(c, s);
}

dg_status dg_adjoint_solve(dg_ctx* ctx, const double* dU0, const double* dlamT, double* dlam0, double* dJdmu,
                           double t0, double dt, int32_t nsteps, int32_t max_snapshots, int64_t* host_counts2,
                           dg_stream stream) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !dU0 || !dlamT || !dlam0 || nsteps < 0 || max_snapshots < 1)
    return afail(c, DG_EINVAL, "dg_adjoint_solve: bad argument");
  if (dlam0 == dU0 || dlamT == dU0) return afail(c, DG_EINVAL, "dg_adjoint_solve: an adjoint aliases the state");
  cudaStream_t s = (cudaStream_t)stream;
  ADJ_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  dg_status st = ensure_adjoint(c);
  if (st != DG_OK) return st;
  const size_t bytes = sizeof(double) * (size_t)c->E * 5 * c->P;
  if (dlam0 != dlamT) ADJ_CUDA(cudaMemcpyAsync(dlam0, dlamT, bytes, cudaMemcpyDeviceToDevice, s), c, "copy");
  if (nsteps == 0) return DG_OK;
  DeviceCheckpoints X;
  X.c = c;
  X.lam = dlam0;
  X.dJdmu = dJdmu;
  X.t0 = t0;
  X.dt = dt;
  X.s = s;
  const int nsnap = max_snapshots < nsteps ? max_snapshots : nsteps;
  try {
    X.snap.assign(nsnap, nullptr);
  } catch (const std::bad_alloc&) {
    return afail(c, DG_ENOMEM, "dg_adjoint_solve: host memory for the snapshot table");
  }
  for (int a = 0; a < nsnap; ++a) {
    cudaError_t e = cudaMalloc(&X.snap[a], bytes);
    if (e != cudaSuccess) {
      for (int b = 0; b < a; ++b) cudaFree(X.snap[b]);
      return afail(c, DG_ENOMEM, "dg_adjoint_solve: snapshot allocation", e);
    }
  }
  long long forward = 0, adjoints = 0;
  cudaError_t e = cudaMemcpyAsync(X.snap[0], dU0, bytes, cudaMemcpyDeviceToDevice, s);
  try {
    st = e == cudaSuccess ? run_schedule(X, nsteps, nsnap, &forward, &adjoints) : afail(c, DG_ECUDA, "copy", e);
  } catch (const std::bad_alloc&) {   // the schedule's interval stack
    st = afail(c, DG_ENOMEM, "dg_adjoint_solve: host memory for the schedule");
  }
  cudaError_t es = cudaStreamSynchronize(s);
  for (double* p : X.snap) cudaFree(p);
  if (st != DG_OK) return st;
  if (es != cudaSuccess) return afail(c, DG_ECUDA, "dg_adjoint_solve: sync", es);
  if (host_counts2) { host_counts2[0] = forward; host_counts2[1] = adjoints; }
  return adj_checked(c, s);
}

dg_status dg_checkpoint_schedule(int32_t nsteps, int32_t max_snapshots, int64_t* host_counts2) {
  if (nsteps < 0 || max_snapshots < 1 || !host_counts2) return DG_EINVAL;
  const int nsnap = max_snapshots < nsteps ? max_snapshots : nsteps;
  long long forward = 0, adjoints = 0;
  if (nsteps > 0) {
    CountOnly X;
    try {
      run_schedule(X, nsteps, nsnap, &forward, &adjoints);
    } catch (const std::bad_alloc&) {
      return DG_ENOMEM;
    }
  }
  host_counts2[0] = forward;
  host_counts2[1] = adjoints;
  return DG_OK;
}

dg_status dg_kinetic_energy(dg_ctx* ctx, const double* dU, double* dgrad, double* host_J, dg_stream stream) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !dU || !host_J) return afail(c, DG_EINVAL, "dg_kinetic_energy: null argument");
  cudaStream_t s = (cudaStream_t)stream;
  ADJ_CUDA(cudaSetDevice(c->device), c, "cudaSetDevice");
  double* d_out = c->d_red + (size_t)(c->red_len) * kRedValues;   // last row of the reduction buffer
  ADJ_CUDA(launch_kinetic(*c, dU, dgrad, d_out, s), c, "kinetic energy");
  ADJ_CUDA(cudaMemcpyAsync(c->h_out, d_out, sizeof(double), cudaMemcpyDeviceToHost, s), c, "copy");
  ADJ_CUDA(cudaStreamSynchronize(s), c, "sync");
  *host_J = c->h_out[0];
  return DG_OK;
}

dg_status dg_set_viscosity(dg_ctx* ctx, double mu) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c || !(mu >= 0.0)) return afail(c, DG_EINVAL, "dg_set_viscosity: bad argument");
  c->prm.mu = mu;
  c->gas.mu = mu;
  set_float_copies(c->gas);
  if (c->graph) {                       // the captured graph holds the old constants
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  return DG_OK;
}

}  // extern "C"
