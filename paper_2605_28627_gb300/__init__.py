"""GB300-native split-form DGSEM hot path (GALAEXI, arXiv 2605.28627).

Thin Python binding over the C ABI declared in ``include/dgsem.h``.  Every
numerical step runs in the CUDA library ``libdgsem.so``; this module only
marshals arguments (device pointers of torch tensors, the current CUDA
stream).  There is no CPU fallback: if the library or a GPU is missing, the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

# DGSEM_CHECKED=1 loads the checked build (every indirect gather index
# bounds-checked, see csrc/dg_check.cuh), for debugging; same API and results.
CHECKED = os.environ.get("DGSEM_CHECKED", "") == "1"
LIB_PATH = _build.LIB_CHECKED if CHECKED else _build.LIB

# dg_status codes
DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_EMESH, DG_ENONFINITE, DG_ETIMEOUT, DG_EUNSUPPORTED = range(8)
STATUS_NAMES = ["DG_OK", "DG_EINVAL", "DG_ENOMEM", "DG_ECUDA", "DG_EMESH", "DG_ENONFINITE", "DG_ETIMEOUT",
                "DG_EUNSUPPORTED"]
FLUX_LLF, FLUX_EC, FLUX_ROE = 0, 1, 2
FP64, FP32OP = 0, 1
SOURCE_NONE, SOURCE_MMS = 0, 1
VISC_CONSTANT, VISC_SUTHERLAND = 0, 1
NODES_LGL, NODES_LG = 0, 1
RK45, RK414 = 0, 1
IC_TGV, IC_MMS = 0, 1
IND_RHO, IND_P, IND_RHOP = 0, 1, 2

# Every symbol that include/dgsem.h declares.
EXPORTS = ["dg_init", "dg_destroy", "dg_state_len", "dg_time_derivative", "dg_rk_step", "dg_advance_host",
           "dg_integrals", "dg_max_dt", "dg_initial_state", "dg_node_coords", "dg_geometry", "dg_profile_stages",
           "dg_probe_peaks", "dg_conserved_totals_noalloc", "dg_ensemble_create", "dg_ensemble_destroy",
           "dg_ensemble_step", "dg_ensemble_plan", "dg_ensemble_last_error", "dg_time_derivative_vjp",
           "dg_adjoint_step", "dg_adjoint_solve", "dg_checkpoint_schedule", "dg_kinetic_energy", "dg_set_viscosity",
           "dg_check_conversions", "dg_check_reciprocals", "dg_indicator", "dg_set_fv_mask", "dg_set_fv_switch",
           "dg_get_fv_mask", "dg_last_error"]


class DGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))


class dg_mesh(C.Structure):
    _fields_ = [("n_elems", C.c_int32), ("ngeo", C.c_int32), ("xgeo", C.POINTER(C.c_double)),
                ("face_nbr", C.POINTER(C.c_int32)), ("n_mortars", C.c_int32), ("mortars", C.POINTER(C.c_int32))]


class dg_params(C.Structure):
    _fields_ = [("N", C.c_int32), ("gamma", C.c_double), ("R", C.c_double), ("Pr", C.c_double),
                ("mu", C.c_double), ("surf_flux", C.c_int32), ("precision", C.c_int32),
                ("source", C.c_int32), ("mms_amp", C.c_double), ("p_ref", C.c_double),
                ("visc_law", C.c_int32), ("T_ref", C.c_double), ("S_suth", C.c_double), ("nodes", C.c_int32),
                ("rk_scheme", C.c_int32)]


_lib = None


def load(build_if_missing: bool = True):
    """Load libdgsem.so (building it in-tree with nvcc if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH) or not _build.up_to_date(CHECKED):
        if not build_if_missing:
            raise RuntimeError("libdgsem.so is not built (run __graft_entry__.build())")
        _build.build(checked=CHECKED)
    L = C.CDLL(LIB_PATH)
    vp, dp, i32, f64 = C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_double
    L.dg_init.argtypes = [C.POINTER(dg_mesh), C.POINTER(dg_params), C.c_int, C.POINTER(vp)]
    L.dg_destroy.argtypes = [vp]
    L.dg_state_len.argtypes = [vp]
    L.dg_state_len.restype = C.c_size_t
    L.dg_time_derivative.argtypes = [vp, vp, vp, f64, vp]
    L.dg_rk_step.argtypes = [vp, vp, vp, f64, f64, i32, vp]
    L.dg_advance_host.argtypes = [vp, vp, f64, f64, i32, vp]
    L.dg_integrals.argtypes = [vp, vp, dp, vp]
    L.dg_max_dt.argtypes = [vp, vp, f64, f64, dp, vp]
    L.dg_initial_state.argtypes = [vp, i32, f64, vp, vp]
    L.dg_node_coords.argtypes = [vp, vp, vp]
    L.dg_geometry.argtypes = [vp, vp, vp, vp]
    L.dg_profile_stages.argtypes = [vp, vp, vp, f64, i32, C.POINTER(C.c_float), vp]
    L.dg_probe_peaks.argtypes = [C.c_int, dp]
    L.dg_check_conversions.argtypes = [vp, i32, vp, vp, vp]
    L.dg_check_reciprocals.argtypes = [vp, i32, vp, vp, vp]
    L.dg_indicator.argtypes = [vp, vp, i32, f64, vp, vp, vp]
    L.dg_set_fv_mask.argtypes = [vp, vp, vp]
    L.dg_set_fv_switch.argtypes = [vp, i32, f64, f64, vp]
    L.dg_get_fv_mask.argtypes = [vp, vp, vp]
    L.dg_conserved_totals_noalloc.argtypes = [vp, vp, i32, i32, i32, vp, vp]
    L.dg_ensemble_create.argtypes = [C.POINTER(vp), i32, C.c_char_p, C.POINTER(vp)]
    L.dg_ensemble_destroy.argtypes = [vp]
    L.dg_ensemble_step.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), dp, dp, i32, vp]
    L.dg_ensemble_plan.argtypes = [vp, C.c_char_p, C.c_size_t]
    L.dg_ensemble_last_error.argtypes = [vp]
    L.dg_ensemble_last_error.restype = C.c_char_p
    L.dg_time_derivative_vjp.argtypes = [vp, vp, vp, vp, vp, f64, vp]
    L.dg_adjoint_step.argtypes = [vp, vp, vp, vp, vp, f64, f64, vp]
    L.dg_adjoint_solve.argtypes = [vp, vp, vp, vp, vp, f64, f64, i32, i32, C.POINTER(C.c_int64), vp]
    L.dg_checkpoint_schedule.argtypes = [i32, i32, C.POINTER(C.c_int64)]
    L.dg_kinetic_energy.argtypes = [vp, vp, vp, dp, vp]
    L.dg_set_viscosity.argtypes = [vp, f64]
    L.dg_last_error.argtypes = [vp]
    L.dg_last_error.restype = C.c_char_p
    for name in ("dg_init", "dg_destroy", "dg_time_derivative", "dg_rk_step", "dg_advance_host", "dg_integrals",
                 "dg_max_dt", "dg_initial_state", "dg_node_coords", "dg_geometry", "dg_profile_stages",
                 "dg_probe_peaks", "dg_conserved_totals_noalloc", "dg_ensemble_create", "dg_ensemble_destroy",
                 "dg_ensemble_step", "dg_ensemble_plan", "dg_time_derivative_vjp", "dg_adjoint_step",
                 "dg_adjoint_solve", "dg_checkpoint_schedule", "dg_kinetic_energy", "dg_set_viscosity",
                 "dg_check_conversions", "dg_check_reciprocals", "dg_indicator", "dg_set_fv_mask",
                 "dg_set_fv_switch", "dg_get_fv_mask"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class Solver:
    """A DGSEM context on one GPU: geometry and work buffers live in the
    library; states are caller-owned float64 CUDA tensors of shape
    ``[E, 5, N+1, N+1, N+1]``."""

    def __init__(self, mesh, N: int, gamma=1.4, R=1.0, Pr=0.72, mu=0.0, surf_flux=FLUX_LLF,
                 precision=FP64, source=SOURCE_NONE, mms_amp=0.1, device: int = 0, p_ref: float = 0.0,
                 visc_law: int = VISC_CONSTANT, T_ref: float = 1.0, S_suth: float = 0.0, nodes: int = NODES_LGL,
                 rk_scheme: int = RK45):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2605_28627_gb300 needs a CUDA GPU; there is no CPU fallback")
        self._L = load()
        self.N, self.n, self.P = N, N + 1, (N + 1) ** 3
        self.device = device
        xgeo = np.ascontiguousarray(mesh.xgeo, dtype=np.float64)
        nbr = np.ascontiguousarray(mesh.face_nbr, dtype=np.int32)
        self.E = int(xgeo.shape[0])
        mortars = getattr(mesh, "mortars", None)
        mortars = None if mortars is None or len(mortars) == 0 else np.ascontiguousarray(mortars, dtype=np.int32)
        m = dg_mesh(self.E, int(xgeo.shape[-1]) - 1, xgeo.ctypes.data_as(C.POINTER(C.c_double)),
                    nbr.ctypes.data_as(C.POINTER(C.c_int32)), 0 if mortars is None else mortars.shape[0],
                    None if mortars is None else mortars.ctypes.data_as(C.POINTER(C.c_int32)))
        p = dg_params(N, gamma, R, Pr, mu, surf_flux, precision, source, mms_amp, p_ref, visc_law, T_ref, S_suth,
                      nodes, rk_scheme)
        h = C.c_void_p()
        torch.cuda.set_device(device)
        st = self._L.dg_init(C.byref(m), C.byref(p), device, C.byref(h))
        if st != DG_OK:
            raise DGError(st, self._L.dg_last_error(None).decode())
        self._h = h
        self.mu = mu

    def close(self):
        if getattr(self, "_h", None):
            self._L.dg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != DG_OK:
            raise DGError(st, self._L.dg_last_error(self._h).decode())

    @property
    def shape(self):
        return (self.E, 5, self.n, self.n, self.n)

    def state_len(self) -> int:
        return int(self._L.dg_state_len(self._h))

    def empty_state(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device="cuda:%d" % self.device)

    def _chk_state(self, U):
        import torch
        if not (isinstance(U, torch.Tensor) and U.is_cuda and U.dtype == torch.float64 and U.is_contiguous()
                and U.numel() == self.state_len()):
            raise ValueError("state must be a contiguous float64 CUDA tensor with %d elements" % self.state_len())

    def time_derivative(self, U, Ut=None, t=0.0, stream=None):
        self._chk_state(U)
        if Ut is None:
            Ut = self.empty_state()
        self._chk_state(Ut)
        self._check(self._L.dg_time_derivative(self._h, _ptr(U), _ptr(Ut), float(t), _stream_handle(stream)))
        return Ut

    def rk_step(self, U, G, t, dt, nsteps=1, stream=None):
        self._chk_state(U)
        self._chk_state(G)
        self._check(self._L.dg_rk_step(self._h, _ptr(U), _ptr(G), float(t), float(dt), int(nsteps),
                                       _stream_handle(stream)))
        return U

    def advance_host(self, U_host, t, dt, nsteps=1, stream=None):
        """End to end through host memory: U_host (float64 numpy array or
        pinned CPU tensor, contiguous) is copied in, advanced and copied back."""
        import torch
        if isinstance(U_host, torch.Tensor):
            assert U_host.device.type == "cpu" and U_host.dtype == torch.float64 and U_host.is_contiguous()
            ptr = C.c_void_p(U_host.data_ptr())
            n = U_host.numel()
        else:
            assert U_host.dtype == np.float64 and U_host.flags["C_CONTIGUOUS"]
            ptr = C.c_void_p(U_host.ctypes.data)
            n = U_host.size
        if n != self.state_len():
            raise ValueError("host state has the wrong size")
        self._check(self._L.dg_advance_host(self._h, ptr, float(t), float(dt), int(nsteps), _stream_handle(stream)))
        return U_host

    def integrals(self, U, stream=None):
        self._chk_state(U)
        out = (C.c_double * 8)()
        self._check(self._L.dg_integrals(self._h, _ptr(U), out, _stream_handle(stream)))
        return np.array(out[:])

    def max_dt(self, U, cfl=0.9, dfl=0.9, stream=None):
        self._chk_state(U)
        dt = C.c_double()
        self._check(self._L.dg_max_dt(self._h, _ptr(U), float(cfl), float(dfl), C.byref(dt), _stream_handle(stream)))
        return dt.value

    def initial_state(self, kind: str, prm0: float, U=None, stream=None):
        if U is None:
            U = self.empty_state()
        self._chk_state(U)
        self._check(self._L.dg_initial_state(self._h, {"tgv": IC_TGV, "mms": IC_MMS}[kind], float(prm0), _ptr(U),
                                             _stream_handle(stream)))
        return U

    def indicator(self, U, var=IND_RHOP, log10_threshold=None, stream=None):
        """Persson modal indicator per element: eta (device float64 [E]) and,
        with a threshold, the troubled-cell flags (device int32 [E])."""
        import torch
        self._chk_state(U)
        eta = torch.empty(self.E, dtype=torch.float64, device="cuda:%d" % self.device)
        flag = None
        if log10_threshold is not None:
            flag = torch.empty(self.E, dtype=torch.int32, device="cuda:%d" % self.device)
        self._check(self._L.dg_indicator(self._h, _ptr(U), int(var),
                                         float(log10_threshold) if log10_threshold is not None else 0.0, _ptr(eta),
                                         _ptr(flag) if flag is not None else None, _stream_handle(stream)))
        return eta, flag

    def set_fv_mask(self, mask, stream=None):
        """Advance the elements with mask[e] != 0 by the FV sub-cell operator
        (device int32 [E], e.g. the flags of ``indicator``; a host array is
        copied to the device first); None restores the pure DG operator."""
        import torch
        if mask is None:
            self._check(self._L.dg_set_fv_mask(self._h, None, _stream_handle(stream)))
            self._fv_mask = None
            return
        m = torch.as_tensor(mask)
        if m.numel() != self.E:
            raise ValueError("FV mask: one entry per element")
        m = (m.reshape(-1) != 0).to(device="cuda:%d" % self.device, dtype=torch.int32).contiguous()
        self._check(self._L.dg_set_fv_mask(self._h, _ptr(m), _stream_handle(stream)))
        self._fv_mask = m   # kept until the stream has passed the copy

    def set_fv_switch(self, var=IND_RHOP, log10_upper=None, log10_lower=None, stream=None):
        """Automatic DG/FV switching before every evaluation of R(U): above
        10^log10_upper an element becomes an FV element, below 10^log10_lower
        (with an admissible nodal state) a DG element; var None turns it off."""
        if var is None:
            self._check(self._L.dg_set_fv_switch(self._h, -1, 0.0, 0.0, _stream_handle(stream)))
            return
        if log10_lower is None:
            log10_lower = log10_upper
        self._check(self._L.dg_set_fv_switch(self._h, int(var), float(log10_upper), float(log10_lower),
                                             _stream_handle(stream)))

    def fv_mask(self, stream=None):
        """The FV mask in effect (device int32 [E])."""
        import torch
        m = torch.empty(self.E, dtype=torch.int32, device="cuda:%d" % self.device)
        self._check(self._L.dg_get_fv_mask(self._h, _ptr(m), _stream_handle(stream)))
        return m

    def node_coords(self, stream=None):
        import torch
        X = torch.empty((self.E, 3, self.P), dtype=torch.float64, device="cuda:%d" % self.device)
        self._check(self._L.dg_node_coords(self._h, _ptr(X), _stream_handle(stream)))
        return X

    def profile_stages(self, U, G, dt, reps=5, stream=None):
        """Average milliseconds per launch of (lifting, face flux, volume)."""
        self._chk_state(U)
        self._chk_state(G)
        ms = (C.c_float * 3)()
        self._check(self._L.dg_profile_stages(self._h, _ptr(U), _ptr(G), float(dt), int(reps), ms,
                                              _stream_handle(stream)))
        return [float(v) for v in ms]

    # ---- discrete adjoint
    def set_viscosity(self, mu):
        self._check(self._L.dg_set_viscosity(self._h, float(mu)))
        self.mu = float(mu)

    def time_derivative_vjp(self, U, v, out=None, dJdmu=None, t=0.0, stream=None):
        """(dR/dU)^T v; dJdmu (1-element float64 CUDA tensor) += v . dR/dmu."""
        self._chk_state(U)
        self._chk_state(v)
        if out is None:
            out = self.empty_state()
        self._check(self._L.dg_time_derivative_vjp(self._h, _ptr(U), _ptr(v), _ptr(out),
                                                   _ptr(dJdmu) if dJdmu is not None else None, float(t),
                                                   _stream_handle(stream)))
        return out

    def adjoint_step(self, U_n, lam_np1, lam_n=None, dJdmu=None, t=0.0, dt=1e-3, stream=None):
        self._chk_state(U_n)
        self._chk_state(lam_np1)
        if lam_n is None:
            lam_n = self.empty_state()
        self._check(self._L.dg_adjoint_step(self._h, _ptr(U_n), _ptr(lam_np1), _ptr(lam_n),
                                            _ptr(dJdmu) if dJdmu is not None else None, float(t), float(dt),
                                            _stream_handle(stream)))
        return lam_n

    def adjoint_solve(self, U0, lamT, t0, dt, nsteps, max_snapshots=16, lam0=None, dJdmu=None, stream=None):
        """Adjoint of nsteps LSERK4-5 steps with binomial checkpointing;
        returns (lam0, (recomputed forward steps, adjoint steps))."""
        self._chk_state(U0)
        self._chk_state(lamT)
        if lam0 is None:
            lam0 = self.empty_state()
        counts = (C.c_int64 * 2)()
        self._check(self._L.dg_adjoint_solve(self._h, _ptr(U0), _ptr(lamT), _ptr(lam0),
                                             _ptr(dJdmu) if dJdmu is not None else None, float(t0), float(dt),
                                             int(nsteps), int(max_snapshots), counts, _stream_handle(stream)))
        return lam0, (int(counts[0]), int(counts[1]))

    def kinetic_energy(self, U, grad=None, stream=None):
        """J = LGL quadrature of 1/2 rho |u|^2; fills grad = dJ/dU if given."""
        self._chk_state(U)
        out = C.c_double()
        self._check(self._L.dg_kinetic_energy(self._h, _ptr(U), _ptr(grad) if grad is not None else None,
                                              C.byref(out), _stream_handle(stream)))
        return out.value

    def geometry(self, stream=None):
        import torch
        Ja = torch.empty((self.E, 3, 3, self.P), dtype=torch.float64, device="cuda:%d" % self.device)
        J = torch.empty((self.E, self.P), dtype=torch.float64, device="cuda:%d" % self.device)
        self._check(self._L.dg_geometry(self._h, _ptr(Ja), _ptr(J), _stream_handle(stream)))
        return Ja, J


def probe_peaks(device: int = 0):
    """Measured FP64 and FP32 FMA throughput in TFLOP/s on `device`."""
    L = load()
    out = (C.c_double * 2)()
    st = L.dg_probe_peaks(int(device), out)
    if st != DG_OK:
        raise DGError(st, "dg_probe_peaks failed")
    return float(out[0]), float(out[1])


def checkpoint_schedule(nsteps: int, max_snapshots: int):
    """(recomputed forward steps, adjoint steps) of the binomial checkpointing
    schedule that ``Solver.adjoint_solve`` runs for these arguments; host
    arithmetic only, no GPU needed."""
    L = load()
    counts = (C.c_int64 * 2)()
    st = L.dg_checkpoint_schedule(int(nsteps), int(max_snapshots), counts)
    if st != 0:
        raise DGError(st, "dg_checkpoint_schedule: bad argument")
    return int(counts[0]), int(counts[1])


def check_conversions(x, stream=None):
    """The FP32 operator's FP64 -> FP32 -> FP64 conversions of the device
    float64 tensor x next to the hardware ones: returns (f_op, f_hw, d_op,
    d_hw) as device tensors."""
    import torch
    L = load()
    x = x.contiguous()
    n = x.numel()
    f = torch.empty(2 * n, dtype=torch.float32, device=x.device)
    d = torch.empty(2 * n, dtype=torch.float64, device=x.device)
    st = L.dg_check_conversions(_ptr(x), n, _ptr(f), _ptr(d), _stream_handle(stream))
    if st != DG_OK:
        raise DGError(st, "dg_check_conversions failed")
    return f[:n], f[n:], d[:n], d[n:]


def check_reciprocals(x, stream=None):
    """The operator kernels' reciprocals of the positive device float64
    tensor x: returns (cubic FP64, quadratic FP64, adjoint FP64, FP32 of x
    rounded to FP32, FP32 quadratic form) as device tensors."""
    import torch
    L = load()
    x = x.contiguous()
    n = x.numel()
    d = torch.empty(3 * n, dtype=torch.float64, device=x.device)
    f = torch.empty(2 * n, dtype=torch.float32, device=x.device)
    st = L.dg_check_reciprocals(_ptr(x), n, _ptr(d), _ptr(f), _stream_handle(stream))
    if st != DG_OK:
        raise DGError(st, "dg_check_reciprocals failed")
    return d[:n], d[n:2 * n], d[2 * n:], f[:n], f[n:]


def conserved_totals_noalloc(U, J, N: int, out=None, stream=None, nodes: int = NODES_LGL):
    """Conservation totals of U (device float64) with Jacobian J (device,
    [E, P]) at the nodes of the node set `nodes` through the allocation-free
    entry point; returns the device tensor `out` (5 doubles)."""
    import torch
    L = load()
    if out is None:
        out = torch.empty(5, dtype=torch.float64, device=U.device)
    st = L.dg_conserved_totals_noalloc(_ptr(U), _ptr(J), int(N), int(nodes), int(J.shape[0]), _ptr(out),
                                       _stream_handle(stream))
    if st != DG_OK:
        raise DGError(st, "dg_conserved_totals_noalloc rejected its arguments")
    return out


class Ensemble:
    """Independent runs (Solver objects on one GPU, same precision) advanced
    together by the batched, autotuned ensemble kernels."""

    def __init__(self, solvers, tune_cache_path=None):
        self._L = load()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s._h.value for s in self.solvers])
        h = C.c_void_p()
        path = tune_cache_path.encode() if tune_cache_path else None
        st = self._L.dg_ensemble_create(arr, len(self.solvers), path, C.byref(h))
        if st != DG_OK:
            raise DGError(st, "dg_ensemble_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.dg_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, Us, Gs, t, dt, nsteps=1, stream=None):
        n = len(self.solvers)
        for s, U, G in zip(self.solvers, Us, Gs):
            s._chk_state(U)
            s._chk_state(G)
        pu = (C.c_void_p * n)(*[U.data_ptr() for U in Us])
        pg = (C.c_void_p * n)(*[G.data_ptr() for G in Gs])
        tt = (C.c_double * n)(*[float(v) for v in t])
        dd = (C.c_double * n)(*[float(v) for v in dt])
        st = self._L.dg_ensemble_step(self._h, pu, pg, tt, dd, int(nsteps), _stream_handle(stream))
        if st != DG_OK:
            raise DGError(st, self._L.dg_ensemble_last_error(self._h).decode())

    def plan(self):
        import json
        buf = C.create_string_buffer(1 << 16)
        if self._L.dg_ensemble_plan(self._h, buf, len(buf)) != DG_OK:
            return None
        return json.loads(buf.value.decode()) if buf.value else None
