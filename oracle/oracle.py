"""ctypes binding of the plain C++ FP64 oracle (test infrastructure only).

The oracle follows the method of GALAEXI Sec. 3.1 (Eqs. 1-3) step by step; see
``dgsem_oracle.cpp`` for the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgsem_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_libs = {}

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")

# -O3, no machine-specific flags (the same source builds on x86-64 and on
# aarch64).  g++'s default contraction of a*b + c into fused multiply-adds
# applies where the target has them (aarch64, not baseline x86-64), so the
# last bits of the two machines' results may differ.
_FLAGS = ["-O3", "-std=c++17", "-shared", "-fPIC"]


def lib_path(omp: bool = False) -> str:
    return _LIB_OMP if omp else _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with g++: the serial library, and the same source
    with OpenMP over the operator's element and face loops (the timed CPU
    baseline on all host cores; bit-identical results)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    for lib, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(os.path.getmtime(_SRC),
                                                                          os.path.getmtime(__file__)):
            tmp = lib + ".tmp%d" % os.getpid()
            subprocess.check_call(["g++", *_FLAGS, *extra, "-o", tmp, _SRC])
            os.replace(tmp, lib)
    return _LIB


def _load(omp: bool = False):
    if omp in _libs:
        return _libs[omp]
    build()
    L = C.CDLL(lib_path(omp))
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _ip, C.c_int, C.c_void_p, _dp, C.c_int, C.c_int,
                             C.c_char_p, C.c_int]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_threads.argtypes = [C.c_int]
    L.orc_threads.restype = C.c_int
    L.orc_nfaces.argtypes = [C.c_void_p]
    L.orc_nfaces.restype = C.c_int
    L.orc_basis.argtypes = [C.c_int, _dp, _dp, _dp]
    L.orc_gauss_basis.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp]
    L.orc_geometry.argtypes = [C.c_void_p, _dp, _dp, _dp]
    L.orc_time_derivative.argtypes = [C.c_void_p, _dp, _dp, C.c_double]
    L.orc_time_derivative_tl.argtypes = [C.c_void_p, _dp, _dp, C.c_double, _dp, _dp, C.c_double]
    L.orc_rk_steps.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, C.c_int]
    L.orc_rk_steps_tl.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_double, C.c_double, C.c_int]
    L.orc_rk_coeffs.argtypes = [_dp, _dp, _dp]
    L.orc_rk14_coeffs.argtypes = [_dp, _dp, _dp]
    L.orc_ec_flux.argtypes = [_dp, _dp, _dp, _dp, _dp]
    L.orc_llf_flux.argtypes = [_dp, _dp, _dp, _dp, _dp]
    L.orc_roe_flux.argtypes = [_dp, _dp, _dp, _dp, _dp]
    L.orc_log_mean.argtypes = [C.c_double, C.c_double]
    L.orc_log_mean.restype = C.c_double
    L.orc_integrals.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_node_coords.argtypes = [C.c_void_p, _dp]
    L.orc_initial_state.argtypes = [C.c_void_p, C.c_int, C.c_double, _dp]
    L.orc_set_vol_flux.argtypes = [C.c_void_p, C.c_int]
    L.orc_set_fv_mask.argtypes = [C.c_void_p, C.c_void_p]
    L.orc_set_fv_mask.restype = C.c_int
    L.orc_lifting.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_volume_term.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_count_ops.argtypes = [C.c_void_p, _dp, C.c_double, _dp]
    L.orc_count_ec_flux_ops.argtypes = [_dp, _dp, _dp, _dp, _dp]
    L.orc_persson_field.argtypes = [C.c_int, _dp, C.c_int, _dp, _dp]
    L.orc_persson.argtypes = [C.c_void_p, _dp, C.c_int, _dp]
    L.orc_set_fv_switch.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double]
    L.orc_set_fv_switch.restype = C.c_int
    L.orc_fv_state.argtypes = [C.c_void_p, C.c_void_p]
    L.orc_fv_state.restype = C.c_double
    _libs[omp] = L
    return L


def set_threads(n: int) -> int:
    """Host threads of the OpenMP build's operator loops (n > 0 sets the
    count); returns the count in effect."""
    return int(_load(omp=True).orc_threads(int(n)))


def gauss_basis(N: int):
    """Legendre-Gauss nodes, weights, D[i, j] = l_j'(x_i), l_j(-1), l_j(+1)."""
    L = _load()
    n = N + 1
    x, w, D, lm, lp = np.zeros(n), np.zeros(n), np.zeros(n * n), np.zeros(n), np.zeros(n)
    L.orc_gauss_basis(N, x, w, D, lm, lp)
    return x, w, D.reshape(n, n), lm, lp


def basis(N: int):
    """LGL nodes, weights and differentiation matrix D[i, j] = l_j'(x_i)."""
    L = _load()
    n = N + 1
    x, w, D = np.zeros(n), np.zeros(n), np.zeros(n * n)
    L.orc_basis(N, x, w, D)
    return x, w, D.reshape(n, n)


def rk14_coeffs():
    L = _load()
    A, B, Cc = np.zeros(14), np.zeros(14), np.zeros(14)
    L.orc_rk14_coeffs(A, B, Cc)
    return A, B, Cc


def rk_coeffs():
    L = _load()
    A, B, Cc = np.zeros(5), np.zeros(5), np.zeros(5)
    L.orc_rk_coeffs(A, B, Cc)
    return A, B, Cc


def _prm(gamma, R, Pr, mu, amp=0.1, visc_law=0, T_ref=1.0, S_suth=0.0, nodes=0, rk=0):
    return np.array([gamma, R, Pr, mu, amp, visc_law, T_ref, S_suth, nodes, rk], dtype=np.float64)


def ec_flux(qL, qR, nv, gamma=1.4):
    out = np.zeros(5)
    _load().orc_ec_flux(_prm(gamma, 1.0, 0.72, 0.0), np.ascontiguousarray(qL, dtype=np.float64),
                        np.ascontiguousarray(qR, dtype=np.float64), np.ascontiguousarray(nv, dtype=np.float64), out)
    return out


def llf_flux(qL, qR, nv, gamma=1.4):
    out = np.zeros(5)
    _load().orc_llf_flux(_prm(gamma, 1.0, 0.72, 0.0), np.ascontiguousarray(qL, dtype=np.float64),
                         np.ascontiguousarray(qR, dtype=np.float64), np.ascontiguousarray(nv, dtype=np.float64), out)
    return out


def roe_flux(qL, qR, nv, gamma=1.4):
    out = np.zeros(5)
    _load().orc_roe_flux(_prm(gamma, 1.0, 0.72, 0.0), np.ascontiguousarray(qL, dtype=np.float64),
                         np.ascontiguousarray(qR, dtype=np.float64), np.ascontiguousarray(nv, dtype=np.float64), out)
    return out


_OP_NAMES = ("add", "mul", "div", "sqrt", "log")


def count_ec_flux_ops(qL, qR, nv, gamma=1.4):
    """Operations of one two-point flux evaluation (from the primitive states
    on), counted by the oracle's counting scalar: dict add/mul/div/sqrt/log."""
    out = np.zeros(5)
    _load().orc_count_ec_flux_ops(_prm(gamma, 1.0, 0.72, 0.0), np.ascontiguousarray(qL, dtype=np.float64),
                                  np.ascontiguousarray(qR, dtype=np.float64),
                                  np.ascontiguousarray(nv, dtype=np.float64), out)
    return dict(zip(_OP_NAMES, (int(v) for v in out)))


def persson_field(N: int, x, q):
    """Persson modal indicator eta of nodal fields q [E, (N+1)^3] given at
    the nodes x (N+1 values per direction)."""
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(q.shape[0], -1)
    out = np.zeros(q.shape[0])
    _load().orc_persson_field(int(N), np.ascontiguousarray(x, dtype=np.float64), q.shape[0], q, out)
    return out


def log_mean(a, b):
    return _load().orc_log_mean(float(a), float(b))


class Oracle:
    """FP64 CPU DGSEM on a mesh in the format of ``workloads.mesh``.

    surf_flux: 0 = local Lax-Friedrichs, 1 = entropy-conservative two-point flux,
    2 = Roe with the Harten-Hyman entropy fix.
    source: 0 = none, 1 = density-wave manufactured solution.
    visc_law: 0 = constant mu, 1 = Sutherland's law mu (T/T_ref)^1.5 (T_ref + S)/(T + S).
    nodes: 0 = LGL nodes with the split form, 1 = Legendre-Gauss nodes with the
    standard weak form (no tangent-linear).
    rk: 0 = LSERK4-5 (Carpenter & Kennedy), 1 = RK4-14 (Niegemann et al.).
    parallel: use the OpenMP build (the FP64 operator's element and face loops
    on the host threads set by ``set_threads``; the same results bit for bit).
    """

    def __init__(self, mesh, N: int, gamma=1.4, R=1.0, Pr=0.72, mu=0.0,
                 surf_flux: int = 0, source: int = 0, mms_amp: float = 0.1,
                 visc_law: int = 0, T_ref: float = 1.0, S_suth: float = 0.0, nodes: int = 0, rk: int = 0,
                 parallel: bool = False):
        L = _load(omp=parallel)
        self.N, self.n, self.P = N, N + 1, (N + 1) ** 3
        self.E = int(mesh.xgeo.shape[0])
        self.gamma, self.R, self.Pr, self.mu = gamma, R, Pr, mu
        self.nodes = nodes
        xgeo = np.ascontiguousarray(mesh.xgeo, dtype=np.float64)
        nbr = np.ascontiguousarray(mesh.face_nbr, dtype=np.int32)
        err = C.create_string_buffer(256)
        mortars = getattr(mesh, "mortars", None)
        self._mortars = None if mortars is None or len(mortars) == 0 else np.ascontiguousarray(mortars, dtype=np.int32)
        nm = 0 if self._mortars is None else self._mortars.shape[0]
        h = L.orc_create(N, self.E, int(mesh.xgeo.shape[-1]) - 1, xgeo, nbr, nm,
                         None if self._mortars is None else self._mortars.ctypes.data,
                         _prm(gamma, R, Pr, mu, mms_amp, visc_law, T_ref, S_suth, nodes, rk), surf_flux, source, err,
                         256)
        if not h:
            raise ValueError("oracle: " + err.value.decode())
        self._h = C.c_void_p(h)
        self._L = L
        self.fv_mask = None

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.orc_destroy(self._h)
            self._h = None

    @property
    def shape(self):
        return (self.E, 5, self.n, self.n, self.n)

    def geometry(self):
        X = np.zeros((self.E, 3, self.P))
        Ja = np.zeros((self.E, 3, 3, self.P))
        J = np.zeros((self.E, self.P))
        self._L.orc_geometry(self._h, X, Ja, J)
        return X, Ja, J

    def time_derivative(self, U, t=0.0):
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = np.zeros_like(U)
        self._L.orc_time_derivative(self._h, U, out, float(t))
        return out

    def _tl_check(self):
        if self.fv_mask is not None:
            raise ValueError("oracle: the tangent-linear is built for the DG operator (no FV elements)")

    def time_derivative_tl(self, U, dU, dmu=0.0, t=0.0):
        self._tl_check()
        U = np.ascontiguousarray(U, dtype=np.float64)
        dU = np.ascontiguousarray(dU, dtype=np.float64)
        Ut, dUt = np.zeros_like(U), np.zeros_like(U)
        self._L.orc_time_derivative_tl(self._h, U, dU, float(dmu), Ut, dUt, float(t))
        return Ut, dUt

    def rk_steps(self, U, t, dt, nsteps):
        U = np.array(U, dtype=np.float64, copy=True, order="C")
        self._L.orc_rk_steps(self._h, U, float(t), float(dt), int(nsteps))
        return U

    def rk_steps_tl(self, U, dU, dmu, t, dt, nsteps):
        self._tl_check()
        U = np.array(U, dtype=np.float64, copy=True, order="C")
        dU = np.array(dU, dtype=np.float64, copy=True, order="C")
        self._L.orc_rk_steps_tl(self._h, U, dU, float(dmu), float(t), float(dt), int(nsteps))
        return U, dU

    def count_ops(self, U, t=0.0):
        """Operations of one R(U) evaluation of this oracle (LGL operator),
        counted by its counting scalar: dict add/mul/div/sqrt/log."""
        out = np.zeros(5)
        self._L.orc_count_ops(self._h, np.ascontiguousarray(U, dtype=np.float64), float(t), out)
        return dict(zip(_OP_NAMES, (int(v) for v in out)))

    def set_vol_flux(self, kind: int):
        self._L.orc_set_vol_flux(self._h, int(kind))

    def set_fv_mask(self, mask):
        """Switch the elements with mask[e] != 0 to the FV sub-cell operator
        ((N+1)^3 sub-cells, MUSCL-minmod reconstruction, LLF sub-face fluxes);
        None restores the pure DG operator.  Either node set."""
        if mask is None:
            self._L.orc_set_fv_mask(self._h, None)
            self.fv_mask = None
            return
        m = np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0, dtype=np.int32)
        if m.shape[0] != self.E:
            raise ValueError("oracle: the FV mask needs one entry per element")
        if self._L.orc_set_fv_mask(self._h, m.ctypes.data) != 0:
            raise ValueError("oracle: an element with a mortar face stays a DG element")
        self.fv_mask = m

    def set_fv_switch(self, var, log10_upper=None, log10_lower=None):
        """Automatic DG/FV switching before every evaluation of R(U): the
        Persson indicator of rho (var 0), p (1) or rho p (2) of the evaluated
        state; above 10^log10_upper an element becomes an FV element, below
        10^log10_lower a DG element, in between it keeps its representation.
        var None turns it off (the mask in effect stays)."""
        if var is None:
            self._L.orc_set_fv_switch(self._h, -1, 0.0, 0.0)
            return
        if log10_lower is None:
            log10_lower = log10_upper
        r = self._L.orc_set_fv_switch(self._h, int(var), float(log10_upper), float(log10_lower))
        if r != 0:
            raise ValueError("oracle: bad switching arguments")

    def fv_state(self):
        """(the FV mask in effect, the smallest distance of a log10 indicator
        value from a switching threshold since the last call)."""
        m = np.zeros(self.E, dtype=np.int32)
        margin = self._L.orc_fv_state(self._h, m.ctypes.data)
        return m, margin

    def lifting(self, U):
        G = np.zeros((self.E, 12, self.P))
        self._L.orc_lifting(self._h, np.ascontiguousarray(U, dtype=np.float64), G)
        return G

    def volume_term(self, U):
        out = np.zeros((self.E, 5, self.P))
        self._L.orc_volume_term(self._h, np.ascontiguousarray(U, dtype=np.float64), out)
        return out

    def persson(self, U, var: int = 2):
        """Persson modal indicator eta per element of rho (var 0), p (1) or
        rho p (2), at the context's nodes."""
        out = np.zeros(self.E)
        self._L.orc_persson(self._h, np.ascontiguousarray(U, dtype=np.float64), int(var), out)
        return out

    def integrals(self, U):
        out = np.zeros(8)
        self._L.orc_integrals(self._h, np.ascontiguousarray(U, dtype=np.float64), out)
        return out

    def node_coords(self):
        X = np.zeros((self.E, 3, self.P))
        self._L.orc_node_coords(self._h, X)
        return X

    def initial_state(self, kind: str, prm0: float):
        U = np.zeros(self.shape)
        self._L.orc_initial_state(self._h, {"tgv": 0, "mms": 1}[kind], float(prm0), U)
        return U
