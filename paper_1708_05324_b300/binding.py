"""Thin ctypes binding of libgmmnlse.so (include/gmmnlse.h).

Argument marshalling only: every step of the propagation runs in the CUDA
library.  Host arrays are numpy complex128 [N][Nt]; device arrays may be
torch complex128 CUDA tensors (used only for memory and streams).  If the
library is missing this module raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgmmnlse.so")

OK, PENDING = 0, 1
E_INVALID, E_NOMEM, E_UNSUPPORTED, E_NOT_CONVERGED = -1, -2, -3, -4
E_NONFINITE, E_CUDA, E_BUSY, E_CANCELLED = -5, -6, -7, -8
FP64, FP32, MIXED_BF16, MIXED_FP16, MIXED_TF32 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": MIXED_BF16, "fp16": MIXED_FP16, "tf32": MIXED_TF32}

# every function include/gmmnlse.h declares
EXPORTS = [
    "gmmnlse_create", "gmmnlse_create_general", "gmmnlse_destroy", "gmmnlse_propagate", "gmmnlse_strerror",
    "gmmnlse_last_error", "gmmnlse_request_bytes", "gmmnlse_server_create",
    "gmmnlse_submit", "gmmnlse_poll", "gmmnlse_server_destroy", "gmmnlse_profile",
    "gmmnlse_propagate_noalloc", "gmmnlse_choose_m",
    "gmmnlse_propagate_rk4ip", "gmmnlse_set_linear_coupling",
    "gmmnlse_set_gain", "gmmnlse_overlap_tensor", "gmmnlse_set_gain_saturation",
    "gmmnlse_set_coupling_profile", "gmmnlse_choose_step", "gmmnlse_cancel",
    "gmmnlse_server_resident_bytes",
]
KERNELS = ["ip_to_time", "pairs_raman", "contract", "integrand", "trapz_norm", "advance"]


class Params(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("Nt", C.c_int), ("dt", C.c_double), ("lambda0", C.c_double),
        ("n2", C.c_double), ("self_steepening", C.c_int), ("precision", C.c_int),
        ("max_iter", C.c_int), ("fixed_iters", C.c_int), ("device", C.c_int),
        ("stream", C.c_void_p), ("io_device", C.c_int),
    ]


class Step(C.Structure):
    _fields_ = [("dz", C.c_double), ("M", C.c_int), ("z_nl", C.c_double), ("z_im", C.c_double),
                ("err_est", C.c_double), ("trials", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [
        ("z", C.c_double), ("long_steps", C.c_int), ("iters_total", C.c_int),
        ("iters_min", C.c_int), ("iters_max", C.c_int), ("iter_hist", C.c_int * 33),
        ("eps_max", C.c_double), ("eps_last", C.c_double),
        ("energy_in", C.c_double), ("energy_out", C.c_double),
        ("photons_in", C.c_double), ("photons_out", C.c_double), ("ms", C.c_double),
        ("coupling_rank", C.c_int),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "iter_hist"}
        d["iter_hist"] = list(self.iter_hist)
        return d


_lib = None


class GmmnlseError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = _lib.gmmnlse_strerror(status).decode() if _lib else str(status)
        if status == E_CUDA and _lib:
            msg += ": " + _lib.gmmnlse_last_error().decode()
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with python -m paper_1708_05324_b300.build")
    lib = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    vp = C.c_void_p
    lib.gmmnlse_create.argtypes = [C.POINTER(Params), vp, vp, vp, C.c_double, vp, C.POINTER(vp)]
    lib.gmmnlse_create_general.argtypes = [C.POINTER(Params), vp, vp, vp, C.c_double, vp, C.POINTER(vp)]
    lib.gmmnlse_destroy.argtypes = [vp]
    lib.gmmnlse_propagate.argtypes = [vp, vp, C.c_double, C.c_double, C.c_int, C.c_double, vp,
                                      C.POINTER(Stats)]
    lib.gmmnlse_strerror.restype = C.c_char_p
    lib.gmmnlse_strerror.argtypes = [C.c_int]
    lib.gmmnlse_last_error.restype = C.c_char_p
    lib.gmmnlse_request_bytes.restype = C.c_size_t
    lib.gmmnlse_request_bytes.argtypes = [vp, C.c_int]
    lib.gmmnlse_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(vp)]
    lib.gmmnlse_submit.argtypes = [vp, vp, vp, C.c_double, C.c_double, C.c_int, C.c_double,
                                   C.POINTER(C.c_uint64)]
    lib.gmmnlse_poll.argtypes = [vp, C.c_uint64, vp, C.POINTER(Stats)]
    lib.gmmnlse_server_destroy.argtypes = [vp]
    lib.gmmnlse_cancel.argtypes = [vp, C.c_uint64]
    lib.gmmnlse_server_resident_bytes.argtypes = [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
    lib.gmmnlse_profile.argtypes = [vp, C.c_int, C.c_int, vp, vp]
    lib.gmmnlse_set_linear_coupling.argtypes = [vp, vp]
    lib.gmmnlse_set_gain.argtypes = [vp, vp]
    lib.gmmnlse_set_gain_saturation.argtypes = [vp, C.c_double]
    lib.gmmnlse_choose_step.argtypes = [vp, vp, C.c_double, C.c_double, C.c_double, vp, C.POINTER(Step)]
    lib.gmmnlse_set_coupling_profile.argtypes = [vp, vp, C.c_int, C.c_double]
    lib.gmmnlse_overlap_tensor.argtypes = [C.c_int, vp, C.c_int, C.c_longlong, C.c_double, vp]
    lib.gmmnlse_propagate_rk4ip.argtypes = [vp, vp, C.c_double, C.c_double, vp, C.POINTER(Stats)]
    lib.gmmnlse_choose_m.argtypes = [vp, vp, C.c_double, C.c_double, vp, C.c_int, C.c_int, vp, vp,
                                     C.POINTER(C.c_int)]
    lib.gmmnlse_propagate_noalloc.argtypes = [vp, vp, C.c_double, C.c_double, C.c_int, C.c_double, vp,
                                              C.POINTER(Stats)]
    del dp
    _lib = lib
    return lib


def _ptr(a):
    """Data pointer of a C-contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def overlap_tensor(F, dA, device=0):
    """gmmnlse_overlap_tensor: S [N][N][N][N] (Eq. 2) from profiles F [N][G]."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    if F.ndim != 2:
        raise ValueError("F must be [N][G]")
    N, G = F.shape
    S = np.empty((N, N, N, N))
    rc = load().gmmnlse_overlap_tensor(int(device), _ptr(F), N, G, float(dA), _ptr(S))
    if rc != OK:
        raise GmmnlseError(rc, "gmmnlse_overlap_tensor")
    return S


class Context:
    """A fiber uploaded to the device (gmmnlse_create; gmmnlse_create_general
    when S^K or S^R is complex)."""

    def __init__(self, N, Nt, dt, lambda0, n2, beta, SK, SR=None, fR=0.0, hR=None,
                 self_steepening=True, precision="fp64", max_iter=0, fixed_iters=0,
                 device=0, stream=None, io_device=False):
        self.lib = load()
        self.N, self.Nt = int(N), int(Nt)
        self._keep = []
        self.beta = np.ascontiguousarray(beta, dtype=np.float64)
        general = np.iscomplexobj(SK) or (SR is not None and np.iscomplexobj(SR))
        dt_s = np.complex128 if general else np.float64
        self.SK = np.ascontiguousarray(SK, dtype=dt_s)
        self.SR = None if SR is None else np.ascontiguousarray(SR, dtype=dt_s)
        self.hR = None if hR is None else np.ascontiguousarray(hR, dtype=np.float64)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.params = Params(self.N, self.Nt, float(dt), float(lambda0), float(n2),
                             1 if self_steepening else 0, prec, int(max_iter), int(fixed_iters),
                             int(device), stream, 1 if io_device else 0)
        h = C.c_void_p()
        create = self.lib.gmmnlse_create_general if general else self.lib.gmmnlse_create
        st = create(C.byref(self.params), _ptr(self.beta), _ptr(self.SK), _ptr(self.SR), float(fR),
                    _ptr(self.hR), C.byref(h))
        if st != OK:
            raise GmmnlseError(st, "gmmnlse_create_general" if general else "gmmnlse_create")
        self.handle = h

    @classmethod
    def from_problem(cls, prob, precision="fp64", **kw):
        return cls(prob.N, prob.Nt, prob.dt, prob.lam0, prob.n2, prob.beta, prob.SK,
                   None if prob.SR is prob.SK else prob.SR, prob.fR,
                   prob.hR if prob.fR else None, prob.self_steepening, precision, **kw)

    def propagate(self, A0, L, dz, M, tol, out=None, check=True):
        """Returns (Aout, stats dict, status).  A0/out: numpy complex128 [N][Nt]
        (or device tensors when the context was made with io_device=True)."""
        if isinstance(A0, np.ndarray):
            A0 = np.ascontiguousarray(A0, dtype=np.complex128)
            if A0.shape != (self.N, self.Nt):
                raise ValueError(f"A0 must be [{self.N}][{self.Nt}]")
            if out is None:
                out = np.empty_like(A0)
        st = Stats()
        rc = self.lib.gmmnlse_propagate(self.handle, _ptr(A0), float(L), float(dz), int(M),
                                        float(tol), _ptr(out), C.byref(st))
        if check and rc not in (OK,):
            raise GmmnlseError(rc, "gmmnlse_propagate")
        return out, st.as_dict(), rc

    def set_linear_coupling(self, Q):
        """gmmnlse_set_linear_coupling: Q [N][N] real (Q[n][p]), or None to remove."""
        if Q is not None:
            Q = np.ascontiguousarray(Q, dtype=np.float64)
            if Q.shape != (self.N, self.N):
                raise ValueError(f"Q must be [{self.N}][{self.N}]")
        rc = self.lib.gmmnlse_set_linear_coupling(self.handle, _ptr(Q))
        if rc != OK:
            raise GmmnlseError(rc, "gmmnlse_set_linear_coupling")

    def set_gain(self, g):
        """gmmnlse_set_gain: g [N] field gain per mode [1/m], or None to remove."""
        if g is not None:
            g = np.ascontiguousarray(g, dtype=np.float64)
            if g.shape != (self.N,):
                raise ValueError(f"g must be [{self.N}]")
        rc = self.lib.gmmnlse_set_gain(self.handle, _ptr(g))
        if rc != OK:
            raise GmmnlseError(rc, "gmmnlse_set_gain")

    def set_gain_saturation(self, sat):
        """gmmnlse_set_gain_saturation: the saturation coefficient (1/I_sat), 0 removes."""
        rc = self.lib.gmmnlse_set_gain_saturation(self.handle, float(sat))
        if rc != OK:
            raise GmmnlseError(rc, "gmmnlse_set_gain_saturation")

    def set_coupling_profile(self, f, fdz=None):
        """gmmnlse_set_coupling_profile: Q(z) = Q f(z), f sampled every fdz [m]; None removes."""
        if f is None:
            rc = self.lib.gmmnlse_set_coupling_profile(self.handle, None, 0, 0.0)
        else:
            f = np.ascontiguousarray(f, dtype=np.float64)
            rc = self.lib.gmmnlse_set_coupling_profile(self.handle, _ptr(f), len(f), float(fdz))
        if rc != OK:
            raise GmmnlseError(rc, "gmmnlse_set_coupling_profile")

    def propagate_rk4ip(self, A0, L, h, out=None, check=True):
        """gmmnlse_propagate_rk4ip: (Aout, stats dict, status); A0/out as for propagate."""
        if isinstance(A0, np.ndarray):
            A0 = np.ascontiguousarray(A0, dtype=np.complex128)
            if A0.shape != (self.N, self.Nt):
                raise ValueError(f"A0 must be [{self.N}][{self.Nt}]")
            if out is None:
                out = np.empty_like(A0)
        st = Stats()
        rc = self.lib.gmmnlse_propagate_rk4ip(self.handle, _ptr(A0), float(L), float(h), _ptr(out), C.byref(st))
        if check and rc != OK:
            raise GmmnlseError(rc, "gmmnlse_propagate_rk4ip")
        return out, st.as_dict(), rc

    def choose_m(self, A0, dz, tol, candidates, trial_substeps, scratch=None):
        """gmmnlse_choose_m: (fastest M, {M: device seconds per substep}).
        A0 and scratch as for propagate (scratch made like A0 if None)."""
        if isinstance(A0, np.ndarray):
            A0 = np.ascontiguousarray(A0, dtype=np.complex128)
            if A0.shape != (self.N, self.Nt):
                raise ValueError(f"A0 must be [{self.N}][{self.Nt}]")
            if scratch is None:
                scratch = np.empty_like(A0)
        elif scratch is None:
            scratch = A0.new_empty(A0.shape)
        cand = np.ascontiguousarray(candidates, dtype=np.int32)
        sec = np.zeros(len(cand))
        best = C.c_int(0)
        rc = self.lib.gmmnlse_choose_m(self.handle, _ptr(A0), float(dz), float(tol), _ptr(cand),
                                       len(cand), int(trial_substeps), _ptr(scratch), _ptr(sec),
                                       C.byref(best))
        if rc != OK:
            raise GmmnlseError(rc, "gmmnlse_choose_m")
        return best.value, {int(m): float(t) for m, t in zip(cand, sec)}

    def choose_step(self, A0, L, rtol, tol, scratch=None):
        """gmmnlse_choose_step: dict of dz, M, z_nl, z_im, err_est, trials.
        A0 as for propagate; scratch [2][N][Nt] made like A0 if None."""
        if isinstance(A0, np.ndarray):
            A0 = np.ascontiguousarray(A0, dtype=np.complex128)
            if scratch is None:
                scratch = np.empty((2,) + A0.shape, dtype=np.complex128)
        elif scratch is None:
            scratch = A0.new_empty((2,) + tuple(A0.shape))
        out = Step()
        rc = self.lib.gmmnlse_choose_step(self.handle, _ptr(A0), float(L), float(rtol), float(tol), _ptr(scratch),
                                          C.byref(out))
        if rc != OK:
            raise GmmnlseError(rc, "gmmnlse_choose_step")
        return out.as_dict()

    def profile(self, M, reps=20):
        """Mean device time [ms] and algorithmic bytes per launch of each
        kernel of one iteration, keyed by KERNELS."""
        ms = np.zeros(6)
        by = np.zeros(6)
        st = self.lib.gmmnlse_profile(self.handle, int(M), int(reps), _ptr(ms), _ptr(by))
        if st != OK:
            raise GmmnlseError(st, "gmmnlse_profile")
        return {k: (float(ms[i]), float(by[i])) for i, k in enumerate(KERNELS)}

    def request_bytes(self, M):
        return int(self.lib.gmmnlse_request_bytes(self.handle, int(M)))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gmmnlse_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (gmmnlse_server_*)."""

    def __init__(self, hbm_budget, max_inflight):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.gmmnlse_server_create(int(hbm_budget), int(max_inflight), C.byref(h))
        if st != OK:
            raise GmmnlseError(st, "gmmnlse_server_create")
        self.handle = h

    def submit(self, ctx: Context, A0, L, dz, M, tol):
        A0 = np.ascontiguousarray(A0, dtype=np.complex128)
        t = C.c_uint64()
        st = self.lib.gmmnlse_submit(self.handle, ctx.handle, _ptr(A0), float(L), float(dz),
                                     int(M), float(tol), C.byref(t))
        if st != OK:
            raise GmmnlseError(st, "gmmnlse_submit")
        return int(t.value)

    def poll(self, ticket, N, Nt):
        out = np.empty((N, Nt), dtype=np.complex128)
        st = Stats()
        rc = self.lib.gmmnlse_poll(self.handle, C.c_uint64(ticket), _ptr(out), C.byref(st))
        return rc, out, st.as_dict()

    def cancel(self, ticket):
        """gmmnlse_cancel: the status code (OK, E_BUSY when already running)."""
        return self.lib.gmmnlse_cancel(self.handle, C.c_uint64(ticket))

    def resident_bytes(self):
        """(now, peak) device bytes held by the server's workspaces."""
        now, peak = C.c_size_t(), C.c_size_t()
        rc = self.lib.gmmnlse_server_resident_bytes(self.handle, C.byref(now), C.byref(peak))
        if rc != OK:
            raise GmmnlseError(rc, "gmmnlse_server_resident_bytes")
        return int(now.value), int(peak.value)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gmmnlse_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
