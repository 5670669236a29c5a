"""Thin ctypes binding of the C ABI in include/elder.h.

Argument marshalling only: every step of the time step runs in the CUDA
kernels of libelder.so.  Tensors are torch CUDA float64 tensors (device
memory and streams come from PyTorch); the calls are ordered on the current
torch stream.  Importing this module fails loudly when the library is
missing; ``paper_1906_01632_gb300.build.build()`` makes it.

Names follow the C ABI: ``elder_config_default``, ``elder_create``,
``elder_step``, ``elder_solve``, ``elder_moments``, ``elder_grad``,
``elder_fields``, ``elder_residual``, ``elder_jacobian``, ``elder_destroy``;
``Elder`` wraps a context with methods of the same names (without prefix).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

SECONDS_PER_YEAR = 365.25 * 86400.0

ELDER_OK, ELDER_EINVAL, ELDER_ENOMEM, ELDER_ECUDA, ELDER_ENOTCONV, ELDER_ETIMEOUT = range(6)
ELDER_FP64, ELDER_MIXED = 0, 1
ELDER_SMOOTH_JACOBI, ELDER_SMOOTH_ZLINE, ELDER_SMOOTH_ILU = 0, 1, 2
SAMPLE_STATUS = {0: "ok", 1: "newton_maxit", 2: "krylov_maxit", 3: "breakdown", 4: "nonfinite",
                 5: "linesearch"}


class elder_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("rho0", ctypes.c_double), ("rho1", ctypes.c_double),
                ("mu", ctypes.c_double), ("g", ctypes.c_double), ("Dm", ctypes.c_double),
                ("bc_mode", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_samples", ctypes.c_int), ("newton_maxit", ctypes.c_int),
                ("newton_tol_c", ctypes.c_double), ("newton_tol_p", ctypes.c_double),
                ("ls_max", ctypes.c_int), ("lin_rtol", ctypes.c_double),
                ("lin_maxit", ctypes.c_int), ("mg_levels", ctypes.c_int),
                ("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double),
                ("coarse_K_harmonic", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("autotune", ctypes.c_int), ("newton_estimate", ctypes.c_int),
                ("smoother", ctypes.c_int), ("omega_line", ctypes.c_double),
                ("mixed_newton_maxit", ctypes.c_int), ("ilu_beta", ctypes.c_double),
                ("omega_ilu", ctypes.c_double)]


class elder_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("newton_iters", ctypes.c_int32),
                ("krylov_iters", ctypes.c_int32), ("ls_cuts", ctypes.c_int32),
                ("res0", ctypes.c_double), ("res", ctypes.c_double),
                ("fp64_retry", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("salt_mass0", ctypes.c_double), ("salt_mass", ctypes.c_double),
                ("salt_inflow", ctypes.c_double)]


K_SMOOTH, K_SPMV, K_MGRES, K_RESIDUAL, K_JACOBIAN, K_SMOOTH0 = range(6)
KERNEL_CLASSES = {K_SMOOTH: "smooth", K_SPMV: "spmv", K_MGRES: "mg_residual",
                  K_RESIDUAL: "residual", K_JACOBIAN: "jacobian", K_SMOOTH0: "smooth0"}


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"libelder.so not found at {path}: run paper_1906_01632_gb300.build.build() "
            "(nvcc, sm_103a) first; there is no CPU fallback")
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.elder_config_default.argtypes = [ctypes.POINTER(elder_config), ip, ip, ip]
    lib.elder_create.argtypes = [ctypes.POINTER(elder_config), ctypes.POINTER(vp)]
    lib.elder_destroy.argtypes = [vp]
    lib.elder_last_error.argtypes = [vp]
    lib.elder_last_error.restype = ctypes.c_char_p
    lib.elder_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int)]
    lib.elder_fields.argtypes = [vp, ip, ip, vp, ctypes.c_double, vp, vp, vp]
    lib.elder_residual.argtypes = [vp, ip, vp, vp, vp, vp, vp, vp, ctypes.c_double, vp, vp]
    lib.elder_jacobian.argtypes = [vp, ip, vp, vp, vp, vp, ctypes.c_double, vp, vp]
    lib.elder_step.argtypes = [vp, ip, vp, vp, vp, vp, ctypes.c_double,
                               ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(elder_stats), vp]
    lib.elder_step_extrapolated.argtypes = [vp, ip, vp, vp, vp, vp, vp, vp, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(elder_stats), vp]
    lib.elder_step_predicted.argtypes = [vp, ip, vp, vp, ip, vp, vp, vp, vp, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(elder_stats), vp]
    lib.elder_solve.argtypes = [vp, ip, vp, vp, vp, vp, ctypes.c_double, ip, vp, vp,
                                ctypes.c_double, ctypes.POINTER(ctypes.c_int32), vp]
    lib.elder_smoother_apply.argtypes = [vp, ip, vp, vp, vp, vp, ctypes.c_double, ip, ip, vp,
                                         vp, vp]
    lib.elder_moments.argtypes = [vp, ip, vp, vp, ctypes.c_double, vp, vp, vp, vp]
    lib.elder_grad.argtypes = [vp, ip, vp, vp, vp, vp, ctypes.c_double, ip, dp, vp, vp, vp]
    lib.elder_initial_state.argtypes = [vp, ip, vp, vp, vp]
    lib.elder_profile.argtypes = [vp, ip]
    lib.elder_profile_read.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int64), dp, dp, dp]
    lib.elder_launch_count.argtypes = [ctypes.POINTER(ctypes.c_int64)]
    lib.elder_measure_peak.argtypes = [ip, dp, vp]
    lib.elder_autotune_choice.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_float)]
    lib.elder_graph_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_char_p)]
    lib.elder_autotune_result.argtypes = [vp, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_float)]
    lib.elder_residual_norms_static.argtypes = [ctypes.POINTER(elder_config), ip, vp, vp, vp, vp,
                                                vp, vp, ctypes.c_double, vp, vp, vp]
    lib.elder_gauss_legendre.argtypes = [ip, dp, dp]
    lib.elder_gpc_indices.argtypes = [ip, ip, ip, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int32), ip]
    lib.elder_gpc_project.argtypes = [ip, ip, vp, ip, ip, vp, vp, ip, vp, vp, vp, vp, vp]
    lib.elder_gpc_exceed.argtypes = [ip, ip, vp, ip, ip, vp, ip, vp, ip, vp, ctypes.c_double,
                                     vp, vp]
    lib.elder_gpc_exceed_engine.argtypes = [ip, ip, ip, vp, ip, ip, vp, ip, vp, ip, vp,
                                            ctypes.c_double, vp, vp]
    del dp
    return lib


_lib = _load()


def lib():
    return _lib


def _ptr(t: torch.Tensor | None, what: str):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: expected a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{what}: must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{what}: must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{what}: must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class ElderError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"elder error {code}: {msg}")
        self.code = code


def elder_config_default(nx, ny, nz, **overrides) -> elder_config:
    cfg = elder_config()
    rc = _lib.elder_config_default(ctypes.byref(cfg), nx, ny, nz)
    if rc != ELDER_OK:
        raise ElderError(rc, "elder_config_default")
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise AttributeError(f"elder_config has no field {k}")
        setattr(cfg, k, v)
    return cfg


def _stats_list(stats):
    return [{"status": s.status, "newton_iters": s.newton_iters,
             "krylov_iters": s.krylov_iters, "ls_cuts": s.ls_cuts, "res0": s.res0,
             "res": s.res, "fp64_retry": s.fp64_retry, "salt_mass0": s.salt_mass0,
             "salt_mass": s.salt_mass, "salt_inflow": s.salt_inflow} for s in stats]


class Elder:
    """A context of the C ABI (owns the hierarchy and device workspace)."""

    def __init__(self, cfg: elder_config):
        h = ctypes.c_void_p()
        rc = _lib.elder_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != ELDER_OK:
            raise ElderError(rc, _lib.elder_last_error(None).decode())
        self._h = h
        self.cfg = cfg
        N = ctypes.c_int64()
        C = ctypes.c_int64()
        L = ctypes.c_int()
        _lib.elder_sizes(h, ctypes.byref(N), ctypes.byref(C), ctypes.byref(L))
        self.N, self.C, self.levels = N.value, C.value, L.value

    def _check(self, rc, allow_notconv=False):
        if rc == ELDER_OK or (allow_notconv and rc == ELDER_ENOTCONV):
            return rc
        raise ElderError(rc, _lib.elder_last_error(self._h).decode())

    def destroy(self):
        if self._h:
            _lib.elder_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # --- entry points -----------------------------------------------------
    def initial_state(self, S, p=None, c=None, device="cuda", stream=None):
        p = p if p is not None else torch.empty(S * self.N, dtype=torch.float64, device=device)
        c = c if c is not None else torch.empty(S * self.N, dtype=torch.float64, device=device)
        self._check(_lib.elder_initial_state(self._h, S, _ptr(p, "p"), _ptr(c, "c"),
                                             _stream(stream)))
        return p, c

    def autotune_result(self):
        b = [ctypes.c_int(), ctypes.c_int(), ctypes.c_int()]
        ms = (ctypes.c_float * 9)()
        self._check(_lib.elder_autotune_result(self._h, *[ctypes.byref(x) for x in b], ms))
        cand = (128, 256, 512)
        names = ("smooth", "spmv", "mg_residual")
        return {"threads_per_block": dict(zip(names, (x.value for x in b))),
                "ms_per_launch": {n: dict(zip(cand, [round(ms[3 * i + q], 4) for q in range(3)]))
                                  for i, n in enumerate(names)}}

    def autotune_choice(self, kernel_class: int):
        """(threads per block, samples per CTA, ms of the 6 candidates) of one class."""
        bs, spc = ctypes.c_int(), ctypes.c_int()
        ms = (ctypes.c_float * 6)()
        self._check(_lib.elder_autotune_choice(self._h, kernel_class, ctypes.byref(bs),
                                               ctypes.byref(spc), ms))
        return bs.value, spc.value, [round(float(v), 4) for v in ms]

    def graph_status(self):
        """Device-controlled steps: (cached step graphs, replays, fallback note)."""
        n = ctypes.c_int()
        r = ctypes.c_int64()
        note = ctypes.c_char_p()
        self._check(_lib.elder_graph_status(self._h, ctypes.byref(n), ctypes.byref(r),
                                            ctypes.byref(note)))
        return n.value, r.value, (note.value or b"").decode()

    def profile(self, on: bool):
        self._check(_lib.elder_profile(self._h, 1 if on else 0))

    def profile_read(self, kernel_class: int):
        n = ctypes.c_int64()
        ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(_lib.elder_profile_read(self._h, kernel_class, ctypes.byref(n),
                                            ctypes.byref(ms), ctypes.byref(by), ctypes.byref(fl)))
        return {"launches": n.value, "ms": ms.value, "bytes": by.value, "flops": fl.value}

    def fields(self, S, kind, params, K_mean=4.845e-13, phi=None, K=None, stream=None):
        dev = params.device
        phi = phi if phi is not None else torch.empty(S * self.C, dtype=torch.float64, device=dev)
        K = K if K is not None else torch.empty(S * self.C, dtype=torch.float64, device=dev)
        self._check(_lib.elder_fields(self._h, S, kind, _ptr(params, "params"), K_mean,
                                      _ptr(phi, "phi"), _ptr(K, "K"), _stream(stream)))
        return phi, K

    def residual(self, S, phi, K, p, c, p_old, c_old, dt, R=None, stream=None):
        R = R if R is not None else torch.empty(S * self.N * 2, dtype=torch.float64, device=p.device)
        self._check(_lib.elder_residual(self._h, S, _ptr(phi, "phi"), _ptr(K, "K"), _ptr(p, "p"),
                                        _ptr(c, "c"), _ptr(p_old, "p_old"), _ptr(c_old, "c_old"),
                                        dt, _ptr(R, "R"), _stream(stream)))
        return R

    def jacobian(self, S, phi, K, p, c, dt, J=None, stream=None):
        J = J if J is not None else torch.empty(S * 27 * self.N * 4, dtype=torch.float64, device=p.device)
        self._check(_lib.elder_jacobian(self._h, S, _ptr(phi, "phi"), _ptr(K, "K"), _ptr(p, "p"),
                                        _ptr(c, "c"), dt, _ptr(J, "J"), _stream(stream)))
        return J

    def step(self, S, phi, K, p, c, dt, stream=None, raise_on_fail=False):
        """One implicit Euler step in place on p, c; returns (status[S], stats list)."""
        status = (ctypes.c_int32 * S)()
        stats = (elder_stats * S)()
        rc = _lib.elder_step(self._h, S, _ptr(phi, "phi"), _ptr(K, "K"), _ptr(p, "p"),
                             _ptr(c, "c"), dt, status, stats, _stream(stream))
        self._check(rc, allow_notconv=not raise_on_fail)
        st = np.frombuffer(status, dtype=np.int32).copy()
        return st, _stats_list(stats)

    def step_extrapolated(self, S, phi, K, p_prev, c_prev, p, c, dt, stream=None,
                          raise_on_fail=False):
        """One implicit Euler step started from 2 u^n - u^{n-1}: p_prev, c_prev
        hold u^{n-1} on entry and u^n on return; p, c hold u^n on entry and
        u^{n+1} on return.  Returns (status[S], stats list) as step."""
        status = (ctypes.c_int32 * S)()
        stats = (elder_stats * S)()
        rc = _lib.elder_step_extrapolated(self._h, S, _ptr(phi, "phi"), _ptr(K, "K"),
                                          _ptr(p_prev, "p_prev"), _ptr(c_prev, "c_prev"),
                                          _ptr(p, "p"), _ptr(c, "c"), dt, status, stats,
                                          _stream(stream))
        self._check(rc, allow_notconv=not raise_on_fail)
        return np.frombuffer(status, dtype=np.int32).copy(), _stats_list(stats)

    def step_predicted(self, S, phi, K, order, p_hist, c_hist, p, c, dt, stream=None,
                       raise_on_fail=False):
        """One implicit Euler step started from the order-1 (2 u^n - u^{n-1}) or
        order-2 (3 u^n - 3 u^{n-1} + u^{n-2}) extrapolation: p_hist, c_hist
        [order][S][N] hold (u^{n-1}[, u^{n-2}]) on entry and (u^n[, u^{n-1}]) on
        return; p, c hold u^n on entry and u^{n+1} on return.  Returns
        (status[S], stats list) as step."""
        for h, what in ((p_hist, "p_hist"), (c_hist, "c_hist")):
            if isinstance(h, torch.Tensor) and h.numel() < int(order) * S * self.N:
                raise ValueError(f"{what}: needs order * S * N = {int(order) * S * self.N} values")
        status = (ctypes.c_int32 * S)()
        stats = (elder_stats * S)()
        rc = _lib.elder_step_predicted(self._h, S, _ptr(phi, "phi"), _ptr(K, "K"), int(order),
                                       _ptr(p_hist, "p_hist"), _ptr(c_hist, "c_hist"),
                                       _ptr(p, "p"), _ptr(c, "c"), dt, status, stats,
                                       _stream(stream))
        self._check(rc, allow_notconv=not raise_on_fail)
        return np.frombuffer(status, dtype=np.int32).copy(), _stats_list(stats)

    def solve(self, S, phi, K, p, c, dt, rhs, transpose=False, rtol=1e-10, x=None, stream=None):
        x = x if x is not None else torch.empty_like(rhs)
        status = (ctypes.c_int32 * S)()
        rc = _lib.elder_solve(self._h, S, _ptr(phi, "phi"), _ptr(K, "K"), _ptr(p, "p"),
                              _ptr(c, "c"), dt, 1 if transpose else 0, _ptr(rhs, "rhs"),
                              _ptr(x, "x"), rtol, status, _stream(stream))
        self._check(rc, allow_notconv=True)
        return x, np.frombuffer(status, dtype=np.int32).copy()

    def smoother_apply(self, S, phi, K, p, c, dt, kind, r, transpose=False, z=None,
                       stream=None):
        """z = P^{-1} r (or P^{-T} r) of the finest level's smoother `kind`
        (ELDER_SMOOTH_*) linearised at (p, c); r, z: [S][N][2] FP64."""
        z = z if z is not None else torch.empty_like(r)
        self._check(_lib.elder_smoother_apply(self._h, S, _ptr(phi, "phi"), _ptr(K, "K"),
                                              _ptr(p, "p"), _ptr(c, "c"), dt, kind,
                                              1 if transpose else 0, _ptr(r, "r"), _ptr(z, "z"),
                                              _stream(stream)))
        return z

    def moments(self, S, c, w=None, threshold=0.5, stream=None):
        dev = c.device
        mean = torch.empty(self.N, dtype=torch.float64, device=dev)
        var = torch.empty_like(mean)
        pexc = torch.empty_like(mean)
        self._check(_lib.elder_moments(self._h, S, _ptr(c, "c"), _ptr(w, "w"), threshold,
                                       _ptr(mean, "mean"), _ptr(var, "var"),
                                       _ptr(pexc, "p_exceed"), _stream(stream)))
        return mean, var, pexc

    def grad(self, n_steps, phi, K, p0, c0, dt, ckpt_every=7, stream=None):
        """Objective J and dJ/dphi, dJ/dK (per cell) by the discrete adjoint."""
        Jv = ctypes.c_double(0.0)
        gphi = torch.empty(self.C, dtype=torch.float64, device=phi.device)
        gK = torch.empty_like(gphi)
        rc = _lib.elder_grad(self._h, n_steps, _ptr(phi, "phi"), _ptr(K, "K"), _ptr(p0, "p0"),
                             _ptr(c0, "c0"), dt, ckpt_every, ctypes.byref(Jv), _ptr(gphi, "dJ_dphi"),
                             _ptr(gK, "dJ_dK"), _stream(stream))
        self._check(rc)
        return Jv.value, gphi, gK


# module-level names of the C ABI
def elder_launch_count() -> int:
    n = ctypes.c_int64()
    _lib.elder_launch_count(ctypes.byref(n))
    return n.value


def elder_measure_peak(kind: str = "fp64", stream=None) -> float:
    """Measured FMA peak of the current device in GFLOP/s ("fp64" or "fp32")."""
    g = ctypes.c_double(0.0)
    rc = _lib.elder_measure_peak({"fp64": 0, "fp32": 1}[kind], ctypes.byref(g), _stream(stream))
    if rc != ELDER_OK:
        raise ElderError(rc, _lib.elder_last_error(None).decode())
    return g.value


def elder_residual_norms_static(cfg: elder_config, S, phi, K, p, c, p_old, c_old, dt,
                                R=None, norms=None, stream=None):
    """Residual and per-sample ||R|| without a context and without any device
    allocation inside the library (its scratch is a fixed 2 MiB device
    array).  R and norms are allocated here by torch unless passed in."""
    N = (cfg.nx + 1) * (cfg.ny + 1) * (cfg.nz + 1)
    dev = p.device
    R = R if R is not None else torch.empty(S * N * 2, dtype=torch.float64, device=dev)
    norms = norms if norms is not None else torch.empty(S, dtype=torch.float64, device=dev)
    for name, t in (("phi", phi), ("K", K), ("c", c), ("p_old", p_old), ("c_old", c_old),
                    ("R", R), ("norms", norms)):
        if isinstance(t, torch.Tensor) and t.device != dev:
            raise ValueError(f"{name} is on {t.device}, p on {dev}: all tensors must share a device")
    # the library launches on the current device: make it the tensors' one
    with torch.cuda.device(dev):
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        rc = _lib.elder_residual_norms_static(ctypes.byref(cfg), S, _ptr(phi, "phi"),
                                              _ptr(K, "K"), _ptr(p, "p"), _ptr(c, "c"),
                                              _ptr(p_old, "p_old"), _ptr(c_old, "c_old"), dt,
                                              _ptr(R, "R"), _ptr(norms, "norms"), _stream(st))
    if rc != ELDER_OK:
        raise ElderError(rc, _lib.elder_last_error(None).decode())
    return R, norms


def _static_check(rc):
    if rc != ELDER_OK:
        raise ElderError(rc, _lib.elder_last_error(None).decode())


def _iptr(t: torch.Tensor | None, what: str):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int32
            and t.is_contiguous()):
        raise ValueError(f"{what}: must be a contiguous int32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


GPC_RULES = {"total": 0, "tensor": 1, "hyperbolic": 2}


def elder_gauss_legendre(q: int):
    """q-point Gauss-Legendre rule on [-1, 1] (host numpy arrays x, w)."""
    x = np.zeros(q)
    w = np.zeros(q)
    dp = ctypes.POINTER(ctypes.c_double)
    _static_check(_lib.elder_gauss_legendre(q, x.ctypes.data_as(dp), w.ctypes.data_as(dp)))
    return x, w


def elder_gpc_indices(M: int, p: int, rule: str = "total") -> np.ndarray:
    """Truncated multi-index set J_{M,p} as an int32 [T, M] host array."""
    n = ctypes.c_int(0)
    _static_check(_lib.elder_gpc_indices(M, p, GPC_RULES[rule], ctypes.byref(n), None, 0))
    beta = np.zeros((n.value, M), dtype=np.int32)
    _static_check(_lib.elder_gpc_indices(M, p, GPC_RULES[rule], ctypes.byref(n),
                                         beta.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                         n.value))
    return beta


def elder_gpc_project(beta: torch.Tensor, theta: torch.Tensor, w: torch.Tensor, u: torch.Tensor,
                      coef=None, mean=None, var=None, stream=None):
    """Expansion coefficients [T, N] (FP64) plus mean and variance [N] from the
    fields u [Nq, N] at the quadrature points theta [Nq, M] with weights w."""
    T, M = beta.shape
    Nq, N = u.shape
    maxdeg = int(beta.max().item()) if beta.numel() else 0
    dev = u.device
    coef = coef if coef is not None else torch.empty(T, N, dtype=torch.float64, device=dev)
    mean = mean if mean is not None else torch.empty(N, dtype=torch.float64, device=dev)
    var = var if var is not None else torch.empty(N, dtype=torch.float64, device=dev)
    _static_check(_lib.elder_gpc_project(M, T, _iptr(beta, "beta"), maxdeg, Nq,
                                         _ptr(theta, "theta"), _ptr(w, "w"), N, _ptr(u, "u"),
                                         _ptr(coef, "coef"), _ptr(mean, "mean"),
                                         _ptr(var, "var"), _stream(stream)))
    return coef, mean, var


GPC_ENGINES = {"auto": 0, "fp32": 1, "tensor": 2}


def elder_gpc_exceed(beta: torch.Tensor, coef: torch.Tensor, theta: torch.Tensor,
                     threshold: float, nodes: torch.Tensor | None = None, out=None, stream=None,
                     engine: str = "auto"):
    """P(u_hat > threshold) per node from the surrogate at the sample points
    theta [Ns, M] (all N nodes, or the int32 node list); engine "auto", "fp32"
    (CUDA cores) or "tensor" (tcgen05 TF32 split product)."""
    T, M = beta.shape
    N = coef.shape[1]
    n_pts = N if nodes is None else nodes.numel()
    maxdeg = int(beta.max().item()) if beta.numel() else 0
    out = out if out is not None else torch.empty(n_pts, dtype=torch.float64, device=coef.device)
    _static_check(_lib.elder_gpc_exceed_engine(GPC_ENGINES[engine], M, T, _iptr(beta, "beta"),
                                               maxdeg, N, _ptr(coef, "coef"), n_pts,
                                               _iptr(nodes, "nodes"), theta.shape[0],
                                               _ptr(theta, "theta"), float(threshold),
                                               _ptr(out, "out"), _stream(stream)))
    return out


def elder_gpc_exceed_engine(engine: str, *a, **k):
    return elder_gpc_exceed(*a, engine=engine, **k)


def elder_initial_state(ctx: Elder, *a, **k):
    return ctx.initial_state(*a, **k)


def elder_autotune_result(ctx: Elder):
    return ctx.autotune_result()


def elder_profile(ctx: Elder, on: bool):
    return ctx.profile(on)


def elder_profile_read(ctx: Elder, kernel_class: int):
    return ctx.profile_read(kernel_class)


def elder_create(cfg: elder_config) -> Elder:
    return Elder(cfg)


def elder_destroy(ctx: Elder):
    ctx.destroy()


def elder_step(ctx: Elder, *a, **k):
    return ctx.step(*a, **k)


def elder_step_extrapolated(ctx: Elder, *a, **k):
    return ctx.step_extrapolated(*a, **k)


def elder_step_predicted(ctx: Elder, *a, **k):
    return ctx.step_predicted(*a, **k)


def elder_solve(ctx: Elder, *a, **k):
    return ctx.solve(*a, **k)


def elder_moments(ctx: Elder, *a, **k):
    return ctx.moments(*a, **k)


def elder_smoother_apply(ctx: Elder, *a, **k):
    return ctx.smoother_apply(*a, **k)


def elder_grad(ctx: Elder, *a, **k):
    return ctx.grad(*a, **k)


def elder_fields(ctx: Elder, *a, **k):
    return ctx.fields(*a, **k)


def elder_residual(ctx: Elder, *a, **k):
    return ctx.residual(*a, **k)


def elder_jacobian(ctx: Elder, *a, **k):
    return ctx.jacobian(*a, **k)


def elder_graph_status(ctx: Elder):
    return ctx.graph_status()


def elder_autotune_choice(ctx: Elder, kernel_class: int):
    return ctx.autotune_choice(kernel_class)


class ElderRollout(torch.autograd.Function):
    """Salt mass below mid-depth after n_steps implicit steps of one sample,
    differentiable w.r.t. the per-cell porosity and permeability through the
    library's discrete adjoint (elder_grad)."""

    @staticmethod
    def forward(ctx, phi, K, p0, c0, elder: Elder, n_steps: int, dt: float, ckpt_every: int = 7):
        J, gphi, gK = elder.grad(n_steps, phi.detach().contiguous(), K.detach().contiguous(),
                                 p0.contiguous(), c0.contiguous(), dt, ckpt_every)
        ctx.save_for_backward(gphi, gK)
        return torch.tensor(J, dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, gout):
        gphi, gK = ctx.saved_tensors
        return gout * gphi, gout * gK, None, None, None, None, None, None
