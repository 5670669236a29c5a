"""FP64 CPU oracle for the implicit Elder step (arXiv:1906.01632).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use this
package; the product path in ``paper_1906_01632_gb300`` never does.  It
shares no code with the CUDA path.

The C sources (``elder_oracle.c``) hold the arithmetic; this module only
compiles them with gcc and marshals numpy arrays through ctypes.  Each C
function cites the passage of the paper it follows (model: Section 2.1,
discretisation: Section 2.3 / 5.1, statistics: Section 3).

Parity status: the discretisation is pinned by the closed forms and
invariants in tests/test_oracle_*.py (1D reduction to the lumped 3-point
scheme, hydrostatic state, salt- and fluid-mass balance, mirror symmetry,
linear-pressure Darcy flux, upwind direction).  The reading of the
"consistent velocity" gravity term has no printed number to pin against in
the paper; it is pinned only by its hydrostatic invariant.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "elder_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lib = None

SECONDS_PER_YEAR = 365.25 * 86400.0  # Julian year: the paper gives no length


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(
                os.path.join(_HERE, "elder_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
                ("Lz", ctypes.c_double), ("rho0", ctypes.c_double),
                ("rho1", ctypes.c_double), ("mu", ctypes.c_double),
                ("g", ctypes.c_double), ("Dm", ctypes.c_double),
                ("bc_mode", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("maxit", ctypes.c_int), ("tol_c", ctypes.c_double),
                ("tol_p", ctypes.c_double), ("lin_rtol", ctypes.c_double),
                ("lin_maxit", ctypes.c_int), ("ls_max", ctypes.c_int),
                ("dense_max", ctypes.c_int), ("smoother", ctypes.c_int),
                ("ilu_beta", ctypes.c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("lin_iters", ctypes.c_int), ("ls_cuts", ctypes.c_int),
                ("res0", ctypes.c_double), ("res", ctypes.c_double)]


@dataclass
class Problem:
    """Elder box problem (Table 1 constants; Dm as in the benchmark configs)."""
    nx: int
    ny: int
    nz: int
    Lx: float = 600.0
    Ly: float = 600.0
    Lz: float = 150.0
    rho0: float = 1000.0
    rho1: float = 1200.0
    mu: float = 1e-3
    g: float = 9.81
    Dm: float = 3.565e-6
    bc_mode: int = 0

    @property
    def N(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def C(self) -> int:
        return self.nx * self.ny * self.nz

    def _c(self) -> _Problem:
        return _Problem(self.nx, self.ny, self.nz, self.Lx, self.Ly, self.Lz,
                        self.rho0, self.rho1, self.mu, self.g, self.Dm,
                        self.bc_mode)


@dataclass
class NewtonOpts:
    maxit: int = 25
    tol_c: float = 1e-12
    tol_p: float = 1e-12 * 1000.0 * 9.81 * 150.0
    lin_rtol: float = 1e-12
    lin_maxit: int = 2000
    ls_max: int = 6
    dense_max: int = 1200
    # 0 point block Jacobi, 1 vertical-line block Jacobi, 2 multicolour
    # block ILU_beta(0) with beta = ilu_beta
    smoother: int = 0
    ilu_beta: float = 0.0

    def _c(self) -> _Opts:
        return _Opts(self.maxit, self.tol_c, self.tol_p, self.lin_rtol,
                     self.lin_maxit, self.ls_max, self.dense_max, self.smoother,
                     self.ilu_beta)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        _lib.orc_objective.restype = ctypes.c_double
        _lib.orc_num_nodes.restype = ctypes.c_int
        del d
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def dirichlet(P: Problem):
    pm = np.zeros(P.N, np.uint8)
    cm = np.zeros(P.N, np.uint8)
    cv = np.zeros(P.N)
    u8 = ctypes.POINTER(ctypes.c_ubyte)
    lib().orc_dirichlet(ctypes.byref(P._c()), pm.ctypes.data_as(u8),
                        cm.ctypes.data_as(u8), _dp(cv))
    return pm.astype(bool), cm.astype(bool), cv


def initial_state(P: Problem):
    p = np.zeros(P.N)
    c = np.zeros(P.N)
    lib().orc_initial_state(ctypes.byref(P._c()), _dp(p), _dp(c))
    return p, c


def residual(P: Problem, phi, K, p, c, p_old, c_old, dt, apply_dirichlet=True):
    phi, K, p, c, p_old, c_old = map(_f64, (phi, K, p, c, p_old, c_old))
    Rp = np.zeros(P.N)
    Rc = np.zeros(P.N)
    lib().orc_residual(ctypes.byref(P._c()), _dp(phi), _dp(K), _dp(p), _dp(c),
                       _dp(p_old), _dp(c_old), ctypes.c_double(dt),
                       ctypes.c_int(1 if apply_dirichlet else 0), _dp(Rp), _dp(Rc))
    return Rp, Rc


def residual_magnitude(P: Problem, phi, K, p, c, c_old, dt) -> float:
    """2-norm of the per-row sums of the magnitudes of the residual's terms
    (its round-off scale); Newton treats ||R|| <= 2 eps times this as solved."""
    lib().orc_residual_magnitude.restype = ctypes.c_double
    return float(lib().orc_residual_magnitude(ctypes.byref(P._c()), _dp(_f64(phi)), _dp(_f64(K)),
                                              _dp(_f64(p)), _dp(_f64(c)), _dp(_f64(c_old)),
                                              ctypes.c_double(dt)))


def jacobian_csr(P: Problem, phi, K, p, c, dt):
    """Exact Jacobian as (rowptr, col, val); unknowns interleaved (p_n, c_n)."""
    phi, K, p, c = map(_f64, (phi, K, p, c))
    L = lib()
    pc = P._c()
    nnz = L.orc_jac_nnz(ctypes.byref(pc))
    rowptr = np.zeros(2 * P.N + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz)
    L.orc_jac_pattern(ctypes.byref(pc), _ip(rowptr), _ip(col))
    L.orc_jacobian(ctypes.byref(pc), _dp(phi), _dp(K), _dp(p), _dp(c),
                   ctypes.c_double(dt), _ip(rowptr), _ip(col), _dp(val))
    return rowptr, col, val


def jacobian_dense(P: Problem, phi, K, p, c, dt) -> np.ndarray:
    rowptr, col, val = jacobian_csr(P, phi, K, p, c, dt)
    n = 2 * P.N
    A = np.zeros((n, n))
    for r in range(n):
        A[r, col[rowptr[r]:rowptr[r + 1]]] += val[rowptr[r]:rowptr[r + 1]]
    return A


def dense_solve(A, b):
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    x = np.array(b, dtype=np.float64, copy=True)
    rc = lib().orc_dense_solve(ctypes.c_int(A.shape[0]), _dp(A), _dp(x))
    if rc != 0:
        raise np.linalg.LinAlgError("zero pivot")
    return x


def bicgstab_ilu0(rowptr, col, val, b, rtol=1e-12, maxit=20000):
    b = _f64(b)
    x = np.zeros_like(b)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    rc = lib().orc_bicgstab_ilu0(ctypes.c_int(b.size), _ip(rowptr), _ip(col),
                                 _dp(_f64(val)), _dp(b), _dp(x), ctypes.c_double(rtol),
                                 ctypes.c_int(maxit), ctypes.byref(it), ctypes.byref(rr))
    return x, rc, it.value, rr.value


def linear_solve(rowptr, col, val, b, opts: NewtonOpts | None = None, transpose=False):
    """Solve J x = b (or J^T x = b) with the oracle's solver choice."""
    opts = opts or NewtonOpts()
    b = _f64(b)
    n = b.size
    if transpose:
        tr = np.zeros(n + 1, np.int32)
        tc = np.zeros(col.size, np.int32)
        tv = np.zeros(col.size)
        lib().orc_csr_transpose(ctypes.c_int(n), _ip(rowptr), _ip(col), _dp(_f64(val)),
                                _ip(tr), _ip(tc), _dp(tv))
        rowptr, col, val = tr, tc, tv
    x = np.zeros(n)
    it = ctypes.c_int(0)
    rc = lib().orc_linear_solve(ctypes.c_int(n), _ip(rowptr), _ip(col), _dp(_f64(val)),
                                _dp(b), _dp(x), ctypes.byref(opts._c()), ctypes.byref(it))
    return x, rc


def mc_rank(P: Problem) -> np.ndarray:
    """Position of every node in the multicolour order (colour = (i&1) +
    2(j&1) + 4(k&1) ascending, node index order within a colour)."""
    rank = np.zeros(P.N, np.int32)
    lib().orc_mc_rank(ctypes.byref(P._c()), _ip(rank))
    return rank


def csr_to_blocks(P: Problem, rowptr, col, val) -> np.ndarray:
    """Block form [N][27][4] of a CSR matrix with the 27-point block pattern:
    [n][s] = block (n, n+d), s = (dx+1) + 3(dy+1) + 9(dz+1), (pp, pc, cp, cc)."""
    B = np.zeros((P.N, 27, 4))
    lib().orc_csr_to_blocks(ctypes.byref(P._c()), _ip(np.ascontiguousarray(rowptr, np.int32)),
                            _ip(np.ascontiguousarray(col, np.int32)), _dp(_f64(val)), _dp(B))
    return B


def mcilu_factor(P: Problem, B, beta=0.0) -> np.ndarray:
    """Multicolour block ILU_beta(0) factors of the block matrix B [N][27][4]
    (slots of earlier-ranked neighbours: L; the others: U, pivots in slot 13)."""
    B = np.ascontiguousarray(B, dtype=np.float64)
    F = np.zeros_like(B)
    rc = lib().orc_mcilu_factor(ctypes.byref(P._c()), _dp(B), ctypes.c_double(beta), _dp(F))
    if rc != 0:
        raise np.linalg.LinAlgError("singular pivot block")
    return F


def mcilu_solve(P: Problem, F, r, transpose=False) -> np.ndarray:
    """z = (L U)^{-1} r, or (L U)^{-T} r, with the factors of mcilu_factor."""
    z = np.zeros(2 * P.N)
    lib().orc_mcilu_solve(ctypes.byref(P._c()), _dp(np.ascontiguousarray(F, dtype=np.float64)),
                          ctypes.c_int(1 if transpose else 0), _dp(_f64(r)), _dp(z))
    return z


def smoother_apply(P: Problem, phi, K, p, c, dt, kind, r, beta=0.0, transpose=False):
    """z = P^{-1} r (or P^{-T} r) for the finest level's smoother at (p, c):
    kind 0 block diagonal, 1 vertical-line block tridiagonal, 2 L U of the
    multicolour block ILU_beta(0); interior unknowns only (Dirichlet
    components of r ignored, of z zero)."""
    z = np.zeros(2 * P.N)
    rc = lib().orc_smoother_apply(ctypes.byref(P._c()), _dp(_f64(phi)), _dp(_f64(K)),
                                  _dp(_f64(p)), _dp(_f64(c)), ctypes.c_double(dt),
                                  ctypes.c_int(kind), ctypes.c_double(beta),
                                  ctypes.c_int(1 if transpose else 0), _dp(_f64(r)), _dp(z))
    if rc != 0:
        raise RuntimeError("orc_smoother_apply failed (singular pivot or coarse grid too large)")
    return z


def newton_step(P: Problem, phi, K, p, c, dt, opts: NewtonOpts | None = None):
    """One implicit Euler step; returns (p_new, c_new, info dict)."""
    opts = opts or NewtonOpts()
    p = np.array(p, dtype=np.float64, copy=True)
    c = np.array(c, dtype=np.float64, copy=True)
    info = _Info()
    lib().orc_newton_step(ctypes.byref(P._c()), _dp(_f64(phi)), _dp(_f64(K)),
                          _dp(p), _dp(c), ctypes.c_double(dt),
                          ctypes.byref(opts._c()), ctypes.byref(info))
    return p, c, {"status": info.status, "newton_iters": info.newton_iters,
                  "lin_iters": info.lin_iters, "ls_cuts": info.ls_cuts,
                  "res0": info.res0, "res": info.res}


def run_steps(P: Problem, phi, K, p, c, dt, n_steps, opts=None):
    infos = []
    for _ in range(n_steps):
        p, c, info = newton_step(P, phi, K, p, c, dt, opts)
        infos.append(info)
    return p, c, infos


def moments(c_samples, w=None, threshold=0.5):
    c_samples = _f64(c_samples)
    S, N = c_samples.shape
    mean = np.zeros(N)
    var = np.zeros(N)
    pexc = np.zeros(N)
    wp = _dp(_f64(w)) if w is not None else None
    lib().orc_moments(ctypes.c_int(S), ctypes.c_int(N), _dp(c_samples), wp,
                      ctypes.c_double(threshold), _dp(mean), _dp(var), _dp(pexc))
    return mean, var, pexc


def fields_sobol(P: Problem, xi, K_mean=4.845e-13):
    phi = np.zeros(P.C)
    K = np.zeros(P.C)
    lib().orc_fields_sobol(ctypes.byref(P._c()), _dp(_f64(xi)), ctypes.c_double(K_mean),
                           _dp(phi), _dp(K))
    return phi, K


def fields_lognormal(P: Problem, Z, K_mean=4.845e-13):
    phi = np.zeros(P.C)
    K = np.zeros(P.C)
    lib().orc_fields_lognormal(ctypes.byref(P._c()), _dp(_f64(Z)), ctypes.c_double(K_mean),
                               _dp(phi), _dp(K))
    return phi, K


def fields_paper3rv(P: Problem, xi, K_mean=4.845e-13):
    phi = np.zeros(P.C)
    K = np.zeros(P.C)
    lib().orc_fields_paper3rv(ctypes.byref(P._c()), _dp(_f64(xi)), ctypes.c_double(K_mean),
                              _dp(phi), _dp(K))
    return phi, K


def objective(P: Problem, phi, c) -> float:
    return float(lib().orc_objective(ctypes.byref(P._c()), _dp(_f64(phi)), _dp(_f64(c))))


def adjoint_gradient(P: Problem, phi, K, p0, c0, dt, n_steps, opts=None):
    """Returns (J, dJ/dphi [C], dJ/dK [C], rc)."""
    opts = opts or NewtonOpts()
    Jv = ctypes.c_double(0.0)
    gphi = np.zeros(P.C)
    gK = np.zeros(P.C)
    rc = lib().orc_adjoint_gradient(ctypes.byref(P._c()), _dp(_f64(phi)), _dp(_f64(K)),
                                    _dp(_f64(p0)), _dp(_f64(c0)), ctypes.c_double(dt),
                                    ctypes.c_int(n_steps), ctypes.byref(opts._c()),
                                    ctypes.byref(Jv), _dp(gphi), _dp(gK))
    return Jv.value, gphi, gK, rc
