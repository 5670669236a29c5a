"""The multigrid smoothers on the GPU against the oracle's (Section 5.1),
element by element, through elder_smoother_apply: z = P^{-1} r (and P^{-T} r)
on the finest level with P the 2x2 block diagonal, the vertical-line block
tridiagonal part, or L U of the multicolour block ILU_beta(0) factors.  The
oracle's smoothers are pinned in tests/test_oracle_ilu.py against dense
linear algebra.

FP64 contexts: agreement to 1e-11 of max |z| (the factorisations are exact up
to rounding order).  ELDER_MIXED: bfloat16 matrices and factors with FP32
arithmetic: a relative 2-norm error of a few 1e-3 per stored rounding;
the bound 3e-2 still fails any indexing or colour-order error (O(1)).

Then the ILU smoother inside the solver: elder_solve (J and J^T) against a
dense LU, and implicit steps against the oracle's states.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

YEAR = O.SECONDS_PER_YEAR
DEV = "cuda:0"
DT = YEAR / 12


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_01632_gb300 import build
    build.build()
    from paper_1906_01632_gb300 import elder
    return elder


def T(a):
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device=DEV)


def H(t):
    return t.detach().cpu().numpy()


def _case(P, S, seed):
    """Per sample: a lognormal porosity field and the state after one oracle
    step from a perturbed initial state (upwinding in every direction)."""
    rng = np.random.default_rng(seed)
    phi = np.zeros((S, P.C))
    K = np.zeros((S, P.C))
    p = np.zeros((S, P.N))
    c = np.zeros((S, P.N))
    p0, c0 = O.initial_state(P)
    for s in range(S):
        phi[s], K[s] = O.fields_lognormal(P, rng.standard_normal(P.C))
        p[s] = p0 + rng.normal(0, 2e3, P.N)
        c[s] = np.clip(c0 + rng.uniform(0, 0.5, P.N), 0, 1)
    return phi, K, p, c


KINDS = {0: "jacobi", 1: "zline", 2: "ilu"}


@pytest.mark.parametrize("dims,bc", [((16, 16, 4), 0), ((12, 10, 6), 2)])
@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("transpose", [False, True])
def test_smoother_apply_fp64_matches_oracle(E, dims, bc, kind, transpose):
    """12x10x6 with the diffusion-column boundary set (it coarsens to 6x5x3):
    13x11x7 nodes, colour classes of unequal sizes."""
    P = O.Problem(*dims, bc_mode=bc)
    S = 3
    phi, K, p, c = _case(P, S, 100 + kind)
    rng = np.random.default_rng(7)
    r = rng.standard_normal((S, 2 * P.N))
    betas = (0.0, 0.5) if kind == 2 else (0.0,)
    for beta in betas:
        ctx = E.elder_create(E.elder_config_default(*dims, max_samples=S, ilu_beta=beta,
                                                    bc_mode=bc))
        z = H(ctx.smoother_apply(S, T(phi), T(K), T(p), T(c), DT, kind, T(r),
                                 transpose=transpose)).reshape(S, -1)
        ctx.destroy()
        for s in range(S):
            ref = O.smoother_apply(P, phi[s], K[s], p[s], c[s], DT, kind, r[s], beta=beta,
                                   transpose=transpose)
            err = np.abs(z[s] - ref).max()
            assert err <= 1e-11 * np.abs(ref).max(), (KINDS[kind], beta, s, err)


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("transpose", [False, True])
def test_smoother_apply_mixed_within_bfloat16_rounding(E, kind, transpose):
    P = O.Problem(16, 16, 4)
    S = 2
    phi, K, p, c = _case(P, S, 200 + kind)
    r = np.random.default_rng(8).standard_normal((S, 2 * P.N))
    ctx = E.elder_create(E.elder_config_default(16, 16, 4, max_samples=S,
                                                precision=E.ELDER_MIXED))
    z = H(ctx.smoother_apply(S, T(phi), T(K), T(p), T(c), DT, kind, T(r),
                             transpose=transpose)).reshape(S, -1)
    ctx.destroy()
    for s in range(S):
        ref = O.smoother_apply(P, phi[s], K[s], p[s], c[s], DT, kind, r[s],
                               transpose=transpose)
        # per component (p and c rows differ in scale by many orders)
        for comp in (0, 1):
            a, b = z[s][comp::2], ref[comp::2]
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert rel <= 3e-2, (KINDS[kind], s, comp, rel)


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
def test_ilu_smoother_solve_matches_dense_lu(E, transpose, precision):
    """The ILU smoother in elder_solve's V-cycle (8x8x4, two smoothed
    levels), J and J^T, against a dense LU of the oracle Jacobian."""
    P = O.Problem(8, 8, 4)
    S = 3
    ctx = E.elder_create(E.elder_config_default(8, 8, 4, max_samples=S, precision=precision,
                                                smoother=E.ELDER_SMOOTH_ILU))
    phi, K, p, c = _case(P, S, 17)
    rhs = np.random.default_rng(18).standard_normal((S, P.N, 2))
    x, st = ctx.solve(S, T(phi), T(K), T(p), T(c), DT, T(rhs), transpose=transpose, rtol=1e-12)
    assert (st == 0).all()
    x = H(x).reshape(S, 2 * P.N)
    for s in range(S):
        A = O.jacobian_dense(P, phi[s], K[s], p[s], c[s], DT)
        ref = O.dense_solve(A.T if transpose else A, rhs[s].ravel())
        scale = np.abs(ref).reshape(-1, 2).max(axis=0)
        err = np.abs(x[s] - ref).reshape(-1, 2).max(axis=0)
        assert (err <= 1e-9 * scale).all(), (err, scale)
    ctx.destroy()


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_steps_with_the_ilu_smoother_match_oracle(E, precision, tol):
    """Five implicit steps at 16x16x4, three samples, with the ILU smoother
    (Krylov rtol 1e-2, V(1,0)), against the oracle's states."""
    P = O.Problem(16, 16, 4)
    S = 3
    rng = np.random.default_rng(9)
    phi = np.zeros((S, P.C))
    K = np.zeros((S, P.C))
    for s in range(S):
        phi[s], K[s] = O.fields_lognormal(P, rng.standard_normal(P.C))
    p0, c0 = O.initial_state(P)
    ctx = E.elder_create(E.elder_config_default(16, 16, 4, max_samples=S, precision=precision,
                                                smoother=E.ELDER_SMOOTH_ILU))
    pt, ct = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
    traj = []
    for _ in range(5):
        st, info = ctx.step(S, T(phi), T(K), pt, ct, DT)
        assert (st == 0).all(), info
        traj.append((H(pt).reshape(S, -1).copy(), H(ct).reshape(S, -1).copy()))
    ctx.destroy()
    pscale = P.rho0 * P.g * P.Lz
    for s in range(S):
        p, c = p0, c0
        for n in range(5):
            p, c, info = O.newton_step(P, phi[s], K[s], p, c, DT)
            assert info["status"] == 0
            assert np.abs(traj[n][1][s] - c).max() <= tol, (s, n)
            assert np.abs(traj[n][0][s] - p).max() <= max(tol, 1e-9) * pscale, (s, n)


def test_smoother_apply_argument_errors(E):
    ctx = E.elder_create(E.elder_config_default(8, 8, 4, max_samples=1))
    P = O.Problem(8, 8, 4)
    phi, K, p, c = _case(P, 1, 3)
    r = T(np.zeros(2 * P.N))
    with pytest.raises(E.ElderError):
        ctx.smoother_apply(1, T(phi), T(K), T(p), T(c), DT, 3, r)
    with pytest.raises(E.ElderError):
        ctx.smoother_apply(2, T(phi), T(K), T(p), T(c), DT, 0, r)
    ctx.destroy()
