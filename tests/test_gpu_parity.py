"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances: c within 1e-10 max-abs per step on the FP64 path and 1e-6 with
mixed precision (Newton on the FP64 residual corrects the FP32 solves).
Pressure within 1e-9 of rho0 g Lz (1.5e-3 Pa): p is pinned only at four top
corner nodes, so the round-off level of the residual leaves ~1e-4 Pa of
solver-dependent noise in it.  Residual and Jacobian agree to round-off.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

YEAR = O.SECONDS_PER_YEAR
DEV = "cuda:0"


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


def _fields(P, S, seed):
    rng = np.random.default_rng(seed)
    phi = np.zeros((S, P.C))
    K = np.zeros((S, P.C))
    for s in range(S):
        phi[s], K[s] = O.fields_lognormal(P, rng.standard_normal(P.C))
    return phi, K


def _random_states(P, S, seed):
    rng = np.random.default_rng(seed)
    p0, c0 = O.initial_state(P)
    p = np.stack([p0 + rng.normal(0, 2e3, P.N) for _ in range(S)])
    c = np.stack([np.clip(c0 + rng.uniform(0, 0.7, P.N), 0, 1) for _ in range(S)])
    return p, c


def _ctx(E, nx, ny, nz, S=1, **kw):
    return E.elder_create(E.elder_config_default(nx, ny, nz, max_samples=S, **kw))


# --------------------------------------------------------------------------
# residual, Jacobian, fields
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims,S", [((8, 8, 2), 1), ((12, 8, 6), 3), ((16, 16, 4), 4)])
def test_residual_matches_oracle(E, dims, S):
    P = O.Problem(*dims)
    ctx = _ctx(E, *dims, S=S)
    phi, K = _fields(P, S, 1)
    p, c = _random_states(P, S, 2)
    po, co = _random_states(P, S, 3)
    dt = YEAR / 12
    R = H(ctx.residual(S, T(phi), T(K), T(p), T(c), T(po), T(co), dt)).reshape(S, P.N, 2)
    for s in range(S):
        Rp, Rc = O.residual(P, phi[s], K[s], p[s], c[s], po[s], co[s], dt)
        scale = max(np.abs(Rp).max(), np.abs(Rc).max())
        assert np.abs(R[s, :, 0] - Rp).max() <= 1e-12 * scale
        assert np.abs(R[s, :, 1] - Rc).max() <= 1e-12 * scale


def _oracle_dia(P, rowptr, col, val):
    """Oracle CSR -> the library's [27][N][4] block layout."""
    D = np.zeros((27, P.N, 4))
    nx1, ny1 = P.nx + 1, P.ny + 1
    for n in range(P.N):
        i, j, k = n % nx1, (n // nx1) % ny1, n // (nx1 * ny1)
        for v in range(2):
            r = 2 * n + v
            for q in range(rowptr[r], rowptr[r + 1]):
                m, w = divmod(int(col[q]), 2)
                mi, mj, mk = m % nx1, (m // nx1) % ny1, m // (nx1 * ny1)
                sl = (mi - i + 1) + 3 * (mj - j + 1) + 9 * (mk - k + 1)
                D[sl, n, 2 * v + w] += val[q]
    return D


def test_jacobian_matches_oracle(E):
    dims, S = (8, 8, 4), 2
    P = O.Problem(*dims)
    ctx = _ctx(E, *dims, S=S)
    phi, K = _fields(P, S, 4)
    p, c = _random_states(P, S, 5)
    dt = YEAR / 12
    J = H(ctx.jacobian(S, T(phi), T(K), T(p), T(c), dt)).reshape(S, 27, P.N, 4)
    for s in range(S):
        D = _oracle_dia(P, *O.jacobian_csr(P, phi[s], K[s], p[s], c[s], dt))
        scale = np.abs(D).max(axis=(0, 2))  # per row node
        err = np.abs(J[s] - D).max(axis=(0, 2)) / scale
        assert err.max() <= 1e-11


def test_fields_match_oracle(E):
    from paper_1906_01632_gb300 import inputs as I
    P = O.Problem(16, 16, 4)
    S = 5
    ctx = _ctx(E, 16, 16, 4, S=S)
    xi = I.sobol_xi(S)
    phi, K = ctx.fields(S, 0, T(xi))
    phi, K = H(phi).reshape(S, -1), H(K).reshape(S, -1)
    for s in range(S):
        rp, rk = O.fields_sobol(P, xi[s])
        np.testing.assert_allclose(phi[s], rp, rtol=1e-14)
        np.testing.assert_allclose(K[s], rk, rtol=1e-13)
    Z = np.stack([I.lognormal_z(P.C, seed=s + 1) for s in range(S)])
    phi, K = ctx.fields(S, 1, T(Z))
    phi, K = H(phi).reshape(S, -1), H(K).reshape(S, -1)
    for s in range(S):
        rp, rk = O.fields_lognormal(P, Z[s])
        np.testing.assert_allclose(phi[s], rp, rtol=1e-14)
        np.testing.assert_allclose(K[s], rk, rtol=1e-13)
    phi, K = ctx.fields(S, 2, T(xi))
    phi, K = H(phi).reshape(S, -1), H(K).reshape(S, -1)
    for s in range(S):
        rp, rk = O.fields_paper3rv(P, xi[s])
        np.testing.assert_allclose(phi[s], rp, rtol=1e-14)
        np.testing.assert_allclose(K[s], rk, rtol=1e-13)


# --------------------------------------------------------------------------
# linear solves: test (d) on 4x4x2 against the oracle's dense LU
# --------------------------------------------------------------------------

@pytest.mark.parametrize("transpose", [False, True])
def test_solve_matches_dense_lu(E, transpose):
    P = O.Problem(4, 4, 2)
    S = 2
    ctx = _ctx(E, 4, 4, 2, S=S)
    phi, K = _fields(P, S, 6)
    p, c = _random_states(P, S, 7)
    rng = np.random.default_rng(8)
    rhs = rng.standard_normal((S, P.N, 2))
    dt = YEAR / 12
    x, st = ctx.solve(S, T(phi), T(K), T(p), T(c), dt, T(rhs), transpose=transpose, rtol=1e-12)
    assert (st == 0).all()
    x = H(x).reshape(S, 2 * P.N)
    for s in range(S):
        A = O.jacobian_dense(P, phi[s], K[s], p[s], c[s], dt)
        ref = O.dense_solve(A.T if transpose else A, rhs[s].ravel())
        scale = np.abs(ref).reshape(-1, 2).max(axis=0)
        err = np.abs(x[s] - ref).reshape(-1, 2).max(axis=0)
        assert (err <= 1e-9 * scale).all(), (err, scale)


@pytest.mark.parametrize("transpose", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
def test_zline_smoother_solve_matches_dense_lu(E, transpose, precision):
    """The z-line smoother (block tridiagonal solve along each vertical
    line) as the multigrid smoother of elder_solve, 8x8x4 (lines of 5 nodes,
    a ragged 81-column batch), against a dense LU of the oracle Jacobian."""
    P = O.Problem(8, 8, 4)
    S = 3
    ctx = _ctx(E, 8, 8, 4, S=S, smoother=E.ELDER_SMOOTH_ZLINE, precision=precision)
    phi, K = _fields(P, S, 16)
    p, c = _random_states(P, S, 17)
    rng = np.random.default_rng(18)
    rhs = rng.standard_normal((S, P.N, 2))
    dt = YEAR / 12
    x, st = ctx.solve(S, T(phi), T(K), T(p), T(c), dt, T(rhs), transpose=transpose, rtol=1e-12)
    assert (st == 0).all()
    x = H(x).reshape(S, 2 * P.N)
    for s in range(S):
        A = O.jacobian_dense(P, phi[s], K[s], p[s], c[s], dt)
        ref = O.dense_solve(A.T if transpose else A, rhs[s].ravel())
        scale = np.abs(ref).reshape(-1, 2).max(axis=0)
        err = np.abs(x[s] - ref).reshape(-1, 2).max(axis=0)
        assert (err <= 1e-9 * scale).all(), (err, scale)


# --------------------------------------------------------------------------
# time steps
# --------------------------------------------------------------------------

def _run_gpu(E, P, phi, K, p, c, steps, dt, **kw):
    S = phi.shape[0]
    ctx = _ctx(E, P.nx, P.ny, P.nz, S=S, **kw)
    pt, ct = T(p), T(c)
    phit, Kt = T(phi), T(K)
    traj = []
    infos = []
    for _ in range(steps):
        st, info = ctx.step(S, phit, Kt, pt, ct, dt)
        assert (st == 0).all(), info
        traj.append((H(pt).reshape(S, -1).copy(), H(ct).reshape(S, -1).copy()))
        infos.append(info)
    return traj, infos


def _oracle_traj(P, phi, K, p, c, steps, dt):
    traj = []
    for _ in range(steps):
        p, c, info = O.newton_step(P, phi, K, p, c, dt)
        assert info["status"] == 0
        traj.append((p.copy(), c.copy()))
    return traj


@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_steps_match_oracle_16x16x4(E, precision, tol, smoother):
    P = O.Problem(16, 16, 4)
    S = 3
    phi, K = _fields(P, S, 9)
    p0, c0 = O.initial_state(P)
    p = np.tile(p0, (S, 1))
    c = np.tile(c0, (S, 1))
    dt = YEAR / 12
    steps = 5
    traj, _ = _run_gpu(E, P, phi, K, p, c, steps, dt, precision=precision, smoother=smoother)
    pscale = P.rho0 * P.g * P.Lz
    for s in range(S):
        ref = _oracle_traj(P, phi[s], K[s], p0, c0, steps, dt)
        for n in range(steps):
            assert np.abs(traj[n][1][s] - ref[n][1]).max() <= tol, (s, n)
            assert np.abs(traj[n][0][s] - ref[n][0]).max() <= max(tol, 1e-9) * pscale, (s, n)


def test_config1_32x32x8_24_steps_fp64(E):
    """32x32x8, uniform phi = 0.1, K = 4.845e-13, dt = 1/12 yr, 24 steps."""
    P = O.Problem(32, 32, 8)
    phi = np.full((1, P.C), 0.1)
    K = np.full((1, P.C), 4.845e-13)
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    steps = 24
    traj, infos = _run_gpu(E, P, phi, K, p0[None], c0[None], steps, dt)
    p, c = p0, c0
    for n in range(steps):
        p, c, info = O.newton_step(P, phi[0], K[0], p, c, dt, O.NewtonOpts(lin_rtol=1e-10))
        assert info["status"] == 0
        assert np.abs(traj[n][1][0] - c).max() <= 1e-10, n
        assert np.abs(traj[n][0][0] - p).max() <= 1e-9 * P.rho0 * P.g * P.Lz, n


def test_moments_match_oracle(E):
    P = O.Problem(16, 16, 4)
    S = 37
    ctx = _ctx(E, 16, 16, 4, S=S)
    rng = np.random.default_rng(10)
    cs = rng.uniform(0, 1, (S, P.N))
    cs[:, :7] = 0.5  # ties at the threshold: strict ">"
    m, v, pe = ctx.moments(S, T(cs))
    mo, vo, po = O.moments(cs)
    np.testing.assert_allclose(H(m), mo, rtol=0, atol=1e-14)
    np.testing.assert_allclose(H(v), vo, rtol=0, atol=1e-14)
    np.testing.assert_allclose(H(pe), po, rtol=0, atol=1e-14)
    w = rng.uniform(0.5, 1.5, S)
    w /= w.sum()
    m, v, pe = ctx.moments(S, T(cs), w=T(w), threshold=0.3)
    mo, vo, po = O.moments(cs, w=w, threshold=0.3)
    np.testing.assert_allclose(H(m), mo, rtol=0, atol=1e-14)
    np.testing.assert_allclose(H(v), vo, rtol=0, atol=1e-14)
    np.testing.assert_allclose(H(pe), po, rtol=0, atol=1e-14)


def test_grad_matches_oracle_adjoint(E):
    P = O.Problem(8, 8, 4)
    # Newton to round-off, as the oracle: J is compared at 1e-10
    ctx = _ctx(E, 8, 8, 4, newton_estimate=0, newton_tol_c=1e-13,
               newton_tol_p=1e-13 * P.rho0 * P.g * P.Lz)
    phi, K = _fields(P, 1, 11)
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    steps = 5
    J, gphi, gK = ctx.grad(steps, T(phi), T(K), T(p0), T(c0), dt, ckpt_every=2)
    Jo, gphio, gKo, rc = O.adjoint_gradient(P, phi[0], K[0], p0, c0, dt, steps)
    assert rc == 0
    assert abs(J - Jo) <= 1e-10 * abs(Jo)
    np.testing.assert_allclose(H(gphi), gphio, rtol=0, atol=1e-7 * np.abs(gphio).max())
    np.testing.assert_allclose(H(gK), gKo, rtol=0, atol=1e-7 * np.abs(gKo).max())


def test_failed_sample_keeps_old_state(E):
    """A NaN porosity in one sample: that sample reports a non-finite status
    and keeps u^n; the other samples advance as usual."""
    P = O.Problem(8, 8, 2)
    S = 2
    phi = np.full((S, P.C), 0.1)
    K = np.full((S, P.C), 4.845e-13)
    phi[1, 5] = np.nan
    p0, c0 = O.initial_state(P)
    ctx = _ctx(E, 8, 8, 2, S=S)
    pt, ct = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
    st, info = ctx.step(S, T(phi), T(K), pt, ct, YEAR / 12)
    assert st[0] == 0 and st[1] == 4
    c = H(ct).reshape(S, -1)
    np.testing.assert_array_equal(c[1], c0)
    _, cref, _ = O.newton_step(P, phi[0], K[0], p0, c0, YEAR / 12)
    assert np.abs(c[0] - cref).max() <= 1e-10


def test_paper_parallelepiped_workload_steps_match_oracle(E):
    """The paper's own workload (Section 5.3): the parallelepiped porosity
    field of eq. poro-paral3RVS at Halton points, dt = 0.005 yr, batched, on a
    16x16x4 grid; c within 1e-10 and p within 1e-9 rho0 g Lz per step."""
    from paper_1906_01632_gb300 import inputs as I
    P = O.Problem(16, 16, 4)
    S = 4
    xi = I.halton_xi(S)
    ctx = _ctx(E, 16, 16, 4, S=S)
    phi_t, K_t = ctx.fields(S, 2, T(xi))
    phi, K = H(phi_t).reshape(S, -1), H(K_t).reshape(S, -1)
    p0, c0 = O.initial_state(P)
    dt = 0.005 * YEAR
    steps = 4
    traj, _ = _run_gpu(E, P, phi, K, np.tile(p0, (S, 1)), np.tile(c0, (S, 1)), steps, dt)
    for s in range(S):
        ref = _oracle_traj(P, phi[s], K[s], p0, c0, steps, dt)
        for n in range(steps):
            assert np.abs(traj[n][1][s] - ref[n][1]).max() <= 1e-10, (s, n)
            assert np.abs(traj[n][0][s] - ref[n][0]).max() <= 1e-9 * P.rho0 * P.g * P.Lz, (s, n)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_fingers_launch_configuration_matches_oracle(E, precision, tol):
    """The launch configuration of the paper's ensemble run (bench.py
    --workload fingers, Section 5.3) on a 16x16x4 grid: the parallelepiped
    field at Halton points, the paper's boundary sets (bc_mode 1: c = 0 on
    the top outside the square, p = 0 on the top edges), dt = 0.005 yr, Newton
    from the quadratic extrapolation (elder_step_predicted, order 2), 8
    steps, against the oracle's states; then the ensemble mean's 0.5 level
    set counted by the bench's plume_lobes on both means."""
    import bench
    from paper_1906_01632_gb300 import inputs as I
    P = O.Problem(16, 16, 4, bc_mode=1)
    S = 4
    xi = I.halton_xi(S)
    ctx = _ctx(E, 16, 16, 4, S=S, bc_mode=1, precision=precision)
    phi_t, K_t = ctx.fields(S, 2, T(xi))
    phi, K = H(phi_t).reshape(S, -1), H(K_t).reshape(S, -1)
    p0, c0 = O.initial_state(P)
    dt = 0.005 * YEAR
    steps = 8
    pt, ct = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
    ph, ch = pt.repeat(2), ct.repeat(2)
    traj = []
    for _ in range(steps):
        st, info = ctx.step_predicted(S, phi_t, K_t, 2, ph, ch, pt, ct, dt)
        assert (st == 0).all(), info
        traj.append((H(pt).reshape(S, -1).copy(), H(ct).reshape(S, -1).copy()))
    mean_gpu = H(ctx.moments(S, ct)[0])
    ctx.destroy()
    pscale = P.rho0 * P.g * P.Lz
    c_end = []
    for s in range(S):
        ref = _oracle_traj(P, phi[s], K[s], p0, c0, steps, dt)
        for n in range(steps):
            assert np.abs(traj[n][1][s] - ref[n][1]).max() <= tol, (s, n)
            assert np.abs(traj[n][0][s] - ref[n][0]).max() <= max(tol, 1e-9) * pscale, (s, n)
        c_end.append(ref[-1][1])
    mean_orc = np.mean(c_end, axis=0)
    assert np.abs(mean_gpu - mean_orc).max() <= tol
    a = bench.plume_lobes(mean_gpu, 16, 16, 4)
    b = bench.plume_lobes(mean_orc, 16, 16, 4)
    assert a["plane_counts_top_down"] == b["plane_counts_top_down"]


def test_step_argument_errors(E):
    """S outside [1, max_samples] and a non-positive dt are rejected with
    ELDER_EINVAL before anything is launched; the state is left untouched."""
    P = O.Problem(8, 8, 4)
    ctx = _ctx(E, 8, 8, 4, S=2)
    phi, K = _fields(P, 2, 31)
    p0, c0 = O.initial_state(P)
    pt, ct = T(np.tile(p0, (2, 1))), T(np.tile(c0, (2, 1)))
    for S, dt in ((0, YEAR / 12), (3, YEAR / 12), (2, 0.0), (2, -1.0)):
        with pytest.raises(E.ElderError) as ei:
            ctx.step(S, T(phi), T(K), pt, ct, dt, raise_on_fail=True)
        assert ei.value.code == E.ELDER_EINVAL
    assert np.array_equal(H(pt), np.tile(p0, 2)) and np.array_equal(H(ct), np.tile(c0, 2))


@pytest.mark.parametrize("smoother", [0, 1])
def test_odd_grid_single_level_matches_oracle(E, smoother):
    """An odd grid (6x10x3, the diffusion-column boundary set) cannot be
    coarsened: the hierarchy is the grid itself and the dense inverse is the
    whole preconditioner.  Ragged node and cell counts against every block
    size; steps against the oracle."""
    P = O.Problem(6, 10, 3, bc_mode=2)
    S = 2
    phi, K = _fields(P, S, 41)
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    traj, _ = _run_gpu(E, P, phi, K, np.tile(p0, (S, 1)), np.tile(c0, (S, 1)), 3, dt,
                       bc_mode=2, smoother=smoother)
    for s in range(S):
        ref = _oracle_traj(P, phi[s], K[s], p0, c0, 3, dt)
        for n in range(3):
            assert np.abs(traj[n][1][s] - ref[n][1]).max() <= 1e-10, (s, n)
            assert np.abs(traj[n][0][s] - ref[n][0]).max() <= 1e-9 * P.rho0 * P.g * P.Lz, (s, n)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_extrapolated_start_marches_to_the_oracle_states(E, precision, tol):
    """elder_step_extrapolated starts Newton from 2 u^n - u^{n-1} but solves
    the same implicit step: a 5-step march matches the oracle's states (which
    start each Newton iteration from u^n), and the history buffers return
    u^n."""
    P = O.Problem(16, 16, 4)
    S = 2
    phi, K = _fields(P, S, 51)
    p0, c0 = O.initial_state(P)
    ctx = _ctx(E, 16, 16, 4, S=S, precision=precision)
    pt, ct = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
    pm, cm = pt.clone(), ct.clone()
    phit, Kt = T(phi), T(K)
    dt = YEAR / 12
    refs = [_oracle_traj(P, phi[s], K[s], p0, c0, 5, dt) for s in range(S)]
    for n in range(5):
        p_before, c_before = H(pt).copy(), H(ct).copy()
        st, _ = ctx.step_extrapolated(S, phit, Kt, pm, cm, pt, ct, dt)
        assert (st == 0).all()
        assert np.array_equal(H(pm), p_before) and np.array_equal(H(cm), c_before)
        for s in range(S):
            c1 = H(ct).reshape(S, -1)[s]
            p1 = H(pt).reshape(S, -1)[s]
            assert np.abs(c1 - refs[s][n][1]).max() <= tol, (s, n)
            assert np.abs(p1 - refs[s][n][0]).max() <= max(tol, 1e-9) * P.rho0 * P.g * P.Lz, (s, n)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-6)])
def test_quadratic_predictor_marches_to_the_oracle_states(E, precision, tol):
    """elder_step_predicted with order 2 starts Newton from 3 u^n - 3 u^{n-1} +
    u^{n-2} and solves the same implicit step: a 5-step march matches the
    oracle's states, and the two history levels shift by one level per call."""
    P = O.Problem(16, 16, 4)
    S = 2
    phi, K = _fields(P, S, 52)
    p0, c0 = O.initial_state(P)
    ctx = _ctx(E, 16, 16, 4, S=S, precision=precision)
    pt, ct = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
    ph, ch = pt.repeat(2), ct.repeat(2)
    phit, Kt = T(phi), T(K)
    dt = YEAR / 12
    nN = S * P.N
    refs = [_oracle_traj(P, phi[s], K[s], p0, c0, 5, dt) for s in range(S)]
    for n in range(5):
        p_before, c_before = H(pt).copy(), H(ct).copy()
        p_lvl0, c_lvl0 = H(ph)[:nN].copy(), H(ch)[:nN].copy()
        st, _ = ctx.step_predicted(S, phit, Kt, 2, ph, ch, pt, ct, dt)
        assert (st == 0).all()
        assert np.array_equal(H(ph)[:nN], p_before) and np.array_equal(H(ch)[:nN], c_before)
        assert np.array_equal(H(ph)[nN:], p_lvl0) and np.array_equal(H(ch)[nN:], c_lvl0)
        for s in range(S):
            c1 = H(ct).reshape(S, -1)[s]
            p1 = H(pt).reshape(S, -1)[s]
            assert np.abs(c1 - refs[s][n][1]).max() <= tol, (s, n)
            assert np.abs(p1 - refs[s][n][0]).max() <= max(tol, 1e-9) * P.rho0 * P.g * P.Lz, (s, n)


def test_predicted_step_rejects_bad_orders_and_short_history(E):
    P = O.Problem(8, 8, 2)
    ctx = _ctx(E, 8, 8, 2, S=1)
    phi, K = _fields(P, 1, 53)
    p0, c0 = O.initial_state(P)
    pt, ct = T(p0), T(c0)
    # the library rejects orders outside {1, 2} (history long enough for 3)
    for order in (0, 3):
        with pytest.raises(Exception):
            ctx.step_predicted(1, T(phi), T(K), order, pt.repeat(3), ct.repeat(3), pt, ct,
                               YEAR / 12)
    # the binding rejects a history shorter than order * S * N
    with pytest.raises(ValueError):
        ctx.step_predicted(1, T(phi), T(K), 2, pt.clone(), ct.clone(), pt, ct, YEAR / 12)


@pytest.mark.parametrize("knob,tier", [(dict(mixed_newton_maxit=1), 1),
                                       (dict(newton_maxit=1), 2)])
def test_failure_tiers_resolve_to_the_oracle_state(E, knob, tier):
    """Failures forced from the host: a Newton cap of 1 on the mixed solve
    alone fails every sample there, and the FP64 re-solve with the
    configured settings succeeds (fp64_retry 1); a cap of 1 on every solve
    fails the FP64 re-solve too, and the last robust FP64 solve succeeds
    (fp64_retry 2).  Either way the returned state is the implicit step's
    solution: the oracle's within 1e-10 in c."""
    P = O.Problem(16, 16, 4)
    S = 3
    phi, K = _fields(P, S, 41)
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    ctx = _ctx(E, 16, 16, 4, S, precision=E.ELDER_MIXED, **knob)
    pt, ct = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
    st, info = ctx.step(S, T(phi), T(K), pt, ct, dt)
    assert (st == 0).all(), info
    assert [i["fp64_retry"] for i in info] == [tier] * S
    pg, cg = H(pt).reshape(S, -1), H(ct).reshape(S, -1)
    for s in range(S):
        pr, cr, oi = O.newton_step(P, phi[s], K[s], p0, c0, dt)
        assert oi["status"] == 0
        assert np.abs(cg[s] - cr).max() <= 1e-10
        assert np.abs(pg[s] - pr).max() <= 1e-9 * P.rho0 * P.g * P.Lz
    ctx.destroy()


def test_measured_fma_peaks(E):
    """The FMA-chain probe that rates the FP64 residual and the FP32
    surrogate evaluation: finite, positive, and FP32 well above FP64 (GB300
    issues FP64 at a small fraction of the FP32 rate)."""
    f64 = E.elder_measure_peak("fp64")
    f32 = E.elder_measure_peak("fp32")
    print(f"FP64 {f64:.0f} GFLOP/s, FP32 {f32:.0f} GFLOP/s")
    assert 0 < f64 < f32 and np.isfinite(f32)


@pytest.mark.parametrize("precision", [0, 1])
def test_device_controlled_step_matches_host_driven_step(E, precision):
    """use_graphs = 2 (the whole step one CUDA graph, its Newton, BiCGStab
    and line-search loops while nodes driven by the per-sample flags on the
    device) runs the same kernels in the same order as the host-driven loop
    (use_graphs = 1): states and iteration counts are bitwise equal over 4
    steps with the quadratic Newton start, and the graph is really used from
    the second step on.  Pointers that change between calls get their own
    captured graph."""
    P = O.Problem(16, 16, 4)
    S = 4
    phi, K = _fields(P, S, 51)
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    out = {}
    for mode in (1, 2):
        ctx = _ctx(E, 16, 16, 4, S, precision=precision, use_graphs=mode)
        ph_t, K_t = T(phi), T(K)
        pt, ct = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
        hp, hc = pt.repeat(2), ct.repeat(2)
        traj = []
        for n in range(4):
            st, info = ctx.step_predicted(S, ph_t, K_t, 2, hp, hc, pt, ct, dt)
            assert (st == 0).all()
            traj.append((H(pt).copy(), H(ct).copy(),
                         [(i["newton_iters"], i["krylov_iters"], i["ls_cuts"]) for i in info]))
        # a second state buffer: a new argument set, a new graph
        p2, c2 = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
        st, _ = ctx.step(S, ph_t, K_t, p2, c2, dt)
        assert (st == 0).all()
        traj.append((H(p2).copy(), H(c2).copy(), None))
        cached, replays, note = ctx.graph_status()
        if mode == 2:
            assert note == "" and replays == 4 and cached == 2, (cached, replays, note)
        else:
            assert replays == 0
        out[mode] = traj
        ctx.destroy()
    for a, b in zip(out[1], out[2]):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert a[2] == b[2]
    # and the marched states are the oracle's
    p, c = p0, c0
    for n in range(4):
        p, c, oi = O.newton_step(P, phi[0], K[0], p, c, dt)
        tol = 1e-10 if precision == 0 else 1e-6
        assert np.abs(out[2][n][1].reshape(S, -1)[0] - c).max() <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_samples_per_cta_variants_are_bitwise_equal(E, precision):
    """Two samples per CTA in the multigrid residual and the z-line sweep
    (autotune = 2) only regroup the same per-node arithmetic: the states and
    iteration counts of 3 steps equal those with one sample per CTA
    (autotune = 0) bit for bit; S = 5 leaves the last CTA half empty."""
    P = O.Problem(16, 16, 4)
    S = 5
    phi, K = _fields(P, S, 61)
    p0, c0 = O.initial_state(P)
    out = {}
    for at in (0, 2):
        ctx = _ctx(E, 16, 16, 4, S, precision=precision, autotune=at)
        pt, ct = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
        hp, hc = pt.repeat(2), ct.repeat(2)
        traj = []
        for _ in range(3):
            st, info = ctx.step_predicted(S, T(phi), T(K), 2, hp, hc, pt, ct, YEAR / 12)
            assert (st == 0).all()
            traj.append((H(pt).copy(), H(ct).copy(), [i["krylov_iters"] for i in info]))
        assert ctx.autotune_choice(E.K_MGRES)[1] == (2 if at == 2 else 1)
        out[at] = traj
        ctx.destroy()
    for a, b in zip(out[0], out[2]):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
