"""Parity at the benchmark configurations' sizes (GPU).

At these sizes the oracle cannot follow every sample, so the checks are:
* properties that hold at any size, evaluated by the oracle on the GPU's
  result: the oracle residual R(u^{n+1}; u^n) at the returned state is at
  the round-off floor (that is what the implicit step's result is), and the
  FP64 and mixed paths give the same state;
* sampled outputs the oracle computes one by one (a few samples of the
  batched run in the launch configuration the bench times);
* the salt-mass balance of every step;
* the adjoint gradient against central finite differences, with the
  perturbed fields batched as samples of one run.
"""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

YEAR = O.SECONDS_PER_YEAR
DEV = "cuda:0"
EPS = 2.220446049250313e-16


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_01632_gb300 import build
    build.build()
    from paper_1906_01632_gb300 import elder
    return elder


@pytest.fixture(scope="module")
def I():
    from paper_1906_01632_gb300 import inputs
    return inputs


def T(a):
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device=DEV)


def H(t):
    return t.detach().cpu().numpy()


def _masses(P, phi, c):
    vscv = (P.Lx / P.nx) * (P.Ly / P.ny) * (P.Lz / P.nz) / 8
    cn = c.reshape(P.nz + 1, P.ny + 1, P.nx + 1)
    ph = phi.reshape(P.nz, P.ny, P.nx)
    parts = []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                cc = cn[dz:dz + P.nz, dy:dy + P.ny, dx:dx + P.nx]
                parts.append((ph * vscv * (P.rho0 + (P.rho1 - P.rho0) * cc) * cc).ravel())
    return math.fsum(np.concatenate(parts))


def _check_solved(P, phi, K, p1, c1, p0, c0, dt, slack=10.0):
    """The oracle residual at the GPU's u^{n+1} is at round-off level."""
    Rp, Rc = O.residual(P, phi, K, p1, c1, p0, c0, dt)
    r = math.sqrt(float((Rp ** 2).sum() + (Rc ** 2).sum()))
    floor = 2 * EPS * O.residual_magnitude(P, phi, K, p1, c1, c0, dt)
    assert r <= slack * floor, (r, floor)


def test_config2_128x128x32_fp64_and_mixed(E):
    """128x128x32 (1,098,306 unknowns, the paper's box mesh), one sample,
    the first steps: both paths solve the implicit step and agree."""
    P = O.Problem(128, 128, 32)
    phi = np.full(P.C, 0.1)
    K = np.full(P.C, 4.845e-13)
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    states = {}
    for prec in (0, 1):
        ctx = E.elder_create(E.elder_config_default(128, 128, 32, max_samples=1, precision=prec))
        pt, ct = T(p0), T(c0)
        traj = []
        for _ in range(2):
            st, info = ctx.step(1, T(phi), T(K), pt, ct, dt)
            assert st[0] == 0, info
            traj.append((H(pt).copy(), H(ct).copy(), info[0]))
        states[prec] = traj
        ctx.destroy()
    pp, cp = p0, c0
    for n in range(2):
        p1, c1, info = states[0][n]
        _check_solved(P, phi, K, p1, c1, pp, cp, dt)
        pm, cm, _ = states[1][n]
        assert np.abs(cm - c1).max() <= 1e-8
        assert np.abs(pm - p1).max() <= 1e-8 * P.rho0 * P.g * P.Lz
        # salt-mass balance of the step (FP64 accumulation on the device)
        m0, m1 = _masses(P, phi, cp), _masses(P, phi, c1)
        assert abs(info["salt_mass0"] - m0) <= 1e-12 * max(m0, 1.0)
        assert abs(info["salt_mass"] - m1) <= 1e-12 * m1
        assert abs(info["salt_mass"] - info["salt_mass0"] - info["salt_inflow"]) <= 1e-9 * m1
        pp, cp = p1, c1


def test_config3_batched_qmc_sampled(E, I):
    """The bench's launch configuration: 64x64x16, 256 Sobol samples, mixed
    precision, one step from the initial state.  Every sample's result
    solves the oracle's implicit step; two sampled samples match the
    oracle's own Newton solution."""
    S = 256
    P = O.Problem(64, 64, 16)
    ctx = E.elder_create(E.elder_config_default(64, 64, 16, max_samples=S, precision=E.ELDER_MIXED))
    xi = I.sobol_xi(S)
    phi_t, K_t = ctx.fields(S, 0, T(xi))
    p_t, c_t = ctx.initial_state(S, device=DEV)
    p0, c0 = H(p_t).reshape(S, -1)[0].copy(), H(c_t).reshape(S, -1)[0].copy()
    dt = YEAR / 12
    st, info = ctx.step(S, phi_t, K_t, p_t, c_t, dt)
    assert (st == 0).all()
    phi = H(phi_t).reshape(S, -1)
    K = H(K_t).reshape(S, -1)
    p1 = H(p_t).reshape(S, -1)
    c1 = H(c_t).reshape(S, -1)
    for s in range(0, S, 8):
        _check_solved(P, phi[s], K[s], p1[s], c1[s], p0, c0, dt, slack=1e4)
    for s in (0, 137):
        pr, cr, oi = O.newton_step(P, phi[s], K[s], p0, c0, dt)
        assert oi["status"] == 0
        assert np.abs(c1[s] - cr).max() <= 1e-6
        assert np.abs(p1[s] - pr).max() <= 1e-6 * P.rho0 * P.g * P.Lz


def test_config4_adjoint_matches_central_fd(E, I):
    """64x64x16, lognormal porosity (median 0.1, sigma_log 0.2, clipped to
    [0.05, 0.2]), Kozeny-Carman K, 40 steps of 1/12 yr, objective = salt
    mass below mid-depth: elder_grad (checkpoints every 7 steps) against
    central differences (h = 1e-5 relative) on 16 cells for phi and 16 for K,
    whose 64 perturbed runs go through one batched step loop.

    Agreement: 1e-5 relative, plus the round-off of the difference of two
    objective values, 1000 eps |J| / (2 h theta_e): each run's state is only
    determined to the Newton round-off floor, and J of the same sample
    differs by ~1e-13 |J| (~450 eps |J|) between runs of different batch
    composition.  The step map is only piecewise smooth (upwinding switches
    with the sign of each face flux), so the quotient approaches the adjoint
    roughly linearly in h: at h = 1e-3 cells on the plume path differ by
    ~1e-3, at 1e-4 by ~6e-5, at 1e-5 by ~1.4e-6; below that the round-off
    term dominates."""
    P = O.Problem(64, 64, 16)
    Z = I.lognormal_z(P.C, seed=1)
    phi, K = O.fields_lognormal(P, Z)
    cand = I.fd_cells(P.C, count=64, seed=2)
    cells = [e for e in cand if 0.05 < phi[e] < 0.2][:16]
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    steps = 40
    # Newton to round-off (no error-estimate stop): a central difference of
    # J at h = 1e-3 moves J by ~1 kg, and a step accepted at |dc| ~ 1e-11
    # leaves ~1e-2 kg of error in J
    ctx = E.elder_create(E.elder_config_default(
        64, 64, 16, max_samples=64, newton_estimate=0, newton_tol_c=1e-13,
        newton_tol_p=1e-13 * P.rho0 * P.g * P.Lz))
    J, gphi, gK = ctx.grad(steps, T(phi), T(K), T(p0), T(c0), dt, ckpt_every=7)
    gphi, gK = H(gphi), H(gK)
    rel = 1e-5
    phis, Ks = [], []
    for e in cells:
        for sgn in (1, -1):
            ph = phi.copy()
            ph[e] *= 1 + sgn * rel
            phis.append(ph)
            Ks.append(K.copy())
    for e in cells:
        for sgn in (1, -1):
            kk = K.copy()
            kk[e] *= 1 + sgn * rel
            phis.append(phi.copy())
            Ks.append(kk)
    S = len(phis)
    phi_b, K_b = T(np.stack(phis)), T(np.stack(Ks))
    pt, ct = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
    for _ in range(steps):
        st, _ = ctx.step(S, phi_b, K_b, pt, ct, dt)
        assert (st == 0).all()
    cfin = H(ct).reshape(S, -1)
    Js = [O.objective(P, phis[s], cfin[s]) for s in range(S)]
    q = 0
    for which, g, base in (("phi", gphi, phi), ("K", gK, K)):
        for e in cells:
            fd = (Js[q] - Js[q + 1]) / (2 * rel * base[e])
            q += 2
            noise = 1000 * EPS * abs(J) / (2 * rel * base[e])
            assert abs(fd - g[e]) <= 1e-5 * abs(g[e]) + noise, (which, e, fd, g[e], noise)


def test_paper_boundary_variant_matches_oracle(E):
    """The paper's own boundary sets (c = 0 on the top outside the square,
    p = 0 on the top edges): GPU steps against the oracle."""
    P = O.Problem(16, 16, 4, bc_mode=1)
    rng = np.random.default_rng(21)
    phi, K = O.fields_lognormal(P, rng.standard_normal(P.C))
    p0, c0 = O.initial_state(P)
    ctx = E.elder_create(E.elder_config_default(16, 16, 4, max_samples=1, bc_mode=1))
    pt, ct = T(p0), T(c0)
    p, c = p0, c0
    for _ in range(3):
        st, info = ctx.step(1, T(phi), T(K), pt, ct, YEAR / 12)
        assert st[0] == 0
        p, c, oi = O.newton_step(P, phi, K, p, c, YEAR / 12)
        assert oi["status"] == 0
        assert np.abs(H(ct) - c).max() <= 1e-10
        assert np.abs(H(pt) - p).max() <= 1e-9 * P.rho0 * P.g * P.Lz
