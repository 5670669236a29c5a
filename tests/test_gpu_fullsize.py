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
import os

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
    """128x128x32 (1,098,306 unknowns, the paper's box mesh of Section 2.1),
    one sample, the first 5 steps of dt = 1/12 yr from the initial state,
    FP64 path and mixed path each against the oracle's own states
    (tests/golden/config2_states.npz, written by the oracle): c within 1e-10
    (FP64) and 1e-6 (mixed) at 16,384 sampled nodes after steps 1-4 and at
    every node after step 5 (every node the oracle left below 1e-13 too);
    p at 4,096 sampled nodes; the oracle residual at every FP64 state at its
    round-off floor; the salt balance of every step."""
    import os as _os
    path = _os.path.join(_os.path.dirname(__file__), "golden", "config2_states.npz")
    if not _os.path.exists(path):
        pytest.skip("config2_states.npz not generated (tests/golden/make_config2_states.py)")
    g = np.load(path)
    P = O.Problem(128, 128, 32)
    phi = np.full(P.C, 0.1)
    K = np.full(P.C, 4.845e-13)
    p0, c0 = O.initial_state(P)
    dt = float(g["dt"])
    assert abs(dt - YEAR / 12) <= 1e-9
    floor = float(g["c_floor"])
    pscale = P.rho0 * P.g * P.Lz
    for prec, tol_c, tol_p in ((0, 1e-10, 1e-9), (1, 1e-6, 1e-6)):
        ctx = E.elder_create(E.elder_config_default(128, 128, 32, max_samples=1, precision=prec))
        pt, ct = T(p0), T(c0)
        pp, cp = p0, c0
        for n in range(1, 6):
            st, info = ctx.step(1, T(phi), T(K), pt, ct, dt)
            assert st[0] == 0, info
            p1, c1 = H(pt).copy(), H(ct).copy()
            idx = g[f"c{n}_idx"]
            dc = np.abs(c1[idx] - g[f"c{n}_val"]).max()
            assert dc <= tol_c, (prec, n, dc)
            if n == 5:
                rest = np.ones(P.N, bool)
                rest[idx] = False
                assert np.abs(c1[rest]).max() <= floor + tol_c
            dp = np.abs(p1[g["p_idx"]] - g[f"p{n}_val"]).max()
            assert dp <= tol_p * pscale, (prec, n, dp)
            if prec == 0:
                _check_solved(P, phi, K, p1, c1, pp, cp, dt)
            m0, m1 = _masses(P, phi, cp), _masses(P, phi, c1)
            assert abs(info[0]["salt_mass0"] - m0) <= 1e-12 * max(m0, 1.0)
            assert abs(info[0]["salt_mass"] - m1) <= 1e-12 * m1
            assert abs(info[0]["salt_mass"] - info[0]["salt_mass0"] - info[0]["salt_inflow"]) \
                <= 1e-9 * m1
            print(f"precision {prec} step {n}: max |c - c_oracle| {dc:.2e}, "
                  f"max |p - p_oracle| {dp:.2e} Pa")
            pp, cp = p1, c1
        ctx.destroy()


def _oracle_trajectory(args):
    """Oracle states after each of `steps` implicit steps of one Sobol sample
    (runs in a spawned worker process)."""
    nx, ny, nz, xi, steps, dt = args
    import oracle as O_
    P = O_.Problem(nx, ny, nz)
    phi, K = O_.fields_sobol(P, xi)
    p, c = O_.initial_state(P)
    out = []
    for _ in range(steps):
        p, c, info = O_.newton_step(P, phi, K, p, c, dt, O_.NewtonOpts(smoother=1,
                                                                        lin_rtol=1e-10))
        if info["status"] != 0:
            raise RuntimeError(info)
        out.append((p.copy(), c.copy()))
    return out


# Newton stops on the size of its correction (max|dc| <= 1e-11, max|dp| <=
# 1e-11 rho0 g Lz, or the same bound on the linear-convergence error
# estimate), not on ||R||: the error it leaves, e <= 1e-11 relative, leaves
# a residual ||J e|| of up to about (1e-11 / 2 eps) ~ 2.3e4 times the
# round-off floor 2 eps ||a|| (a: the row sums of the terms' magnitudes,
# ~ |J| |u| row by row).  The FP64-path tests run Newton to the floor itself.
NEWTON_SLACK = 1e-11 / (2 * EPS)


def test_config3_batched_qmc_sampled(E, I):
    """The bench's launch configuration: 64x64x16, 256 Sobol samples, mixed
    precision, Newton from the quadratic extrapolation (elder_step_predicted,
    order 2), the first 3 steps from the initial state.  Every sample's
    result solves the oracle's implicit step (residual within the bound the
    Newton tolerance sets); 12 samples spread over the batch match the
    oracle's own 3-step trajectories within 1e-6 in c, step by step."""
    import multiprocessing as mp
    S, steps = 256, 3
    P = O.Problem(64, 64, 16)
    dt = YEAR / 12
    xi = I.sobol_xi(S)
    picks = list(range(0, S, 23))[:12]
    pool = mp.get_context("spawn").Pool(min(len(picks), os.cpu_count() or 1))
    ref = pool.map_async(_oracle_trajectory, [(64, 64, 16, xi[s], steps, dt) for s in picks],
                         chunksize=1)
    ctx = E.elder_create(E.elder_config_default(64, 64, 16, max_samples=S, precision=E.ELDER_MIXED))
    phi_t, K_t = ctx.fields(S, 0, T(xi))
    p_t, c_t = ctx.initial_state(S, device=DEV)
    ph, ch = p_t.repeat(2), c_t.repeat(2)
    p0, c0 = H(p_t).reshape(S, -1)[0].copy(), H(c_t).reshape(S, -1)[0].copy()
    phi = H(phi_t).reshape(S, -1)
    K = H(K_t).reshape(S, -1)
    traj = []
    for n in range(steps):
        st, info = ctx.step_predicted(S, phi_t, K_t, 2, ph, ch, p_t, c_t, dt)
        assert (st == 0).all()
        traj.append((H(p_t).reshape(S, -1).copy(), H(c_t).reshape(S, -1).copy()))
    pp, cp = np.tile(p0, (S, 1)), np.tile(c0, (S, 1))
    for n in range(steps):
        p1, c1 = traj[n]
        for s in range(0, S, 8):
            _check_solved(P, phi[s], K[s], p1[s], c1[s], pp[s], cp[s], dt, slack=NEWTON_SLACK)
        pp, cp = p1, c1
    ref = ref.get(timeout=1800)
    pool.close()
    worst = 0.0
    for q, s in enumerate(picks):
        for n in range(steps):
            pr, cr = ref[q][n]
            dc = np.abs(traj[n][1][s] - cr).max()
            worst = max(worst, dc)
            assert dc <= 1e-6, (s, n, dc)
            assert np.abs(traj[n][0][s] - pr).max() <= 1e-6 * P.rho0 * P.g * P.Lz
    print(f"max |c - c_oracle| over {len(picks)} samples x {steps} steps: {worst:.2e}")


def test_config5_uneven_batch_both_grid_sizes(E, I):
    """The uneven ensemble's two grid sizes, one context each, one step of
    dt = 1/24 yr in mixed precision with the bench's Newton start: the first
    two of its 64 Sobol samples at 128x128x32 (1,098,306 unknowns each) and
    its first 256x256x64 sample (sample 48; 8,586,370 unknowns, the paper's
    largest box mesh of 4,194,304 cells).  Every result solves the oracle's
    implicit step within the bound the Newton tolerance sets, and the salt
    balance of the step holds."""
    xi = I.sobol_xi(64)
    dt = YEAR / 24
    for (nx, ny, nz), ids in (((128, 128, 32), [0, 1]), ((256, 256, 64), [48])):
        S = len(ids)
        P = O.Problem(nx, ny, nz)
        ctx = E.elder_create(E.elder_config_default(nx, ny, nz, max_samples=S,
                                                    precision=E.ELDER_MIXED))
        phi_t, K_t = ctx.fields(S, 0, T(xi[ids]))
        p_t, c_t = ctx.initial_state(S, device=DEV)
        p0, c0 = H(p_t).reshape(S, -1)[0].copy(), H(c_t).reshape(S, -1)[0].copy()
        ph, ch = p_t.repeat(2), c_t.repeat(2)
        st, info = ctx.step_predicted(S, phi_t, K_t, 2, ph, ch, p_t, c_t, dt)
        assert (st == 0).all(), info
        phi = H(phi_t).reshape(S, -1)
        K = H(K_t).reshape(S, -1)
        p1 = H(p_t).reshape(S, -1)
        c1 = H(c_t).reshape(S, -1)
        ctx.destroy()
        for q in range(S):
            ph_o, K_o = O.fields_sobol(P, xi[ids[q]])
            np.testing.assert_allclose(phi[q], ph_o, rtol=1e-14, atol=0)
            _check_solved(P, phi[q], K[q], p1[q], c1[q], p0, c0, dt, slack=NEWTON_SLACK)
            m0, m1 = _masses(P, phi[q], c0), _masses(P, phi[q], c1[q])
            assert abs(info[q]["salt_mass"] - m1) <= 1e-12 * m1
            assert abs(info[q]["salt_mass"] - info[q]["salt_mass0"] - info[q]["salt_inflow"]) \
                <= 1e-8 * m1
        print((nx, ny, nz), [(i["newton_iters"], i["krylov_iters"], i["fp64_retry"])
                             for i in info])


def test_config4_adjoint_matches_central_fd(E, I):
    """64x64x16, lognormal porosity (median 0.1, sigma_log 0.2, clipped to
    [0.05, 0.2]), Kozeny-Carman K, 40 steps of 1/12 yr, objective = salt
    mass below mid-depth: elder_grad (checkpoints every 7 steps) against
    central differences at h = 1e-6 relative, the configured step, all
    perturbed runs batched as the samples of one step loop.

    (1) Per cell, on 32 random cells (unclipped), for phi and for K: a
    single cell moves J by ~h theta_e |g_e| ~ 1e-11 |J|, while each run's J is
    determined only to the Newton round-off floor (~1e-13 |J|, ~450 eps |J|,
    between runs of different batch composition).  The quotient therefore
    carries a round-off term 1000 eps |J| / (2 h theta_e); a cell passes when
    |fd - g| <= 1e-5 |g| + that term, and the test reports how many pass on
    1e-5 |g| alone.
    (2) Along random +-1 directions over all cells (one for phi, one for K):
    (J(theta (1 + h v)) - J(theta (1 - h v))) / 2h against sum_e g_e theta_e
    v_e.  The perturbation moves J by ~h |J|, so round-off enters at ~1e-7
    and the adjoint is checked at the configured step to 1e-5 of
    sum_e |g_e theta_e|.  The step map is only piecewise smooth (upwinding
    switches with the sign of each face flux): quotients approach the
    adjoint roughly linearly in h, ~1e-7 relative at h = 1e-6."""
    P = O.Problem(64, 64, 16)
    Z = I.lognormal_z(P.C, seed=1)
    phi, K = O.fields_lognormal(P, Z)
    cand = I.fd_cells(P.C, count=96, seed=2)
    cells = [e for e in cand if 0.05 < phi[e] < 0.2][:32]
    assert len(cells) == 32
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    steps = 40
    rel = 1e-6
    rng = np.random.default_rng(3)
    v_phi = rng.choice([-1.0, 1.0], P.C)
    v_K = rng.choice([-1.0, 1.0], P.C)
    phis, Ks = [], []
    for which in ("phi", "K"):
        for e in cells:
            for sgn in (1, -1):
                ph, kk = phi.copy(), K.copy()
                (ph if which == "phi" else kk)[e] *= 1 + sgn * rel
                phis.append(ph)
                Ks.append(kk)
    for sgn in (1, -1):
        phis.append(phi * (1 + sgn * rel * v_phi))
        Ks.append(K.copy())
    for sgn in (1, -1):
        phis.append(phi.copy())
        Ks.append(K * (1 + sgn * rel * v_K))
    S = len(phis)
    # Newton to round-off (no error-estimate stop): a step accepted at
    # |dc| ~ 1e-11 would leave ~1e-2 kg of error in J
    ctx = E.elder_create(E.elder_config_default(
        64, 64, 16, max_samples=S, newton_estimate=0, newton_tol_c=1e-13,
        newton_tol_p=1e-13 * P.rho0 * P.g * P.Lz))
    J, gphi, gK = ctx.grad(steps, T(phi), T(K), T(p0), T(c0), dt, ckpt_every=7)
    gphi, gK = H(gphi), H(gK)
    phi_b, K_b = T(np.stack(phis)), T(np.stack(Ks))
    pt, ct = T(np.tile(p0, (S, 1))), T(np.tile(c0, (S, 1)))
    for _ in range(steps):
        st, _ = ctx.step(S, phi_b, K_b, pt, ct, dt)
        assert (st == 0).all()
    cfin = H(ct).reshape(S, -1)
    Js = [O.objective(P, phis[s], cfin[s]) for s in range(S)]
    q = 0
    alone = 0
    for which, g, base in (("phi", gphi, phi), ("K", gK, K)):
        for e in cells:
            fd = (Js[q] - Js[q + 1]) / (2 * rel * base[e])
            q += 2
            noise = 1000 * EPS * abs(J) / (2 * rel * base[e])
            err = abs(fd - g[e])
            alone += err <= 1e-5 * abs(g[e])
            assert err <= 1e-5 * abs(g[e]) + noise, (which, e, fd, g[e], noise)
    print(f"per-cell quotients at h = {rel}: {alone} of 64 within 1e-5 |g| without the "
          f"round-off term")
    for which, g, base, v in (("phi", gphi, phi, v_phi), ("K", gK, K, v_K)):
        fd = (Js[q] - Js[q + 1]) / (2 * rel)
        q += 2
        want = float(np.sum(g * base * v))
        scale = float(np.sum(np.abs(g * base)))
        print(f"directional {which}: fd {fd:.9e} adjoint {want:.9e} rel {abs(fd - want) / scale:.2e}")
        assert abs(fd - want) <= 1e-5 * scale, (which, fd, want, scale)


def test_autograd_rollout_matches_elder_grad_and_a_forward_run(E):
    """ElderRollout (torch.autograd.Function over elder_grad): J equals the
    objective of an independent forward run (elder_step, objective by the
    oracle), phi.grad / K.grad equal elder_grad's gradients, the incoming
    gradient scales them, and a Kozeny-Carman K(phi) written in torch chains
    through to dJ/dphi + dJ/dK dK/dphi of the oracle's own adjoint."""
    P = O.Problem(16, 16, 4)
    rng = np.random.default_rng(31)
    phi_np, K_np = O.fields_lognormal(P, rng.standard_normal(P.C))
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    steps = 3
    kw = dict(newton_estimate=0, newton_tol_c=1e-13, newton_tol_p=1e-13 * P.rho0 * P.g * P.Lz)
    ctx = E.elder_create(E.elder_config_default(16, 16, 4, max_samples=1, **kw))
    phi = T(phi_np).requires_grad_(True)
    K = T(K_np).requires_grad_(True)
    J = E.ElderRollout.apply(phi, K, T(p0), T(c0), ctx, steps, dt)
    (3.0 * J).backward()
    Jr, gphi, gK = ctx.grad(steps, T(phi_np), T(K_np), T(p0), T(c0), dt)
    assert float(J.detach()) == Jr
    torch.testing.assert_close(phi.grad, 3.0 * gphi, rtol=0, atol=0)
    torch.testing.assert_close(K.grad, 3.0 * gK, rtol=0, atol=0)
    pt, ct = T(p0), T(c0)
    for _ in range(steps):
        st, _ = ctx.step(1, T(phi_np), T(K_np), pt, ct, dt)
        assert st[0] == 0
    assert abs(O.objective(P, phi_np, H(ct)) - Jr) <= 1e-12 * abs(Jr)
    # chain rule through a torch Kozeny-Carman map
    ph = T(phi_np).requires_grad_(True)
    Kc = 4.845e-13 * (ph ** 3 / (1 - ph) ** 2) / (0.1 ** 3 / 0.9 ** 2)
    Jc = E.ElderRollout.apply(ph, Kc, T(p0), T(c0), ctx, steps, dt)
    Jc.backward()
    Kc_np = H(Kc.detach())
    Jo, go_phi, go_K, rc = O.adjoint_gradient(P, phi_np, Kc_np, p0, c0, dt, steps,
                                              O.NewtonOpts(tol_c=1e-15, tol_p=1e-9, maxit=40))
    assert rc == 0
    dK = 4.845e-13 / (0.1 ** 3 / 0.9 ** 2) * (3 * phi_np ** 2 / (1 - phi_np) ** 2
                                               + 2 * phi_np ** 3 / (1 - phi_np) ** 3)
    total = go_phi + go_K * dK
    got = H(ph.grad)
    assert np.abs(got - total).max() <= 1e-7 * np.abs(total).max()
    ctx.destroy()


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
