"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each checks a closed form, an
invariant or a reduction to a textbook scheme that a plausible mistake in the
oracle (a dropped term, a wrong sign or index, a transposed operand) breaks.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

YEAR = O.SECONDS_PER_YEAR
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _uniform(P, phi=0.1, K=4.845e-13):
    return np.full(P.C, phi), np.full(P.C, K)


def _node_xyz(P):
    k, j, i = np.meshgrid(np.arange(P.nz + 1), np.arange(P.ny + 1),
                          np.arange(P.nx + 1), indexing="ij")
    return (i.ravel() * P.Lx / P.nx, j.ravel() * P.Ly / P.ny,
            k.ravel() * P.Lz / P.nz, i.ravel(), j.ravel(), k.ravel())


# --------------------------------------------------------------------------
# counts printed in the paper
# --------------------------------------------------------------------------

def test_paper_dof_count():
    """Section 2.1: 524,288 hexahedra carry 1,098,306 DoFs (c and p at the
    nodes of the vertex-centred scheme), i.e. the 128x128x32 box."""
    g = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))
    P = O.Problem(128, 128, 32)
    assert P.C == g["box_mesh"]["cells"]
    assert 2 * O.lib().orc_num_nodes(__import__("ctypes").byref(P._c())) == g["box_mesh"]["dofs"]
    assert O.Problem(256, 256, 64).C == g["largest_box_mesh"]["cells"]


# --------------------------------------------------------------------------
# Jacobian = derivative of the residual
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(4, 8, 2), (8, 4, 4)])
def test_jacobian_matches_central_fd(dims):
    P = O.Problem(*dims)
    rng = np.random.default_rng(1)
    phi = 0.1 * np.exp(0.2 * rng.standard_normal(P.C))
    K = 4.845e-13 * (phi / 0.1) ** 3
    p0, c0 = O.initial_state(P)
    p = p0 + rng.normal(0, 3e3, P.N)
    c = np.clip(c0 + rng.uniform(0, 0.6, P.N), 0, 1)
    dt = YEAR / 12
    A = O.jacobian_dense(P, phi, K, p, c, dt)
    n = 2 * P.N
    worst = 0.0
    for jcol in range(n):
        h = 1e-2 if jcol % 2 == 0 else 1e-7
        up, uc = p.copy(), c.copy()
        dn_p, dn_c = p.copy(), c.copy()
        if jcol % 2 == 0:
            up[jcol // 2] += h
            dn_p[jcol // 2] -= h
        else:
            uc[jcol // 2] += h
            dn_c[jcol // 2] -= h
        Rp1, Rc1 = O.residual(P, phi, K, up, uc, p0, c0, dt)
        Rp0, Rc0 = O.residual(P, phi, K, dn_p, dn_c, p0, c0, dt)
        fd = np.empty(n)
        fd[0::2] = (Rp1 - Rp0) / (2 * h)
        fd[1::2] = (Rc1 - Rc0) / (2 * h)
        scale = np.abs(A).max(axis=1)
        worst = max(worst, float(np.max(np.abs(A[:, jcol] - fd) / scale)))
    assert worst < 1e-6


# --------------------------------------------------------------------------
# (a) pure diffusion: exact reduction to the 1D lumped scheme, and erfc
# --------------------------------------------------------------------------

def _thomas(a, b, c, d):
    """Tridiagonal solve (sub a, diag b, super c)."""
    n = len(b)
    cp, dp = np.zeros(n), np.zeros(n)
    cp[0] = c[0] / b[0]
    dp[0] = d[0] / b[0]
    for i in range(1, n):
        m = b[i] - a[i] * cp[i - 1]
        cp[i] = c[i] / m if i < n - 1 else 0.0
        dp[i] = (d[i] - a[i] * dp[i - 1]) / m
    x = np.zeros(n)
    x[-1] = dp[-1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def _layered_1d_step(cz, phi_layer, h, dt, Dm):
    """Implicit Euler, lumped mass, 3-point flux for
    d/dt(phi c) = d/dz(phi Dm dc/dz), c=0 at k=0 and c=1 at k=nz."""
    nz = len(cz) - 1
    a = np.zeros(nz + 1)
    b = np.ones(nz + 1)
    cc = np.zeros(nz + 1)
    d = np.zeros(nz + 1)
    d[0], d[nz] = 0.0, 1.0
    for k in range(1, nz):
        m = 0.5 * (phi_layer[k - 1] + phi_layer[k]) * h / dt
        fl, fu = phi_layer[k - 1] * Dm / h, phi_layer[k] * Dm / h
        a[k], b[k], cc[k] = -fl, m + fl + fu, -fu
        d[k] = m * cz[k]
    return _thomas(a, b, cc, d)


def test_diffusion_reduces_exactly_to_1d_scheme():
    """rho1 = rho0 gives q = 0 (Darcy law with constant density and the
    hydrostatic pressure), so for x,y-uniform data the box scheme must equal
    the 1D lumped-mass 3-point implicit Euler scheme in every column, also
    with z-layered porosity."""
    P = O.Problem(4, 4, 12, rho1=1000.0, bc_mode=2)
    k_cell = np.repeat(np.arange(P.nz), P.nx * P.ny)
    phi_layer = 0.08 + 0.04 * np.sin(np.arange(P.nz) + 0.3) ** 2
    phi = phi_layer[k_cell]
    K = np.full(P.C, 4.845e-13)
    p, c = O.initial_state(P)
    dt = YEAR / 12
    cz = np.zeros(P.nz + 1)
    cz[-1] = 1.0
    for _ in range(4):
        p, c, info = O.newton_step(P, phi, K, p, c, dt)
        assert info["status"] == 0
        cz = _layered_1d_step(cz, phi_layer, P.Lz / P.nz, dt, P.Dm)
    col = c.reshape(P.nz + 1, P.ny + 1, P.nx + 1)
    for j in range(P.ny + 1):
        for i in range(P.nx + 1):
            np.testing.assert_allclose(col[:, j, i], cz, rtol=0, atol=1e-13)


def test_diffusion_converges_to_erfc():
    """Continuum solution of the pure-diffusion column with c=1 at the top:
    c = erfc((Lz - z) / (2 sqrt(Dm t))).  Refining h by 2 and dt by 4 must
    cut the max error by about 4 (O(h^2 + dt))."""
    errs = []
    T = 1.2e6
    for nz, nt in ((16, 4), (32, 16), (64, 64)):
        P = O.Problem(2, 2, nz, Lx=1.0, Ly=1.0, Lz=16.0, rho1=1000.0, bc_mode=2)
        phi, K = _uniform(P)
        p, c = O.initial_state(P)
        for _ in range(nt):
            p, c, info = O.newton_step(P, phi, K, p, c, T / nt)
        z = np.arange(nz + 1) * P.Lz / nz
        exact = np.array([math.erfc((P.Lz - zz) / (2 * math.sqrt(P.Dm * T))) for zz in z])
        errs.append(np.abs(c.reshape(nz + 1, 3, 3)[:, 1, 1] - exact).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
    assert errs[2] < 5e-3


# --------------------------------------------------------------------------
# (b) hydrostatic states
# --------------------------------------------------------------------------

def test_uniform_concentration_is_hydrostatic():
    """Uniform c, no c Dirichlet data: q = 0, p = rho(c) g (Lz - z) exactly,
    c unchanged (eqs. e_Darcy_vel, e_lin_density with g = (0,0,-g))."""
    P = O.Problem(8, 8, 4, bc_mode=3)
    rng = np.random.default_rng(3)
    phi = 0.1 * np.exp(0.2 * rng.standard_normal(P.C))
    K = 4.845e-13 * np.exp(rng.standard_normal(P.C))
    cbar = 0.37
    c = np.full(P.N, cbar)
    p = np.zeros(P.N)  # far from the answer on purpose
    p1, c1, info = O.newton_step(P, phi, K, p, c, YEAR / 12)
    assert info["status"] == 0
    z = _node_xyz(P)[2]
    rho = P.rho0 + (P.rho1 - P.rho0) * cbar
    exact = rho * P.g * (P.Lz - z)
    assert np.max(np.abs(p1 - exact)) <= 1e-12 * rho * P.g * P.Lz
    assert np.max(np.abs(c1 - cbar)) <= 1e-14


def test_stratified_concentration_has_discrete_hydrostatic_pressure():
    """c depending on z only and no diffusion (Dm = 0), so c is static and
    the fluid-mass storage term vanishes: horizontal uniformity keeps
    q_x = q_y = 0 and the consistent gravity term must give q_z = 0 on every
    vertical edge, i.e. p_k - p_{k+1} = g h (rho_k + rho_{k+1}) / 2 with
    p = 0 on top.  (With Dm > 0 the density changes in time and the
    d(phi rho)/dt term of eq. e_cont_eq drives a flow.)"""
    P = O.Problem(4, 4, 8, Dm=0.0, bc_mode=3)
    phi, K = _uniform(P)
    z = _node_xyz(P)[2]
    c = 0.5 + 0.4 * np.cos(np.pi * z / P.Lz)
    p = np.zeros(P.N)
    p1, c1, info = O.newton_step(P, phi, K, p, c, YEAR / 12)
    assert info["status"] == 0
    assert np.max(np.abs(c1 - c)) < 1e-14  # static
    cz = c1.reshape(P.nz + 1, -1)
    rho = P.rho0 + (P.rho1 - P.rho0) * cz[:, 0]
    h = P.Lz / P.nz
    pz = np.zeros(P.nz + 1)
    for k in range(P.nz - 1, -1, -1):
        pz[k] = pz[k + 1] + P.g * h * 0.5 * (rho[k] + rho[k + 1])
    got = p1.reshape(P.nz + 1, -1)
    assert np.max(np.abs(got - pz[:, None])) <= 1e-12 * P.rho0 * P.g * P.Lz


# --------------------------------------------------------------------------
# (c) conservation
# --------------------------------------------------------------------------

def _masses(P, phi, c):
    """Salt and fluid mass of the lumped storage, summed cell by cell with
    math.fsum: sum_e sum_corners phi_e |scv| rho(c) (c)."""
    vscv = (P.Lx / P.nx) * (P.Ly / P.ny) * (P.Lz / P.nz) / 8
    cn = c.reshape(P.nz + 1, P.ny + 1, P.nx + 1)
    ph = phi.reshape(P.nz, P.ny, P.nx)
    salt, fluid = [], []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                cc = cn[dz:dz + P.nz, dy:dy + P.ny, dx:dx + P.nx]
                rho = P.rho0 + (P.rho1 - P.rho0) * cc
                salt.append((ph * vscv * rho * cc).ravel())
                fluid.append((ph * vscv * rho).ravel())
    return math.fsum(np.concatenate(salt)), math.fsum(np.concatenate(fluid))


def test_salt_and_fluid_mass_balance():
    """Summing the raw FV balances over all nodes, the face fluxes telescope,
    so sum_i R_i = (M^{n+1} - M^n)/dt for salt and fluid; at the converged
    step the interior balances vanish and the change of mass equals the
    Dirichlet-node fluxes."""
    P = O.Problem(8, 8, 4)
    rng = np.random.default_rng(5)
    phi, K = O.fields_lognormal(P, rng.standard_normal(P.C))
    p, c = O.initial_state(P)
    dt = YEAR / 12
    for _ in range(2):
        p_old, c_old = p, c
        p, c, info = O.newton_step(P, phi, K, p, c, dt)
        assert info["status"] == 0
    Rp, Rc = O.residual(P, phi, K, p, c, p_old, c_old, dt, apply_dirichlet=False)
    s1, f1 = _masses(P, phi, c)
    s0, f0 = _masses(P, phi, c_old)
    scale_s = math.fsum(np.abs(Rc)) + abs(s1 / dt)
    scale_f = math.fsum(np.abs(Rp)) + abs(f1 / dt)
    assert abs(math.fsum(Rc) - (s1 - s0) / dt) <= 1e-12 * scale_s
    assert abs(math.fsum(Rp) - (f1 - f0) / dt) <= 1e-12 * scale_f
    pm, cm, _ = O.dirichlet(P)
    # converged: interior balances vanish, Dirichlet fluxes carry the change
    assert abs(math.fsum(Rc[cm]) - (s1 - s0) / dt) <= 1e-10 * scale_s
    assert abs(math.fsum(Rp[pm]) - (f1 - f0) / dt) <= 1e-10 * scale_f


# --------------------------------------------------------------------------
# mirror symmetry of the benchmark problem
# --------------------------------------------------------------------------

def test_mirror_symmetry():
    """Uniform phi, K: the top square and the boundary sets are invariant
    under x -> Lx - x, y -> Ly - y and x <-> y, so the solution is too."""
    P = O.Problem(8, 8, 4)
    phi, K = _uniform(P)
    p, c = O.initial_state(P)
    for _ in range(3):
        p, c, info = O.newton_step(P, phi, K, p, c, YEAR / 12)
        assert info["status"] == 0
    for f in (p, c):
        a = f.reshape(P.nz + 1, P.ny + 1, P.nx + 1)
        tol = 1e-12 * max(1.0, np.abs(a).max())
        assert np.max(np.abs(a - a[:, :, ::-1])) <= tol
        assert np.max(np.abs(a - a[:, ::-1, :])) <= tol
        assert np.max(np.abs(a - a.transpose(0, 2, 1))) <= tol


# --------------------------------------------------------------------------
# closed-form fluxes
# --------------------------------------------------------------------------

def test_linear_pressure_gives_uniform_darcy_flux():
    """Uniform c and a linear p give a uniform Darcy flux q (eq. e_Darcy_vel).
    Its divergence vanishes, so each node's balance equals minus the outflow
    through the boundary part of its control volume:
    R_p,i = -rho sum_b (q.n_b) A_b and R_c,i = c R_p,i."""
    P = O.Problem(4, 6, 2, bc_mode=3)
    cbar = 0.25
    phi, K = _uniform(P, 0.1, 3e-13)
    x, y, z, i, j, k = _node_xyz(P)
    a, b, d = 3.0, -5.0, -11000.0
    p = a * x + b * y + d * z + 7.0
    c = np.full(P.N, cbar)
    Rp, Rc = O.residual(P, phi, K, p, c, p, c, 1.0, apply_dirichlet=False)
    rho = P.rho0 + (P.rho1 - P.rho0) * cbar
    q = -(3e-13 / P.mu) * np.array([a, b, d + rho * P.g])
    h = np.array([P.Lx / P.nx, P.Ly / P.ny, P.Lz / P.nz])
    idx = np.stack([i, j, k], 1)
    nmax = np.array([P.nx, P.ny, P.nz])
    expect = np.zeros(P.N)
    for node in range(P.N):
        ext = np.where((idx[node] == 0) | (idx[node] == nmax), h / 2, h)
        for dd in range(3):
            area = np.prod(np.delete(ext, dd))
            if idx[node, dd] == 0:
                expect[node] -= rho * (-q[dd]) * area
            if idx[node, dd] == nmax[dd]:
                expect[node] -= rho * (q[dd]) * area
    scale = rho * np.abs(q).max() * h.max() ** 2
    np.testing.assert_allclose(Rp, expect, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(Rc, cbar * expect, rtol=0, atol=1e-11 * scale)


def test_upwind_direction_and_diffusion_closed_form():
    """Constant density, flow in +x (p = a x with a < 0), c = (x/Lx)^2 and no
    time change: at interior nodes the full-upwind advective balance is
    m (c_i - c_{i-1}) and the diffusive one -rho phi Dm A (c_{i+1} - 2c_i +
    c_{i-1})/h.  A downwind choice would give m (c_{i+1} - c_i)."""
    P = O.Problem(6, 4, 2, rho1=1000.0, bc_mode=3)
    phi, K = _uniform(P, 0.12, 4e-13)
    x, y, z, i, j, k = _node_xyz(P)
    a = -2000.0
    p = a * x + P.rho0 * P.g * (P.Lz - z)
    c = (x / P.Lx) ** 2
    Rp, Rc = O.residual(P, phi, K, p, c, p, c, 1.0, apply_dirichlet=False)
    hx, hy, hz = P.Lx / P.nx, P.Ly / P.ny, P.Lz / P.nz
    A = hy * hz
    m = P.rho0 * (-(4e-13 / P.mu) * a) * A
    interior = (i > 0) & (i < P.nx) & (j > 0) & (j < P.ny) & (k > 0) & (k < P.nz)
    cm = ((i - 1) * hx / P.Lx) ** 2
    cpl = ((i + 1) * hx / P.Lx) ** 2
    expect = m * (c - cm) - P.rho0 * 0.12 * P.Dm * A * (cpl - 2 * c + cm) / hx
    np.testing.assert_allclose(Rc[interior], expect[interior], rtol=1e-12, atol=0)
    np.testing.assert_allclose(Rp[interior], 0.0, atol=1e-12 * abs(m))


# --------------------------------------------------------------------------
# (d) linear solvers
# --------------------------------------------------------------------------

def test_dense_and_iterative_solves_on_4x4x2():
    P = O.Problem(4, 4, 2)
    rng = np.random.default_rng(7)
    phi, K = O.fields_lognormal(P, rng.standard_normal(P.C))
    p0, c0 = O.initial_state(P)
    c = np.clip(c0 + rng.uniform(0, 0.5, P.N), 0, 1)
    rowptr, col, val = O.jacobian_csr(P, phi, K, p0, c, YEAR / 12)
    A = O.jacobian_dense(P, phi, K, p0, c, YEAR / 12)
    b = rng.standard_normal(2 * P.N)
    x = O.dense_solve(A, b)
    assert np.linalg.norm(A @ x - b) <= 1e-13 * np.linalg.norm(b) * np.linalg.cond(A) ** 0.5
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9,
                               atol=1e-12 * np.abs(x).max())
    xi, rc, it, rr = O.bicgstab_ilu0(rowptr, col, val, b, rtol=1e-13)
    assert rc == 0 and rr <= 1e-12
    np.testing.assert_allclose(xi, x, rtol=0, atol=1e-8 * np.abs(x).max())
    # transposed solve: <A^-1 b, w> = <b, A^-T w>
    w = rng.standard_normal(2 * P.N)
    y, rc = O.linear_solve(rowptr, col, val, w, transpose=True)
    assert rc == 0
    assert abs(x @ w - b @ y) <= 1e-10 * abs(x @ w)


# --------------------------------------------------------------------------
# statistics and sample fields
# --------------------------------------------------------------------------

def test_moments_match_numpy():
    rng = np.random.default_rng(11)
    cs = rng.uniform(0, 1, (37, 101))
    mean, var, pexc = O.moments(cs, threshold=0.5)
    np.testing.assert_allclose(mean, cs.mean(0), rtol=1e-14)
    np.testing.assert_allclose(var, cs.var(0), rtol=1e-12)
    np.testing.assert_allclose(pexc, (cs > 0.5).mean(0), rtol=1e-14)
    w = rng.uniform(0.5, 1.5, 37)
    w /= w.sum()
    mean, var, pexc = O.moments(cs, w=w, threshold=0.3)
    np.testing.assert_allclose(mean, np.average(cs, 0, w), rtol=1e-13)
    np.testing.assert_allclose(var, np.average((cs - np.average(cs, 0, w)) ** 2, 0, w), rtol=1e-11)
    np.testing.assert_allclose(pexc, (w[:, None] * (cs > 0.3)).sum(0), rtol=1e-13)
    # strict ">" (exceedance estimate of Section 3.3)
    _, _, pe = O.moments(np.full((4, 3), 0.5))
    assert np.all(pe == 0.0)


def test_sample_fields_properties():
    """Kozeny-Carman normalised so that K(E phi) = E K (eq.
    e_perm_Kozeny_Carman); the Sobol field has mean level 0.1 at xi = 0 and
    stays within 0.1*(1 +- 0.3); the lognormal field is clipped to
    [0.05, 0.2]."""
    P = O.Problem(8, 8, 4)
    phi, K = O.fields_sobol(P, [0.0, 0.0, 0.0])
    assert np.all(phi == 0.1)
    np.testing.assert_allclose(K, 4.845e-13, rtol=1e-15)
    phi, K = O.fields_sobol(P, [1.0, -1.0, 1.0])
    assert phi.min() >= 0.07 - 1e-15 and phi.max() <= 0.13 + 1e-15
    np.testing.assert_allclose(K, 4.845e-13 * (phi ** 3 / (1 - phi) ** 2) / (0.1 ** 3 / 0.9 ** 2), rtol=1e-14)
    Z = np.linspace(-20, 20, P.C)
    phi, K = O.fields_lognormal(P, Z)
    assert phi.min() == 0.05 and phi.max() == 0.2
    phi, K = O.fields_lognormal(P, np.zeros(P.C))
    assert np.all(phi == 0.1)


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------

def test_adjoint_gradient_matches_central_fd():
    P = O.Problem(8, 8, 4)
    rng = np.random.default_rng(13)
    phi, K = O.fields_lognormal(P, rng.standard_normal(P.C))
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    steps = 3
    # tight Newton so that the FD quotient is not limited by the solve; the
    # FD step is 1e-3 relative: J is ~1e6 kg, so at 1e-6 relative the FP64
    # round-off of J alone moves the quotient by ~1e-4 relative.
    opts = O.NewtonOpts(tol_c=1e-15, tol_p=1e-9, maxit=40)
    J, gphi, gK, rc = O.adjoint_gradient(P, phi, K, p0, c0, dt, steps, opts)
    assert rc == 0

    def J_of(ph, KK):
        p, c, _ = O.run_steps(P, ph, KK, p0, c0, dt, steps, opts)
        return O.objective(P, ph, c)

    assert abs(J_of(phi, K) - J) <= 1e-13 * abs(J)
    cells = rng.choice(P.C, 8, replace=False)
    for e in cells:
        for which, g in (("phi", gphi), ("K", gK)):
            base = phi if which == "phi" else K
            h = 1e-3 * base[e]
            up, dn = base.copy(), base.copy()
            up[e] += h
            dn[e] -= h
            if which == "phi":
                fd = (J_of(up, K) - J_of(dn, K)) / (2 * h)
            else:
                fd = (J_of(phi, up) - J_of(phi, dn)) / (2 * h)
            scale = np.abs(g).max()
            assert abs(fd - g[e]) <= 1e-5 * max(abs(g[e]), 1e-3 * scale), (which, e, fd, g[e])


# --------------------------------------------------------------------------
# the paper's parallelepiped porosity field (Section 5.3, eq. poro-paral3RVS)
# --------------------------------------------------------------------------

def _kc(phi, K_mean=4.845e-13):
    return K_mean * (phi ** 3 / (1 - phi) ** 2) / (0.1 ** 3 / 0.9 ** 2)


def test_paper3rv_field_closed_forms():
    """eq. poro-paral3RVS: phi = 0.1 + 0.01 (xi1 sx + xi2 sy + xi3 sz + xi1 sx sy
    + xi2 sx sz) with sx = sin(pi x/600), sy = sin(pi y/600), sz = sin(pi
    z/150) at the cell centre.  On a 6x6x2 grid the centres sit at x, y in
    {50, 150, ..., 550} and z in {37.5, 112.5}, where the sines have closed
    forms: sin(pi/12) = (sqrt6 - sqrt2)/4, sin(pi/4) = sqrt2/2, sin(5pi/12) =
    (sqrt6 + sqrt2)/4, and sz = sqrt2/2 in both layers.  Expected values are
    written from those surds, not from the oracle's expression."""
    P = O.Problem(6, 6, 2)
    r2, r6 = math.sqrt(2.0), math.sqrt(6.0)
    s = {0: (r6 - r2) / 4, 1: r2 / 2, 2: (r6 + r2) / 4}  # sin of the centre of cell i (i<=2)

    def cell(i, j, k):
        return i + P.nx * (j + P.ny * k)

    phi0, K0 = O.fields_paper3rv(P, [0.0, 0.0, 0.0])
    assert np.all(phi0 == 0.1)
    np.testing.assert_allclose(K0, 4.845e-13, rtol=1e-15)
    sz = r2 / 2
    cases = [  # (xi, cell (i, j, k), expected phi)
        ((1.0, 0.0, 0.0), (1, 0, 0), 0.1 + 0.01 * (s[1] + s[1] * s[0])),
        ((1.0, 0.0, 0.0), (0, 2, 1), 0.1 + 0.01 * (s[0] + s[0] * s[2])),
        ((0.0, 1.0, 0.0), (2, 0, 0), 0.1 + 0.01 * (s[0] + s[2] * sz)),
        ((0.0, 1.0, 0.0), (0, 1, 1), 0.1 + 0.01 * (s[1] + s[0] * sz)),
        ((0.0, 0.0, 1.0), (2, 1, 0), 0.1 + 0.01 * sz),
        ((-1.0, 0.5, 1.0), (1, 2, 1),
         0.1 + 0.01 * (-s[1] + 0.5 * s[2] + sz - s[1] * s[2] + 0.5 * s[1] * sz)),
    ]
    for xi, (i, j, k), want in cases:
        phi, K = O.fields_paper3rv(P, list(xi))
        assert abs(phi[cell(i, j, k)] - want) <= 1e-16, (xi, (i, j, k), phi[cell(i, j, k)], want)
        assert abs(K[cell(i, j, k)] - _kc(want)) <= 1e-14 * _kc(want)


def test_paper3rv_field_mirror_symmetries():
    """All three sines are symmetric under x -> 600 - x, y -> 600 - y and
    z -> 150 - z (sin(pi - a) = sin a), so the field is too, for every xi;
    the cross terms are not symmetric under x <-> y (xi2 multiplies sx sz, not
    sy sz), which a swapped argument would make them."""
    P = O.Problem(8, 12, 4)
    rng = np.random.default_rng(3)
    for _ in range(4):
        phi, _ = O.fields_paper3rv(P, rng.uniform(-1, 1, 3))
        a = phi.reshape(P.nz, P.ny, P.nx)
        np.testing.assert_allclose(a, a[:, :, ::-1], rtol=0, atol=1e-16)
        np.testing.assert_allclose(a, a[:, ::-1, :], rtol=0, atol=1e-16)
        np.testing.assert_allclose(a, a[::-1, :, :], rtol=0, atol=1e-16)
    Q = O.Problem(8, 8, 4)
    phi, _ = O.fields_paper3rv(Q, [0.0, 1.0, 0.0])
    a = phi.reshape(Q.nz, Q.ny, Q.nx)
    assert np.abs(a - a.transpose(0, 2, 1)).max() > 1e-4


# --------------------------------------------------------------------------
# the plume functional (salt mass below mid-depth)
# --------------------------------------------------------------------------

def test_objective_closed_forms():
    """J = sum over the cells whose centre lies below Lz/2 of sum over their
    8 corners of phi_e |scv| rho(c) c, |scv| = hx hy hz / 8.  Closed forms on
    an even nz (the mid-plane is a grid plane):
      c = 1 everywhere:   J = rho1 phi Lx Ly Lz / 2;
      c = 0.5 everywhere: J = rho(0.5) 0.5 phi Lx Ly Lz / 2;
      c = 0 everywhere:   J = 0;
      c = 1 on nodes with z > Lz/2 only: J = 0 (no lower cell has such a corner);
      c = 1 on nodes with z >= Lz/2: only the upper corners of the top lower
        layer count, 4 per cell: J = rho1 phi Lx Ly hz / 2;
    and with phi different per layer only the lower layers count."""
    P = O.Problem(8, 6, 4)
    phi = np.full(P.C, 0.13)
    x, y, z, i, j, k = _node_xyz(P)
    V = P.Lx * P.Ly * P.Lz
    hz = P.Lz / P.nz
    rho = lambda cc: P.rho0 + (P.rho1 - P.rho0) * cc  # noqa: E731
    tol = 1e-13
    assert abs(O.objective(P, phi, np.ones(P.N)) - P.rho1 * 0.13 * V / 2) <= tol * P.rho1 * V
    assert abs(O.objective(P, phi, np.full(P.N, 0.5)) - rho(0.5) * 0.5 * 0.13 * V / 2) \
        <= tol * P.rho1 * V
    assert O.objective(P, phi, np.zeros(P.N)) == 0.0
    assert O.objective(P, phi, (z > P.Lz / 2).astype(float)) == 0.0
    want = P.rho1 * 0.13 * P.Lx * P.Ly * hz / 2
    assert abs(O.objective(P, phi, (z >= P.Lz / 2 - 1e-9).astype(float)) - want) <= tol * want
    # layered porosity: layers k = 0, 1 (below) weigh in, layers 2, 3 do not
    lay = np.array([0.05, 0.07, 0.11, 0.19])
    phil = np.repeat(lay, P.nx * P.ny)
    want = P.rho1 * (lay[0] + lay[1]) * P.Lx * P.Ly * hz
    assert abs(O.objective(P, phil, np.ones(P.N)) - want) <= tol * want


# --------------------------------------------------------------------------
# boundary sets (Section 2.1 and the caption of Fig. 1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(8, 8, 4), (12, 16, 2), (4, 8, 3)])
def test_dirichlet_sets_counts(dims):
    """Paper variant (bc_mode 1): p = 0 on the four top edges, i.e. 2(nx+1) +
    2(ny+1) - 4 nodes; c prescribed on every top and every bottom node and
    nowhere else, with c = 1 on the closed square [Lx/4, 3Lx/4] x [Ly/4,
    3Ly/4] of the top, (nx/2 + 1)(ny/2 + 1) nodes, and c = 0 on the rest.
    Benchmark (bc_mode 0): p = 0 at the four top corners only; c prescribed
    on the square and on the bottom only."""
    nx, ny, nz = dims
    for mode in (0, 1):
        P = O.Problem(nx, ny, nz, bc_mode=mode)
        pm, cm, cv = O.dirichlet(P)
        x, y, z, i, j, k = _node_xyz(P)
        top, bottom = k == nz, k == 0
        sq = top & (4 * i >= nx) & (4 * i <= 3 * nx) & (4 * j >= ny) & (4 * j <= 3 * ny)
        assert sq.sum() == (nx // 2 + 1) * (ny // 2 + 1)
        edge = top & ((i == 0) | (i == nx) | (j == 0) | (j == ny))
        corner = top & ((i == 0) | (i == nx)) & ((j == 0) | (j == ny))
        if mode == 1:
            assert pm.sum() == 2 * (nx + 1) + 2 * (ny + 1) - 4
            assert np.array_equal(pm, edge)
            assert np.array_equal(cm, top | bottom)
        else:
            assert pm.sum() == 4 and np.array_equal(pm, corner)
            assert np.array_equal(cm, sq | bottom)
        assert np.array_equal(cv == 1.0, sq)
        assert np.all(cv[~sq] == 0.0)


def test_mirror_symmetry_paper_boundary_variant():
    """bc_mode 1 is invariant under x -> Lx - x, y -> Ly - y and x <-> y as
    well, so the solution is too (uniform phi, K)."""
    P = O.Problem(8, 8, 4, bc_mode=1)
    phi, K = _uniform(P)
    p, c = O.initial_state(P)
    for _ in range(3):
        p, c, info = O.newton_step(P, phi, K, p, c, YEAR / 12)
        assert info["status"] == 0
    for f in (p, c):
        a = f.reshape(P.nz + 1, P.ny + 1, P.nx + 1)
        tol = 1e-12 * max(1.0, np.abs(a).max())
        assert np.max(np.abs(a - a[:, :, ::-1])) <= tol
        assert np.max(np.abs(a - a[:, ::-1, :])) <= tol
        assert np.max(np.abs(a - a.transpose(0, 2, 1))) <= tol
    # Dirichlet rows (R = u - u_D) hold c at its prescribed values: 1 on the
    # square, 0 on the rest of the top and on the bottom
    pm, cm, cv = O.dirichlet(P)
    assert np.abs(c[cm] - cv[cm]).max() <= 1e-15
    assert np.abs(p[pm]).max() <= 1e-9


def test_line_smoother_reaches_the_same_step():
    """The oracle's two multigrid smoothers only change the path of the
    linear solves: the converged implicit step (and a transposed solve) agree
    to round-off.  16x16x4 has 2890 unknowns, above the dense-LU limit."""
    P = O.Problem(16, 16, 4)
    rng = np.random.default_rng(17)
    phi, K = O.fields_lognormal(P, rng.standard_normal(P.C))
    p0, c0 = O.initial_state(P)
    dt = YEAR / 12
    out = []
    for sm in (0, 1):
        p, c, info = O.newton_step(P, phi, K, p0, c0, dt, O.NewtonOpts(smoother=sm))
        assert info["status"] == 0
        out.append((p, c, info["lin_iters"]))
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-13
    assert np.abs(out[0][0] - out[1][0]).max() <= 1e-9 * P.rho0 * P.g * P.Lz
    # the adjoint's transposed multigrid solves (two steps)
    g = []
    for sm in (0, 1):
        J, gphi, gK, rc = O.adjoint_gradient(P, phi, K, p0, c0, dt, 2, O.NewtonOpts(smoother=sm))
        assert rc == 0
        g.append((J, gphi, gK))
    assert abs(g[0][0] - g[1][0]) <= 1e-13 * abs(g[0][0])
    # the gradients go through the states' Jacobians, so they inherit the
    # states' round-off differences amplified by the solves: 1e-6 of the
    # largest entry (the FD pins hold the adjoint to 1e-5)
    for q in (1, 2):
        np.testing.assert_allclose(g[1][q], g[0][q], rtol=0, atol=1e-6 * np.abs(g[0][q]).max())
