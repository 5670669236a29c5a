"""gPC surrogate on the GPU (Section 3) against the oracle, through the C ABI.

Projection, mean and variance are FP64 and compared element by element.  The
exceedance estimate evaluates the surrogate in FP32, so the decision
"u_hat > c*" is compared where it is unique: the GPU count must lie between
the oracle's FP64 counts at c* + delta and c* - delta, delta the FP32
evaluation bound 16 T 2^-24 sum_t |u_t| per node."""
import numpy as np
import pytest

import oracle as O
from oracle import gpc as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
YEAR = O.SECONDS_PER_YEAR


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_01632_gb300 import build
    build.build()
    from paper_1906_01632_gb300 import elder
    return elder


def Td(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def Ti(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.int32, device=DEV)


@pytest.mark.parametrize("M,p,q,N", [(3, 4, 5, 5003), (3, 2, 3, 129), (2, 6, 7, 1), (4, 3, 4, 777)])
def test_projection_matches_oracle(E, M, p, q, N):
    beta = G.multi_indices(M, p)
    th, w = G.tensor_grid(q, M)
    rng = np.random.default_rng(M * 100 + p)
    u = rng.uniform(0, 1, (th.shape[0], N))
    coef, mean, var = E.elder_gpc_project(Ti(beta), Td(th), Td(w), Td(u))
    c_ref = G.project(u, th, w, beta)
    m_ref, v_ref = G.mean_var(c_ref, beta)
    assert np.abs(coef.cpu().numpy() - c_ref).max() < 1e-13
    assert np.abs(mean.cpu().numpy() - m_ref).max() < 1e-14
    assert np.abs(var.cpu().numpy() - v_ref).max() < 1e-14


def _bracket_check(E, beta, coef, theta, thr, nodes=None, engine="auto"):
    cg = E.elder_gpc_exceed(Ti(beta), Td(coef), Td(theta), thr,
                            None if nodes is None else Ti(nodes), engine=engine).cpu().numpy()
    sel = coef if nodes is None else coef[:, nodes]
    Ns = theta.shape[0]
    delta = 16 * beta.shape[0] * 2.0**-24 * np.abs(sel).sum(0)
    vals = G.evaluate(sel, beta, theta)
    lo = (vals > thr + delta).sum(0)
    hi = (vals > thr - delta).sum(0)
    got = np.rint(cg * Ns).astype(np.int64)
    assert np.allclose(cg * Ns, got, atol=1e-6)
    assert ((got >= lo) & (got <= hi)).all()
    return got, lo, hi


# (3, 4): 35 terms (the bench's surrogate, padded to 36, 4 nodes per thread);
# (3, 3): 20 terms; (3, 5) and (5, 3): 56 terms (2 nodes per thread)
@pytest.mark.parametrize("M,p,engine", [(3, 4, "fp32"), (3, 3, "fp32"), (3, 5, "fp32"),
                                        (5, 3, "fp32"), (3, 4, "tensor"), (3, 3, "tensor"),
                                        (2, 6, "tensor"), (4, 2, "tensor"), (3, 5, "auto")])
def test_exceedance_brackets_oracle(E, M, p, engine):
    beta = G.multi_indices(M, p)
    rng = np.random.default_rng(7 + 10 * M + p)
    N = 300
    # coefficients of smooth responses: decaying with degree, mean near the threshold
    deg = beta.sum(1)
    coef = rng.standard_normal((beta.shape[0], N)) * (0.3 ** deg)[:, None]
    coef[0] = rng.uniform(0.3, 0.7, N)
    theta = rng.uniform(-1, 1, (20011, M))  # ragged: not a multiple of the chunk
    got, lo, hi = _bracket_check(E, beta, coef, theta, 0.5, engine=engine)
    assert (hi - lo).max() <= 24  # the FP32 band holds at most a few samples
    nodes = np.array([5, 0, 299, 17, 17, 123], dtype=np.int32)
    _bracket_check(E, beta, coef, theta, 0.5, nodes, engine=engine)
    if engine == "tensor":  # the two engines agree but for samples inside the band
        cf = E.elder_gpc_exceed(Ti(beta), Td(coef), Td(theta), 0.5, engine="fp32").cpu().numpy()
        assert np.abs(np.rint(cf * theta.shape[0]) - got).max() <= (hi - lo).max()


def test_tensor_engine_basis_in_other_order(E):
    """The total-degree-4 basis in 3 variables with its terms permuted (the
    kernel builds the canonical order from registers and any other order from
    the Legendre table): the count still lies in the oracle bracket, and
    agrees with the canonical order but for samples inside the band."""
    beta = G.multi_indices(3, 4)
    rng = np.random.default_rng(31)
    N = 300
    deg = beta.sum(1)
    coef = rng.standard_normal((beta.shape[0], N)) * (0.3 ** deg)[:, None]
    coef[0] = rng.uniform(0.3, 0.7, N)
    theta = rng.uniform(-1, 1, (20011, 3))
    perm = rng.permutation(beta.shape[0])
    got, lo, hi = _bracket_check(E, beta[perm], coef[perm], theta, 0.5, engine="tensor")
    canon, _, _ = _bracket_check(E, beta, coef, theta, 0.5, engine="tensor")
    assert np.abs(got - canon).max() <= (hi - lo).max()


def test_exceedance_closed_form(E):
    """u_hat = theta_1 on a midpoint grid: exactly 35% exceed 0.3 (the FP32
    band is empty there: no grid point within 1e-6 of 0.3)."""
    beta = G.multi_indices(2, 2)
    coef = np.zeros((beta.shape[0], 3))
    t1 = [t for t, b in enumerate(beta) if tuple(b) == (1, 0)][0]
    coef[t1, 0] = 1.0
    coef[0, 1] = 0.25
    coef[0, 2] = 0.75
    K = 100000
    g = -1 + (np.arange(K) + 0.5) * 2 / K
    theta = np.stack([g, np.zeros(K)], 1)
    for engine in ("fp32", "tensor"):
        pe = E.elder_gpc_exceed(Ti(beta), Td(coef), Td(theta), 0.3, engine=engine).cpu().numpy()
        assert pe[0] == 0.35 and pe[1] == 0.0 and pe[2] == 1.0, engine


def test_surrogate_workflow_matches_oracle_and_qmc(E):
    """Section 3 workflow at 8x8x2: the batched step at the 27 points of the
    3^3 Gauss-Legendre grid, projection onto total degree <= 2, mean and
    variance of c; against the oracle's steps and projection at 1e-9, and
    the gPC mean against a 64-point scrambled-Sobol QMC mean of the GPU
    step within 5e-3 (a validation, as in the paper, not a parity check)."""
    from paper_1906_01632_gb300 import inputs as I
    P = O.Problem(8, 8, 2)
    M, p, q = 3, 2, 3
    beta = G.multi_indices(M, p)
    th, w = G.tensor_grid(q, M)
    S = th.shape[0]
    dt, steps = YEAR / 12, 4
    ctx = E.elder_create(E.elder_config_default(8, 8, 2, max_samples=64))
    phi, K = ctx.fields(S, 0, Td(th.ravel()))
    p_, c_ = ctx.initial_state(S, device=DEV)
    for _ in range(steps):
        st, _ = ctx.step(S, phi, K, p_, c_, dt)
        assert (st == 0).all()
    u = c_.reshape(S, -1)
    coef, mean, var = E.elder_gpc_project(Ti(beta), Td(th), Td(w), u)
    # oracle pipeline
    p0, c0 = O.initial_state(P)
    cref = np.zeros((S, P.N))
    for s in range(S):
        ph, kk = O.fields_sobol(P, th[s])
        pp, cc = p0, c0
        for _ in range(steps):
            pp, cc, info = O.newton_step(P, ph, kk, pp, cc, dt)
            assert info["status"] == 0
        cref[s] = cc
    m_ref, v_ref = G.mean_var(G.project(cref, th, w, beta), beta)
    assert np.abs(mean.cpu().numpy() - m_ref).max() < 1e-9
    assert np.abs(var.cpu().numpy() - v_ref).max() < 1e-9
    # QMC validation
    Sq = 64
    xi = Td(I.sobol_xi(Sq, seed=0).ravel())
    phq, kq = ctx.fields(Sq, 0, xi)
    pq, cq = ctx.initial_state(Sq, device=DEV)
    for _ in range(steps):
        st, _ = ctx.step(Sq, phq, kq, pq, cq, dt)
        assert (st == 0).all()
    qmc_mean = cq.reshape(Sq, -1).mean(0).cpu().numpy()
    assert np.abs(mean.cpu().numpy() - qmc_mean).max() < 5e-3


def test_tensor_engine_many_tiles_and_slices(E):
    """The tensor-core count at a size with many node tiles (1,000 nodes: 8
    tiles, the last ragged) and many sample chunks per CTA (300,017 points,
    the last chunk ragged), against the FP32 engine and the oracle bracket at
    sampled nodes; nodes listed in reverse order."""
    beta = G.multi_indices(3, 4)
    rng = np.random.default_rng(99)
    N = 1000
    deg = beta.sum(1)
    coef = rng.standard_normal((beta.shape[0], N)) * (0.3 ** deg)[:, None]
    coef[0] = rng.uniform(0.3, 0.7, N)
    theta = rng.uniform(-1, 1, (300017, 3))
    nodes = np.arange(N - 1, -1, -1).astype(np.int32)
    tc = E.elder_gpc_exceed(Ti(beta), Td(coef), Td(theta), 0.5, Ti(nodes), engine="tensor")
    f32 = E.elder_gpc_exceed(Ti(beta), Td(coef), Td(theta), 0.5, Ti(nodes), engine="fp32")
    tc, f32 = tc.cpu().numpy(), f32.cpu().numpy()
    assert np.isfinite(tc).all()
    Ns = theta.shape[0]
    assert np.abs(np.rint(tc * Ns) - np.rint(f32 * Ns)).max() <= 24
    pick = np.array([0, 1, 127, 128, 500, 998, 999])
    sub = coef[:, nodes[pick]]
    vals = G.evaluate(sub, beta, theta)
    delta = 16 * beta.shape[0] * 2.0**-24 * np.abs(sub).sum(0)
    lo = (vals > 0.5 + delta).sum(0)
    hi = (vals > 0.5 - delta).sum(0)
    got = np.rint(tc[pick] * Ns)
    assert ((got >= lo) & (got <= hi)).all()
