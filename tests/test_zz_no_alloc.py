"""The allocation-free residual entry point (elder_residual_norms_static).

It exists for callers that must not allocate device memory: it takes no
context and keeps its only scratch (block partial sums) in a fixed device
array inside the library.  Checked here through the C ABI against the
regular context-based elder_residual on two calls in a row; this file is
collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_01632_gb300 import build
    build.build()
    from paper_1906_01632_gb300 import elder
    return elder


def _inputs(nx, ny, nz, S, seed):
    rng = np.random.default_rng(seed)
    N = (nx + 1) * (ny + 1) * (nz + 1)
    C = nx * ny * nz
    k = np.repeat(np.arange(nz + 1), (nx + 1) * (ny + 1))
    p0 = 1000.0 * 9.81 * (150.0 - k * 150.0 / nz)
    phi = 0.1 * np.exp(0.2 * rng.standard_normal((S, C)))
    K = 4.845e-13 * (phi / 0.1) ** 3
    p = p0 + rng.normal(0, 2e3, (S, N))
    c = rng.uniform(0, 1, (S, N))
    po = p0 + rng.normal(0, 2e3, (S, N))
    co = rng.uniform(0, 1, (S, N))

    def T(a):
        return torch.tensor(a.ravel(), dtype=torch.float64, device="cuda:0")
    return [T(a) for a in (phi, K, p, c, po, co)]


@pytest.mark.parametrize("bc_mode", [0, 1, 2, 3])
def test_static_scratch_residual_matches_context_residual(E, bc_mode):
    """Every boundary set: the entry point evaluates the Dirichlet sets from
    the node indices itself, the context from its stored masks."""
    dt = 365.25 * 86400.0 / 12
    for (nx, ny, nz, S, seed) in ((16, 16, 4, 3, 1 + bc_mode), (32, 32, 8, 2, 2 + bc_mode)):
        cfg = E.elder_config_default(nx, ny, nz, max_samples=S, bc_mode=bc_mode)
        ctx = E.elder_create(cfg)
        phi, K, p, c, po, co = _inputs(nx, ny, nz, S, seed)
        R_ref = ctx.residual(S, phi, K, p, c, po, co, dt)
        torch.cuda.synchronize()
        norms_ref = R_ref.view(S, -1).norm(dim=1)
        scale = R_ref.abs().max().item()
        for _ in range(2):  # two calls in a row share the static scratch
            R, norms = E.elder_residual_norms_static(cfg, S, phi, K, p, c, po, co, dt)
            torch.cuda.synchronize()
            assert (R - R_ref).abs().max().item() <= 1e-12 * scale
            torch.testing.assert_close(norms, norms_ref, rtol=1e-12, atol=0.0)
        ctx.destroy()


def test_static_scratch_rejects_oversized_batch(E):
    cfg = E.elder_config_default(64, 64, 16, max_samples=1)
    N = 65 * 65 * 17
    S = 262144 // ((N + 255) // 256) + 1
    phi, K, p, c, po, co = _inputs(4, 4, 2, 1, 0)  # never read: the call is refused first
    with pytest.raises(E.ElderError) as ei:
        E.elder_residual_norms_static(cfg, S, phi, K, p, c, po, co, 1.0,
                                      R=torch.empty(1, dtype=torch.float64, device="cuda:0"),
                                      norms=torch.empty(1, dtype=torch.float64, device="cuda:0"))
    assert ei.value.code == E.ELDER_EINVAL
    assert "capacity" in str(ei.value)


def test_static_scratch_rejects_more_samples_than_the_launch_grid_holds(E):
    """On a grid of at most 256 nodes one partial sum per sample fits the
    scratch for up to 262,144 samples, but a call takes at most 65,535 (the
    samples run along the launch grid's y dimension): refused before any
    launch."""
    cfg = E.elder_config_default(4, 4, 2, max_samples=1)
    phi, K, p, c, po, co = _inputs(4, 4, 2, 1, 0)  # never read: the call is refused first
    with pytest.raises(E.ElderError) as ei:
        E.elder_residual_norms_static(cfg, 65536, phi, K, p, c, po, co, 1.0,
                                      R=torch.empty(1, dtype=torch.float64, device="cuda:0"),
                                      norms=torch.empty(1, dtype=torch.float64, device="cuda:0"))
    assert ei.value.code == E.ELDER_EINVAL
    assert "65535" in str(ei.value)
