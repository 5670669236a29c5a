"""Pins of the oracle's multicolour block ILU_beta(0) smoother (Section 5.1
names the multigrid smoother ILU_beta and does not define it; the reading is
block ILU(0) in the 8-colour node order, beta lumping the dropped fill onto
the diagonal block).  Each property below follows from the definition of the
factorisation, not from the oracle's code:

- beta = 0: L U agrees with A on every block of A's pattern (ILU(0));
- beta = 1: every block row sum of L U equals A's (modified ILU);
- the colour classes are independent sets of the 27-point stencil;
- the triangular solves equal a dense solve with L U and with (L U)^T;
- beta = 0: the factors of A^T are the transposes of A's (L'U' = (L U)^T);
- the smoother applications (kinds 0, 1, 2) equal dense linear algebra on
  the interior Jacobian: the block diagonal, the vertical-line block
  tridiagonal part, and L U;
- Newton with the ILU smoother reaches the state the other smoothers reach
  (at 16x16x4 with V(1,1): 24 BiCGStab iterations for the step with beta = 0,
  38 with the line smoother, 52 with point Jacobi).
"""
import numpy as np
import pytest

import oracle as O

DT = O.SECONDS_PER_YEAR / 12


@pytest.fixture(scope="module", params=[(8, 8, 4, 0), (6, 10, 3, 2)],
                ids=["8x8x4-benchmark", "6x10x3-column"])
def case(request):
    """A box after one implicit step (a physical, nonsymmetric Jacobian with
    upwinding and Dirichlet rows): 8x8x4 with the benchmark boundary sets,
    and 6x10x3 (odd node counts in y and z, colour classes of unequal
    sizes) with the diffusion-column set."""
    O.build()
    nx, ny, nz, bc = request.param
    P = O.Problem(nx, ny, nz, bc_mode=bc)
    rng = np.random.default_rng(5)
    phi = 0.1 * (1 + 0.2 * rng.uniform(-1, 1, P.C))
    K = 4.845e-13 * (phi / 0.1) ** 3 * (0.9 / (1 - phi)) ** 2
    p, c = O.initial_state(P)
    p1, c1, info = O.newton_step(P, phi, K, p, c, DT)
    assert info["status"] == 0
    return P, phi, K, p1, c1


def _interior_dense(P, phi, K, p, c):
    """The Jacobian with Dirichlet rows and columns replaced by the identity."""
    A = O.jacobian_dense(P, phi, K, p, c, DT)
    pm, cm, _ = O.dirichlet(P)
    dm = np.zeros(2 * P.N, bool)
    dm[0::2], dm[1::2] = pm, cm
    A[dm, :] = 0.0
    A[:, dm] = 0.0
    A[dm, dm] = 1.0
    return A, dm


def _blocks_to_dense(P, B):
    A = np.zeros((2 * P.N, 2 * P.N))
    sx, sy = P.nx + 1, P.ny + 1
    for n in range(P.N):
        i, j, k = n % sx, (n // sx) % sy, n // (sx * sy)
        for s in range(27):
            a, b, c = i + s % 3 - 1, j + (s // 3) % 3 - 1, k + s // 9 - 1
            if 0 <= a <= P.nx and 0 <= b <= P.ny and 0 <= c <= P.nz:
                m = a + sx * (b + sy * c)
                A[2 * n:2 * n + 2, 2 * m:2 * m + 2] = B[n, s].reshape(2, 2)
    return A


def _lu_dense(P, F):
    """Dense L (unit block diagonal) and U from the factor storage."""
    rank = O.mc_rank(P)
    FD = _blocks_to_dense(P, F)
    L = np.eye(2 * P.N)
    U = np.zeros_like(FD)
    for n in range(P.N):
        for m in range(P.N):
            blk = FD[2 * n:2 * n + 2, 2 * m:2 * m + 2]
            if rank[m] < rank[n]:
                L[2 * n:2 * n + 2, 2 * m:2 * m + 2] = blk
            else:
                U[2 * n:2 * n + 2, 2 * m:2 * m + 2] = blk
    return L, U


def _pattern(P):
    """Block pattern of the 27-point stencil as a dense boolean (2N x 2N)."""
    ones = np.zeros((P.N, 27, 4))
    rp, ci, _ = O.jacobian_csr(P, np.full(P.C, 0.1), np.full(P.C, 1e-12),
                               *O.initial_state(P), DT)
    ones = O.csr_to_blocks(P, rp, ci, np.ones(ci.size))
    return _blocks_to_dense(P, ones) != 0


def test_colour_classes_are_independent_sets():
    P = O.Problem(8, 8, 4)
    rank = O.mc_rank(P)
    assert sorted(rank) == list(range(P.N))
    sx, sy = P.nx + 1, P.ny + 1
    ijk = [(n % sx, (n // sx) % sy, n // (sx * sy)) for n in range(P.N)]
    colour = np.array([(i & 1) + 2 * (j & 1) + 4 * (k & 1) for i, j, k in ijk])
    # ranks ascend with the colour, then with the node index
    order = np.argsort(rank)
    assert np.all(np.diff(colour[order]) >= 0)
    for col in range(8):
        nodes = order[colour[order] == col]
        assert np.all(np.diff(nodes) > 0)
        pts = np.array([ijk[n] for n in nodes])
        d = np.abs(pts[:, None, :] - pts[None, :, :]).max(axis=2)
        np.fill_diagonal(d, 9)
        assert d.min() >= 2      # no two nodes of one colour share a cell


def test_ilu0_reproduces_A_on_its_pattern(case):
    P, phi, K, p, c = case
    A, _ = _interior_dense(P, phi, K, p, c)
    rp, ci, val = O.jacobian_csr(P, phi, K, p, c, DT)
    B = O.csr_to_blocks(P, rp, ci, val)
    assert np.array_equal(_blocks_to_dense(P, B), O.jacobian_dense(P, phi, K, p, c, DT))
    Bi = _dense_to_blocks(P, A)
    L, U = _lu_dense(P, O.mcilu_factor(P, Bi, 0.0))
    R = L @ U - A
    pat = _pattern(P)
    scale = np.abs(A).max(axis=1, keepdims=True)
    assert np.abs(R[pat] / np.broadcast_to(scale, R.shape)[pat]).max() < 1e-13
    # the factorisation is incomplete: fill outside the pattern is dropped
    assert np.abs(R[~pat]).max() > 1e-6 * np.abs(A).max()


def _dense_to_blocks(P, A):
    B = np.zeros((P.N, 27, 4))
    sx, sy = P.nx + 1, P.ny + 1
    for n in range(P.N):
        i, j, k = n % sx, (n // sx) % sy, n // (sx * sy)
        for s in range(27):
            a, b, c = i + s % 3 - 1, j + (s // 3) % 3 - 1, k + s // 9 - 1
            if 0 <= a <= P.nx and 0 <= b <= P.ny and 0 <= c <= P.nz:
                m = a + sx * (b + sy * c)
                B[n, s] = A[2 * n:2 * n + 2, 2 * m:2 * m + 2].ravel()
    return B


def test_modified_ilu_keeps_block_row_sums(case):
    P, phi, K, p, c = case
    A, _ = _interior_dense(P, phi, K, p, c)
    L, U = _lu_dense(P, O.mcilu_factor(P, _dense_to_blocks(P, A), 1.0))
    LU = L @ U
    # block row sums: sum over the block columns of each 2x2 row block
    rs = lambda M: M.reshape(2 * P.N, P.N, 2).sum(axis=1)
    scale = np.abs(A).sum(axis=1, keepdims=True)
    assert np.abs((rs(LU) - rs(A)) / scale).max() < 1e-13
    # beta = 1 differs from beta = 0 (fill was dropped and lumped)
    L0, U0 = _lu_dense(P, O.mcilu_factor(P, _dense_to_blocks(P, A), 0.0))
    assert np.abs(L0 @ U0 - LU).max() > 1e-6 * np.abs(A).max()


@pytest.mark.parametrize("beta", [0.0, 0.5])
def test_triangular_solves_equal_dense_solves(case, beta):
    P, phi, K, p, c = case
    A, _ = _interior_dense(P, phi, K, p, c)
    F = O.mcilu_factor(P, _dense_to_blocks(P, A), beta)
    L, U = _lu_dense(P, F)
    r = np.random.default_rng(1).standard_normal(2 * P.N)
    z = O.mcilu_solve(P, F, r)
    assert np.allclose(z, np.linalg.solve(L @ U, r), rtol=1e-11, atol=1e-11 * np.abs(z).max())
    zt = O.mcilu_solve(P, F, r, transpose=True)
    assert np.allclose(zt, np.linalg.solve((L @ U).T, r), rtol=1e-11,
                       atol=1e-11 * np.abs(zt).max())


def test_ilu0_of_the_transpose_is_the_transpose(case):
    P, phi, K, p, c = case
    A, _ = _interior_dense(P, phi, K, p, c)
    L, U = _lu_dense(P, O.mcilu_factor(P, _dense_to_blocks(P, A), 0.0))
    Lt, Ut = _lu_dense(P, O.mcilu_factor(P, _dense_to_blocks(P, A.T), 0.0))
    d = Lt @ Ut - (L @ U).T
    assert np.abs(d).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("transpose", [False, True])
def test_smoother_kinds_equal_dense_linear_algebra(case, transpose):
    P, phi, K, p, c = case
    A, dm = _interior_dense(P, phi, K, p, c)
    At = A.T if transpose else A
    r = np.random.default_rng(2).standard_normal(2 * P.N)
    ri = np.where(dm, 0.0, r)
    tol = lambda z: dict(rtol=1e-10, atol=1e-10 * np.abs(z).max())
    # kind 0: the 2x2 block diagonal
    D = np.zeros_like(At)
    for n in range(P.N):
        D[2 * n:2 * n + 2, 2 * n:2 * n + 2] = At[2 * n:2 * n + 2, 2 * n:2 * n + 2]
    z0 = O.smoother_apply(P, phi, K, p, c, DT, 0, r, transpose=transpose)
    ref = np.where(dm, 0.0, np.linalg.solve(D, ri))
    assert np.allclose(z0, ref, **tol(ref))
    # kind 1: the blocks of vertical neighbours (same i, j) and the diagonal
    sz = (P.nx + 1) * (P.ny + 1)
    T = np.zeros_like(At)
    for n in range(P.N):
        for m in (n - sz, n, n + sz):
            if 0 <= m < P.N:
                T[2 * n:2 * n + 2, 2 * m:2 * m + 2] = At[2 * n:2 * n + 2, 2 * m:2 * m + 2]
    z1 = O.smoother_apply(P, phi, K, p, c, DT, 1, r, transpose=transpose)
    ref = np.where(dm, 0.0, np.linalg.solve(T, ri))
    assert np.allclose(z1, ref, **tol(ref))
    # kind 2: L U of the untransposed matrix's factors, transposed for the
    # transposed solve (beta = 1 is left out here: the pressure rows of A sum
    # to about 0 (the Darcy fluxes depend on pressure differences), so the
    # modified factorisation's pivots are nearly singular and a dense solve
    # with L U is not an accurate reference)
    for beta in (0.0, 0.5):
        L, U = _lu_dense(P, O.mcilu_factor(P, _dense_to_blocks(P, A), beta))
        LU = L @ U
        z2 = O.smoother_apply(P, phi, K, p, c, DT, 2, r, beta=beta, transpose=transpose)
        ref = np.where(dm, 0.0, np.linalg.solve(LU.T if transpose else LU, ri))
        assert np.allclose(z2, ref, **tol(ref))


def test_newton_with_the_ilu_smoother_reaches_the_same_state():
    """16x16x4 (above the dense-solve size): the converged step does not
    depend on the multigrid smoother."""
    P = O.Problem(16, 16, 4)
    phi = np.full(P.C, 0.1)
    K = np.full(P.C, 4.845e-13)
    p, c = O.initial_state(P)
    out = {}
    # (beta = 1 is not a usable smoother here: its pivots are nearly singular,
    # see test_smoother_kinds_equal_dense_linear_algebra)
    for sm, beta in ((1, 0.0), (2, 0.0), (2, 0.5)):
        opts = O.NewtonOpts(smoother=sm, ilu_beta=beta, dense_max=0, lin_rtol=1e-11)
        p1, c1, info = O.newton_step(P, phi, K, p, c, DT, opts)
        assert info["status"] == 0 and info["lin_iters"] > 0
        out[(sm, beta)] = (p1, c1, info["lin_iters"])
    pr, cr, _ = out[(1, 0.0)]
    for key in ((2, 0.0), (2, 0.5)):
        p1, c1, _ = out[key]
        assert np.abs(c1 - cr).max() < 1e-10
        assert np.abs(p1 - pr).max() < 1e-10 * np.abs(pr).max()
