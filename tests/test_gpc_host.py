"""Host-side gPC entry points of the C ABI (no GPU needed): the
Gauss-Legendre rule and the multi-index sets against the oracle."""
import numpy as np
import pytest

from oracle import gpc as G


@pytest.fixture(scope="module")
def E():
    from paper_1906_01632_gb300 import elder
    return elder


@pytest.mark.parametrize("q", [1, 2, 3, 5, 9, 17, 40, 64])
def test_gauss_legendre_matches_library_rule(E, q):
    x, w = E.elder_gauss_legendre(q)
    xr, wr = G.gauss_legendre(q)
    assert np.abs(x - xr).max() < 2e-15 and np.abs(w - wr).max() < 5e-15
    assert abs(w.sum() - 2.0) < 1e-14


@pytest.mark.parametrize("rule", ["total", "tensor", "hyperbolic"])
@pytest.mark.parametrize("M,p", [(1, 6), (2, 4), (3, 4), (3, 5), (4, 3)])
def test_multi_indices_match_oracle(E, rule, M, p):
    assert np.array_equal(E.elder_gpc_indices(M, p, rule), G.multi_indices(M, p, rule))


def test_total_degree_4_basis_in_3_variables_is_in_canonical_order(E):
    """The tensor-core count builds the total-degree-4 basis in 3 variables
    from Legendre values in registers when the index set comes in this order
    (total degree, then the first variable's degree, then the second's);
    any other order takes the shared-memory table.  The library's index set
    for (3, 4) must keep this order, so that the bench's surrogate takes the
    register builder."""
    want = [(a, b, s - a - b) for s in range(5) for a in range(s + 1) for b in range(s - a + 1)]
    got = [tuple(int(v) for v in row) for row in E.elder_gpc_indices(3, 4)]
    assert got == want


def test_gpc_argument_errors(E):
    with pytest.raises(E.ElderError):
        E.elder_gauss_legendre(0)
    with pytest.raises(E.ElderError):
        E.elder_gpc_indices(9, 2)
