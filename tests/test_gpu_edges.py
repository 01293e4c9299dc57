"""Parity with the CPU oracle on the method's degenerate inputs (CUDA path,
through the C ABI): the Gamma point, whose G = 0 plane wave has K = 0, and
k-points whose ball |k+G| <= K_max holds one or two plane waves."""
import numpy as np
import pytest

import oracle
import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs

from helpers import TOL_EMU, TOL_F64, ab_block, herm_relerr, lower_to_full, oracle_hs, run_hs, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fl.build()
    torch = torch_cuda()
    assert torch.cuda.is_available()


METHODS = {
    "from_ab": dict(operands=fl.OPERANDS_FROM_AB),
    "factored": dict(operands=fl.OPERANDS_FACTORED),
    "s_legendre": dict(operands=fl.OPERANDS_FACTORED, s_method=fl.S_LEGENDRE),
    "h_alg3": dict(operands=fl.OPERANDS_FACTORED, h_method=fl.H_ALG3),
}


@pytest.mark.parametrize("precision,tol", [(fl.PREC_FP64, TOL_F64), (fl.PREC_EMU, TOL_EMU)])
@pytest.mark.parametrize("method", list(METHODS))
def test_gamma_point(precision, tol, method):
    """k = 0: the first plane wave is G = 0 with K = 0 (K_hat taken as z;
    only l = 0 is non-zero there)."""
    p = inputs.small(29, n_atoms=3, n_types=2, lmax=4, n_target=(250,))
    p.k_frac = np.zeros_like(p.k_frac)
    h, Hs, Ss, (A, B) = run_hs(p, precision, **METHODS[method])
    assert np.array_equal(h.gvectors(0)[0], [0, 0, 0])
    Ho, So = oracle_hs(p)
    ng = Ho.shape[0]
    assert herm_relerr(lower_to_full(Hs[0], ng, 0), Ho) <= tol
    assert herm_relerr(lower_to_full(Ss[0], ng, 0), So) <= tol
    if method == "from_ab":
        # the G = 0 column of A and B: zero for l >= 1, the oracle's for l = 0
        Ao, Bo = oracle.build_ab(p, 0, h.gvectors(0), [0])
        a = ab_block(p, h, A, 0)[:, :, 0]
        b = ab_block(p, h, B, 0)[:, :, 0]
        assert np.all(a[:, 1:] == 0) and np.all(b[:, 1:] == 0)
        assert np.abs(a - Ao[:, :, 0]).max() <= 1e-13 * np.abs(Ao).max()
        assert np.abs(b - Bo[:, :, 0]).max() <= 1e-13 * np.abs(Bo).max()


@pytest.mark.parametrize("precision,tol", [(fl.PREC_FP64, TOL_F64), (fl.PREC_EMU, TOL_EMU)])
@pytest.mark.parametrize("layout", [fl.LAYOUT_LOWER_FULL, fl.LAYOUT_LOWER_PACKED])
@pytest.mark.parametrize("n_g", [1, 2])
def test_one_or_two_plane_waves(precision, tol, layout, n_g):
    """The smallest problems: every tile is almost all padding."""
    p = inputs.small(40, n_atoms=2, n_types=2, lmax=3, n_target=(n_g,))
    h, Hs, Ss, _ = run_hs(p, precision, layout=layout, operands=fl.OPERANDS_FACTORED)
    assert h.num_g(0) == n_g
    Ho, So = oracle_hs(p)
    assert herm_relerr(lower_to_full(Hs[0], n_g, layout), Ho) <= tol
    assert herm_relerr(lower_to_full(Ss[0], n_g, layout), So) <= tol
