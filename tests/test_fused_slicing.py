"""The default emulated path forms the S and H operand rows from the
type-level operands and slices them in one pass each (no FP64 operand).
Every slice count 4..8 against the oracle, with sigma = -1 rows and
slots different from types.  The error of the split-precision product
falls by about 2^7 per slice (measured 4.9e-12 at s = 6 and 3.9e-14 at s = 7
on config 2); the bound here is 20x that rate, with an FP64 floor."""
import numpy as np
import pytest

import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs

from helpers import herm_relerr, lower_to_full, oracle_hs, run_hs, torch_cuda

pytestmark = pytest.mark.gpu


def tol(s):
    return max(20 * 4e-14 * 128.0 ** (7 - s), 1e-13)


@pytest.fixture(scope="module", autouse=True)
def _built():
    fl.build()
    assert torch_cuda().cuda.is_available()


@pytest.mark.parametrize("n_slices", [4, 5, 6, 8])
def test_every_slice_count(n_slices):
    # l_max 8: the literal T (I + 0.1 random Hermitian, 162 x 162) is indefinite
    p = inputs.small(91, n_atoms=3, n_types=2, lmax=8, n_target=(330, 97))
    p.atom_slot = (np.arange(p.n_atoms) % p.n_slots).astype(np.int32)[::-1].copy()
    h, Hs, Ss, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, n_slices=n_slices)
    assert h.stats()["n_neg"] > 0          # the literal T is indefinite
    for k in range(p.n_k):
        Ho, So = oracle_hs(p, k)
        ng = Ho.shape[0]
        eh = herm_relerr(lower_to_full(Hs[k], ng, 0), Ho)
        es = herm_relerr(lower_to_full(Ss[k], ng, 0), So)
        assert eh <= tol(n_slices) and es <= tol(n_slices), (n_slices, k, eh, es)


def test_fused_and_fp64_operand_paths_agree():
    # the same problem through the FP64 operands and the slicer (A/B operands)
    p = inputs.small(92, n_atoms=4, n_types=2, lmax=5, n_target=(610,))
    h, Hf, Sf, AB = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED)
    _, Ha, Sa, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FROM_AB, h=h, AB=AB)
    ng = h.num_g(0)
    Ho, So = oracle_hs(p)
    for X, Y, R in ((Hf[0], Ha[0], Ho), (Sf[0], Sa[0], So)):
        a, b = lower_to_full(X, ng, 0), lower_to_full(Y, ng, 0)
        assert herm_relerr(a, b) <= 2e-13
        assert herm_relerr(a, R) <= 1e-12
