"""S by the addition theorem (FLAPW_S_LEGENDRE) against the oracle's S, which
sums Eq. (def_overlap) term by term; H still comes from the contraction."""
import numpy as np
import pytest

import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs

from helpers import (TOL_EMU, TOL_F64, columns_from_lower, herm_relerr, lower_to_full,
                     oracle_hs, run_hs, torch_cuda)
import oracle

pytestmark = pytest.mark.gpu

TOL_LEG = 1e-13   # FP64 Legendre sums


@pytest.fixture(scope="module", autouse=True)
def _built():
    fl.build()
    assert torch_cuda().cuda.is_available()


@pytest.mark.parametrize("precision,tol", [(fl.PREC_FP64, TOL_F64), (fl.PREC_EMU, TOL_EMU)])
@pytest.mark.parametrize("layout", [fl.LAYOUT_LOWER_FULL, fl.LAYOUT_LOWER_PACKED])
def test_config1_full(precision, tol, layout):
    p = inputs.config1()
    h, Hs, Ss, _ = run_hs(p, precision, layout=layout, operands=fl.OPERANDS_FACTORED,
                          s_method=fl.S_LEGENDRE)
    Ho, So = oracle_hs(p)
    ng = Ho.shape[0]
    assert herm_relerr(lower_to_full(Ss[0], ng, layout), So) <= TOL_LEG
    assert herm_relerr(lower_to_full(Hs[0], ng, layout), Ho) <= tol
    st = h.stats()
    assert st["ms_s"] > 0 and st["ms_s"] <= st["ms_contract"]


@pytest.mark.parametrize("lmax,n_atoms,n_types,n_target", [(3, 3, 2, (333, 190)), (12, 3, 2, (230,)),
                                                           (0, 1, 1, (20,)), (6, 40, 2, (410,))])
def test_small_multi_k(lmax, n_atoms, n_types, n_target):
    # ragged sizes, several k-points, more than one 16-atom chunk per type,
    # slots different from types
    p = inputs.small(41 + lmax, n_atoms=n_atoms, n_types=n_types, lmax=lmax, n_target=n_target)
    p.atom_slot = (np.arange(n_atoms) % p.n_slots).astype(np.int32)[::-1].copy()
    h, Hs, Ss, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, s_method=fl.S_LEGENDRE)
    for k in range(p.n_k):
        Ho, So = oracle_hs(p, k)
        ng = Ho.shape[0]
        assert herm_relerr(lower_to_full(Ss[k], ng, 0), So) <= TOL_LEG, k
        assert herm_relerr(lower_to_full(Hs[k], ng, 0), Ho) <= TOL_EMU, k


def test_config2_sampled_columns():
    p = inputs.config2()
    h, Hs, Ss, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, s_method=fl.S_LEGENDRE)
    n3 = h.gvectors(0)
    ng = len(n3)
    cols = np.array([0, 1, 777, 2000, ng - 1])
    Ho, So = oracle.hs_columns(p, 0, n3, cols)
    Sg = columns_from_lower(Ss[0], ng, 0, cols)
    Hg = columns_from_lower(Hs[0], ng, 0, cols)
    assert np.linalg.norm(Sg - So) / np.linalg.norm(So) <= TOL_LEG
    assert np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho) <= TOL_EMU


@pytest.mark.parametrize("lmax,hpd", [(8, False), (8, True), (12, False), (2, False)])
def test_cluster_factorisation_matches_single_cta(lmax, hpd):
    # with S by the addition theorem each T slot is factorised by a cluster of
    # CTAs; the pivot decisions and every element's arithmetic are those of
    # the one-CTA kernel, so the factors agree (to the compiler's choice of
    # fused multiply-adds; a different pivot sequence would differ at O(1))
    p = inputs.small(95 + lmax, n_atoms=3, n_types=3, lmax=lmax, n_target=(120,), hpd=hpd)
    h1, _, _, _ = run_hs(p, fl.PREC_FP64, operands=fl.OPERANDS_FACTORED)
    f1 = [h1.factor(s) for s in range(p.n_slots)]
    h8, _, _, _ = run_hs(p, fl.PREC_FP64, operands=fl.OPERANDS_FACTORED, s_method=fl.S_LEGENDRE)
    for slot in range(p.n_slots):
        CH, npos, nneg = h8.factor(slot)
        assert (npos, nneg) == f1[slot][1:]
        assert np.abs(CH - f1[slot][0]).max() <= 1e-13 * np.abs(f1[slot][0]).max()
        n = CH.shape[0]
        sig = np.concatenate([np.ones(npos), -np.ones(nneg), np.zeros(n - npos - nneg)])
        R = CH.conj().T @ (sig[:, None] * CH)
        assert np.linalg.norm(R - p.T[slot]) <= 1e-13 * np.linalg.norm(p.T[slot])
    assert h8.stats()["n_pivot2"] == h1.stats()["n_pivot2"]


def test_zero_pivots_dropped_in_both_factorisations():
    # T with two zero rows and columns: the elimination meets zero columns
    # (zero pivots, rows dropped from the operand) in the one-CTA and the
    # cluster factorisation alike; H still equals the oracle's
    p = inputs.small(93, n_atoms=3, n_types=2, lmax=8, n_target=(140,))
    T = p.T.copy()
    for slot in range(p.n_slots):
        for i in (5, 97):
            T[slot][i, :] = 0
            T[slot][:, i] = 0
    p.T = T
    h1, H1, _, _ = run_hs(p, fl.PREC_FP64, operands=fl.OPERANDS_FACTORED)
    h8, H8, _, _ = run_hs(p, fl.PREC_FP64, operands=fl.OPERANDS_FACTORED, s_method=fl.S_LEGENDRE)
    n = 2 * p.n_L
    for slot in range(p.n_slots):
        CH1, np1, nn1 = h1.factor(slot)
        CH8, np8, nn8 = h8.factor(slot)
        assert (np8, nn8) == (np1, nn1) and np1 + nn1 == n - 2
        assert np.abs(CH8 - CH1).max() <= 1e-13 * np.abs(CH1).max()
    Ho, _ = oracle_hs(p)
    ng = Ho.shape[0]
    for H in (H1, H8):
        assert herm_relerr(lower_to_full(H[0], ng, 0), Ho) <= TOL_F64


def test_requires_factored_operands():
    p = inputs.config1()
    bad = fl.default_options(operands=fl.OPERANDS_FROM_AB, s_method=fl.S_LEGENDRE)
    with pytest.raises(fl.FlapwError) as e:
        fl.from_problem(p, bad)
    assert e.value.code == -1
