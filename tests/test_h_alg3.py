"""H by the paper's Alg. 3 operation sequence (FLAPW_H_ALG3, Sec. 5.1): the
zhemm/zgemm operand steps X_a = T^BA A_a + T^BB B_a / 2, Y_a = T^AA A_a and
the zher2k + zherkx contraction H = X^H B + B^H X + A^H Y, evaluated as one
lower-triangle contraction L^H R with L_a = [X_a; B_a; A_a] and
R_a = [B_a; X_a; Y_a].  Compared with the oracle's H, which sums
Eq. (def_hamilton) term by term."""
import numpy as np
import pytest

import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs

from helpers import (TOL_EMU, TOL_F64, columns_from_lower, herm_relerr, lower_to_full,
                     oracle_hs, run_hs, torch_cuda)
import oracle


def test_stacked_operands_reproduce_h():
    """The L/R stacking the operand kernels write gives H (host, numpy)."""
    p = inputs.small(52, n_atoms=3, n_types=2, lmax=3, n_target=(120,))
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    A, B = oracle.build_ab(p, 0, n3)
    nl = p.n_L
    Ls, Rs = [], []
    for a in range(p.n_atoms):
        T = p.T[p.atom_slot[a]]
        X = T[nl:, :nl] @ A[a] + 0.5 * T[nl:, nl:] @ B[a]
        Y = T[:nl, :nl] @ A[a]
        Ls.append(np.vstack([X, B[a], A[a]]))
        Rs.append(np.vstack([B[a], X, Y]))
    L, R = np.vstack(Ls), np.vstack(Rs)
    assert L.shape[0] == 3 * p.n_atoms * nl
    H = L.conj().T @ R
    Ho, _ = oracle.hs_full(p, 0, n3)
    assert np.linalg.norm(H - Ho) / np.linalg.norm(Ho) < 1e-13


gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def _built():
    fl.build()
    assert torch_cuda().cuda.is_available()


@gpu
@pytest.mark.parametrize("precision,tol", [(fl.PREC_FP64, TOL_F64), (fl.PREC_EMU, TOL_EMU)])
@pytest.mark.parametrize("layout", [fl.LAYOUT_LOWER_FULL, fl.LAYOUT_LOWER_PACKED])
@pytest.mark.parametrize("operands", [fl.OPERANDS_FROM_AB, fl.OPERANDS_FACTORED])
def test_config1(_built, precision, tol, layout, operands):
    p = inputs.config1()
    h, Hs, Ss, _ = run_hs(p, precision, layout=layout, operands=operands, h_method=fl.H_ALG3)
    Ho, So = oracle_hs(p)
    ng = Ho.shape[0]
    assert herm_relerr(lower_to_full(Hs[0], ng, layout), Ho) <= tol
    assert herm_relerr(lower_to_full(Ss[0], ng, layout), So) <= tol
    st = h.stats()
    assert st["k_total"] == 3 * p.n_atoms * p.n_L
    assert st["n_pos"] == st["k_total"] and st["n_neg"] == 0 and st["n_pivot2"] == 0
    with pytest.raises(fl.FlapwError) as e:
        h.factor(0)
    assert e.value.code == -6


@gpu
@pytest.mark.parametrize("lmax,n_atoms,n_types,n_target", [(3, 3, 2, (333, 190)), (12, 3, 2, (230,)),
                                                           (0, 1, 1, (20,)), (6, 40, 2, (410,))])
def test_small_multi_k(_built, lmax, n_atoms, n_types, n_target):
    # ragged sizes, several k-points, slots different from types; 40 atoms of
    # lmax 6 give K = 5880 (92 K chunks, more than one unit)
    p = inputs.small(61 + lmax, n_atoms=n_atoms, n_types=n_types, lmax=lmax, n_target=n_target)
    p.atom_slot = (np.arange(n_atoms) % p.n_slots).astype(np.int32)[::-1].copy()
    for precision, tol in [(fl.PREC_EMU, TOL_EMU), (fl.PREC_FP64, TOL_F64)]:
        h, Hs, Ss, _ = run_hs(p, precision, operands=fl.OPERANDS_FACTORED, h_method=fl.H_ALG3)
        for k in range(p.n_k):
            Ho, So = oracle_hs(p, k)
            ng = Ho.shape[0]
            assert herm_relerr(lower_to_full(Hs[k], ng, 0), Ho) <= tol, (precision, k)
            assert herm_relerr(lower_to_full(Ss[k], ng, 0), So) <= tol, (precision, k)


@gpu
def test_hpd_t_and_legendre_s(_built):
    # T scaled to be positive definite (the paper's "in theory" case), with S
    # by the addition theorem beside the Alg. 3 H
    p = inputs.small(77, n_atoms=5, n_types=2, lmax=5, n_target=(700,), hpd=True)
    h, Hs, Ss, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, h_method=fl.H_ALG3,
                          s_method=fl.S_LEGENDRE)
    Ho, So = oracle_hs(p)
    ng = Ho.shape[0]
    assert herm_relerr(lower_to_full(Hs[0], ng, 0), Ho) <= TOL_EMU
    assert herm_relerr(lower_to_full(Ss[0], ng, 0), So) <= 1e-13


@gpu
def test_config2_sampled_columns_and_factored_agreement(_built):
    p = inputs.config2()
    h, Hs, Ss, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, h_method=fl.H_ALG3)
    n3 = h.gvectors(0)
    ng = len(n3)
    cols = np.array([0, 1, 777, 2000, ng - 1])
    Ho, So = oracle.hs_columns(p, 0, n3, cols)
    Hg = columns_from_lower(Hs[0], ng, 0, cols)
    Sg = columns_from_lower(Ss[0], ng, 0, cols)
    assert np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho) <= TOL_EMU
    assert np.linalg.norm(Sg - So) / np.linalg.norm(So) <= TOL_EMU
    # the same H through the factorised single-operand form, on the same handle
    _, Hf, _, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, h=h)
    a = lower_to_full(Hs[0], ng, 0)
    b = lower_to_full(Hf[0], ng, 0)
    assert herm_relerr(a, b) <= 2 * TOL_EMU


@gpu
def test_rejects_unknown_h_method(_built):
    p = inputs.config1()
    with pytest.raises(fl.FlapwError) as e:
        fl.from_problem(p, fl.default_options(h_method=2))
    assert e.value.code == -1
