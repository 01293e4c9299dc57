"""H by the paper's Alg. 1 (FLAPW_H_ALG1, Sec. 3): H_AB+BA+BB by the zher2k of
Z_a = T^BA A_a + T^BB B_a / 2 with B_a, and H_AA per atom by the Cholesky
factorisation T^AA = C C^H where it succeeds ((C^H A_a)^H (C^H A_a), the
paper's ztrmm + zherk) and by A_a^H (T^AA A_a) where it fails (zhemm +
zgemm).  Evaluated on the stacked contraction of Alg. 3 with the third block
of L_a and R_a both C^H A_a, or A_a and T^AA A_a.  Compared with the
oracle's H of Eq. (def_hamilton), with T blocks whose T^AA factorises, fails
at its first pivot, or fails at its last one."""
import numpy as np
import pytest

import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs

from helpers import (TOL_EMU, TOL_F64, columns_from_lower, herm_relerr, lower_to_full,
                     oracle_hs, run_hs, torch_cuda)
import oracle


def _mixed_T(p, fail_at):
    """Slot 0 keeps the recipe's T (T^AA positive definite at l_max <= 4);
    slot 1's T^AA gets a negative pivot: the whole diagonal shifted by -3
    ("first") or only its last entry by -40 ("last")."""
    nl = p.n_L
    T = p.T.copy()
    if fail_at == "first":
        T[1, np.arange(nl), np.arange(nl)] -= 3.0
    else:
        T[1, nl - 1, nl - 1] -= 40.0
    return T


def test_alg1_stacking_reproduces_h():
    """The L/R stacking of Alg. 1, with numpy's Cholesky deciding per slot,
    gives the oracle's H (host)."""
    p = inputs.small(71, n_atoms=3, n_types=2, lmax=3, n_target=(130,))
    p.T = _mixed_T(p, "last")
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    A, B = oracle.build_ab(p, 0, n3)
    nl = p.n_L
    Ls, Rs, ok = [], [], []
    for a in range(p.n_atoms):
        T = p.T[p.atom_slot[a]]
        Taa = np.tril(T[:nl, :nl]) + np.tril(T[:nl, :nl], -1).conj().T
        X = T[nl:, :nl] @ A[a] + 0.5 * T[nl:, nl:] @ B[a]
        try:
            C = np.linalg.cholesky(Taa)
            Y = C.conj().T @ A[a]
            Ls.append(np.vstack([X, B[a], Y]))
            Rs.append(np.vstack([B[a], X, Y]))
            ok.append(True)
        except np.linalg.LinAlgError:
            Ls.append(np.vstack([X, B[a], A[a]]))
            Rs.append(np.vstack([B[a], X, Taa @ A[a]]))
            ok.append(False)
    assert any(ok) and not all(ok)
    H = np.vstack(Ls).conj().T @ np.vstack(Rs)
    Ho, _ = oracle.hs_full(p, 0, n3)
    assert np.linalg.norm(H - Ho) / np.linalg.norm(Ho) < 1e-13


gpu = pytest.mark.gpu


@gpu
@pytest.mark.parametrize("precision,tol", [(fl.PREC_FP64, TOL_F64), (fl.PREC_EMU, TOL_EMU)])
@pytest.mark.parametrize("operands", [fl.OPERANDS_FROM_AB, fl.OPERANDS_FACTORED])
def test_config1_every_slot_factorises(precision, tol, operands):
    torch_cuda()
    p = inputs.config1()
    h, Hs, Ss, _ = run_hs(p, precision, operands=operands, h_method=fl.H_ALG1)
    Ho, So = oracle_hs(p)
    ng = Ho.shape[0]
    assert herm_relerr(lower_to_full(Hs[0], ng, 0), Ho) <= tol
    assert herm_relerr(lower_to_full(Ss[0], ng, 0), So) <= tol
    st = h.stats()
    assert st["n_chol"] == p.T.shape[0]
    assert st["k_total"] == 3 * p.n_atoms * p.n_L


@gpu
@pytest.mark.parametrize("fail_at", ["first", "last"])
@pytest.mark.parametrize("layout", [fl.LAYOUT_LOWER_FULL, fl.LAYOUT_LOWER_PACKED])
def test_mixed_slots(fail_at, layout):
    # slot 0 factorises, slot 1 does not; ragged k-points, slots != types
    torch_cuda()
    p = inputs.small(73, n_atoms=4, n_types=2, lmax=4, n_target=(310, 170))
    p.T = _mixed_T(p, fail_at)
    p.atom_slot = np.array([1, 0, 0, 1], dtype=np.int32)
    for precision, tol in [(fl.PREC_EMU, TOL_EMU), (fl.PREC_FP64, TOL_F64)]:
        for operands in (fl.OPERANDS_FACTORED, fl.OPERANDS_FROM_AB):
            h, Hs, Ss, _ = run_hs(p, precision, layout=layout, operands=operands, h_method=fl.H_ALG1)
            assert h.stats()["n_chol"] == 1
            for k in range(p.n_k):
                Ho, So = oracle_hs(p, k)
                ng = Ho.shape[0]
                assert herm_relerr(lower_to_full(Hs[k], ng, layout), Ho) <= tol, (precision, operands, k)
                assert herm_relerr(lower_to_full(Ss[k], ng, layout), So) <= tol


@gpu
def test_config2_sampled_and_against_alg3():
    torch_cuda()
    p = inputs.config2()
    h1, H1, S1, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, h_method=fl.H_ALG1)
    n_chol = h1.stats()["n_chol"]
    assert 0 <= n_chol <= p.T.shape[0]
    n3 = h1.gvectors(0)
    ng = len(n3)
    cols = [0, 1, 64, 1999, ng - 1]
    Ho, _ = oracle.hs_columns(p, 0, n3, cols)
    eh = np.linalg.norm(columns_from_lower(H1[0], ng, 0, cols) - Ho) / np.linalg.norm(Ho)
    assert eh <= TOL_EMU, eh
    h3, H3, _, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, h_method=fl.H_ALG3)
    d = np.linalg.norm(columns_from_lower(H1[0], ng, 0, cols) - columns_from_lower(H3[0], ng, 0, cols))
    assert d / np.linalg.norm(Ho) <= 2 * TOL_EMU
