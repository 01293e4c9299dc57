"""The generalised eigenproblem H c = lambda S c of Sec. 2 (flapw_eigh) on
matrices the library built, against scipy's generalised Hermitian solver on
the same matrices and on the oracle's H and S of Eqs. (def_hamilton) and
(def_overlap), plus the residual and the S-orthonormality of the vectors.
The muffin-tin S alone is positive definite only where 2 N_A N_L >= N_G:
the small cell below has K = 288 for N_G 148 (S's condition number about
1.5e5); config 1 (K 100 < N_G 298) must be refused with FLAPW_ERR_FACTOR."""
import numpy as np
import pytest
import scipy.linalg as sl

import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs

from helpers import alloc_out, lower_to_full, oracle_hs, run_ab, torch_cuda

pytestmark = pytest.mark.gpu


def _built(precision):
    p = inputs.small(62, n_atoms=4, n_types=2, lmax=5, n_target=(150,))
    h = fl.from_problem(p, fl.default_options(precision=precision, operands=fl.OPERANDS_FACTORED))
    _, A, B = run_ab(p, h)
    ng = h.num_g(0)
    H, S = alloc_out(ng, 0), alloc_out(ng, 0)
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
    h.sync()
    return p, h, ng, H, S


@pytest.mark.parametrize("precision", [fl.PREC_EMU, fl.PREC_FP64])
def test_eigh_matches_scipy_and_the_oracle(precision):
    torch = torch_cuda()
    p, h, ng, H, S = _built(precision)
    Hf, Sf = lower_to_full(H, ng, 0), lower_to_full(S, ng, 0)
    assert np.linalg.eigvalsh(Sf).min() > 0
    w = h.eigh(ng, H, ng, S, ng)
    C = H.cpu().numpy().reshape(ng, ng).T          # column j: eigenvector j
    L = np.tril(S.cpu().numpy().reshape(ng, ng).T)
    scale = np.abs(w).max()
    # the same matrices in scipy (LAPACK zhegvd): eigenvalues within the
    # solvers' rounding times the condition of S
    wr = sl.eigh(Hf, Sf, eigvals_only=True)
    assert np.all(np.diff(w) >= 0)
    assert np.abs(w - wr).max() <= 1e-9 * scale, np.abs(w - wr).max() / scale
    # the oracle's H and S: within the build's error (<= 1e-12 relative) times cond(S)
    Ho, So = oracle_hs(p, 0)
    wo = sl.eigh(Ho, So, eigvals_only=True)
    assert np.abs(w - wo).max() <= 1e-7 * scale, np.abs(w - wo).max() / scale
    # residual, S-orthonormal vectors, and S = L L^H
    R = Hf @ C - Sf @ C * w[None, :]
    den = np.linalg.norm(Hf) * np.linalg.norm(C) + np.linalg.norm(Sf) * np.linalg.norm(C) * scale
    assert np.linalg.norm(R) <= 1e-11 * den, np.linalg.norm(R) / den
    assert np.abs(C.conj().T @ Sf @ C - np.eye(ng)).max() <= 1e-9
    assert np.abs(L @ L.conj().T - Sf).max() <= 1e-12 * np.abs(Sf).max()
    # eigenvalues only: the same values
    H2, S2 = torch.tensor(Hf.T.reshape(-1).copy(), device="cuda"), torch.tensor(Sf.T.reshape(-1).copy(), device="cuda")
    w2 = h.eigh(ng, H2, ng, S2, ng, vectors=False)
    assert np.abs(w2 - w).max() <= 1e-9 * scale
    h.destroy()


def test_eigh_refuses_an_indefinite_S():
    # config 1: K = 2 N_A N_L = 100 < N_G = 298, S has rank 100
    p = inputs.config1()
    h = fl.from_problem(p, fl.default_options(precision=fl.PREC_FP64, operands=fl.OPERANDS_FACTORED))
    _, A, B = run_ab(p, h)
    ng = h.num_g(0)
    H, S = alloc_out(ng, 0), alloc_out(ng, 0)
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
    h.sync()
    with pytest.raises(fl.FlapwError) as e:
        h.eigh(ng, H, ng, S, ng)
    assert e.value.code == -4 and "positive definite" in str(e.value)
    with pytest.raises(fl.FlapwError) as e:
        h.eigh(ng, H, ng - 1, S, ng)
    assert e.value.code == -1
    h.destroy()
