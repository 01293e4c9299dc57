"""The factored form of H on the host (no GPU): T = C diag(sigma) C^H from a
Bunch-Kaufman LDL^H with each 2x2 block of D split by its eigenvectors
(scipy), then H = sum_a Z_a^H diag(sigma) Z_a with Z_a = C^H [A_a; B_a] and
S = sum_a Z_S,a^H Z_S,a with Z_S,a = [A_a; U B_a].  This is the identity the
library's single Hermitian rank-K update rests on (Sec. 3, Alg. 1's Cholesky
step generalised to indefinite T); it is checked here against the oracle's
element-by-element H and S, for indefinite and for positive definite T."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1712_07206_gb300 import inputs


def factor_signature(T):
    """C, sigma with T = C diag(sigma) C^H (sigma = +-1; zero pivots dropped)."""
    lu, d, perm = sl.ldl(T, lower=True, hermitian=True)
    n = T.shape[0]
    cols, sig = [], []
    i = 0
    while i < n:
        if i + 1 < n and d[i + 1, i] != 0:      # a 2x2 block
            lam, V = np.linalg.eigh(d[i:i + 2, i:i + 2])
            for j in range(2):
                cols.append(lu[:, i:i + 2] @ V[:, j] * np.sqrt(abs(lam[j])))
                sig.append(np.sign(lam[j]))
            i += 2
        else:
            if d[i, i].real != 0:
                cols.append(lu[:, i] * np.sqrt(abs(d[i, i].real)))
                sig.append(np.sign(d[i, i].real))
            i += 1
    return np.stack(cols, axis=1), np.array(sig)


@pytest.mark.parametrize("hpd", [False, True])
def test_factored_form_reproduces_t_and_the_oracle(hpd):
    p = inputs.small(61, n_atoms=3, n_types=2, lmax=8, n_target=(150,), hpd=hpd)
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    A, B = oracle.build_ab(p, 0, n3)
    ls = np.concatenate([[l] * (2 * l + 1) for l in range(p.lmax + 1)])
    factors = []
    for T in p.T:
        C, sig = factor_signature(T)
        assert np.linalg.norm(C * sig @ C.conj().T - T) < 1e-13 * np.linalg.norm(T)
        ev = np.linalg.eigvalsh(T)
        assert np.sum(sig < 0) == np.sum(ev < 0)        # Sylvester: the signature is T's inertia
        assert len(sig) == T.shape[0]                    # no zero pivots here
        if hpd:
            assert np.all(sig > 0)
        else:                                            # negative signs and 2x2 pivots occur
            assert np.sum(sig < 0) > 0 and np.any(np.diag(sl.ldl(T, hermitian=True)[1], -1) != 0)
        factors.append((C, sig))
    ng = len(n3)
    H = np.zeros((ng, ng), complex)
    S = np.zeros((ng, ng), complex)
    for a in range(p.n_atoms):
        C, sig = factors[p.atom_slot[a]]
        Z = C.conj().T @ np.vstack([A[a], B[a]])
        H += Z.conj().T @ (sig[:, None] * Z)
        Zs = np.vstack([A[a], p.U[p.atom_type[a], ls][:, None] * B[a]])
        S += Zs.conj().T @ Zs
    Ho, So = oracle.hs_full(p, 0, n3)
    assert np.linalg.norm(H - Ho) / np.linalg.norm(Ho) < 1e-13
    assert np.linalg.norm(S - So) / np.linalg.norm(So) < 1e-13


def test_default_t_needs_the_indefinite_factorisation():
    """The default T of the l_max 8 workloads is indefinite: a Cholesky
    factorisation (Alg. 1's first choice) fails, the signature form does not."""
    p = inputs.config2()
    for T in p.T:
        with pytest.raises(np.linalg.LinAlgError):
            np.linalg.cholesky(T)
        C, sig = factor_signature(T)
        assert np.sum(sig < 0) > 0
        assert np.linalg.norm(C * sig @ C.conj().T - T) < 1e-13 * np.linalg.norm(T)
