"""H with the spherical part of T by the addition theorem (FLAPW_H_SPHERICAL,
the H half of the compression the Conclusions point to): with
T = T_sph + rest, T_sph l-diagonal per slot (T^XY_{L'L} = t^XY_l delta_{L'L}),
H = (4 pi / Omega) sum_c rho_c sum_l (2l+1) P_l [t^AA a'a + t^BB b'b
+ t^AB a'b + t^BA b'a]_l plus the contraction of the factorised rest.  A rest
confined to r rows and columns of each slot contracts over r rows per atom; a
zero rest runs no contraction.  Both against the oracle's H of the whole T
(Eq. (def_hamilton))."""
import numpy as np
import pytest

import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs

from helpers import TOL_EMU, TOL_F64, alloc_out, columns_from_lower, herm_relerr, lower_to_full, oracle_hs, run_ab

pytestmark = pytest.mark.gpu


def _spherical_plus_rest(p, r, seed):
    """T = spherical part + a Hermitian rest on r random rows/columns per slot;
    returns (T, t_sph[slot][l][4])."""
    rng = np.random.default_rng(seed)
    nl, L1, n = p.n_L, p.lmax + 1, 2 * p.n_L
    ns = p.T.shape[0]
    t = np.zeros((ns, L1, 4))
    t[..., 0] = rng.uniform(0.5, 1.5, (ns, L1))
    t[..., 1] = rng.uniform(0.5, 1.5, (ns, L1))
    t[..., 2:] = rng.uniform(-0.3, 0.3, (ns, L1, 2))
    T = np.zeros((ns, n, n), complex)
    for s in range(ns):
        for l in range(L1):
            for L in range(l * l, (l + 1) * (l + 1)):
                tba = t[s, l, 2] + 1j * t[s, l, 3]
                T[s, L, L] = t[s, l, 0]
                T[s, nl + L, nl + L] = t[s, l, 1]
                T[s, nl + L, L] = tba
                T[s, L, nl + L] = np.conj(tba)
        if r:
            idx = rng.choice(n, size=r, replace=False)
            X = rng.uniform(-1, 1, (r, r)) + 1j * rng.uniform(-1, 1, (r, r))
            T[s][np.ix_(idx, idx)] += 0.2 * (X + X.conj().T)
    return T, t


@pytest.mark.parametrize("precision,tol", [(fl.PREC_EMU, TOL_EMU), (fl.PREC_FP64, TOL_F64)])
@pytest.mark.parametrize("r", [0, 5])
def test_spherical_split_matches_oracle(precision, tol, r):
    p = inputs.small(41, n_atoms=3, n_types=2, lmax=4, n_target=(600, 333))
    p.atom_slot = np.array([1, 0, 1], dtype=np.int32)
    p.T, t_sph = _spherical_plus_rest(p, r, seed=3 + r)
    opt = fl.default_options(precision=precision, operands=fl.OPERANDS_FACTORED, h_method=fl.H_SPHERICAL)
    h = fl.from_problem(p, opt)
    _, A, B = run_ab(p, h)
    h.set_spherical_T(t_sph)
    Hs = [alloc_out(h.num_g(k), 0) for k in range(p.n_k)]
    Ss = [alloc_out(h.num_g(k), 0) for k in range(p.n_k)]
    h.build_HS(p.T, p.atom_slot, p.U, A, B, Hs, Ss)
    h.sync()
    st = h.stats()
    assert st["n_pos"] + st["n_neg"] == p.n_atoms * r      # only the rest is contracted
    for k in range(p.n_k):
        Ho, So = oracle_hs(p, k)
        ng = Ho.shape[0]
        assert herm_relerr(lower_to_full(Hs[k], ng, 0), Ho) <= tol, (k, herm_relerr(lower_to_full(Hs[k], ng, 0), Ho))
        assert herm_relerr(lower_to_full(Ss[k], ng, 0), So) <= tol


def test_spherical_split_any_t_sph_gives_the_same_H():
    # linearity in T: a t_sph that is not T's spherical part moves work
    # between the two terms (the rest becomes full) but not the result
    p = inputs.small(43, n_atoms=2, n_types=1, lmax=3, n_target=(420,))
    _, t_sph = _spherical_plus_rest(p, 0, seed=9)
    opt = fl.default_options(precision=fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, h_method=fl.H_SPHERICAL)
    h = fl.from_problem(p, opt)
    _, A, B = run_ab(p, h)
    h.set_spherical_T(t_sph)                     # p.T is the dense random T of the recipe
    ng = h.num_g(0)
    H, S = alloc_out(ng, 0), alloc_out(ng, 0)
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
    h.sync()
    Ho, So = oracle_hs(p, 0)
    assert herm_relerr(lower_to_full(H, ng, 0), Ho) <= TOL_EMU


def test_spherical_split_needs_t_sph():
    p = inputs.small(43, n_atoms=2, n_types=1, lmax=3, n_target=(200,))
    opt = fl.default_options(precision=fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, h_method=fl.H_SPHERICAL)
    h = fl.from_problem(p, opt)
    _, A, B = run_ab(p, h)
    ng = h.num_g(0)
    with pytest.raises(fl.FlapwError) as e:
        h.build_HS(p.T, p.atom_slot, p.U, A, B, [alloc_out(ng, 0)], [alloc_out(ng, 0)])
    assert e.value.code == -6


@pytest.mark.parametrize("precision,tol", [(fl.PREC_EMU, TOL_EMU), (fl.PREC_FP64, TOL_F64)])
def test_config2_with_spherical_T_has_no_H_contraction(precision, tol):
    # config 2 with T replaced by its spherical part (per slot and l the mean
    # over m of each block's diagonal): H comes from the addition theorem alone
    # (double-float on the emulated path, FP64 on the other), S from the
    # contraction; sampled full columns against the oracle of the same T
    import oracle
    p = inputs.config2()
    nl, L1 = p.n_L, p.lmax + 1
    t = np.zeros((p.T.shape[0], L1, 4))
    Ts = np.zeros_like(p.T)
    for s in range(p.T.shape[0]):
        for l in range(L1):
            L = np.arange(l * l, (l + 1) * (l + 1))
            tba = np.mean(p.T[s, nl + L, L])
            t[s, l] = (np.mean(p.T[s, L, L].real), np.mean(p.T[s, nl + L, nl + L].real), tba.real, tba.imag)
            Ts[s, L, L] = t[s, l, 0]
            Ts[s, nl + L, nl + L] = t[s, l, 1]
            Ts[s, nl + L, L] = tba
            Ts[s, L, nl + L] = np.conj(tba)
    p.T = Ts
    opt = fl.default_options(precision=precision, operands=fl.OPERANDS_FACTORED, h_method=fl.H_SPHERICAL)
    h = fl.from_problem(p, opt)
    _, A, B = run_ab(p, h)
    h.set_spherical_T(t)
    ng = h.num_g(0)
    H, S = alloc_out(ng, 0), alloc_out(ng, 0)
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
    h.sync()
    st = h.stats()
    assert st["n_pos"] + st["n_neg"] == 0
    n3 = h.gvectors(0)
    cols = [0, 1, 63, 64, 1777, 2048, ng - 2, ng - 1]
    Ho, So = oracle.hs_columns(p, 0, n3, cols)
    eh = np.linalg.norm(columns_from_lower(H, ng, 0, cols) - Ho) / np.linalg.norm(Ho)
    es = np.linalg.norm(columns_from_lower(S, ng, 0, cols) - So) / np.linalg.norm(So)
    assert eh <= tol and es <= tol, (eh, es)
    h.destroy()


@pytest.mark.parametrize("precision,tol", [(fl.PREC_EMU, TOL_EMU), (fl.PREC_FP64, TOL_F64)])
@pytest.mark.parametrize("r", [0, 5])
def test_spherical_split_host_outputs(precision, tol, r):
    # H and S into pinned host memory: the H work (the contraction of the rest
    # and the addition theorem, or the addition theorem alone) runs in two
    # launches split by column so that the first part's columns go back while
    # the second runs; the second k-point has fewer than 64 plane waves, so
    # its first part is empty
    p = inputs.small(47, n_atoms=3, n_types=2, lmax=4, n_target=(700, 40))
    p.T, t_sph = _spherical_plus_rest(p, r, seed=11 + r)
    opt = fl.default_options(precision=precision, operands=fl.OPERANDS_FACTORED, h_method=fl.H_SPHERICAL)
    h = fl.from_problem(p, opt)
    _, A, B = run_ab(p, h)
    h.set_spherical_T(t_sph)
    Hs = [alloc_out(h.num_g(k), 0, True) for k in range(p.n_k)]
    Ss = [alloc_out(h.num_g(k), 0, True) for k in range(p.n_k)]
    h.build_HS(p.T, p.atom_slot, p.U, A, B, Hs, Ss)
    h.sync()
    assert h.num_g(1) < 64
    for k in range(p.n_k):
        Ho, So = oracle_hs(p, k)
        ng = Ho.shape[0]
        assert herm_relerr(lower_to_full(Hs[k], ng, 0), Ho) <= tol, k
        assert herm_relerr(lower_to_full(Ss[k], ng, 0), So) <= tol, k
    h.destroy()
