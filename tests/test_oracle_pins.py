"""Pins for the CPU oracle: each test checks it against something other than itself.

  * library special functions (scipy) for j_l, j_l' and Y_lm,
  * closed forms: the addition theorem and the Rayleigh plane-wave expansion,
  * continuity of value and slope of the LAPW basis with the plane wave at the
    muffin-tin boundary (Sec. 2, Eq. (basis)), which fixes A, B completely,
  * brute-force quadruple sums of Eqs. (def_overlap)/(def_hamilton) on tiny
    inputs, written independently with scipy,
  * the Legendre closed form of H and S for l-diagonal T (an independent
    O(N_G^2) algorithm through the addition theorem),
  * the paper's own operation sequence (Alg. 3, refined HSDLA) in numpy BLAS,
  * invariants: Hermiticity, positive semi-definiteness and rank of S,
    inertia of H (Sylvester), lattice-translation invariance.
"""
import numpy as np
import pytest
import scipy.special as sp

import oracle
from paper_1712_07206_gb300 import inputs


# ---------------------------------------------------------------- helpers

def recip(lat):
    return 2 * np.pi * np.linalg.inv(lat).T


def kvec(p, kidx, n3):
    return (n3 + p.k_frac[kidx]) @ recip(p.lattice)


def ab_scipy(p, kidx, n3):
    """A, B written independently from Sec. 2 with scipy special functions."""
    K = kvec(p, kidx, n3)
    kabs = np.linalg.norm(K, axis=1)
    theta = np.where(kabs > 0, np.arctan2(np.hypot(K[:, 0], K[:, 1]), K[:, 2]), 0.0)
    phi = np.where(kabs > 0, np.arctan2(K[:, 1], K[:, 0]), 0.0)
    omega = abs(np.linalg.det(p.lattice))
    nl = p.n_L
    A = np.zeros((p.n_atoms, nl, len(n3)), complex)
    B = np.zeros_like(A)
    for a in range(p.n_atoms):
        t = p.atom_type[a]
        R = p.mt_radius[t]
        ph = np.exp(2j * np.pi * ((n3 + p.k_frac[kidx]) @ p.pos_frac[a]))
        for l in range(p.lmax + 1):
            u, up, ud, udp = p.radial[t, l]
            j = sp.spherical_jn(l, kabs * R)
            dj = kabs * sp.spherical_jn(l, kabs * R, derivative=True)
            M = np.array([[u, ud], [up, udp]])
            al, bl = np.linalg.solve(M, np.vstack([j, dj]))
            for m in range(-l, l + 1):
                f = 4 * np.pi / np.sqrt(omega) * ph * (1j ** l) * np.conj(sp.sph_harm_y(l, m, theta, phi))
                A[a, l * l + l + m] = f * al
                B[a, l * l + l + m] = f * bl
    return A, B


def hs_from_ab(p, A, B):
    """Eqs. (h), (s) with numpy matmul: H = sum_a W^H T W, S = sum_a A^H A + B^H U^2 B."""
    ng = A.shape[2]
    H = np.zeros((ng, ng), complex)
    S = np.zeros((ng, ng), complex)
    for a in range(p.n_atoms):
        W = np.vstack([A[a], B[a]])
        H += W.conj().T @ p.T[p.atom_slot[a]] @ W
        u2 = np.repeat(p.U[p.atom_type[a]] ** 2, [2 * l + 1 for l in range(p.lmax + 1)])
        S += A[a].conj().T @ A[a] + B[a].conj().T @ (u2[:, None] * B[a])
    return H, S


def relerr(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


# ------------------------------------------------------ special functions

@pytest.mark.parametrize("l", range(0, 13))
def test_bessel_vs_scipy(l):
    for x in np.concatenate([[0.0, 1e-6, 0.05], np.linspace(0.1, 14.0, 57)]):
        j, dj = oracle.sph_bessel(l, x)
        jr = sp.spherical_jn(l, x)
        djr = sp.spherical_jn(l, x, derivative=True)
        assert abs(j - jr) <= 1e-13 * abs(jr) + 1e-17, (l, x, j, jr)
        assert abs(dj - djr) <= 1e-12 * abs(djr) + 1e-16, (l, x, dj, djr)


def test_ylm_vs_scipy():
    rng = np.random.default_rng(7)
    for theta, phi in list(rng.uniform([0, -np.pi], [np.pi, np.pi], size=(20, 2))) + [(0.0, 0.0), (np.pi, 1.0)]:
        Y = oracle.ylm(10, theta, phi)
        for l in range(11):
            for m in range(-l, l + 1):
                ref = sp.sph_harm_y(l, m, theta, phi)
                assert abs(Y[l * l + l + m] - ref) < 1e-13, (l, m, theta, phi)


def test_addition_theorem():
    """sum_m Y*_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(cos gamma)."""
    rng = np.random.default_rng(11)
    lmax = 30
    for _ in range(10):
        ta, pa, tb, pb = rng.uniform([0, -np.pi, 0, -np.pi], [np.pi, np.pi, np.pi, np.pi])
        Ya, Yb = oracle.ylm(lmax, ta, pa), oracle.ylm(lmax, tb, pb)
        ua = np.array([np.sin(ta) * np.cos(pa), np.sin(ta) * np.sin(pa), np.cos(ta)])
        ub = np.array([np.sin(tb) * np.cos(pb), np.sin(tb) * np.sin(pb), np.cos(tb)])
        cg = ua @ ub
        for l in range(lmax + 1):
            s = np.sum(np.conj(Ya[l * l:(l + 1) ** 2]) * Yb[l * l:(l + 1) ** 2])
            ref = (2 * l + 1) / (4 * np.pi) * sp.eval_legendre(l, cg)
            assert abs(s - ref) < 1e-12 * (2 * l + 1), (l, s, ref)


def test_rayleigh_expansion():
    """exp(i K.r) = 4 pi sum_lm i^l j_l(K r) Y*_lm(K_hat) Y_lm(r_hat), truncated at l=40."""
    rng = np.random.default_rng(3)
    lmax = 40
    for _ in range(8):
        K = rng.normal(size=3) * 2.5
        r = rng.normal(size=3)
        r *= rng.uniform(1.0, 2.4) / np.linalg.norm(r)
        kk, rr = np.linalg.norm(K), np.linalg.norm(r)
        angles = lambda v: (np.arctan2(np.hypot(v[0], v[1]), v[2]), np.arctan2(v[1], v[0]))
        YK, Yr = oracle.ylm(lmax, *angles(K)), oracle.ylm(lmax, *angles(r))
        s = 0
        for l in range(lmax + 1):
            j, _ = oracle.sph_bessel(l, kk * rr)
            s += 4 * np.pi * (1j ** l) * j * np.sum(np.conj(YK[l * l:(l + 1) ** 2]) * Yr[l * l:(l + 1) ** 2])
        assert abs(s - np.exp(1j * K @ r)) < 1e-12


# ------------------------------------------------- matching coefficients

def test_radial_inputs_satisfy_wronskian():
    for cfg in (inputs.config1(), inputs.config2(), inputs.small(5)):
        for t in range(cfg.n_types):
            R = cfg.mt_radius[t]
            for l in range(cfg.lmax + 1):
                u, up, ud, udp = cfg.radial[t, l]
                assert abs(ud * up - u * udp - 1 / R ** 2) < 1e-13


def test_basis_continuity_at_sphere_boundary():
    """Value and slope of phi_G inside sphere a equal those of the plane wave
    Omega^{-1/2} exp(i (k+G).r) at |r - tau_a| = R (Sec. 2, Eq. (basis)).
    A large l_max makes the truncation negligible; this pins A, B completely,
    including the 4 pi / sqrt(Omega) normalisation and the Y_lm conventions."""
    p = inputs.small(21, n_atoms=2, n_types=2, lmax=34, n_target=(40,))
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    sel = np.array([0, 3, 7, len(n3) - 1])
    A, B = oracle.build_ab(p, 0, n3, sel)
    K = kvec(p, 0, n3[sel])
    omega = abs(np.linalg.det(p.lattice))
    rng = np.random.default_rng(5)
    for a in range(p.n_atoms):
        t = p.atom_type[a]
        R = p.mt_radius[t]
        tau = p.pos_frac[a] @ p.lattice
        rad = p.radial[t]
        ls = np.concatenate([[l] * (2 * l + 1) for l in range(p.lmax + 1)])
        for _ in range(4):
            rh = rng.normal(size=3)
            rh /= np.linalg.norm(rh)
            Y = oracle.ylm(p.lmax, np.arctan2(np.hypot(rh[0], rh[1]), rh[2]), np.arctan2(rh[1], rh[0]))
            for gi in range(len(sel)):
                val = np.sum((A[a, :, gi] * rad[ls, 0] + B[a, :, gi] * rad[ls, 2]) * Y)
                slope = np.sum((A[a, :, gi] * rad[ls, 1] + B[a, :, gi] * rad[ls, 3]) * Y)
                pw = np.exp(1j * K[gi] @ (tau + R * rh)) / np.sqrt(omega)
                assert abs(val - pw) < 1e-11, (a, gi, val, pw)
                assert abs(slope - 1j * (K[gi] @ rh) * pw) < 1e-10, (a, gi)


def test_ab_vs_scipy_restatement():
    p = inputs.small(8, n_atoms=3, n_types=2, lmax=6, n_target=(120,))
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    A, B = oracle.build_ab(p, 0, n3)
    A2, B2 = ab_scipy(p, 0, n3)
    assert relerr(A, A2) < 1e-13 and relerr(B, B2) < 1e-13


# ------------------------------------------------------------ plane waves

def test_gvector_set_is_the_kmax_ball():
    p = inputs.small(9, n_target=(400,))
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    K = kvec(p, 0, n3)
    k2 = np.sum(K ** 2, axis=1)
    assert np.all(k2 <= p.kmax[0] ** 2 * (1 + 1e-12))
    assert np.all(np.diff(k2) >= -1e-9 * p.kmax[0] ** 2)     # ascending |k+G|
    # brute force over a generous box finds the same set
    rng = np.arange(-25, 26)
    g = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    kk = np.sum(((g + p.k_frac[0]) @ recip(p.lattice)) ** 2, axis=1)
    inside = g[kk <= p.kmax[0] ** 2]
    assert len(inside) == len(n3)
    assert {tuple(x) for x in inside} == {tuple(x) for x in n3}


# ------------------------------------------------------------- H and S

def brute_force_hs(p, n3):
    """Eqs. (def_overlap), (def_hamilton) as literal loops over G', G, a, L', L."""
    ng, nl = len(n3), p.n_L
    assert ng <= 40
    A, B = ab_scipy(p, 0, n3)
    H = np.zeros((ng, ng), complex)
    S = np.zeros((ng, ng), complex)
    for gp in range(ng):
        for g in range(ng):
            h = s = 0
            for a in range(p.n_atoms):
                T = p.T[p.atom_slot[a]]
                t = p.atom_type[a]
                for Lp in range(nl):
                    lp = int(np.sqrt(Lp))
                    s += np.conj(A[a, Lp, gp]) * A[a, Lp, g] + np.conj(B[a, Lp, gp]) * B[a, Lp, g] * p.U[t, lp] ** 2
                    for L in range(nl):
                        h += np.conj(A[a, Lp, gp]) * T[Lp, L] * A[a, L, g]
                        h += np.conj(A[a, Lp, gp]) * T[Lp, nl + L] * B[a, L, g]
                        h += np.conj(B[a, Lp, gp]) * T[nl + Lp, L] * A[a, L, g]
                        h += np.conj(B[a, Lp, gp]) * T[nl + Lp, nl + L] * B[a, L, g]
            H[gp, g], S[gp, g] = h, s
    return H, S


def test_brute_force_quadruple_sum():
    p = inputs.small(13, n_atoms=2, n_types=2, lmax=2, n_target=(24,))
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    H, S = brute_force_hs(p, n3)
    Ho, So = oracle.hs_full(p, 0, n3)
    assert relerr(Ho, H) < 1e-13
    assert relerr(So, S) < 1e-13


def test_gamma_point_with_the_k0_plane_wave():
    """k = 0: the plane wave G = 0 has K = 0, where K_hat is undefined and only
    l = 0 survives (j_l(0) = 0 for l >= 1, K j_l'(K R) = 0); the oracle agrees
    with the brute-force sums there, and its G = 0 row of A, B is zero for l >= 1."""
    p = inputs.small(29, n_atoms=2, n_types=2, lmax=2, n_target=(24,))
    p.k_frac = np.zeros_like(p.k_frac)
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    assert np.array_equal(n3[0], [0, 0, 0])
    A, B = oracle.build_ab(p, 0, n3)
    assert np.all(A[:, 1:, 0] == 0) and np.all(B[:, 1:, 0] == 0)
    assert np.all(A[:, 0, 0] != 0)
    H, S = brute_force_hs(p, n3)
    Ho, So = oracle.hs_full(p, 0, n3)
    assert relerr(Ho, H) < 1e-13
    assert relerr(So, S) < 1e-13


def legendre_closed_form(p, kidx, n3, t_l):
    """H_{G'G} = 4 pi/Omega sum_a e^{i(K-K').tau_a} sum_l (2l+1) P_l(K'.K/|K'||K|)
    [a'a t^AA + a'b t^AB + b'a t^BA + b'b t^BB]_l, for T diagonal in L with
    entries depending on l only (addition theorem applied to Eq. (def_hamilton))."""
    K = kvec(p, kidx, n3)
    kabs = np.linalg.norm(K, axis=1)
    Kh = K / kabs[:, None]
    cosg = np.clip(Kh @ Kh.T, -1, 1)
    omega = abs(np.linalg.det(p.lattice))
    ng = len(n3)
    H = np.zeros((ng, ng), complex)
    for a in range(p.n_atoms):
        t = p.atom_type[a]
        R = p.mt_radius[t]
        ph = np.exp(2j * np.pi * ((n3 + p.k_frac[kidx]) @ p.pos_frac[a]))
        pair = np.conj(ph)[:, None] * ph[None, :]
        acc = np.zeros((ng, ng), complex)
        for l in range(p.lmax + 1):
            u, up, ud, udp = p.radial[t, l]
            j = sp.spherical_jn(l, kabs * R)
            dj = kabs * sp.spherical_jn(l, kabs * R, derivative=True)
            al, bl = np.linalg.solve(np.array([[u, ud], [up, udp]]), np.vstack([j, dj]))
            taa, tab, tba, tbb = t_l(a, t, l)
            blk = (taa * np.outer(al, al) + tab * np.outer(al, bl) + tba * np.outer(bl, al)
                   + tbb * np.outer(bl, bl))
            acc += (2 * l + 1) * sp.eval_legendre(l, cosg) * blk
        H += pair * acc
    return 4 * np.pi / omega * H


def test_legendre_closed_form_S_and_ldiagonal_H():
    p = inputs.config1()
    # l-diagonal T with complex off-diagonal blocks, one per slot
    rng = np.random.default_rng(17)
    tl = rng.uniform(0.5, 1.5, size=(p.n_slots, p.lmax + 1, 2))
    tab = rng.normal(size=(p.n_slots, p.lmax + 1)) + 1j * rng.normal(size=(p.n_slots, p.lmax + 1))
    nl = p.n_L
    ls = np.concatenate([[l] * (2 * l + 1) for l in range(p.lmax + 1)])
    T = np.zeros_like(p.T)
    for s in range(p.n_slots):
        T[s][np.arange(nl), np.arange(nl)] = tl[s, ls, 0]
        T[s][nl + np.arange(nl), nl + np.arange(nl)] = tl[s, ls, 1]
        T[s][np.arange(nl), nl + np.arange(nl)] = tab[s, ls]
        T[s][nl + np.arange(nl), np.arange(nl)] = np.conj(tab[s, ls])
    p.T = T
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    Ho, So = oracle.hs_full(p, 0, n3)
    Sref = legendre_closed_form(p, 0, n3, lambda a, t, l: (1.0, 0.0, 0.0, p.U[t, l] ** 2))
    s_of = lambda a: p.atom_slot[a]
    Href = legendre_closed_form(p, 0, n3, lambda a, t, l: (tl[s_of(a), l, 0], tab[s_of(a), l],
                                                            np.conj(tab[s_of(a), l]), tl[s_of(a), l, 1]))
    assert relerr(So, Sref) < 1e-12
    assert relerr(Ho, Href) < 1e-12


def test_paper_algorithm3_sequence_matches():
    """Alg. 3 (refined HSDLA): S = A^H A; X = U B; S += X^H X;
    Z_a = T^BA A_a + 1/2 T^BB B_a; H = Z^H B + B^H Z; X_a = T^AA A_a; H += A^H X."""
    p = inputs.small(31, n_atoms=3, n_types=2, lmax=4, n_target=(150,))
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    A, B = oracle.build_ab(p, 0, n3)
    nl = p.n_L
    ls = np.concatenate([[l] * (2 * l + 1) for l in range(p.lmax + 1)])
    Ast = np.vstack(list(A))
    Bst = np.vstack(list(B))
    X = np.vstack([p.U[p.atom_type[a], ls][:, None] * B[a] for a in range(p.n_atoms)])
    S = Ast.conj().T @ Ast + X.conj().T @ X
    Z = np.vstack([p.T[p.atom_slot[a]][nl:, :nl] @ A[a] + 0.5 * p.T[p.atom_slot[a]][nl:, nl:] @ B[a]
                   for a in range(p.n_atoms)])
    H = Z.conj().T @ Bst + Bst.conj().T @ Z
    X = np.vstack([p.T[p.atom_slot[a]][:nl, :nl] @ A[a] for a in range(p.n_atoms)])
    H += Ast.conj().T @ X
    Ho, So = oracle.hs_full(p, 0, n3)
    assert relerr(So, S) < 1e-13
    assert relerr(Ho, H) < 1e-13


def test_hermitian_psd_rank_inertia():
    p = inputs.config1()
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    Ho, So = oracle.hs_full(p, 0, n3)
    assert np.abs(Ho - Ho.conj().T).max() < 1e-13 * np.abs(Ho).max()
    assert np.abs(So - So.conj().T).max() < 1e-13 * np.abs(So).max()
    K = 2 * p.n_atoms * p.n_L          # rank of S and H: 2 N_A N_L < N_G here
    ev = np.linalg.eigvalsh(So)
    assert ev.min() > -1e-12 * ev.max()
    assert np.sum(ev > 1e-10 * ev.max()) == K
    # Sylvester: H = W^H blkdiag(T) W with W of full row rank -> inertia of T's
    hv = np.linalg.eigvalsh(Ho)
    tv = np.concatenate([np.linalg.eigvalsh(p.T[s]) for s in p.atom_slot])
    tol = 1e-9 * np.abs(hv).max()
    assert np.sum(hv > tol) == np.sum(tv > 0)
    assert np.sum(hv < -tol) == np.sum(tv < 0)


def test_translation_invariants():
    p = inputs.small(41, n_atoms=3, n_types=2, lmax=3, n_target=(90,))
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    H0, S0 = oracle.hs_full(p, 0, n3)
    # (i) moving one atom by a lattice vector changes nothing
    p.pos_frac = p.pos_frac.copy()
    p.pos_frac[1] += np.array([1.0, -2.0, 3.0])
    H1, S1 = oracle.hs_full(p, 0, n3)
    assert relerr(H1, H0) < 1e-13 and relerr(S1, S0) < 1e-13
    # (ii) a common shift d multiplies element (G', G) by exp(i (G - G').d)
    d = np.array([0.137, -0.291, 0.405])
    p.pos_frac = p.pos_frac + d
    H2, S2 = oracle.hs_full(p, 0, n3)
    ph = np.exp(2j * np.pi * (n3 @ d))
    F = np.conj(ph)[:, None] * ph[None, :]
    assert relerr(H2, F * H0) < 1e-12 and relerr(S2, F * S0) < 1e-12


def test_herk_step_alone_small_exact():
    """Z^H diag(sigma) Z on small integers equals the integer brute force."""
    rng = np.random.default_rng(2)
    Z = rng.integers(-5, 6, size=(7, 5)) + 1j * rng.integers(-5, 6, size=(7, 5))
    sig = np.array([1, -1, 1, 1, -1, 1, 1.0])
    M = oracle.herk_lower(Z, sig)
    for i in range(5):
        for j in range(5):
            ref = sum(np.conj(Z[k, i]) * sig[k] * Z[k, j] for k in range(7))
            assert M[i, j] == ref


# ------------------------------------------------------- stored fixtures

def _golden(name):
    import os
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)


def test_golden_plane_wave_counts():
    rows = np.loadtxt(_golden("gcounts.txt"))
    for c, k, kmax, ng in rows:
        p = inputs.CONFIGS[int(c)]()
        assert abs(p.kmax[int(k)] - kmax) < 1e-12
        if int(c) in (1, 2, 4):
            assert len(oracle.gvectors(p.lattice, p.k_frac[int(k)], kmax)) == int(ng)


def test_golden_c1_elements():
    rows = np.loadtxt(_golden("c1_hs.txt"))
    p = inputs.config1()
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    cols = sorted({int(c) for c in rows[:, 1]})
    H, S = oracle.hs_columns(p, 0, n3, cols)
    for r, c, hr, hi, sr, si in rows:
        ci = cols.index(int(c))
        assert abs(H[ci, int(r)] - (hr + 1j * hi)) < 1e-13
        assert abs(S[ci, int(r)] - (sr + 1j * si)) < 1e-13
