"""The seeded synthetic workloads (no GPU): shapes, determinism, and the
physical conditions the method assumes of its inputs -- muffin-tin spheres
that do not overlap (Sec. 2), Hermitian T blocks, positive U."""
import numpy as np
import pytest

from paper_1712_07206_gb300 import inputs

# config: (atoms, types, l_max, k-points, cell diagonal in bohr)
SHAPES = {
    1: (2, 1, 4, 1, (6.0, 6.0, 6.0)),
    2: (16, 2, 8, 1, (12.0, 12.0, 14.0)),
    3: (64, 4, 10, 1, (20.0, 20.0, 20.0)),
    4: (27, 3, 8, 32, (16.0, 16.0, 16.0)),
    5: (256, 4, 8, 1, (32.0, 32.0, 32.0)),
}


@pytest.fixture(scope="module")
def problems():
    return {c: inputs.CONFIGS[c]() for c in SHAPES}


@pytest.mark.parametrize("cfg", sorted(SHAPES))
def test_workload_shapes(problems, cfg):
    p = problems[cfg]
    n_atoms, n_types, lmax, n_k, cell = SHAPES[cfg]
    assert (p.n_atoms, p.n_types, p.lmax, p.n_k) == (n_atoms, n_types, lmax, n_k)
    assert np.allclose(p.lattice, np.diag(cell))
    assert p.n_L == (lmax + 1) ** 2
    assert sorted(set(p.atom_type.tolist())) == list(range(n_types))
    assert p.T.shape == (p.n_slots, 2 * p.n_L, 2 * p.n_L)
    assert p.radial.shape == (n_types, lmax + 1, 4) and p.U.shape == (n_types, lmax + 1)
    assert np.all((p.pos_frac >= -0.5) & (p.pos_frac <= 1.5))


@pytest.mark.parametrize("cfg", sorted(SHAPES))
def test_muffin_tin_spheres_do_not_overlap(problems, cfg):
    """|tau_i - tau_j + R| >= r_i + r_j over all pairs and lattice vectors R
    (including an atom and its own images), by brute force over neighbour cells."""
    p = problems[cfg]
    cart = p.pos_frac @ p.lattice
    r = p.mt_radius[p.atom_type]
    shifts = np.array([[i, j, k] for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)],
                      dtype=np.float64) @ p.lattice
    frac_d = p.pos_frac[:, None, :] - p.pos_frac[None, :, :]
    d0 = (frac_d - np.round(frac_d)) @ p.lattice            # nearest image in the cell frame
    dist = np.linalg.norm(d0[:, :, None, :] + shifts[None, None, :, :], axis=-1).min(axis=2)
    np.fill_diagonal(dist, np.inf)
    own = np.linalg.norm(shifts[np.any(shifts != 0, axis=1)], axis=1).min()
    need = r[:, None] + r[None, :]
    assert np.all(dist >= need), float((dist - need).min())
    assert own >= 2 * r.max()
    assert np.all(np.isfinite(cart))


@pytest.mark.parametrize("cfg", sorted(SHAPES))
def test_inputs_are_seeded(problems, cfg):
    q = inputs.CONFIGS[cfg]()
    p = problems[cfg]
    for f in ("lattice", "pos_frac", "atom_type", "mt_radius", "k_frac", "kmax", "radial", "U", "T"):
        assert np.array_equal(getattr(p, f), getattr(q, f)), f


@pytest.mark.parametrize("cfg", sorted(SHAPES))
def test_t_hermitian_u_positive(problems, cfg):
    p = problems[cfg]
    for T in p.T:
        assert np.array_equal(T, T.conj().T)
    assert np.all((p.U >= 0.1) & (p.U <= 1.0))
    assert np.all(p.mt_radius > 0)


def test_t_definiteness_default_and_hpd():
    """The default T (identity plus a 0.1-scaled Hermitian perturbation) is
    indefinite on the l_max 8 and 10 workloads (2 N_L = 162, 242: the
    perturbation's spectral radius grows like sqrt(N_L)) and positive definite
    at l_max 4 (2 N_L = 50); the hpd variant is positive definite."""
    for cfg in (2, 3):
        p = inputs.CONFIGS[cfg]()
        assert all(np.linalg.eigvalsh(T).min() < 0 for T in p.T), cfg
    q = inputs.config2(hpd=True)
    assert all(np.linalg.eigvalsh(T).min() > 0 for T in q.T)
    small = inputs.config1()
    assert all(np.linalg.eigvalsh(T).min() > 0 for T in small.T)


def test_kmax_from_target_counts():
    """K_max = (6 pi^2 N / Omega)^(1/3) holds N plane waves on average; config 4's
    32 k-points draw their targets from 2500..6000."""
    p = inputs.config4()
    n = p.kmax ** 3 * p.volume / (6 * np.pi ** 2)
    assert np.all((n >= 2500 - 1e-6) & (n <= 6000 + 1e-6))
    assert len(np.unique(np.round(n))) > 16
    for cfg, target in ((1, 300), (2, 4000), (5, 24000)):
        q = inputs.CONFIGS[cfg]()
        m = float(q.kmax[0] ** 3 * q.volume / (6 * np.pi ** 2))
        assert abs(m - target) / target < 0.01, (cfg, m)
