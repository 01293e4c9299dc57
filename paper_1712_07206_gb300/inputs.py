"""Seeded synthetic inputs for the muffin-tin H/S build.

This module is shared by the CUDA path, the CPU oracle, the tests and the
benchmark.  It draws random numbers and lays out crystal geometry; it holds
none of the method's arithmetic (no Bessel functions, spherical harmonics,
phases, matching, factorisation or contraction).

The paper's own test systems (NaCl, AuAg, TiO2 in the problem-size table of
Sec. 5.2) are FLEUR inputs that are not available; the five workloads below
stand in for them with the same shapes (atoms, l_max, number of plane waves).

Conventions (Sec. 2, Eq. (basis) and Eqs. (h)/(s)):
  lattice     3x3, rows are the real-space lattice vectors a1, a2, a3 (bohr)
  pos_frac    [n_atoms][3] fractional atom positions
  atom_type   [n_atoms] type index (radial data, U and radius are per type)
  mt_radius   [n_types] muffin-tin radius R_t
  radial      [n_types][lmax+1][4] = u_l(R), u_l'(R), udot_l(R), udot_l'(R)
  U           [n_types][lmax+1] = ||udot_l||, the diagonal of U in Eq. (s)
  T           [n_slots][2N_L][2N_L] complex Hermitian, rows/cols ordered
              [A-part L=0..N_L-1, B-part L=0..N_L-1]; block (X,Y) is T^[XY]
  atom_slot   [n_atoms] which T block an atom uses (default: its type)
  k_frac      [n_k][3] k-points in fractional reciprocal coordinates
  kmax        [n_k] plane-wave cut-off |k+G| <= kmax per k-point
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Problem:
    name: str
    lattice: np.ndarray
    pos_frac: np.ndarray
    atom_type: np.ndarray
    mt_radius: np.ndarray
    lmax: int
    k_frac: np.ndarray
    kmax: np.ndarray
    radial: np.ndarray
    U: np.ndarray
    T: np.ndarray
    atom_slot: np.ndarray
    layout: str = "full"        # "full" lower column-major or "packed" lower
    n_target: tuple = ()

    @property
    def n_atoms(self) -> int:
        return int(self.pos_frac.shape[0])

    @property
    def n_types(self) -> int:
        return int(self.mt_radius.shape[0])

    @property
    def n_L(self) -> int:
        return (self.lmax + 1) ** 2

    @property
    def n_k(self) -> int:
        return int(self.k_frac.shape[0])

    @property
    def n_slots(self) -> int:
        return int(self.T.shape[0])

    @property
    def volume(self) -> float:
        return abs(float(np.linalg.det(self.lattice)))


def kmax_for_count(n_target: float, volume: float) -> float:
    """Cut-off whose free-electron sphere holds about n_target plane waves.

    A sphere of radius K in reciprocal space holds K^3 Omega / (6 pi^2)
    lattice points on average, so K = (6 pi^2 N / Omega)^(1/3).
    """
    return (6.0 * math.pi ** 2 * n_target / volume) ** (1.0 / 3.0)


def _radial(rng, n_types, lmax, radii):
    """u, u', udot drawn U[0.2, 1.5]; udot' fixed by udot u' - u udot' = 1/R^2."""
    rad = np.empty((n_types, lmax + 1, 4))
    for t in range(n_types):
        for l in range(lmax + 1):
            u, up, ud = rng.uniform(0.2, 1.5, size=3)
            R = radii[t]
            udp = (ud * up - 1.0 / (R * R)) / u
            rad[t, l] = (u, up, ud, udp)
    return rad


def _t_blocks(rng, n_slots, n_L, hpd=False):
    """T = I + 0.1 (X + X^H)/2, Re X, Im X ~ U[-1, 1], one block per slot.

    With hpd=True the Hermitian perturbation is rescaled to spectral norm 0.5,
    so T is Hermitian positive definite.
    """
    n = 2 * n_L
    T = np.empty((n_slots, n, n), dtype=np.complex128)
    for s in range(n_slots):
        X = rng.uniform(-1, 1, size=(n, n)) + 1j * rng.uniform(-1, 1, size=(n, n))
        W = (X + X.conj().T) / 2
        if hpd:
            W = W * (0.5 / np.abs(np.linalg.eigvalsh(W)).max())
            T[s] = np.eye(n) + W
        else:
            T[s] = np.eye(n) + 0.1 * W
    return T


def _min_image_sep(frac, lattice):
    n = frac.shape[0]
    best = np.inf
    for i in range(n):
        for j in range(i + 1, n):
            d = frac[i] - frac[j]
            d -= np.round(d)
            best = min(best, float(np.linalg.norm(d @ lattice)))
    return best


def _finish(name, rng, lattice, pos_frac, atom_type, radii, lmax, k_frac, n_target,
            layout="full", hpd=False, kmax=None):
    n_types = len(radii)
    vol = abs(float(np.linalg.det(lattice)))
    if kmax is None:
        kmax = np.array([kmax_for_count(n, vol) for n in n_target])
    radial = _radial(rng, n_types, lmax, radii)
    U = rng.uniform(0.1, 1.0, size=(n_types, lmax + 1))
    T = _t_blocks(rng, n_types, (lmax + 1) ** 2, hpd=hpd)
    return Problem(name=name, lattice=np.ascontiguousarray(lattice, dtype=np.float64),
                   pos_frac=np.ascontiguousarray(pos_frac, dtype=np.float64),
                   atom_type=np.ascontiguousarray(atom_type, dtype=np.int32),
                   mt_radius=np.asarray(radii, dtype=np.float64), lmax=int(lmax),
                   k_frac=np.ascontiguousarray(k_frac, dtype=np.float64),
                   kmax=np.asarray(kmax, dtype=np.float64), radial=radial, U=U, T=T,
                   atom_slot=np.ascontiguousarray(atom_type, dtype=np.int32),
                   layout=layout, n_target=tuple(n_target))


def with_kpoints(p: Problem, copies: int, seed: int = 3000) -> Problem:
    """The workload over `copies` sets of its k-points, the job of `copies`
    independent callers: the first set is p's own, the others seeded k-points
    of the same crystal (uniform in the cube of reciprocal coordinates
    [-1/2, 1/2)^3), each with the K_max of the k-point whose place it takes, so
    that N_G stays close.  The name stays the workload's."""
    if copies <= 1:
        return p
    rng = np.random.Generator(np.random.PCG64(seed))
    extra = rng.uniform(-0.5, 0.5, size=((copies - 1) * p.n_k, 3))
    return dataclasses.replace(p, k_frac=np.ascontiguousarray(np.vstack([p.k_frac, extra])),
                               kmax=np.tile(np.asarray(p.kmax, dtype=np.float64), copies),
                               n_target=tuple(p.n_target) * copies)


def subset_kpoints(p: Problem, ks) -> Problem:
    """The same crystal and data with only the k-points ks (in that order)."""
    ks = list(ks)
    return dataclasses.replace(p, k_frac=np.ascontiguousarray(p.k_frac[ks]),
                               kmax=np.asarray(p.kmax, dtype=np.float64)[ks],
                               n_target=tuple(p.n_target[k] for k in ks) if p.n_target else ())


def config1(hpd=False) -> Problem:
    """2 atoms, one type, simple-cubic a=6 bohr, l_max=4, ~300 plane waves."""
    rng = np.random.Generator(np.random.PCG64(1001))
    lat = np.eye(3) * 6.0
    while True:
        pos = rng.uniform(0, 1, size=(2, 3))
        if _min_image_sep(pos, lat) >= 4.6:
            break
    k = rng.uniform(-0.5, 0.5, size=(1, 3))
    return _finish("c1_sc6_2at_l4_ng300", rng, lat, pos, [0, 0], [2.2], 4, k, [300], hpd=hpd)


def config2(hpd=False) -> Problem:
    """16 atoms in 2 types (bcc 2x2x2 of 6x6x7 cells), l_max=8, ~4000 plane waves."""
    rng = np.random.Generator(np.random.PCG64(1002))
    lat = np.diag([12.0, 12.0, 14.0])
    pos, typ = [], []
    for i in range(2):
        for j in range(2):
            for l in range(2):
                pos.append([i / 2, j / 2, l / 2]); typ.append(0)
                pos.append([(i + 0.5) / 2, (j + 0.5) / 2, (l + 0.5) / 2]); typ.append(1)
    pos = np.array(pos)
    jit = rng.uniform(-0.2, 0.2, size=pos.shape) / np.array([12.0, 12.0, 14.0])
    pos = (pos + jit) % 1.0
    k = rng.uniform(-0.5, 0.5, size=(1, 3))
    return _finish("c2_ortho_16at_l8_ng4000", rng, lat, pos, typ, [2.0, 2.4], 8, k, [4000], hpd=hpd)


def _sc_grid(n, a, jitter, rng):
    g = (np.arange(n) + 0.5) / n
    pos = np.array([[x, y, z] for x in g for y in g for z in g])
    pos = pos + rng.uniform(-jitter, jitter, size=pos.shape) / a
    return pos % 1.0


def config3(hpd=False) -> Problem:
    """64 atoms in 4 types, cubic a=20 bohr, l_max=10, ~12000 plane waves."""
    rng = np.random.Generator(np.random.PCG64(1003))
    a = 20.0
    pos = _sc_grid(4, a, 0.1, rng)
    typ = rng.permutation(np.repeat(np.arange(4), 16))
    radii = [1.9, 1.9 + 0.5 / 3, 1.9 + 1.0 / 3, 2.4]
    k = rng.uniform(-0.5, 0.5, size=(1, 3))
    return _finish("c3_sc20_64at_l10_ng12000", rng, np.eye(3) * a, pos, typ, radii, 10, k,
                   [12000], hpd=hpd)


def config4(hpd=False) -> Problem:
    """27 atoms in 3 types, cubic a=16 bohr, l_max=8, 32 k-points with 2500..6000 plane waves."""
    rng = np.random.Generator(np.random.PCG64(1004))
    a = 16.0
    pos = _sc_grid(3, a, 0.3, rng)
    typ = np.repeat(np.arange(3), 9)
    ks, nt = [], []
    for i in range(32):
        r = np.random.Generator(np.random.PCG64(2000 + i))
        ks.append(r.uniform(-0.5, 0.5, size=3))
        nt.append(int(r.integers(2500, 6001)))
    return _finish("c4_sc16_27at_l8_32k", rng, np.eye(3) * a, pos, typ, [2.0, 2.1, 2.2], 8,
                   np.array(ks), nt, hpd=hpd)


def config5(hpd=False) -> Problem:
    """256 atoms in 4 types (fcc 4x4x4 of 8-bohr cubes), l_max=8, ~24000 plane waves, packed output."""
    rng = np.random.Generator(np.random.PCG64(1005))
    a = 32.0
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    pos = np.array([(np.array([i, j, l]) + b + 0.25) / 4 for i in range(4) for j in range(4)
                    for l in range(4) for b in basis])
    pos = (pos + rng.uniform(-0.2, 0.2, size=pos.shape) / a) % 1.0
    typ = rng.permutation(np.repeat(np.arange(4), 64))
    radii = [1.9, 1.9 + 0.5 / 3, 1.9 + 1.0 / 3, 2.4]
    k = rng.uniform(-0.5, 0.5, size=(1, 3))
    return _finish("c5_sc32_256at_l8_ng24000", rng, np.eye(3) * a, pos, typ, radii, 8, k,
                   [24000], layout="packed", hpd=hpd)


CONFIGS = {1: config1, 2: config2, 3: config3, 4: config4, 5: config5}


def small(seed: int, n_atoms=3, n_types=2, lmax=3, n_target=(200,), cell=(7.0, 8.0, 9.0),
          hpd=False, layout="full", skew=0.15) -> Problem:
    """A small random triclinic cell for tests (ragged sizes, several types)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lat = np.diag(cell) + rng.uniform(-skew, skew, size=(3, 3)) * np.array(cell)[:, None]
    pos = rng.uniform(0, 1, size=(n_atoms, 3))
    typ = np.arange(n_atoms) % n_types
    radii = list(rng.uniform(1.6, 2.2, size=n_types))
    k = rng.uniform(-0.5, 0.5, size=(len(n_target), 3))
    return _finish(f"small_s{seed}", rng, lat, pos, typ, radii, lmax, k, list(n_target),
                   hpd=hpd, layout=layout)
