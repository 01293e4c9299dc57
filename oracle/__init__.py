"""CPU oracle for the FLAPW muffin-tin H/S build (test infrastructure only).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package.  The product path (the CUDA library and its binding) never
imports, links or runs anything here, and nothing here imports the product.

The arithmetic lives in ``oracle.c`` (plain C, FP64 with long-double special
functions), which follows the paper's definitions:

  * the plane-wave set |k+G| <= K_max (Sec. 2),
  * the LAPW matching coefficients A, B (Sec. 2, Eq. (basis), continuity of
    value and slope at the muffin-tin boundary, via the Rayleigh expansion),
  * S and H element by element (Eqs. (def_overlap), (def_hamilton), i.e.
    Eqs. (h), (s)), evaluated column by column.

``herk_lower`` below is the contraction step alone, Z^H diag(sigma) Z, written
with one numpy matmul (a library primitive) and nothing else.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i = ctypes.c_double, ctypes.c_int
            lib.oracle_gvectors.argtypes = [P(d), P(d), d, i, P(i)]
            lib.oracle_gvectors.restype = i
            lib.oracle_sph_bessel.argtypes = [i, d, P(d), P(d)]
            lib.oracle_ylm.argtypes = [i, d, d, P(d)]
            lib.oracle_build_ab.argtypes = [P(d), i, P(d), P(i), i, P(d), i, P(d), P(d), P(i), i,
                                            P(i), P(d), P(d)]
            lib.oracle_build_ab.restype = i
            lib.oracle_hs_columns.argtypes = [P(d), i, P(d), P(i), i, P(d), i, P(d), P(d), P(d),
                                              P(d), P(i), i, P(i), i, P(i), P(d), P(d)]
            lib.oracle_hs_columns.restype = i
            lib.oracle_max_threads.restype = i
            lib.oracle_set_threads.argtypes = [i]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def gvectors(lattice, k_frac, kmax) -> np.ndarray:
    """Integer triples n of the plane waves |(n+k).B| <= kmax, in the fixed order."""
    lib = _load()
    lat = _f64(lattice).reshape(9)
    k = _f64(k_frac).reshape(3)
    n = lib.oracle_gvectors(_dp(lat), _dp(k), float(kmax), 0, None)
    out = np.zeros((n, 3), dtype=np.int32)
    lib.oracle_gvectors(_dp(lat), _dp(k), float(kmax), n, _ip(out))
    return out


def sph_bessel(l: int, x: float):
    """(j_l(x), j_l'(x))."""
    j, dj = ctypes.c_double(), ctypes.c_double()
    _load().oracle_sph_bessel(int(l), float(x), ctypes.byref(j), ctypes.byref(dj))
    return j.value, dj.value


def ylm(lmax: int, theta: float, phi: float) -> np.ndarray:
    """Y_lm(theta, phi) at index L = l*l + l + m, complex128[(lmax+1)^2]."""
    out = np.zeros(2 * (lmax + 1) ** 2)
    _load().oracle_ylm(int(lmax), float(theta), float(phi), _dp(out))
    return out.view(np.complex128)


def build_ab(p, kidx: int, n3: np.ndarray, g_idx=None):
    """A, B as complex128 [n_atoms][N_L][len(g_idx)] for k-point kidx."""
    lib = _load()
    n3 = _i32(n3)
    g_idx = _i32(np.arange(n3.shape[0]) if g_idx is None else g_idx)
    nl = p.n_L
    A = np.zeros((p.n_atoms, nl, len(g_idx), 2))
    B = np.zeros_like(A)
    lat, pos, rad = _f64(p.lattice), _f64(p.pos_frac), _f64(p.mt_radius)
    typ, radial, k = _i32(p.atom_type), _f64(p.radial), _f64(p.k_frac[kidx])
    rc = lib.oracle_build_ab(_dp(lat), p.n_atoms, _dp(pos), _ip(typ), p.n_types, _dp(rad),
                             p.lmax, _dp(k), _dp(radial), _ip(n3), len(g_idx), _ip(g_idx),
                             _dp(A), _dp(B))
    assert rc == 0
    return A.view(np.complex128)[..., 0], B.view(np.complex128)[..., 0]


def hs_columns(p, kidx: int, n3: np.ndarray, cols):
    """Columns of H and S: arrays [len(cols)][N_G] with out[c][G'] = X_{G', cols[c]}."""
    lib = _load()
    n3 = _i32(n3)
    cols = _i32(cols)
    ng = n3.shape[0]
    H = np.zeros((len(cols), ng, 2))
    S = np.zeros_like(H)
    lat, pos, rad = _f64(p.lattice), _f64(p.pos_frac), _f64(p.mt_radius)
    typ, radial, k = _i32(p.atom_type), _f64(p.radial), _f64(p.k_frac[kidx])
    U = _f64(p.U)
    T = np.ascontiguousarray(p.T, dtype=np.complex128).view(np.float64)
    slot = _i32(p.atom_slot)
    rc = lib.oracle_hs_columns(_dp(lat), p.n_atoms, _dp(pos), _ip(typ), p.n_types, _dp(rad),
                               p.lmax, _dp(k), _dp(radial), _dp(U), _dp(T), _ip(slot), ng,
                               _ip(n3), len(cols), _ip(cols), _dp(H), _dp(S))
    assert rc == 0
    return H.view(np.complex128)[..., 0], S.view(np.complex128)[..., 0]


def hs_full(p, kidx: int, n3: np.ndarray):
    """Full Hermitian H and S (both triangles) as [N_G][N_G] with [G'][G]."""
    ng = n3.shape[0]
    Hc, Sc = hs_columns(p, kidx, n3, np.arange(ng))
    return Hc.T.copy(), Sc.T.copy()


def herk_lower(Z: np.ndarray, sigma=None) -> np.ndarray:
    """Z^H diag(sigma) Z for Z of shape [K][N] (the contraction step alone).

    Returns the full N x N product; callers compare its lower triangle.
    """
    Zs = Z if sigma is None else Z * np.asarray(sigma, dtype=np.float64)[:, None]
    return Z.conj().T @ Zs
