"""GB300 (sm_103a) builder of the FLAPW muffin-tin Hamiltonian and overlap.

Python binding of the C ABI declared in include/flapw.h: the same entry
points, argument marshalling only.  Host arrays are numpy arrays; device
buffers are anything with a ``data_ptr()`` (torch tensors) or a raw integer
address; streams are ``torch.cuda.Stream`` objects, raw handles or None.
Every computation runs in the CUDA library; if it has not been built the
binding raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

__all__ = ["FlapwError", "Options", "Stats", "Handle", "load", "library_path", "build",
           "default_options", "enumerate_g", "hs_create", "engine_create", "herk_noalloc", "partition",
           "declared_symbols",
           "PREC_FP64", "PREC_EMU", "LAYOUT_LOWER_FULL", "LAYOUT_LOWER_PACKED",
           "OPERANDS_FROM_AB", "OPERANDS_FACTORED", "S_CONTRACTION", "S_LEGENDRE",
           "H_FACTORED", "H_ALG3", "H_SPHERICAL", "H_ALG1"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_HEADER = os.path.join(os.path.dirname(_HERE), "include", "flapw.h")

PREC_FP64, PREC_EMU = 0, 1
LAYOUT_LOWER_FULL, LAYOUT_LOWER_PACKED = 0, 1
OPERANDS_FROM_AB, OPERANDS_FACTORED = 0, 1
S_CONTRACTION, S_LEGENDRE = 0, 1
H_FACTORED, H_ALG3, H_SPHERICAL, H_ALG1 = 0, 1, 2, 3
ERR = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_FACTOR",
       -5: "ERR_TIMEOUT", -6: "ERR_STATE", -7: "ERR_UNSUPPORTED"}


class FlapwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("n_slices", ctypes.c_int), ("layout", ctypes.c_int),
                ("operands", ctypes.c_int), ("use_graph", ctypes.c_int), ("autotune", ctypes.c_int),
                ("tile_order", ctypes.c_int), ("s_method", ctypes.c_int), ("h_method", ctypes.c_int),
                ("pipeline", ctypes.c_int), ("tile_cover", ctypes.c_int),
                ("wait_us", ctypes.c_int), ("mem_cap_mb", ctypes.c_int),
                ("part_count", ctypes.c_int), ("part_index", ctypes.c_int),
                ("reserved", ctypes.c_int * 1)]


class Stats(ctypes.Structure):
    _fields_ = [("ms_ab", ctypes.c_double), ("ms_factor", ctypes.c_double),
                ("ms_operands", ctypes.c_double), ("ms_slice", ctypes.c_double),
                ("ms_contract", ctypes.c_double), ("ms_hs_total", ctypes.c_double),
                ("flops_herk", ctypes.c_double), ("flops_tensor", ctypes.c_double),
                ("k_total", ctypes.c_int64), ("n_pos", ctypes.c_int), ("n_neg", ctypes.c_int),
                ("n_pivot2", ctypes.c_int), ("n_slices", ctypes.c_int), ("n_tiles", ctypes.c_int),
                ("tile_order", ctypes.c_int), ("graph_replays", ctypes.c_int),
                ("tile_cover", ctypes.c_int), ("pipeline", ctypes.c_int),
                ("copy_ops", ctypes.c_int), ("bytes_d2h", ctypes.c_int64),
                ("n_chol", ctypes.c_int),
                ("reserved", ctypes.c_int * 3), ("ms_s", ctypes.c_double),
                ("ms_ab_assemble", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return os.path.join(_HERE, "_build", "libflapw.so")


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (nvcc) into this package's _build/."""
    from . import _build
    return _build.build(force=force)


def load():
    """The loaded C library; raises FlapwError if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise FlapwError(-2, f"CUDA library not built: {path} is missing "
                                 "(run paper_1712_07206_gb300.build())")
        lib = ctypes.CDLL(path)
        P, c_int, c_void_p = ctypes.POINTER, ctypes.c_int, ctypes.c_void_p
        dp, ip, h = P(ctypes.c_double), P(c_int), c_void_p
        sig = {
            "flapw_default_options": (None, [P(Options)]),
            "flapw_enumerate_g": (c_int, [dp, dp, ctypes.c_double, c_int, ip, ip]),
            "flapw_hs_create": (c_int, [dp, c_int, dp, ip, c_int, dp, c_int, c_int, dp, dp,
                                        P(Options), P(h)]),
            "flapw_engine_create": (c_int, [P(Options), P(h)]),
            "flapw_partition": (c_int, [c_int, ip, c_int, ip]),
            "flapw_set_spherical_T": (c_int, [h, dp, c_int]),
            "flapw_set_options": (c_int, [h, P(Options)]),
            "flapw_num_g": (c_int, [h, c_int, ip]),
            "flapw_get_gvectors": (c_int, [h, c_int, ip]),
            "flapw_ab_offset": (c_int, [h, c_int, P(ctypes.c_int64)]),
            "flapw_build_AB": (c_int, [h, dp, c_void_p, c_void_p, c_void_p]),
            "flapw_build_HS": (c_int, [h, dp, c_int, ip, dp, c_void_p, c_void_p, P(c_void_p),
                                       P(c_void_p), c_void_p]),
            "flapw_herk": (c_int, [h, c_void_p, ctypes.c_int64, c_int, c_int, ip, c_void_p,
                                   ctypes.c_int64, c_void_p]),
            "flapw_herk_noalloc": (c_int, [c_void_p, ctypes.c_int64, c_int, c_int, ip, c_void_p,
                                           ctypes.c_int64, c_int, c_int, c_void_p]),
            "flapw_eigh": (c_int, [h, c_int, c_void_p, ctypes.c_int64, c_void_p, ctypes.c_int64, dp,
                                   c_int, c_void_p]),
            "flapw_sync": (c_int, [h]),
            "flapw_get_stats": (c_int, [h, P(Stats)]),
            "flapw_get_factor": (c_int, [h, c_int, dp, ip, ip]),
            "flapw_last_error": (ctypes.c_char_p, [h]),
            "flapw_destroy": (c_int, [h]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def declared_symbols():
    """Names of the entry points declared in include/flapw.h."""
    txt = open(_HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(flapw_\w+)\s*\(", txt)))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _addr(x):
    """Raw address of a device tensor, numpy array, integer or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(getattr(s, "cuda_stream"))


def _check(rc, handle=None):
    if rc != 0:
        lib = load()
        msg = lib.flapw_last_error(handle)
        raise FlapwError(rc, msg.decode() if msg else "")


def default_options(**kw) -> Options:
    o = Options()
    load().flapw_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def enumerate_g(lattice, k_frac, kmax) -> np.ndarray:
    """Plane waves of one k-point as int32 triples (host only)."""
    lib = load()
    lat, k = _f64(lattice).reshape(9), _f64(k_frac).reshape(3)
    n = ctypes.c_int()
    _check(lib.flapw_enumerate_g(_dp(lat), _dp(k), float(kmax), 0, None, ctypes.byref(n)))
    out = np.zeros((n.value, 3), dtype=np.int32)
    _check(lib.flapw_enumerate_g(_dp(lat), _dp(k), float(kmax), n.value, _ip(out), ctypes.byref(n)))
    return out


class Handle:
    """A crystal (or an engine-only handle) on the current CUDA device."""

    def __init__(self, raw, n_k=0, n_atoms=0, n_L=0, n_types=0, lmax=0):
        self._h = raw
        self.n_k, self.n_atoms, self.n_L, self.n_types, self.lmax = n_k, n_atoms, n_L, n_types, lmax

    def _call(self, name, *args):
        rc = getattr(load(), name)(self._h, *args)
        _check(rc, self._h)

    def set_options(self, opt: Options):
        self._call("flapw_set_options", ctypes.byref(opt))

    def num_g(self, k: int) -> int:
        n = ctypes.c_int()
        self._call("flapw_num_g", int(k), ctypes.byref(n))
        return n.value

    def gvectors(self, k: int) -> np.ndarray:
        out = np.zeros((self.num_g(k), 3), dtype=np.int32)
        self._call("flapw_get_gvectors", int(k), _ip(out))
        return out

    def ab_offset(self, k: int) -> int:
        o = ctypes.c_int64()
        self._call("flapw_ab_offset", int(k), ctypes.byref(o))
        return o.value

    def build_AB(self, radial, A, B, stream=None):
        rad = _f64(radial)
        self._call("flapw_build_AB", _dp(rad), _addr(A), _addr(B), _stream(stream))

    def build_HS(self, T, atom_slot, U, A, B, H, S, stream=None):
        T = np.ascontiguousarray(T, dtype=np.complex128)
        Tv = T.view(np.float64)
        slot, Uf = _i32(atom_slot), _f64(U)
        Hp = (ctypes.c_void_p * len(H))(*[_addr(x) for x in H])
        Sp = (ctypes.c_void_p * len(S))(*[_addr(x) for x in S])
        self._call("flapw_build_HS", _dp(Tv), int(T.shape[0]), _ip(slot), _dp(Uf), _addr(A),
                   _addr(B), Hp, Sp, _stream(stream))

    def herk(self, Z, ldz, K, N, sigma, H, ldh, stream=None):
        sig = None if sigma is None else _i32(sigma)
        self._call("flapw_herk", _addr(Z), int(ldz), int(K), int(N),
                   None if sig is None else _ip(sig), _addr(H), int(ldh), _stream(stream))

    def eigh(self, n, H, ldh, S, lds, vectors=True, stream=None):
        """flapw_eigh: H c = lambda S c in place on device matrices (H becomes
        the eigenvectors, S its Cholesky factor); returns the eigenvalues."""
        w = np.zeros(int(n), dtype=np.float64)
        self._call("flapw_eigh", int(n), _addr(H), int(ldh), _addr(S), int(lds), _dp(w),
                   1 if vectors else 0, _stream(stream))
        return w

    def set_spherical_T(self, t_sph):
        """flapw_set_spherical_T: t_sph [n_slots][lmax+1][4] = t^AA, t^BB,
        Re t^BA, Im t^BA (None clears)."""
        if t_sph is None:
            self._call("flapw_set_spherical_T", None, 0)
            return
        t = _f64(t_sph)
        self._call("flapw_set_spherical_T", _dp(t), int(t.shape[0]))

    def sync(self):
        self._call("flapw_sync")

    def stats(self) -> dict:
        s = Stats()
        self._call("flapw_get_stats", ctypes.byref(s))
        return s.as_dict()

    def factor(self, slot: int):
        n = 2 * self.n_L
        CH = np.zeros((n, n), dtype=np.complex128)
        npos, nneg = ctypes.c_int(), ctypes.c_int()
        self._call("flapw_get_factor", int(slot), _dp(CH.view(np.float64)), ctypes.byref(npos),
                   ctypes.byref(nneg))
        return CH, npos.value, nneg.value

    def destroy(self):
        if self._h:
            _check(load().flapw_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def hs_create(lattice, pos_frac, atom_type, mt_radius, lmax, k_frac, kmax,
              options: Options | None = None) -> Handle:
    lib = load()
    lat, pos, rad = _f64(lattice).reshape(9), _f64(pos_frac), _f64(mt_radius)
    typ, kf, km = _i32(atom_type), _f64(k_frac), _f64(kmax)
    raw = ctypes.c_void_p()
    rc = lib.flapw_hs_create(_dp(lat), int(pos.shape[0]), _dp(pos), _ip(typ), int(rad.shape[0]),
                             _dp(rad), int(lmax), int(kf.shape[0]), _dp(kf), _dp(km),
                             None if options is None else ctypes.byref(options), ctypes.byref(raw))
    _check(rc)
    return Handle(raw, n_k=int(kf.shape[0]), n_atoms=int(pos.shape[0]),
                  n_L=(int(lmax) + 1) ** 2, n_types=int(rad.shape[0]), lmax=int(lmax))


def herk_noalloc(Z, ldz, K, N, sigma, H, ldh, layout=LAYOUT_LOWER_FULL, n_slices=0, stream=None):
    """flapw_herk_noalloc: the emulated contraction with no device allocation
    (workspaces in the library's static 64 MiB device array)."""
    sig = None if sigma is None else _i32(sigma)
    _check(load().flapw_herk_noalloc(_addr(Z), int(ldz), int(K), int(N),
                                     None if sig is None else _ip(sig), _addr(H), int(ldh),
                                     int(layout), int(n_slices), _stream(stream)))


def partition(n_g, part_count) -> np.ndarray:
    """flapw_partition: the part owning each k-point (-1 for all when the
    k-points are shared by tiles).  Host only."""
    ng = _i32(n_g)
    owner = np.zeros(len(ng), dtype=np.int32)
    _check(load().flapw_partition(len(ng), _ip(ng), int(part_count), _ip(owner)))
    return owner


def engine_create(options: Options | None = None) -> Handle:
    lib = load()
    raw = ctypes.c_void_p()
    _check(lib.flapw_engine_create(None if options is None else ctypes.byref(options),
                                   ctypes.byref(raw)))
    return Handle(raw)


def from_problem(p, options: Options | None = None) -> Handle:
    """hs_create for an inputs.Problem."""
    return hs_create(p.lattice, p.pos_frac, p.atom_type, p.mt_radius, p.lmax, p.k_frac, p.kmax,
                     options)
