"""C-ABI library: loads without a GPU, exports what include/flapw.h declares,
and its host-side logic (plane-wave set, argument checks) is right."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def _built():
    fl.build()


def test_library_exports_every_declared_symbol():
    lib = fl.load()
    syms = fl.declared_symbols()
    assert len(syms) >= 16
    for s in syms:
        assert hasattr(lib, s), s


def test_default_options():
    o = fl.default_options()
    assert (o.precision, o.n_slices, o.layout, o.operands, o.use_graph) == (
        fl.PREC_EMU, 7, fl.LAYOUT_LOWER_FULL, fl.OPERANDS_FROM_AB, 0)


@pytest.mark.parametrize("cfg", [1, 2, 3, 4, 5])
def test_plane_wave_set_matches_oracle(cfg):
    p = inputs.CONFIGS[cfg]()
    for k in range(p.n_k):
        a = fl.enumerate_g(p.lattice, p.k_frac[k], p.kmax[k])
        b = oracle.gvectors(p.lattice, p.k_frac[k], p.kmax[k])
        assert a.shape == b.shape
        assert np.array_equal(a, b)


def test_plane_wave_set_triclinic_and_ties():
    for seed in range(5):
        p = inputs.small(100 + seed, n_target=(700,), skew=0.3)
        a = fl.enumerate_g(p.lattice, p.k_frac[0], p.kmax[0])
        assert np.array_equal(a, oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0]))
    # k = 0 in a cubic cell: large groups of exactly equal |G|
    lat = np.eye(3) * 7.0
    a = fl.enumerate_g(lat, [0, 0, 0], 3.1)
    assert np.array_equal(a, oracle.gvectors(lat, [0, 0, 0], 3.1))
    assert tuple(a[0]) == (0, 0, 0)


def test_enumerate_g_errors():
    with pytest.raises(fl.FlapwError) as e:
        fl.enumerate_g(np.zeros((3, 3)), [0, 0, 0], 3.0)
    assert e.value.code == -1
    with pytest.raises(fl.FlapwError):
        fl.enumerate_g(np.eye(3), [0, 0, 0], -1.0)
    lib = fl.load()
    assert lib.flapw_enumerate_g(None, None, 1.0, 0, None, None) == -1
    assert b"NULL" in lib.flapw_last_error(None)


def test_eigh_checks_its_arguments_first():
    # no handle, no matrices: refused on the host before any CUDA call
    lib = fl.load()
    w = np.zeros(4)
    dp = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.flapw_eigh(None, 4, None, 4, None, 4, dp, 1, None) == -1
    assert b"NULL" in lib.flapw_last_error(None)


def test_enumerate_g_writes_at_most_max_g():
    """The count is always the full one; only the first max_g triples are written."""
    lib = fl.load()
    lat = np.ascontiguousarray(np.eye(3) * 7.0)
    k = np.array([0.1, 0.2, 0.3])
    full = fl.enumerate_g(lat, k, 3.1)
    assert len(full) > 10
    buf = np.full((len(full), 3), -99, dtype=np.int32)
    n = ctypes.c_int()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.flapw_enumerate_g(dp(lat), dp(k), 3.1, 5, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 ctypes.byref(n)) == 0
    assert n.value == len(full)
    assert np.array_equal(buf[:5], full[:5]) and np.all(buf[5:] == -99)


def test_handleless_errors_are_per_thread():
    """Each thread reads the message of its own last handle-less call."""
    import threading
    lib = fl.load()
    lat = np.ascontiguousarray(np.zeros(9))
    k = np.zeros(3)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    go = threading.Barrier(2)
    seen = {}

    def null_args():
        assert lib.flapw_enumerate_g(None, None, 1.0, 0, None, None) == -1
        go.wait()
        go.wait()
        seen["null"] = lib.flapw_last_error(None)

    def singular():
        go.wait()
        n = ctypes.c_int()
        assert lib.flapw_enumerate_g(dp(lat), dp(k), 1.0, 0, None, ctypes.byref(n)) == -1
        go.wait()
        seen["singular"] = lib.flapw_last_error(None)

    threads = [threading.Thread(target=f) for f in (null_args, singular)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert b"NULL" in seen["null"] and b"singular" in seen["singular"], seen


def test_herk_noalloc_rejects_bad_arguments_before_touching_the_device():
    """Argument checks that come before any CUDA call (the pointers are never
    dereferenced: each case fails first)."""
    lib = fl.load()
    Z = H = 4096
    good = dict(Z=Z, ldz=8, K=8, N=4, sigma=None, H=H, ldh=4, layout=fl.LAYOUT_LOWER_FULL, n_slices=0)
    bad = [dict(Z=None), dict(H=None), dict(K=0), dict(N=0), dict(ldz=7),
           dict(layout=2), dict(ldh=3), dict(n_slices=3), dict(n_slices=9)]
    for change in bad:
        a = dict(good, **change)
        rc = lib.flapw_herk_noalloc(a["Z"], a["ldz"], a["K"], a["N"], a["sigma"], a["H"], a["ldh"],
                                    a["layout"], a["n_slices"], None)
        assert rc == -1, change
        # the message names the argument (the calling thread's handle-less error)
        assert lib.flapw_last_error(None), change
    # K at or above 2^17 is refused like the other contraction entry points
    rc = lib.flapw_herk_noalloc(Z, 1 << 17, 1 << 17, 1, None, H, 1, fl.LAYOUT_LOWER_FULL, 0, None)
    assert rc == -7
    assert b"131072" in lib.flapw_last_error(None)
    rc = lib.flapw_herk_noalloc(Z, 8, 8, 4, None, H, 3, fl.LAYOUT_LOWER_FULL, 0, None)
    assert rc == -1 and b"ldh" in lib.flapw_last_error(None)


def test_create_rejects_bad_arguments_before_touching_the_device():
    p = inputs.config1()
    with pytest.raises(fl.FlapwError) as e:
        fl.hs_create(p.lattice, p.pos_frac, p.atom_type, p.mt_radius, 13, p.k_frac, p.kmax)
    assert e.value.code == -7
    with pytest.raises(fl.FlapwError) as e:
        fl.hs_create(p.lattice, p.pos_frac, [0, 5], p.mt_radius, 4, p.k_frac, p.kmax)
    assert e.value.code == -1
    with pytest.raises(fl.FlapwError) as e:
        fl.hs_create(p.lattice, p.pos_frac, p.atom_type, [-1.0], 4, p.k_frac, p.kmax)
    assert e.value.code == -1
    bad = fl.default_options(n_slices=3)
    with pytest.raises(fl.FlapwError):
        fl.hs_create(p.lattice, p.pos_frac, p.atom_type, p.mt_radius, 4, p.k_frac, p.kmax, bad)
    # option values outside their ranges are rejected before any device work
    for kw in (dict(pipeline=3), dict(h_method=4), dict(h_method=2), dict(s_method=2), dict(tile_order=7), dict(tile_cover=3),
               dict(wait_us=-1), dict(mem_cap_mb=-1),
               dict(operands=fl.OPERANDS_FROM_AB, s_method=fl.S_LEGENDRE)):
        with pytest.raises(fl.FlapwError) as e:
            fl.hs_create(p.lattice, p.pos_frac, p.atom_type, p.mt_radius, 4, p.k_frac, p.kmax,
                         fl.default_options(**kw))
        assert e.value.code == -1, kw


def test_structs_match_header_layout(tmp_path):
    # the ctypes mirrors against the C compiler's view of include/flapw.h
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "flapw.h"
int main(void) {
  printf("%zu %zu\\n", sizeof(flapw_options), sizeof(flapw_stats));
  printf("%zu %zu %zu %zu\\n", offsetof(flapw_options, tile_order), offsetof(flapw_options, s_method),
         offsetof(flapw_options, tile_cover), offsetof(flapw_options, reserved));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", offsetof(flapw_stats, flops_tensor), offsetof(flapw_stats, k_total),
         offsetof(flapw_stats, graph_replays), offsetof(flapw_stats, tile_cover),
         offsetof(flapw_stats, pipeline), offsetof(flapw_stats, ms_s), offsetof(flapw_stats, copy_ops),
         offsetof(flapw_stats, bytes_d2h));
  return 0;
}
""")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals[0] == ctypes.sizeof(fl.Options) and vals[1] == ctypes.sizeof(fl.Stats)
    assert vals[2:6] == [fl.Options.tile_order.offset, fl.Options.s_method.offset,
                         fl.Options.tile_cover.offset, fl.Options.reserved.offset]
    assert vals[6:14] == [fl.Stats.flops_tensor.offset, fl.Stats.k_total.offset,
                          fl.Stats.graph_replays.offset, fl.Stats.tile_cover.offset,
                          fl.Stats.pipeline.offset, fl.Stats.ms_s.offset, fl.Stats.copy_ops.offset,
                          fl.Stats.bytes_d2h.offset]
