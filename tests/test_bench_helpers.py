"""Host-side helpers of bench.py (no GPU): launch counts per mode, the
spherical part of T, the measured-peak file and the traffic table."""
import importlib.util
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


class Args:
    def __init__(self, operands="factored", s_method="contraction", h_method="factored"):
        self.operands, self.s_method, self.h_method = operands, s_method, h_method


@pytest.mark.parametrize("operands,s_method,h_method,n", [
    ("factored", "contraction", "factored", 14),
    ("factored", "legendre", "factored", 13),
    ("from_ab", "contraction", "factored", 10),
    ("factored", "contraction", "alg3", 15),
    ("from_ab", "contraction", "alg3", 10),
    ("factored", "contraction", "alg1", 15),
    ("factored", "contraction", "spherical", 8),
])
def test_launches_per_step(bench, operands, s_method, h_method, n):
    assert bench.launches_per_step(Args(operands, s_method, h_method)) == n


def test_peaks_and_traffic_table(bench):
    bf16, bf16_sus, hbm, src = bench.peaks()
    assert bf16 > 0 and bf16_sus > 0 and hbm > 0 and src in ("measured", "fallback")
    for (name, slices, s_method, h_method, cover, order, pipe), v in bench.MEASURED_TRAFFIC.items():
        assert 4 <= slices <= 8 and s_method in ("contraction", "legendre")
        assert h_method in ("factored", "alg3") and v["bytes"] > 0
        assert cover in (1, 2) and 0 <= order <= 5 and pipe in (1, 2)
        assert len(v["kernel_sha"]) == 16
    # a capture is reported only for the kernel sources it was taken on
    key = next(iter(bench.MEASURED_TRAFFIC))
    rec = bench.MEASURED_TRAFFIC[key]
    if rec["kernel_sha"] == bench.kernel_source_hash():
        assert bench.measured_traffic(*key) == rec["bytes"]
    saved = rec["kernel_sha"]
    rec["kernel_sha"] = "0" * 16
    try:
        assert bench.measured_traffic(*key) is None
    finally:
        rec["kernel_sha"] = saved


def test_columns_from_lower_matches_full_matrix(bench):
    import numpy as np
    rng = np.random.default_rng(3)
    ng = 37
    X = rng.normal(size=(ng, ng)) + 1j * rng.normal(size=(ng, ng))
    X = X + X.conj().T
    cols = np.array([0, 5, 36])
    full = X.T.reshape(-1)                      # full layout, column-major
    packed = np.concatenate([X[j:, j] for j in range(ng)])
    assert np.allclose(bench.columns_from_lower(full, ng, 0, cols), X[:, cols].T)
    assert np.allclose(bench.columns_from_lower(packed, ng, 1, cols), X[:, cols].T)


class _Handle:
    """Stand-in for the library handle: only the plane-wave list is read."""

    def __init__(self, n3):
        self.n3 = n3

    def gvectors(self, k):
        return self.n3


def _lower(X, layout, fl):
    """Lower triangle of a full Hermitian matrix in the library's host layouts."""
    import numpy as np
    ng = X.shape[0]
    if layout == fl.LAYOUT_LOWER_PACKED:
        return np.concatenate([X[j:, j] for j in range(ng)])
    return X.T.reshape(-1).copy()  # column j holds rows 0..ng-1


@pytest.mark.parametrize("layout_name", ["LAYOUT_LOWER_FULL", "LAYOUT_LOWER_PACKED"])
def test_cpu_baseline_calibrates_and_measures_parity(bench, layout_name):
    """The CPU baseline sizes its sample from a timed warm-up (cpu_cols 0),
    always samples the first and last column, and its relative errors are
    zero for exact results and large for a planted error."""
    import numpy as np
    import oracle
    import paper_1712_07206_gb300 as fl
    from paper_1712_07206_gb300 import inputs

    layout = getattr(fl, layout_name)
    p = inputs.CONFIGS[1]()
    oracle.build()
    n3 = oracle.gvectors(p.lattice, p.k_frac[0], p.kmax[0])
    ng = len(n3)
    Hf, Sf = oracle.hs_full(p, 0, n3)
    H, S = [_lower(Hf, layout, fl)], [_lower(Sf, layout, fl)]

    class A:
        cpu_cols, cpu_seconds = 0, 0.05

    out = bench.cpu_baseline(p, _Handle(n3), H, S, layout, [ng], A, H64=H, S64=S)
    n = int(out["sample"].split()[0])
    assert 16 <= n <= ng and out["sample"].endswith(" s")
    assert out["kind"] == "oracle" and out["cores"] >= 1 and out["value"] > 0
    for key in ("parity_rel_err", "parity_rel_err_fp64_path"):
        assert out[key]["H"] < 1e-15 and out[key]["S"] < 1e-15

    A.cpu_cols = 20
    Hbad = [H[0].copy()]
    Hbad[0][0] += 1.0  # H(0,0), in column 0, which every sample holds
    out = bench.cpu_baseline(p, _Handle(n3), Hbad, S, layout, [ng], A)
    assert int(out["sample"].split()[0]) <= 20
    assert out["parity_rel_err"]["H"] > 1e-6 and out["parity_rel_err"]["S"] < 1e-15
    assert "parity_rel_err_fp64_path" not in out


def test_spherical_part_is_a_projection(bench):
    import numpy as np
    import paper_1712_07206_gb300 as fl
    assert bench.H_METHODS == {"factored": fl.H_FACTORED, "alg3": fl.H_ALG3, "spherical": fl.H_SPHERICAL,
                               "alg1": fl.H_ALG1}
    from paper_1712_07206_gb300 import inputs
    p = inputs.small(5, n_atoms=2, n_types=2, lmax=3)
    Ts, t = bench.spherical_part(p.T, p.lmax)
    nl = p.n_L
    assert t.shape == (p.T.shape[0], p.lmax + 1, 4)
    assert np.allclose(Ts, np.conj(np.transpose(Ts, (0, 2, 1))))
    # l-diagonal: nonzero only where both indices have the same L
    idx = np.arange(2 * nl) % nl
    assert np.all(Ts[:, idx[:, None] != idx[None, :]] == 0)
    # a second projection changes nothing
    Ts2, t2 = bench.spherical_part(Ts, p.lmax)
    assert np.allclose(Ts2, Ts, rtol=0, atol=1e-15) and np.allclose(t2, t, rtol=0, atol=1e-15)
    # the l = 1 entries are the mean over m of T's diagonal entries
    L = np.arange(1, 4)
    assert np.isclose(t[0, 1, 0], np.mean(p.T[0, L, L].real))
    assert np.isclose(t[1, 1, 2] + 1j * t[1, 1, 3], np.mean(p.T[1, nl + L, L]))
