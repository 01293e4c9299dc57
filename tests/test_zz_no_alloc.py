"""flapw_herk_noalloc, the contraction entry point for callers that cannot
allocate device memory (a fixed memory budget, or a framework's caching
allocator that owns the GPU): it must give the same lower triangle as the
regular entry point, flapw_herk, on two calls in a row (the second reuses
the static scratch the first left behind), and reject problems that do not
fit its 64 MiB scratch array before doing any work.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import paper_1712_07206_gb300 as fl

from helpers import TOL_EMU, alloc_out, herm_relerr, lower_to_full, torch_cuda

pytestmark = pytest.mark.gpu


def _regular(Zd, K, N, sig, layout):
    h = fl.engine_create(fl.default_options(precision=fl.PREC_EMU, layout=layout))
    H = alloc_out(N, layout)
    h.herk(Zd, K, K, N, sig, H, N)
    h.sync()
    h.destroy()
    return lower_to_full(H, N, layout)


@pytest.mark.parametrize("layout", [fl.LAYOUT_LOWER_FULL, fl.LAYOUT_LOWER_PACKED])
def test_noalloc_matches_regular_entry_point_twice(layout):
    torch = torch_cuda()
    fl.build()
    for call, (K, N, seed) in enumerate([(900, 260, 1), (1300, 333, 2)]):
        rng = np.random.default_rng(seed)
        Z = rng.normal(size=(K, N)) + 1j * rng.normal(size=(K, N))
        Z *= np.exp(rng.uniform(-2, 2, size=(1, N)))
        sig = np.where(rng.uniform(size=K) < 0.25, -1, 1).astype(np.int32)
        Zd = torch.from_numpy(np.asfortranarray(Z).ravel(order="F")).cuda()
        H = alloc_out(N, layout)
        fl.herk_noalloc(Zd, K, K, N, sig, H, N, layout=layout)
        torch.cuda.synchronize()
        G = lower_to_full(H, N, layout)
        R = _regular(Zd, K, N, sig, layout)
        assert herm_relerr(G, R) <= TOL_EMU, (call, herm_relerr(G, R))
        # and against the exact product
        E = Z.conj().T @ (sig[:, None] * Z)
        assert herm_relerr(G, E) <= TOL_EMU


@pytest.mark.parametrize("case", ["deep_pipeline", "all_negative", "ldh_above_n"])
def test_noalloc_edge_cases(case):
    # N above 8192 with a short K (the 5-stage load pipeline), every sigma = -1
    # (no positive rows), and the full layout with ldh > N; each against the
    # regular entry point and the exact product
    torch = torch_cuda()
    fl.build()
    K, N, ldh = {"deep_pipeline": (48, 8500, 8500), "all_negative": (700, 300, 300),
                 "ldh_above_n": (500, 250, 331)}[case]
    rng = np.random.default_rng({"deep_pipeline": 3, "all_negative": 4, "ldh_above_n": 5}[case])
    Z = rng.normal(size=(K, N)) + 1j * rng.normal(size=(K, N))
    sig = (-np.ones(K) if case == "all_negative" else np.where(rng.uniform(size=K) < 0.3, -1, 1))
    sig = sig.astype(np.int32)
    Zd = torch.from_numpy(np.asfortranarray(Z).ravel(order="F")).cuda()
    H = torch.zeros(ldh * N, dtype=torch.complex128, device="cuda")
    fl.herk_noalloc(Zd, K, K, N, sig, H, ldh)
    torch.cuda.synchronize()
    M = H.cpu().numpy().reshape(N, ldh)[:, :N].T     # column j at j * ldh
    L = np.tril(M)
    G = L + np.tril(L, -1).conj().T
    assert np.all(H.cpu().numpy().reshape(N, ldh)[:, N:] == 0)   # rows past N untouched
    R = _regular(Zd, K, N, sig, fl.LAYOUT_LOWER_FULL)
    assert herm_relerr(G, R) <= TOL_EMU, herm_relerr(G, R)
    if case != "deep_pipeline":
        E = Z.conj().T @ (sig[:, None] * Z)
        assert herm_relerr(G, E) <= TOL_EMU
    else:
        # sampled columns of the exact product at this size
        cols = [0, 4097, N - 1]
        E = Z.conj().T @ (sig[:, None] * Z[:, cols])
        assert np.linalg.norm(G[:, cols] - E) <= TOL_EMU * np.linalg.norm(E)


def test_noalloc_rejects_problems_beyond_its_scratch():
    torch = torch_cuda()
    K, N = 8192, 4096                       # ~1.5 GB of workspace: far above 64 MiB
    Zd = torch.zeros(K * N, dtype=torch.complex128, device="cuda")
    H = torch.zeros(N * N, dtype=torch.complex128, device="cuda")
    with pytest.raises(fl.FlapwError) as e:
        fl.herk_noalloc(Zd, K, K, N, None, H, N)
    assert e.value.code == -7
    assert float(H.abs().max()) == 0.0      # nothing was enqueued
