"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: A, B within 1e-13 of the largest entry; H and S within 1e-12
relative Frobenius error (the bound stated for the emulated path) and 1e-13
for the FP64 path; integer-valued contractions bit-exact.
"""
import numpy as np
import pytest

import oracle
import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs

from helpers import (TOL_EMU, TOL_F64, alloc_out, ab_block, columns_from_lower, herm_relerr,
                     lower_to_full, oracle_hs, run_ab, run_hs, torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    fl.build()
    torch = torch_cuda()
    assert torch.cuda.is_available()


# ------------------------------------------------------------- A and B

@pytest.mark.parametrize("seed,lmax,nt", [(1, 4, (300, 170)), (2, 8, (500,)), (3, 0, (40,)),
                                          (4, 12, (90,))])
def test_ab_matches_oracle(seed, lmax, nt):
    p = inputs.small(seed, n_atoms=3, n_types=2, lmax=lmax, n_target=nt)
    h, A, B = run_ab(p)
    for k in range(p.n_k):
        n3 = h.gvectors(k)
        assert np.array_equal(n3, oracle.gvectors(p.lattice, p.k_frac[k], p.kmax[k]))
        Ao, Bo = oracle.build_ab(p, k, n3)
        Ag, Bg = ab_block(p, h, A, k), ab_block(p, h, B, k)
        assert np.abs(Ag - Ao).max() <= 1e-13 * np.abs(Ao).max()
        assert np.abs(Bg - Bo).max() <= 1e-13 * np.abs(Bo).max()
        # every (atom, L) row against its own size too, so that the small rows
        # of high l (j_l(KR) ~ (KR)^l / (2l+1)!!) are checked in relative terms
        for X, Xo in ((Ag, Ao), (Bg, Bo)):
            num = np.linalg.norm(X - Xo, axis=2)
            den = np.linalg.norm(Xo, axis=2)
            assert (den > 0).all()
            assert (num / den).max() <= 1e-12, (num / den).max()


def test_ab_config2_sampled():
    p = inputs.config2()
    h, A, B = run_ab(p)
    n3 = h.gvectors(0)
    sel = np.array([0, 1, 2, 100, 1234, 2999, len(n3) - 2, len(n3) - 1])
    Ao, Bo = oracle.build_ab(p, 0, n3, sel)
    Ag, Bg = ab_block(p, h, A, 0)[:, :, sel], ab_block(p, h, B, 0)[:, :, sel]
    assert np.abs(Ag - Ao).max() <= 1e-13 * np.abs(Ao).max()
    assert np.abs(Bg - Bo).max() <= 1e-13 * np.abs(Bo).max()


# ------------------------------------------------------ factorisation

@pytest.mark.parametrize("hpd", [False, True])
def test_factor_reconstructs_T(hpd):
    p = inputs.config2(hpd=hpd)
    h, Hs, Ss, _ = run_hs(p, fl.PREC_FP64)
    st = h.stats()
    for slot in range(p.n_slots):
        CH, npos, nneg = h.factor(slot)
        n = CH.shape[0]
        sig = np.concatenate([np.ones(npos), -np.ones(nneg), np.zeros(n - npos - nneg)])
        R = CH.conj().T @ (sig[:, None] * CH)
        assert np.linalg.norm(R - p.T[slot]) <= 1e-13 * np.linalg.norm(p.T[slot])
        ev = np.linalg.eigvalsh(p.T[slot])
        assert npos == np.sum(ev > 0) and nneg == np.sum(ev < 0)
    if hpd:
        assert st["n_neg"] == 0


# ------------------------------------------------------ H and S, full

@pytest.mark.parametrize("precision,tol", [(fl.PREC_FP64, TOL_F64), (fl.PREC_EMU, TOL_EMU)])
@pytest.mark.parametrize("layout", [fl.LAYOUT_LOWER_FULL, fl.LAYOUT_LOWER_PACKED])
def test_hs_config1_full(precision, tol, layout):
    p = inputs.config1()
    h, Hs, Ss, _ = run_hs(p, precision, layout)
    Ho, So = oracle_hs(p)
    ng = Ho.shape[0]
    eh = herm_relerr(lower_to_full(Hs[0], ng, layout), Ho)
    es = herm_relerr(lower_to_full(Ss[0], ng, layout), So)
    assert eh <= tol and es <= tol, (eh, es)


@pytest.mark.parametrize("precision,tol", [(fl.PREC_FP64, TOL_F64), (fl.PREC_EMU, TOL_EMU)])
@pytest.mark.parametrize("operands", [fl.OPERANDS_FROM_AB, fl.OPERANDS_FACTORED])
def test_hs_small_multi_k_ragged(precision, tol, operands):
    # 2 k-points, N_G not multiples of the tiles, 3 atoms of 2 types, slots != types
    p = inputs.small(7, n_atoms=3, n_types=2, lmax=3, n_target=(333, 190))
    p.atom_slot = np.array([1, 0, 1], dtype=np.int32)
    h, Hs, Ss, _ = run_hs(p, precision, operands=operands)
    for k in range(p.n_k):
        Ho, So = oracle_hs(p, k)
        ng = Ho.shape[0]
        eh = herm_relerr(lower_to_full(Hs[k], ng, 0), Ho)
        es = herm_relerr(lower_to_full(Ss[k], ng, 0), So)
        assert eh <= tol and es <= tol, (k, eh, es)


@pytest.mark.parametrize("precision", [fl.PREC_FP64, fl.PREC_EMU])
def test_hs_edge_one_atom_lmax0_tiny(precision):
    p = inputs.small(9, n_atoms=1, n_types=1, lmax=0, n_target=(20,))
    h, Hs, Ss, _ = run_hs(p, precision)
    Ho, So = oracle_hs(p)
    ng = Ho.shape[0]
    tol = TOL_EMU if precision == fl.PREC_EMU else TOL_F64
    assert herm_relerr(lower_to_full(Hs[0], ng, 0), Ho) <= tol
    assert herm_relerr(lower_to_full(Ss[0], ng, 0), So) <= tol


@pytest.mark.parametrize("precision,tol", [(fl.PREC_FP64, TOL_F64), (fl.PREC_EMU, TOL_EMU)])
def test_hs_lmax12_longest_operand_reduction(precision, tol):
    # lmax 12: 2 N_L = 338 rows of C^H, the H operand product's reduction padded
    # to 384 terms, the most that one exact FP32 accumulation per slice level
    # allows; 3 atoms in 2 (slot, type) combinations, one of them shared
    p = inputs.small(13, n_atoms=3, n_types=2, lmax=12, n_target=(230,))
    p.atom_slot = np.array([0, 1, 0], dtype=np.int32)
    h, Hs, Ss, _ = run_hs(p, precision, operands=fl.OPERANDS_FACTORED)
    Ho, So = oracle_hs(p)
    ng = Ho.shape[0]
    assert herm_relerr(lower_to_full(Hs[0], ng, 0), Ho) <= tol
    assert herm_relerr(lower_to_full(Ss[0], ng, 0), So) <= tol


@pytest.mark.parametrize("layout", [fl.LAYOUT_LOWER_FULL, fl.LAYOUT_LOWER_PACKED])
def test_hs_split_last_wave_full_parity(layout):
    # N_G ~1600: more 256 x 64 tiles than co-resident CTA pairs, so the
    # partly empty last wave is split into K parts over several pairs
    p = inputs.small(17, n_atoms=2, n_types=2, lmax=3, n_target=(1600,))
    h, Hs, Ss, _ = run_hs(p, fl.PREC_EMU, layout=layout, operands=fl.OPERANDS_FACTORED)
    Ho, So = oracle_hs(p)
    ng = Ho.shape[0]
    assert herm_relerr(lower_to_full(Hs[0], ng, layout), Ho) <= TOL_EMU
    assert herm_relerr(lower_to_full(Ss[0], ng, layout), So) <= TOL_EMU


def test_hs_hpd_T_has_no_negative_rows():
    p = inputs.small(11, n_atoms=2, n_types=2, lmax=3, n_target=(260,), hpd=True)
    h, Hs, Ss, _ = run_hs(p, fl.PREC_EMU)
    assert h.stats()["n_neg"] == 0
    Ho, So = oracle_hs(p)
    assert herm_relerr(lower_to_full(Hs[0], Ho.shape[0], 0), Ho) <= TOL_EMU


def test_upper_triangle_untouched():
    p = inputs.config1()
    torch = torch_cuda()
    h = fl.from_problem(p, fl.default_options(precision=fl.PREC_EMU))
    _, A, B = run_ab(p, h)
    ng = h.num_g(0)
    H = torch.full((ng * ng,), 7.0 + 3.0j, dtype=torch.complex128, device="cuda")
    S = torch.full((ng * ng,), 7.0 + 3.0j, dtype=torch.complex128, device="cuda")
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
    h.sync()
    M = H.cpu().numpy().reshape(ng, ng).T  # [row][col]
    assert np.all(M[np.triu_indices(ng, 1)] == 7.0 + 3.0j)


# --------------------------------------------- the contraction step alone

@pytest.mark.parametrize("precision", [fl.PREC_FP64, fl.PREC_EMU])
@pytest.mark.parametrize("K,N", [(1, 1), (37, 200), (1000, 129), (2100, 321)])
def test_herk_step_vs_numpy(precision, K, N):
    torch = torch_cuda()
    rng = np.random.default_rng(K * 1000 + N)
    Z = rng.normal(size=(K, N)) + 1j * rng.normal(size=(K, N))
    Z *= np.exp(rng.uniform(-3, 3, size=(1, N)))          # uneven column scales
    sig = np.where(rng.uniform(size=K) < 0.2, -1, 1).astype(np.int32)
    h = fl.engine_create(fl.default_options(precision=precision))
    Zd = torch.from_numpy(np.asfortranarray(Z).ravel(order="F")).cuda()
    H = alloc_out(N, 0)
    h.herk(Zd, K, K, N, sig, H, N)
    h.sync()
    R = oracle.herk_lower(Z, sig)
    tol = TOL_EMU if precision == fl.PREC_EMU else TOL_F64
    assert herm_relerr(lower_to_full(H, N, 0), R) <= tol


@pytest.mark.parametrize("K", [64, 1024, 1025, 2049, 4096, 4097, 9000])
def test_herk_integer_data_bit_exact(K):
    """Entries m/128 with |m| <= 127: the leading slice carries them exactly,
    so the emulated product must equal the exact (integer-valued) sum bit for
    bit, with leading digits near their largest (exactness of the FP32
    tensor-core accumulation over 1024 terms of up to 2^14 and of the drain)."""
    torch = torch_cuda()
    N = 192
    rng = np.random.default_rng(K)
    M = rng.integers(-127, 128, size=(K, N)) + 1j * rng.integers(-127, 128, size=(K, N))
    M[:, :3] = 127 + 127j                                   # saturate some columns
    M[0, :] = 127 + 127j                                    # and make every row max reach 127/128
    Z = M / 128.0
    h = fl.engine_create(fl.default_options(precision=fl.PREC_EMU, n_slices=4))
    Zd = torch.from_numpy(np.asfortranarray(Z).ravel(order="F")).cuda()
    H = alloc_out(N, 0)
    h.herk(Zd, K, K, N, None, H, N)
    h.sync()
    R = (M.conj().T @ M) / 16384.0                          # exact in FP64 (integers < 2^53)
    G = lower_to_full(H, N, 0)
    assert np.array_equal(np.tril(G), np.tril(R))


# ------------------------------------------------ larger configs, sampled

@pytest.mark.parametrize("precision,tol", [(fl.PREC_FP64, TOL_F64), (fl.PREC_EMU, TOL_EMU)])
@pytest.mark.parametrize("operands", [fl.OPERANDS_FROM_AB, fl.OPERANDS_FACTORED])
def test_hs_config2_sampled_columns(precision, tol, operands):
    # the factored emulated case is the configuration bench.py times
    p = inputs.config2()
    h, Hs, Ss, _ = run_hs(p, precision, operands=operands)
    n3 = h.gvectors(0)
    ng = len(n3)
    cols = [0, 1, 63, 64, 127, 128, 1000, 2047, ng - 65, ng - 1]
    Ho, So = oracle.hs_columns(p, 0, n3, cols)
    Hg = columns_from_lower(Hs[0], ng, 0, cols)
    Sg = columns_from_lower(Ss[0], ng, 0, cols)
    eh = np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho)
    es = np.linalg.norm(Sg - So) / np.linalg.norm(So)
    assert eh <= tol and es <= tol, (eh, es)


# --------------------------------------------- options: autotune, graph, host buffers

def test_autotune_keeps_results_and_picks_a_configuration():
    p = inputs.config1()
    opt = fl.default_options(precision=fl.PREC_EMU)
    opt.autotune = 1
    h = fl.from_problem(p, opt)
    _, A, B = run_ab(p, h)
    ng = h.num_g(0)
    H, S = alloc_out(ng, 0), alloc_out(ng, 0)
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
    h.sync()
    st = h.stats()
    assert 0 <= st["tile_order"] <= 5 and st["tile_cover"] in (1, 2) and st["pipeline"] in (1, 2)
    Ho, So = oracle_hs(p)
    assert herm_relerr(lower_to_full(H, ng, 0), Ho) <= TOL_EMU
    assert herm_relerr(lower_to_full(S, ng, 0), So) <= TOL_EMU
    # the next call runs with the tuned choice, and gives the same results
    H2, S2 = alloc_out(ng, 0), alloc_out(ng, 0)
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H2], [S2])
    h.sync()
    st2 = h.stats()
    assert (st2["tile_order"], st2["tile_cover"], st2["pipeline"]) == \
        (st["tile_order"], st["tile_cover"], st["pipeline"])
    assert herm_relerr(lower_to_full(H2, ng, 0), Ho) <= TOL_EMU


AUTOTUNE_CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs
p = inputs.small(int(sys.argv[2]), n_atoms=2, n_types=1, lmax=3, n_target=(int(sys.argv[3]),))
opt = fl.default_options(precision=fl.PREC_EMU, operands=fl.OPERANDS_FACTORED)
opt.autotune = 1
h = fl.from_problem(p, opt)
A = torch.zeros(h.ab_offset(1), dtype=torch.complex128, device="cuda")
B = torch.zeros_like(A)
h.build_AB(p.radial, A, B)
ng = h.num_g(0)
H = torch.zeros(ng * ng, dtype=torch.complex128, device="cuda")
S = torch.zeros_like(H)
h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
h.sync()
st = h.stats()
print(json.dumps([st["tile_cover"], st["tile_order"], st["pipeline"]]))
"""


def test_autotune_cache_file(tmp_path):
    # FLAPW_AUTOTUNE_CACHE: a fresh process tunes a new shape and appends one
    # line; another process with the same shape reads the choice back (no new
    # line); a new shape appends a second line
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    env = dict(os.environ, FLAPW_AUTOTUNE_CACHE=str(cache))
    child = tmp_path / "child.py"
    child.write_text(AUTOTUNE_CHILD)

    def run(seed, ng):
        r = subprocess.run([sys.executable, str(child), root, str(seed), str(ng)], env=env,
                           capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        return json.loads(r.stdout.strip().splitlines()[-1])

    c1 = run(5, 700)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1
    key, cover, order, pipe = lines[0].split()
    assert [int(cover), int(order), int(pipe)] == c1
    assert run(5, 700) == c1
    assert len(cache.read_text().splitlines()) == 1
    run(6, 1500)
    assert len(cache.read_text().splitlines()) == 2


@pytest.mark.parametrize("cover", [1, 2])
@pytest.mark.parametrize("order", range(6))
def test_every_tile_order(order, cover):
    # the order only schedules the tiles of a cover; the cyclic cover writes
    # the blocks above a strip's diagonal conjugate-transposed, the aligned one
    # computes 256-row blocks and writes their lower parts: every combination
    # must give the oracle's H and S (2 k-points, ragged N_G, an even and an
    # odd number of 64-row blocks, more row blocks than any band)
    p = inputs.small(19, n_atoms=3, n_types=2, lmax=4, n_target=(2300, 700))
    opt = fl.default_options(precision=fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, tile_order=order + 1,
                             tile_cover=cover)
    h = fl.from_problem(p, opt)
    h, Hs, Ss, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, tile_order=order + 1, h=h,
                          tile_cover=cover)
    st = h.stats()
    assert st["tile_order"] == order and st["tile_cover"] == cover
    for k in range(p.n_k):
        Ho, So = oracle_hs(p, k)
        ng = Ho.shape[0]
        assert herm_relerr(lower_to_full(Hs[k], ng, 0), Ho) <= TOL_EMU, (order, cover, k)
        assert herm_relerr(lower_to_full(Ss[k], ng, 0), So) <= TOL_EMU, (order, cover, k)


@pytest.mark.parametrize("h_method", [fl.H_FACTORED, fl.H_ALG3])
def test_pipeline_shapes_identical(h_method):
    # the 3-stage and the 5-stage load pipelines run the same MMAs and drains:
    # bit-identical H and S (the 5-stage one is the default above N_G 8192)
    p = inputs.small(23, n_atoms=3, n_types=2, lmax=5, n_target=(1500, 333))
    h, H1, S1, AB = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, h_method=h_method,
                           pipeline=1)
    H1 = [x.clone() for x in H1]
    S1 = [x.clone() for x in S1]
    _, H2, S2, _ = run_hs(p, fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, h_method=h_method,
                          pipeline=2, h=h, AB=AB)
    for k in range(p.n_k):
        ng = h.num_g(k)
        assert np.array_equal(lower_to_full(H1[k], ng, 0), lower_to_full(H2[k], ng, 0)), k
        assert np.array_equal(lower_to_full(S1[k], ng, 0), lower_to_full(S2[k], ng, 0)), k
        Ho, So = oracle_hs(p, k)
        assert herm_relerr(lower_to_full(H2[k], ng, 0), Ho) <= TOL_EMU
        assert herm_relerr(lower_to_full(S2[k], ng, 0), So) <= TOL_EMU


@pytest.mark.parametrize("precision", [fl.PREC_FP64, fl.PREC_EMU])
def test_graph_replay_matches(precision):
    p = inputs.small(17, n_atoms=2, n_types=2, lmax=3, n_target=(210, 150))
    opt = fl.default_options(precision=precision, use_graph=1)
    h = fl.from_problem(p, opt)
    _, A, B = run_ab(p, h)
    Hs = [alloc_out(h.num_g(k), 0) for k in range(p.n_k)]
    Ss = [alloc_out(h.num_g(k), 0) for k in range(p.n_k)]
    for rep in range(3):
        for X in Hs + Ss:
            X.zero_()
        h.build_HS(p.T, p.atom_slot, p.U, A, B, Hs, Ss)
        h.sync()
    assert h.stats()["graph_replays"] >= 2
    tol = TOL_EMU if precision == fl.PREC_EMU else TOL_F64
    for k in range(p.n_k):
        Ho, So = oracle_hs(p, k)
        ng = Ho.shape[0]
        assert herm_relerr(lower_to_full(Hs[k], ng, 0), Ho) <= tol
        assert herm_relerr(lower_to_full(Ss[k], ng, 0), So) <= tol


@pytest.mark.parametrize("precision", [fl.PREC_FP64, fl.PREC_EMU])
def test_back_to_back_build_hs_with_different_T(precision):
    # build_HS returns after enqueueing: two calls with different T blocks on
    # one handle and no synchronisation between them (the second stages its T
    # in the other pinned slot while the first call's work runs); both must give
    # their own oracle's H and S
    import copy
    p = inputs.small(29, n_atoms=3, n_types=2, lmax=4, n_target=(900, 420))
    p2 = copy.deepcopy(p)
    rng = np.random.default_rng(7)
    n = p.T.shape[1]
    for t in range(p2.T.shape[0]):
        X = rng.uniform(-1, 1, (n, n)) + 1j * rng.uniform(-1, 1, (n, n))
        p2.T[t] = p2.T[t] + 0.05 * (X + X.conj().T)
    opt = fl.default_options(precision=precision, operands=fl.OPERANDS_FACTORED)
    h = fl.from_problem(p, opt)
    _, A, B = run_ab(p, h)
    out = []
    for q in (p, p2):
        Hs = [alloc_out(h.num_g(k), 0) for k in range(q.n_k)]
        Ss = [alloc_out(h.num_g(k), 0) for k in range(q.n_k)]
        h.build_HS(q.T, q.atom_slot, q.U, A, B, Hs, Ss)
        out.append((q, Hs, Ss))
    h.sync()
    tol = TOL_EMU if precision == fl.PREC_EMU else TOL_F64
    for q, Hs, Ss in out:
        for k in range(q.n_k):
            Ho, So = oracle_hs(q, k)
            ng = Ho.shape[0]
            assert herm_relerr(lower_to_full(Hs[k], ng, 0), Ho) <= tol
            assert herm_relerr(lower_to_full(Ss[k], ng, 0), So) <= tol


def test_host_buffers_through_the_abi():
    torch = torch_cuda()
    p = inputs.config1()
    h = fl.from_problem(p, fl.default_options(precision=fl.PREC_EMU))
    n = h.ab_offset(p.n_k)
    A = torch.zeros(n, dtype=torch.complex128).pin_memory()
    B = torch.zeros(n, dtype=torch.complex128).pin_memory()
    h.build_AB(p.radial, A, B)
    ng = h.num_g(0)
    H = np.zeros(ng * ng, dtype=np.complex128)     # pageable host memory
    S = torch.zeros(ng * ng, dtype=torch.complex128).pin_memory()
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
    h.sync()
    Ao, _ = oracle.build_ab(p, 0, h.gvectors(0))
    assert np.abs(A.numpy().reshape(p.n_atoms, p.n_L, ng) - Ao).max() <= 1e-13 * np.abs(Ao).max()
    Ho, So = oracle_hs(p)
    assert herm_relerr(lower_to_full(H, ng, 0), Ho) <= TOL_EMU
    assert herm_relerr(lower_to_full(S, ng, 0), So) <= TOL_EMU


def _nan_outputs(torch, h, p, layout, memory):
    Hs, Ss = [], []
    for k in range(p.n_k):
        ng = h.num_g(k)
        n = ng * (ng + 1) // 2 if layout == fl.LAYOUT_LOWER_PACKED else ng * ng
        for lst in (Hs, Ss):
            if memory == "pinned":
                lst.append(torch.full((n,), float("nan"), dtype=torch.complex128).pin_memory())
            else:
                lst.append(np.full(n, np.nan, dtype=np.complex128))
    return Hs, Ss


def _host(x):
    return x.numpy() if hasattr(x, "numpy") else x


@pytest.mark.parametrize("memory", ["pinned", "pageable"])
@pytest.mark.parametrize("layout", [fl.LAYOUT_LOWER_FULL, fl.LAYOUT_LOWER_PACKED])
@pytest.mark.parametrize("precision,tol", [(fl.PREC_EMU, TOL_EMU), (fl.PREC_FP64, TOL_F64)])
def test_host_outputs_every_lower_element_copied(layout, precision, tol, memory):
    # host outputs (pinned or pageable) filled with NaN must receive every
    # lower element of every k-point (ragged N_G, one N_G above 64 x 32 so that
    # the column blocks are wider than 64), both precisions: staged on the
    # device and copied back in column blocks, H contracted in two launches
    # split by column
    torch = torch_cuda()
    p = inputs.small(88, n_atoms=3, n_types=2, lmax=3, n_target=(2100, 150, 65))
    h = fl.from_problem(p, fl.default_options(precision=precision, layout=layout,
                                              operands=fl.OPERANDS_FACTORED))
    _, A, B = run_ab(p, h)
    Hs, Ss = _nan_outputs(torch, h, p, layout, memory)
    h.build_HS(p.T, p.atom_slot, p.U, A, B, Hs, Ss)
    h.sync()
    for k in range(p.n_k):
        Ho, So = oracle_hs(p, k)
        ng = Ho.shape[0]
        assert herm_relerr(lower_to_full(Hs[k], ng, layout), Ho) <= tol, k
        assert herm_relerr(lower_to_full(Ss[k], ng, layout), So) <= tol, k
    # the library's count of what reached host memory: every lower element,
    # and with block copies of the full layout at most one block-sized
    # triangle per block more
    st = h.stats()
    lower = 2 * 16 * sum(h.num_g(k) * (h.num_g(k) + 1) // 2 for k in range(p.n_k))
    if layout == fl.LAYOUT_LOWER_PACKED:
        assert st["bytes_d2h"] == lower
    else:
        assert lower < st["bytes_d2h"] <= 1.25 * lower
    assert 2 * p.n_k <= st["copy_ops"] <= 320 + p.n_k


@pytest.mark.parametrize("memory", ["pinned", "pageable"])
def test_many_host_outputs(memory):
    # 48 k-points into host memory (pinned or pageable) in one call: the
    # column blocks widen (5 per matrix instead of 32) so that the call
    # enqueues at most ~320 copies and returns before they run (the device's
    # work queue holds about a thousand operations); every lower element must
    # still arrive
    torch = torch_cuda()
    sizes = tuple(300 + 37 * (i % 11) for i in range(48))
    p = inputs.small(91, n_atoms=2, n_types=2, lmax=2, n_target=sizes)
    h = fl.from_problem(p, fl.default_options(precision=fl.PREC_EMU, operands=fl.OPERANDS_FACTORED))
    _, A, B = run_ab(p, h)
    Hs, Ss = _nan_outputs(torch, h, p, fl.LAYOUT_LOWER_FULL, memory)
    h.build_HS(p.T, p.atom_slot, p.U, A, B, Hs, Ss)
    h.sync()
    st = h.stats()
    lower = 2 * 16 * sum(h.num_g(k) * (h.num_g(k) + 1) // 2 for k in range(p.n_k))
    assert st["copy_ops"] <= 320 + p.n_k, st["copy_ops"]
    assert lower < st["bytes_d2h"] <= 1.6 * lower
    for k in (0, 1, 17, 46, 47):
        Ho, So = oracle_hs(p, k)
        ng = Ho.shape[0]
        assert herm_relerr(lower_to_full(Hs[k], ng, 0), Ho) <= TOL_EMU, k
        assert herm_relerr(lower_to_full(Ss[k], ng, 0), So) <= TOL_EMU, k
    for k in range(p.n_k):
        ng = h.num_g(k)
        L = np.tril(np.ones((ng, ng), dtype=bool))
        for X in (Hs[k], Ss[k]):
            assert not np.isnan(_host(X).reshape(ng, ng).T[L]).any(), k


def test_bad_calls_return_codes_not_faults():
    p = inputs.config1()
    h = fl.from_problem(p)
    with pytest.raises(fl.FlapwError) as e:
        h.build_HS(p.T, [0, 7], p.U, None, None, [None], [None])
    assert e.value.code == -1
    opt = fl.default_options(operands=fl.OPERANDS_FACTORED)
    h2 = fl.from_problem(p, opt)
    ng = h2.num_g(0)
    with pytest.raises(fl.FlapwError) as e:
        h2.build_HS(p.T, p.atom_slot, p.U, None, None, [alloc_out(ng, 0)], [alloc_out(ng, 0)])
    assert e.value.code == -6          # factored operands need build_AB's radial data first
    eng = fl.engine_create()
    with pytest.raises(fl.FlapwError) as e:
        eng.num_g(0)
    assert e.value.code == -6


# ------------------------------------------- full-size workloads, sampled columns

def _sampled_check(p, Hs, Ss, h, layout, ks, tol, n_cols=6, seed=0):
    rng = np.random.default_rng(seed)
    for k in ks:
        n3 = h.gvectors(k)
        ng = len(n3)
        cols = np.unique(np.concatenate([[0, ng - 1], rng.integers(0, ng, size=n_cols - 2)]))
        Ho, So = oracle.hs_columns(p, k, n3, cols)
        Hg = columns_from_lower(Hs[k], ng, layout, cols)
        Sg = columns_from_lower(Ss[k], ng, layout, cols)
        eh = np.linalg.norm(Hg - Ho) / np.linalg.norm(Ho)
        es = np.linalg.norm(Sg - So) / np.linalg.norm(So)
        assert eh <= tol and es <= tol, (k, eh, es)


@pytest.mark.parametrize("precision,tol", [(fl.PREC_EMU, TOL_EMU), (fl.PREC_FP64, TOL_F64)])
def test_config3_sampled(precision, tol):
    p = inputs.config3()
    h, Hs, Ss, _ = run_hs(p, precision, operands=fl.OPERANDS_FACTORED)
    _sampled_check(p, Hs, Ss, h, fl.LAYOUT_LOWER_FULL, [0], tol, n_cols=32)


@pytest.mark.parametrize("precision,tol", [(fl.PREC_EMU, TOL_EMU), (fl.PREC_FP64, TOL_F64)])
def test_config4_batched_32k_sampled(precision, tol):
    p = inputs.config4()
    h, Hs, Ss, _ = run_hs(p, precision, operands=fl.OPERANDS_FACTORED, use_graph=1)
    ngs = [h.num_g(k) for k in range(p.n_k)]
    assert min(ngs) >= 2500 and max(ngs) <= 6000 and len(set(ngs)) > 20
    _sampled_check(p, Hs, Ss, h, fl.LAYOUT_LOWER_FULL, list(range(p.n_k)), tol, n_cols=2)


def test_config5_packed_sampled():
    torch = torch_cuda()
    p = inputs.config5()
    h, Hs, Ss, _ = run_hs(p, fl.PREC_EMU, layout=fl.LAYOUT_LOWER_PACKED,
                          operands=fl.OPERANDS_FACTORED)
    ng = h.num_g(0)
    assert Hs[0].numel() == ng * (ng + 1) // 2
    _sampled_check(p, Hs, Ss, h, fl.LAYOUT_LOWER_PACKED, [0], TOL_EMU, n_cols=32)
    del Hs, Ss
    torch.cuda.empty_cache()


def test_config5_fp64_tile_subset():
    # the FP64 path on config 5 would take hours; part 0 of 4096 parts (every
    # 4096th 64 x 64 tile, the tile split of the job partition) computes 17
    # blocks of each lower triangle, compared element by element with the
    # oracle on one column of each of four blocks
    torch = torch_cuda()
    p = inputs.config5()
    parts = 4096
    opt = fl.default_options(precision=fl.PREC_FP64, layout=fl.LAYOUT_LOWER_PACKED,
                             operands=fl.OPERANDS_FACTORED, part_count=parts, part_index=0)
    h = fl.from_problem(p, opt)
    _, A, B = run_ab(p, h)
    del A, B
    ng = h.num_g(0)
    H, S = alloc_out(ng, fl.LAYOUT_LOWER_PACKED), alloc_out(ng, fl.LAYOUT_LOWER_PACKED)
    h.build_HS(p.T, p.atom_slot, p.U, None, None, [H], [S])
    h.sync()
    nb = (ng + 63) // 64
    blocks = [(ib, jb) for ib in range(nb) for jb in range(ib + 1)][::parts]   # part 0's tiles
    assert len(blocks) >= 17
    pick = [blocks[i] for i in (0, 5, 11, len(blocks) - 1)]
    n3 = h.gvectors(0)
    cols = [jb * 64 + 7 for ib, jb in pick]
    Ho, So = oracle.hs_columns(p, 0, n3, cols)
    Hg = columns_from_lower(H, ng, fl.LAYOUT_LOWER_PACKED, cols)
    Sg = columns_from_lower(S, ng, fl.LAYOUT_LOWER_PACKED, cols)
    for X, R in ((Hg, Ho), (Sg, So)):
        got = np.concatenate([X[c, ib * 64:min(ng, ib * 64 + 64)] for c, (ib, jb) in enumerate(pick)])
        ref = np.concatenate([R[c, ib * 64:min(ng, ib * 64 + 64)] for c, (ib, jb) in enumerate(pick)])
        assert np.linalg.norm(got - ref) <= TOL_F64 * np.linalg.norm(ref)
    del H, S
    h.destroy()
    torch.cuda.empty_cache()
