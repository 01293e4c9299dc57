"""A job split over independent parts (options.part_count / part_index; the
paper's multi-device split, Sec. 5, with k-points and output tiles as the
independent units).  The parts run one after the other on cuda:0, as separate
callers would on separate GPUs (no part waits on another): with several
k-points each part computes whole k-points and leaves the others' outputs
alone (they may be NULL); with one k-point each part computes every P-th tile
and the parts' zero-initialised outputs sum to the oracle's H and S, on the
device and in host memory (where other parts' blocks come back as zeros)."""
import numpy as np
import pytest

import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs

from helpers import TOL_EMU, TOL_F64, alloc_out, herm_relerr, lower_to_full, oracle_hs, run_ab

pytestmark = pytest.mark.gpu


def _run_parts(p, precision, parts, host=False, layout=fl.LAYOUT_LOWER_FULL):
    """Every part on its own handle; returns per part the [H_k], [S_k] lists
    (None for k-points of other parts) and the owner list."""
    owner = fl.partition([fl.enumerate_g(p.lattice, p.k_frac[k], p.kmax[k]).shape[0]
                          for k in range(p.n_k)], parts)
    res = []
    for r in range(parts):
        opt = fl.default_options(precision=precision, operands=fl.OPERANDS_FACTORED, layout=layout,
                                 part_count=parts, part_index=r)
        h = fl.from_problem(p, opt)
        _, A, B = run_ab(p, h)
        mine = [owner[k] < 0 or owner[k] == r for k in range(p.n_k)]
        Hs = [alloc_out(h.num_g(k), layout, host) if mine[k] else None for k in range(p.n_k)]
        Ss = [alloc_out(h.num_g(k), layout, host) if mine[k] else None for k in range(p.n_k)]
        h.build_HS(p.T, p.atom_slot, p.U, A, B, Hs, Ss)
        h.sync()
        res.append((Hs, Ss))
        h.destroy()
    return res, owner


@pytest.mark.parametrize("precision", [fl.PREC_EMU, fl.PREC_FP64])
def test_kpoint_split_two_parts(precision):
    p = inputs.small(31, n_atoms=2, n_types=2, lmax=3, n_target=(700, 650, 420, 380))
    res, owner = _run_parts(p, precision, 2)
    assert sorted(set(owner.tolist())) == [0, 1]          # whole k-points, both parts busy
    tol = TOL_EMU if precision == fl.PREC_EMU else TOL_F64
    for k in range(p.n_k):
        Hs, Ss = res[owner[k]]
        Ho, So = oracle_hs(p, k)
        ng = Ho.shape[0]
        assert herm_relerr(lower_to_full(Hs[k], ng, 0), Ho) <= tol
        assert herm_relerr(lower_to_full(Ss[k], ng, 0), So) <= tol
        other = res[1 - owner[k]][0][k]
        assert other is None


@pytest.mark.parametrize("precision,host,layout", [(fl.PREC_EMU, False, fl.LAYOUT_LOWER_FULL),
                                                  (fl.PREC_EMU, True, fl.LAYOUT_LOWER_FULL),
                                                  (fl.PREC_EMU, False, fl.LAYOUT_LOWER_PACKED),
                                                  (fl.PREC_FP64, False, fl.LAYOUT_LOWER_FULL)])
@pytest.mark.parametrize("parts", [2, 3])
def test_tile_split_parts_sum_to_oracle(precision, host, layout, parts):
    p = inputs.small(33, n_atoms=3, n_types=2, lmax=4, n_target=(1900,))
    res, owner = _run_parts(p, precision, parts, host=host, layout=layout)
    assert owner.tolist() == [-1]                       # one k-point: shared by tiles
    Ho, So = oracle_hs(p, 0)
    ng = Ho.shape[0]
    H = sum(r[0][0].cpu().numpy() for r in res)
    S = sum(r[1][0].cpu().numpy() for r in res)
    tol = TOL_EMU if precision == fl.PREC_EMU else TOL_F64
    assert herm_relerr(lower_to_full(H, ng, layout), Ho) <= tol
    assert herm_relerr(lower_to_full(S, ng, layout), So) <= tol
    # no part computed everything: each leaves blocks to the others
    for r in res:
        assert np.count_nonzero(r[0][0].cpu().numpy()) < 0.9 * ng * (ng + 1) // 2
