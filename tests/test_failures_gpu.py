"""Failure paths of the library, made in the allowed forms: a device wait
that runs out because its bound is set to microseconds, and a device-memory
cap that makes a call fail with FLAPW_ERR_OOM.  No GPU fault is made: the
bounded waits stop the tensor-core kernels cleanly (the pair lets its copies
and MMAs finish, frees TMEM and exits) and the cap refuses allocations on
the host.  After each failure the same handle must give the oracle's H and S
(the factorisation may fail too, Sec. 3, Alg. 1, and the paper's dynamic
hybrid scheme runs out of memory on its largest case, Sec. 6: the library
reports both kinds of failure and stays usable)."""
import numpy as np
import pytest

import oracle
import paper_1712_07206_gb300 as fl
from paper_1712_07206_gb300 import inputs

from helpers import TOL_EMU, alloc_out, columns_from_lower, run_ab, torch_cuda

pytestmark = pytest.mark.gpu


def _sampled_parity(p, h, H, S):
    n3 = h.gvectors(0)
    ng = len(n3)
    cols = [0, 1, 64, 1000, ng - 1]
    Ho, So = oracle.hs_columns(p, 0, n3, cols)
    eh = np.linalg.norm(columns_from_lower(H, ng, 0, cols) - Ho) / np.linalg.norm(Ho)
    es = np.linalg.norm(columns_from_lower(S, ng, 0, cols) - So) / np.linalg.norm(So)
    assert eh <= TOL_EMU and es <= TOL_EMU, (eh, es)


def test_wait_bound_runs_out_then_the_handle_recovers():
    torch = torch_cuda()
    fl.build()
    p = inputs.config2()
    opt = fl.default_options(precision=fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, wait_us=1)
    h = fl.from_problem(p, opt)
    _, A, B = run_ab(p, h)
    ng = h.num_g(0)
    H, S = alloc_out(ng, 0), alloc_out(ng, 0)
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])     # enqueued: the failure is on the device
    with pytest.raises(fl.FlapwError) as e:
        h.sync()
    assert e.value.code == -5, e.value
    torch.cuda.synchronize()                              # nothing is left waiting
    # the default bound on the same handle: the oracle's results
    h.set_options(fl.default_options(precision=fl.PREC_EMU, operands=fl.OPERANDS_FACTORED))
    H.zero_()
    S.zero_()
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
    h.sync()
    _sampled_parity(p, h, H, S)
    h.destroy()


def test_memory_cap_gives_oom_then_the_handle_recovers():
    torch = torch_cuda()
    fl.build()
    p = inputs.config2()
    cap = fl.default_options(precision=fl.PREC_EMU, operands=fl.OPERANDS_FACTORED, mem_cap_mb=64)
    h = fl.from_problem(p, cap)
    _, A, B = run_ab(p, h)                                # A/B tables: a few MB, under the cap
    ng = h.num_g(0)
    H, S = alloc_out(ng, 0), alloc_out(ng, 0)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free_before = torch.cuda.mem_get_info()[0]
    # the slices alone are ~0.3 GB: refused before anything is enqueued
    with pytest.raises(fl.FlapwError) as e:
        h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
    assert e.value.code == -3, e.value
    assert float(H.abs().max()) == 0.0
    # a larger cap on the same handle proceeds
    h.set_options(fl.default_options(precision=fl.PREC_EMU, operands=fl.OPERANDS_FACTORED))
    h.build_HS(p.T, p.atom_slot, p.U, A, B, [H], [S])
    h.sync()
    _sampled_parity(p, h, H, S)
    # every workspace stays owned by the handle and goes back at destroy (torch's
    # own temporaries released too; a few MB for kernel code loaded on first use)
    h.destroy()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    assert torch.cuda.mem_get_info()[0] >= free_before - (16 << 20)
