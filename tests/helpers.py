"""Shared helpers of the GPU tests: run the CUDA path, read back outputs and
compare them with the oracle."""
import numpy as np

import oracle
import paper_1712_07206_gb300 as fl

TOL_EMU = 1e-12   # relative Frobenius error bound stated for H and S
TOL_F64 = 1e-13


def torch_cuda():
    import torch
    return torch


def run_ab(p, h=None, stream=None):
    """build_AB on the GPU; returns (handle, A_dev, B_dev)."""
    torch = torch_cuda()
    h = h or fl.from_problem(p)
    total = h.ab_offset(p.n_k)
    A = torch.zeros(total, dtype=torch.complex128, device="cuda")
    B = torch.zeros_like(A)
    h.build_AB(p.radial, A, B, stream)
    return h, A, B


def ab_block(p, h, X, k):
    """[n_atoms][N_L][N_G] view of k-point k's block of an A/B buffer (host numpy)."""
    ng = h.num_g(k)
    o0 = h.ab_offset(k)
    x = X[o0:o0 + p.n_atoms * p.n_L * ng]
    x = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    return x.reshape(p.n_atoms, p.n_L, ng)


def alloc_out(ng, layout, host=False):
    torch = torch_cuda()
    n = ng * (ng + 1) // 2 if layout == fl.LAYOUT_LOWER_PACKED else ng * ng
    if host:
        return torch.zeros(n, dtype=torch.complex128).pin_memory()
    return torch.zeros(n, dtype=torch.complex128, device="cuda")


def run_hs(p, precision, layout=fl.LAYOUT_LOWER_FULL, operands=fl.OPERANDS_FROM_AB, n_slices=7,
           T=None, h=None, AB=None, use_graph=0, tile_order=0, s_method=fl.S_CONTRACTION,
           h_method=fl.H_FACTORED, pipeline=0, tile_cover=0):
    """build_AB + build_HS; returns (handle, [H_k], [S_k]) as device tensors."""
    opt = fl.default_options(precision=precision, layout=layout, operands=operands,
                             n_slices=n_slices, use_graph=use_graph, tile_order=tile_order,
                             s_method=s_method, h_method=h_method, pipeline=pipeline,
                             tile_cover=tile_cover)
    if h is None:
        h = fl.from_problem(p, opt)
    else:
        h.set_options(opt)
    if AB is None:
        _, A, B = run_ab(p, h)
    else:
        A, B = AB
    Hs = [alloc_out(h.num_g(k), layout) for k in range(p.n_k)]
    Ss = [alloc_out(h.num_g(k), layout) for k in range(p.n_k)]
    h.build_HS(p.T if T is None else T, p.atom_slot, p.U, A, B, Hs, Ss)
    h.sync()
    return h, Hs, Ss, (A, B)


def lower_to_full(x, ng, layout):
    """Full Hermitian matrix [G'][G] from the library's lower-triangle output."""
    x = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    if layout == fl.LAYOUT_LOWER_PACKED:
        M = np.zeros((ng, ng), complex)
        o = 0
        for j in range(ng):
            M[j:, j] = x[o:o + ng - j]
            o += ng - j
    else:
        M = x.reshape(ng, ng).T.copy()   # column-major: element (i, j) at j*ng + i
    L = np.tril(M)
    return L + np.tril(L, -1).conj().T


def herm_relerr(X, R):
    """Relative Frobenius error over the full Hermitian matrices."""
    return float(np.linalg.norm(X - R) / np.linalg.norm(R))


def columns_from_lower(x, ng, layout, cols):
    """Full columns cols[c] of the Hermitian matrix, as [len(cols)][ng]."""
    x = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    out = np.zeros((len(cols), ng), complex)

    def at(i, j):  # i >= j
        if layout == fl.LAYOUT_LOWER_PACKED:
            return x[j * ng - j * (j - 1) // 2 + (i - j)]
        return x[j * ng + i]

    for c, g in enumerate(cols):
        i = np.arange(ng)
        lo = i >= g
        if layout == fl.LAYOUT_LOWER_PACKED:
            out[c, lo] = x[g * ng - g * (g - 1) // 2 + (i[lo] - g)]
            hi = i[~lo]
            out[c, ~lo] = np.conj(x[hi * ng - hi * (hi - 1) // 2 + (g - hi)])
        else:
            out[c, lo] = x[g * ng + i[lo]]
            out[c, ~lo] = np.conj(x[i[~lo] * ng + g])
    return out


def oracle_hs(p, k=0):
    n3 = oracle.gvectors(p.lattice, p.k_frac[k], p.kmax[k])
    return oracle.hs_full(p, k, n3)
