"""The allocation-free FP32 pair sum (ctr_pair_sum_fp32_static) against ctr_ibim_matvec.

Callers that cannot allocate device memory (code running under an allocator
that owns all of the device's memory, or a loop that must not stall on an
allocation) use ctr_pair_sum_fp32_static, whose scratch is a fixed device
array.  Its output must equal the dense pair part of ctr_ibim_matvec's FP32
operator (the matvec minus its diagonal and its correction) within the FP32
operator tolerance of the parity tests, on two calls in a row with different
densities (the second call must not see the first call's scratch), and the
second call must leave the device's free memory unchanged (the first call may
load the library's device code, which brings the fixed array with it).
"""
import ctypes
import math

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


def _pair_part_from_matvec(G, ctr, x, h, kappa, eps_in, eps_out):
    """ctr_ibim_matvec(x) minus Lambda x and minus the correction (from the exported Omega)."""
    M = G.M
    y = G.matvec(x, ctr.FP32_REFINE)
    ptr, node, w = G.corrections()
    _, _, W = G.geometry()
    lam1 = 0.5 * (1 + eps_out / eps_in)
    lam2 = 0.5 * (1 + eps_in / eps_out)
    rows = np.repeat(np.arange(M), np.diff(ptr))
    Wm = W[node]
    c1 = Wm * (h * h * w[0] * x[node] - h ** 3 * w[3] * x[M + node])
    c2 = Wm * (h * h * w[1] * x[node] - h * h * w[2] * x[M + node])
    corr1 = np.bincount(rows, weights=c1, minlength=M)
    corr2 = np.bincount(rows, weights=c2, minlength=M)
    return np.concatenate([y[:M] - lam1 * x[:M] - corr1, y[M:] - lam2 * x[M:] - corr2])


def test_static_scratch_pair_sum_matches_matvec():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03699_gb300 as ctr
    L = ctr.lib
    L.ctr_pair_sum_fp32_static.restype = ctypes.c_int
    L.ctr_pair_sum_fp32_static.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    prob = syn.ellipsoid_problem(h=0.2)
    G = ctr.CtrIbim.from_problem(prob)
    M, h = G.M, prob.grid.h
    P, n, W = G.geometry()
    ptr, node, _ = G.corrections()
    excl = np.concatenate([np.sort(node[ptr[i]:ptr[i + 1]]) for i in range(M)]).astype(np.int32)
    d_ptr = torch.tensor(ptr.astype(np.int32), device="cuda")
    d_excl = torch.tensor(excl, device="cuda")
    scale = h * h * h / (4.0 * math.pi)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    calls = []
    for seed in (21, 22):                       # two calls in a row, different densities
        x = syn.random_density(M, seed=seed, smooth_points=P)
        src = np.empty((M, 8), dtype=np.float32)
        src[:, 0:3] = P
        src[:, 3] = scale * W * x[:M]
        src[:, 4:7] = n
        src[:, 7] = scale * W * x[M:]
        d_src = torch.tensor(src.ravel(), device="cuda")
        out = torch.full((2 * M,), float("nan"), dtype=torch.float64, device="cuda")
        calls.append((x, d_src, out))           # every caller buffer exists before the first call
    torch.cuda.synchronize()
    free = []
    for x, d_src, out in calls:
        st = L.ctr_pair_sum_fp32_static(M, ctypes.c_void_p(d_src.data_ptr()), ctypes.c_void_p(d_ptr.data_ptr()),
                                        ctypes.c_void_p(d_excl.data_ptr()), prob.eps_out / prob.eps_in, prob.kappa,
                                        ctypes.c_void_p(out.data_ptr()), stream)
        assert st == 0, L.ctr_last_error()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    assert free[1] == free[0], f"the second call changed the free device memory by {free[0] - free[1]} bytes"
    for x, d_src, out in calls:
        got = out.cpu().numpy()
        ref = _pair_part_from_matvec(G, ctr, x, h, prob.kappa, prob.eps_in, prob.eps_out)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 2e-5
    # more nodes than the fixed scratch holds is rejected before any device work
    st = L.ctr_pair_sum_fp32_static(2 ** 21, ctypes.c_void_p(d_src.data_ptr()), ctypes.c_void_p(d_ptr.data_ptr()),
                                    ctypes.c_void_p(d_excl.data_ptr()), 80.0, 0.1, ctypes.c_void_p(out.data_ptr()),
                                    stream)
    assert st == -8
    G.close()
