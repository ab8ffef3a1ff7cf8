"""The allocation-free energy entry point, pfm_potts_energy_noalloc.

It exists for callers that cannot call cudaMalloc (device memory owned by an
outer allocator that has claimed the budget, or latency-critical loops where
an allocation may synchronise the device).  Its per-block partial sums live
in a fixed device array inside the library.  These tests call it through
the C ABI on buffers the caller already holds and check that two calls in a
row each give what pfm_energy gives for the same state.  This file sorts
last so that a run stopping at its first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from helpers import gpu_problem


def _lib():
    import paper_1501_07844_gb300 as pfm
    return pfm.lib()


def _call(L, prob, u, q, D, S, norm, out, stream):
    spatial = prob.spatial
    ndim = len(spatial)
    dims = (C.c_int64 * 3)(spatial[-1], spatial[-2], spatial[0] if ndim == 3 else 1)
    s_label = None
    if prob.s_node is not None:
        arr = np.ascontiguousarray(prob.s_node, dtype=np.float32)
        s_label = arr.ctypes.data_as(C.POINTER(C.c_float))
    return L.pfm_potts_energy_noalloc(ndim, dims, prob.n_leaf, u.data_ptr(), q.data_ptr(), D.data_ptr(),
                                      None if S is None else S.data_ptr(), s_label, norm, out.data_ptr(),
                                      stream)


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["3d_field_iso", "2d_labels_aniso", "3d_ragged_16"])
def test_noalloc_energy_matches_pfm_energy(case):
    import torch
    if case == "3d_field_iso":
        prob, norm = synth.potts3d_problem(seed=2200, nl=8, shape=(33, 40, 52)), 0
    elif case == "2d_labels_aniso":
        prob, norm = synth.random_problem(2201, (70, 90), nl=5, s_kind="node"), 1
    else:
        prob, norm = synth.random_problem(2202, (9, 17, 23), nl=16, s_kind="both"), 0
    L = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    with gpu_problem(prob, norm=norm, stream=stream) as gp:
        gp.iterate(17)
        E_ref, P_ref = gp.energy()
        u, q = gp.labels(), gp.flows()
    D = torch.from_numpy(prob.D).cuda()
    S = None if prob.S_field is None else torch.from_numpy(prob.S_field).cuda()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        assert _call(L, prob, u, q, D, S, norm, out, stream) == 0, L.pfm_last_error()
        torch.cuda.synchronize()
        E, P = out.tolist()
        assert abs(E - E_ref) <= 1e-6 * abs(E_ref), (E, E_ref)
        assert abs(P - P_ref) <= 1e-6 * abs(P_ref) + 1e-6, (P, P_ref)


@pytest.mark.gpu
def test_noalloc_energy_matches_the_oracle():
    """E and P of a GPU state through the allocation-free entry point against
    the FP64 oracle's E(u) (Eq. potts_original) and P(q) (Eq. potts_pseudo)
    of the same state."""
    import torch
    import oracle
    prob = synth.potts3d_problem(seed=2203, nl=8, shape=(21, 30, 44))
    L = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    with gpu_problem(prob, stream=stream) as gp:
        gp.iterate(25)
        u, q = gp.labels(), gp.flows()
    D = torch.from_numpy(prob.D).cuda()
    S = torch.from_numpy(prob.S_field).cuda()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    assert _call(L, prob, u, q, D, S, 0, out, stream) == 0, L.pfm_last_error()
    torch.cuda.synchronize()
    E, P = out.tolist()
    E_o, P_o = oracle.potts_energy(prob.D.astype(np.float64), u.cpu().numpy().astype(np.float64),
                                   q.cpu().numpy().astype(np.float64), S_field=prob.S_field.astype(np.float64))
    assert abs(E - E_o) <= 1e-6 * abs(E_o) and abs(P - P_o) <= 1e-6 * abs(P_o) + 1e-6, (E, E_o, P, P_o)


@pytest.mark.gpu
def test_noalloc_energy_at_the_largest_accepted_grid():
    """A grid of exactly PFM_NOALLOC_MAX_VOXELS voxels (256^3, two labels):
    every block of the fixed scratch is used, the last partial sits just
    before the flag word; twice in a row, against pfm_energy."""
    import torch
    prob = synth.potts3d_problem(seed=2204, nl=2, shape=(256, 256, 256))
    assert int(np.prod(prob.spatial)) == 16777216
    L = _lib()
    stream = torch.cuda.current_stream().cuda_stream
    with gpu_problem(prob, stream=stream) as gp:
        gp.iterate(5)
        E_ref, P_ref = gp.energy()
        u, q = gp.labels(), gp.flows()
    D = torch.from_numpy(prob.D).cuda()
    S = torch.from_numpy(prob.S_field).cuda()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(float("nan"))
        assert _call(L, prob, u, q, D, S, 0, out, stream) == 0, L.pfm_last_error()
        torch.cuda.synchronize()
        E, P = out.tolist()
        assert abs(E - E_ref) <= 1e-6 * abs(E_ref) and abs(P - P_ref) <= 1e-6 * abs(P_ref) + 1e-6
    del u, q, D, S
    torch.cuda.empty_cache()


def test_noalloc_rejects_grid_beyond_scratch():
    """A grid larger than the fixed scratch allows is refused on the host,
    before any device work (the pointers are never dereferenced)."""
    L = _lib()
    dims = (C.c_int64 * 3)(257, 256, 256)
    fake = C.c_void_p(256)
    st = L.pfm_potts_energy_noalloc(3, dims, 8, fake, fake, fake, None, None, 0, fake, None)
    assert st == 1
    assert b"PFM_NOALLOC_MAX_VOXELS" in L.pfm_last_error()
    dims_ok_labels_bad = (C.c_int64 * 3)(8, 8, 8)
    assert L.pfm_potts_energy_noalloc(3, dims_ok_labels_bad, 17, fake, fake, fake, None, None, 0, fake, None) == 8
