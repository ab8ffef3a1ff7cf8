"""Host-side checks of the C ABI: the library builds and loads without a GPU,
exports every function include/pfm.h declares, and rejects malformed input
before touching the device."""
import json
import os
import re
import subprocess

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pfm():
    import paper_1501_07844_gb300 as pfm
    pfm.lib()
    return pfm


def declared_functions():
    text = open(os.path.join(ROOT, "include", "pfm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pfm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(pfm):
    names = declared_functions()
    assert len(names) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", pfm.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b[TW] (pfm_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # nothing but the C ABI is exported
    assert all(e.startswith("pfm_") for e in re.findall(r"\bT (\w+)", out) if not e.startswith("_"))


def test_version_and_defaults(pfm):
    L = pfm.lib()
    assert L.pfm_version() == 1
    p = pfm.binding.params()
    assert (p.c, p.tau, p.norm, p.grad_source, p.storage, p.schedule, p.check_every, p.gap_tol) == \
        (0.5, 0.11, 0, 0, 0, 0, 10, 1e-4)


def test_footprint_counts(pfm):
    nn, edges = synth.hmf_tree(3, 4)
    nb, nbuf, nl = pfm.binding.footprint((8, 8, 8), nn, edges, has_S_field=False, schedule=pfm.INPLACE)
    assert nl == 12
    assert nbuf == 12 * (1 + 1) + 15 * 3            # u + D per leaf, 3 flow components per node
    assert nb == 4 * 512 * nbuf
    nb2, nbuf2, _ = pfm.binding.footprint((8, 8, 8), nn, edges, schedule=pfm.FUSED)
    assert nbuf2 == 12 * 3 + 15 * 6                 # double-buffered u and q
    nb3, _, _ = pfm.binding.footprint((8, 8, 8), nn, edges, schedule=pfm.FUSED, storage=pfm.BF16)
    assert nb3 == 2 * 512 * (12 * 2 + 15 * 6) + 4 * 512 * 12


def test_in_place_buffers_within_paper_counts(pfm):
    """The paper's pseudo-flow counts (Section 3.3: 5 per end-label, 4 per
    inner node, 1 accumulator; Section 3.1: 4 for the binary model) bound
    what the in-place schedule allocates for 3-D problems (the excess d and
    the accumulator stay on chip)."""
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_buffer_counts.json")))
    dg = g["dagmf"]
    rng = np.random.default_rng(0)
    for _ in range(5):
        nn, edges = synth.random_dag(rng, 4, 10, 2)
        nl = nn - 4
        _, nbuf, _ = pfm.binding.footprint((4, 4, 4), nn, edges, schedule=pfm.INPLACE)
        paper = dg["pseudo_flow_per_end_label"] * nl + dg["pseudo_flow_per_inner_node"] * (nn - nl) + dg["pseudo_flow_extra"]
        full = dg["full_flow_per_end_label"] * nl + dg["full_flow_per_inner_node"] * (nn - nl) + dg["full_flow_extra"]
        assert nbuf <= paper < full
    # binary model in 2-D: u, D and two flow components per label -> 2 labels; the paper's
    # binary pseudo-flow stores one labelling, one flow field pair and the two data terms
    _, nbuf2, _ = pfm.binding.footprint((4, 4), 2, [(-1, 0, 1.0), (-1, 1, 1.0)], schedule=pfm.INPLACE)
    assert nbuf2 == 8


@pytest.mark.parametrize("edges,n", [
    ([(-1, 0, 1.0), (0, 1, 1.0), (1, 0, 1.0)], 2),        # cycle
    ([(-1, 0, 1.0)], 2),                                   # node without parent
    ([(-1, 0, 1.0), (0, 7, 1.0)], 2),                      # index out of range
    ([(-1, 0, 1.0), (-1, 1, 0.0)], 2),                     # non-positive weight
    ([(-1, 0, 1.0), (0, 1, 0.5), (0, 2, 1.0)], 3),         # W_(S,leaf) = 0.5
])
def test_malformed_dag_rejected_on_host(pfm, edges, n):
    with pytest.raises(pfm.PfmError) as ei:
        pfm.binding.footprint((4, 4), n, edges)
    assert ei.value.name == "PFM_EDAG"


def test_bad_params_rejected_on_host(pfm):
    for kw in ({"c": 0.0}, {"tau": -1.0}, {"norm": 5}, {"storage": 9}, {"schedule": 3}, {"check_every": 0}):
        with pytest.raises(pfm.PfmError) as ei:
            pfm.binding.footprint((4, 4), 2, [(-1, 0, 1.0), (-1, 1, 1.0)], **kw)
        assert ei.value.name == "PFM_EINVAL"
    with pytest.raises(pfm.PfmError) as ei:
        pfm.binding.footprint((4, 4), 17, [(-1, L, 1.0) for L in range(17)])
    assert ei.value.name == "PFM_EUNSUPPORTED"
    with pytest.raises(pfm.PfmError):
        pfm.binding.footprint((4, 4), 2, [(-1, 0, 1.0), (-1, 1, 1.0)], s_node=[0.1, -0.2])


def test_create_validates_before_device_work(pfm):
    """A malformed problem is rejected by pfm_create on a machine without a GPU."""
    D = np.zeros((2, 4, 4), dtype=np.float32)
    with pytest.raises(pfm.PfmError) as ei:
        pfm.Problem(D, n_nodes=2, edges=[(-1, 0, 1.0), (0, 1, 1.0), (1, 0, 1.0)])
    assert ei.value.name == "PFM_EDAG"


def test_null_handles_rejected_on_host(pfm):
    """Entry points on a NULL problem or batch return PFM_EINVAL (or -1 for
    the counters) without touching the device."""
    import ctypes as C
    L = pfm.lib()
    zc = C.c_int(-7)
    assert L.pfm_tune(None, 3, C.byref(zc)) == 1 and zc.value == -7
    assert L.pfm_adjoint_steps(None, 2, None, None, None, None, None, None, None) == 1
    assert L.pfm_set_chunk_length(None, 8) == 1
    assert L.pfm_chunk_length(None) == -1
    assert L.pfm_iterate(None, 1) == 1
    assert L.pfm_iterations_done(None) == -1 and L.pfm_launch_count(None) == -1
    assert L.pfm_batch_launch_count(None) == -1
    E, P = C.c_double(), C.c_double()
    assert L.pfm_energy(None, C.byref(E), C.byref(P)) == 1
    assert b"NULL" in L.pfm_last_error()
