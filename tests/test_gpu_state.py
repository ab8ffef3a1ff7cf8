"""Checkpoint / resume through the state blob (pfm_get_state /
pfm_set_state): a problem restored from a blob continues bit for bit as the
saved one would have, iteration counter and step parameters included."""
import numpy as np
import pytest

import synth
from helpers import gpu_problem

pytestmark = pytest.mark.gpu


def _cases():
    return [
        ("potts3d_f32", synth.random_problem(6100, (11, 20, 45), nl=5, s_kind="both"), dict()),
        ("potts3d_bf16", synth.random_problem(6101, (9, 17, 38), nl=4, s_kind="field"), dict(storage=1)),
        ("hmf3d_f16", synth.hmf_problem(seed=6106, shape=(7, 9, 29)), dict(storage=2)),
        ("potts2d_literal", synth.random_problem(6102, (23, 37), nl=3, s_kind="node"), dict(grad_source=1)),
        ("potts3d_inplace", synth.random_problem(6103, (10, 16, 33), nl=8, s_kind="field"), dict(schedule=1)),
        ("hmf3d", synth.hmf_problem(seed=6104, shape=(9, 12, 34)), dict()),
        ("ishikawa3d", synth.ishikawa_problem(6105, (8, 12, 40), nlev=5), dict()),
    ]


@pytest.mark.parametrize("idx", range(7), ids=[c[0] for c in _cases()])
@pytest.mark.parametrize("where", ["host", "device"])
def test_resume_is_bitwise(idx, where):
    import torch
    name, prob, kw = _cases()[idx]
    with gpu_problem(prob, **kw) as a:
        a.iterate(7)
        a.set_step(0.35, 0.12)                    # a continuation step before the save
        a.iterate(2)
        if where == "host":
            blob = a.get_state()
        else:
            blob = torch.empty(a.state_size(), dtype=torch.uint8, device="cuda")
            a.get_state(out=blob)
        a.iterate(6)
        ua, qa, it_a = a.labels().cpu().numpy(), a.flows().cpu().numpy(), a.iterations
        Ea = a.energy()
    with gpu_problem(prob, **kw) as b:
        b.iterate(3)                              # a state that the import replaces
        b.set_state(blob)
        assert b.iterations == 9
        b.iterate(6)
        assert b.iterations == it_a == 15
        assert np.array_equal(b.labels().cpu().numpy(), ua), name
        assert np.array_equal(b.flows().cpu().numpy(), qa), name
        assert b.energy() == Ea


def test_state_blob_layout_and_rejections():
    import paper_1501_07844_gb300 as pfm
    prob = synth.random_problem(6200, (6, 10, 17), nl=3, s_kind="field")
    with gpu_problem(prob) as a:
        a.iterate(4)
        blob = a.get_state()
        n = 6 * 10 * 17
        assert blob.nbytes == 128 + 4 * (3 * n + 3 * 3 * n)
        assert bytes(blob[:8]) == b"PFMSTATE"
        hdr = blob[:128]
        assert int(hdr[8:12].view(np.int32)[0]) == 1                      # version
        assert list(hdr[32:56].view(np.int64)) == [17, 10, 6]            # dims
        assert int(hdr[56:64].view(np.int64)[0]) == 4                     # iterations
        assert float(hdr[64:72].view(np.float64)[0]) == prob.c
        # the blob's arrays are the getters' dense arrays, bit for bit
        u = blob[128:128 + 4 * 3 * n].view(np.float32).reshape((3,) + prob.spatial)
        assert np.array_equal(u, a.labels().cpu().numpy())
        with pytest.raises(pfm.PfmError):
            a.set_state(blob[:-4])                                        # truncated
        bad = blob.copy()
        bad[0] = ord("X")
        with pytest.raises(pfm.PfmError):
            a.set_state(bad)                                              # magic
        assert a.iterations == 4                                          # nothing changed
    with gpu_problem(prob, storage=1) as b:                               # storage mismatch
        with pytest.raises(pfm.PfmError):
            b.set_state(blob)
    other = synth.random_problem(6201, (6, 10, 18), nl=3, s_kind="field")
    with gpu_problem(other) as c:                                         # shape mismatch
        with pytest.raises(pfm.PfmError):
            c.set_state(np.concatenate([blob, np.zeros(48 * 6 * 10, np.uint8)]))  # size fits, shape not
