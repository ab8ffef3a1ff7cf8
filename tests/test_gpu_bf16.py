"""BF16 storage of u and q (FP32 arithmetic) against the FP64 oracle.

The error is reported per result.  The bounds are those of BF16 rounding
(8-bit significand, relative 2^-9 per store) accumulated over the run, not
the FP32 parity bounds: measured on GB300 after 60 iterations, max |du| is
1.4e-2..1.7e-2 (Potts) and 4.3e-2 (HMF), the thresholded labels agree on
>= 99.97 % of voxels, and the primal energy is off by 0.5..1.5 % because
the total variation of a labelling stored with 8 significant bits carries
quantisation noise of ~2^-8 per voxel in flat regions."""
import numpy as np
import pytest

import synth
from helpers import compare, gpu_problem

pytestmark = pytest.mark.gpu

BF16_TOL = dict(tol_u=6e-2, tol_e=3e-2, tol_argmax=0.999)


@pytest.mark.parametrize("sched", [0, 1, 2], ids=["fused_tma", "inplace", "fused_plain"])
def test_potts3d_bf16(sched):
    prob = synth.potts3d_problem(seed=2300, nl=8, shape=(28, 33, 48))
    with gpu_problem(prob, storage=1, schedule=sched) as gp:
        res = compare(prob, gp, 60, **BF16_TOL)
        print("bf16 potts", gp.variant, {k: "%.2e" % v for k, v in res.items()})


def test_hmf_bf16():
    prob = synth.hmf_problem(seed=3300, shape=(20, 24, 36))
    with gpu_problem(prob, storage=1) as gp:
        res = compare(prob, gp, 60, **BF16_TOL)
        print("bf16 hmf", gp.variant, {k: "%.2e" % v for k, v in res.items()})


def test_bf16_resume_bit_exact():
    prob = synth.potts3d_problem(seed=2301, nl=8, shape=(12, 16, 32))
    with gpu_problem(prob, storage=1) as a:
        a.iterate(14)
        ref = a.labels().cpu().numpy()
    with gpu_problem(prob, storage=1) as b:
        b.iterate(6)
        u, q = b.labels().cpu().numpy(), b.flows().cpu().numpy()
    with gpu_problem(prob, storage=1) as c:
        c.set_labels(u)
        c.set_flows(q)
        c.iterate(8)
        assert np.array_equal(c.labels().cpu().numpy(), ref)
