"""16-bit storage of u and q (BF16 or F16; FP32 arithmetic) against the FP64
oracle.

The error is reported per result; the bounds are those of the storage
rounding accumulated over the run, not the FP32 parity bounds.
BF16 (8-bit significand, relative 2^-9 per store): measured on GB300 after 60
iterations, max |du| 1.4e-2..1.7e-2 (Potts) and 4.3e-2 (HMF), thresholded
labels equal on >= 99.97 % of voxels, primal energy off by 0.5..1.5 % (the
total variation of a labelling stored with 8 significant bits carries
quantisation noise of ~2^-8 per voxel in flat regions).
F16 (11-bit significand, labelling floored at 2^-24): on the Potts volume
eight times finer than BF16 (max |du| 1.5e-3); on HMF much coarser (labels
agree on 98.9 % of voxels after 60 iterations): F16's narrow exponent range
leaves a small labelling value only absolute precision (2^-24 in the
subnormal range), so the ratios of small labels, which the multiplicative
update amplifies, are lost.  An emulation of F16 rounding of the stored
state applied to the FP64 iteration gives the same agreement (98.92 %), so
this is the storage format, not the kernels."""
import numpy as np
import pytest

import synth
from helpers import compare, gpu_problem

pytestmark = pytest.mark.gpu

TOL = {1: dict(tol_u=6e-2, tol_e=3e-2, tol_argmax=0.999),
       2: dict(tol_u=8e-3, tol_e=4e-3, tol_argmax=0.999)}
TOL_HMF_F16 = dict(tol_u=1.0, tol_e=3e-2, tol_argmax=0.985)
NAME = {1: "bf16", 2: "f16"}


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
@pytest.mark.parametrize("sched", [0, 1, 2], ids=["fused_tma", "inplace", "fused_plain"])
def test_potts3d_lowp(sched, storage):
    prob = synth.potts3d_problem(seed=2300, nl=8, shape=(28, 33, 48))
    with gpu_problem(prob, storage=storage, schedule=sched) as gp:
        res = compare(prob, gp, 60, **TOL[storage])
        print("%s potts" % NAME[storage], gp.variant, {k: "%.2e" % v for k, v in res.items()})


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
def test_hmf_lowp(storage):
    prob = synth.hmf_problem(seed=3300, shape=(20, 24, 36))
    with gpu_problem(prob, storage=storage) as gp:
        res = compare(prob, gp, 60, **(TOL[storage] if storage == 1 else TOL_HMF_F16))
        print("%s hmf" % NAME[storage], gp.variant, {k: "%.2e" % v for k, v in res.items()})


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
def test_lowp_resume_bit_exact(storage):
    prob = synth.potts3d_problem(seed=2301, nl=8, shape=(12, 16, 32))
    with gpu_problem(prob, storage=storage) as a:
        a.iterate(14)
        ref = a.labels().cpu().numpy()
    with gpu_problem(prob, storage=storage) as b:
        b.iterate(6)
        u, q = b.labels().cpu().numpy(), b.flows().cpu().numpy()
    with gpu_problem(prob, storage=storage) as c:
        c.set_labels(u)
        c.set_flows(q)
        c.iterate(8)
        assert np.array_equal(c.labels().cpu().numpy(), ref)


@pytest.mark.parametrize("sched", [0, 1, 2], ids=["fused_tma", "inplace", "fused_plain"])
def test_f16_labelling_floor(sched):
    """With zero capacity the flows stay zero and the labelling follows
    u <- u exp(-D/c) / sum; labels whose exact value falls below 2^-24 are
    held at the floor 2^-24 (they would otherwise round to an F16 zero that
    never recovers), the others follow the closed form softmax(-k D / c) to
    F16 rounding."""
    prob = synth.random_problem(2310, (7, 9, 40), nl=4, s_kind="field")
    prob.S_field = np.zeros_like(prob.S_field)
    prob.D = (prob.D * 4.0).astype(np.float32)          # data gaps up to 4: fast decay
    k = 12
    with gpu_problem(prob, storage=2, schedule=sched) as gp:
        gp.iterate(k)
        u = gp.labels().cpu().numpy().astype(np.float64)
        assert not np.any(gp.flows().cpu().numpy())
    z = -k * prob.D.astype(np.float64) / prob.c
    z -= z.max(0, keepdims=True)
    exact = np.exp(z) / np.exp(z).sum(0, keepdims=True)
    floor = 2.0 ** -24
    assert u.min() == floor and np.any(exact < floor / 4)
    big = exact >= 1e-3
    assert np.all(np.abs(u[big] - exact[big]) <= 4e-3 * exact[big] + 2 * floor)
    assert np.all(u[exact < floor / 4] == floor)
    assert np.abs(u.sum(0) - 1).max() <= 4 * 2.0 ** -11
