"""Parity at the benchmark's full size, in the launch configuration bench.py
times (3-D Potts 256^3 x 8 labels, TMA-staged fused kernel at the tuned
chunk length, steps of 10 iterations whose last also reduces E and P):
every voxel against the FP64 oracle after the workload's own 500
iterations, FP32 and BF16 storage; then the workload's stopping rule (relative
primal-dual gap <= 1e-4, checked every 10 iterations) from there; and
properties that hold at any size."""
import numpy as np
import pytest

import synth
from helpers import TOL_ARGMAX, TOL_E, TOL_U, gpu_problem, oracle_run

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ITERS = 500                       # the 3-D Potts workload's fixed count
# 16-bit storage of u and q after 500 iterations, against the FP64 oracle,
# stated per result.  Measured on GB300: BF16 max |du| 0.38 at 0.014 % of
# the voxels (near-ties whose winner the 8-bit rounding decides), 99.99th
# percentile 2.5e-3, relative E 2.2e-5, labels equal on 99.996 %; F16 max
# |du| 0.049, 99.99th percentile 2.2e-4, relative E 8e-5, labels 99.9998 %.
LOWP_BOUNDS = {1: dict(p9999=1e-2, dE=1e-4, agree=0.9999), 2: dict(p9999=1e-3, dE=3e-4, agree=0.9999)}


@pytest.fixture(scope="module")
def bench_problem():
    return synth.potts3d_problem(seed=2000, nl=8, shape=(256, 256, 256))


@pytest.fixture(scope="module")
def oracle_500(bench_problem):
    """The oracle after 499 iterations (E, P of the state the 500th starts
    from: what the bench's last gap check reports) and after 500."""
    prob = bench_problem
    u, q, E499, P499 = oracle_run(prob, ITERS - 1)
    u, q, E, P = oracle_run(prob, 1, state=(u, q))
    return dict(u=u, q=q, E=E, P=P, E499=E499, P499=P499)


def _step_like_bench(gp, iters):
    """iters iterations in the bench's steps (9 plain + 1 with the reduction)."""
    EP = None
    for _ in range(iters // 10):
        gp.iterate(9)
        EP = gp.iterate_energy(1)
    return EP


def test_fullsize_every_voxel_after_500_iterations(bench_problem, oracle_500):
    prob, o = bench_problem, oracle_500
    with gpu_problem(prob) as gp:
        assert gp.variant == "fused_tma"
        zc = gp.tune(3)                          # as the bench: tuned chunk length, state reset
        E_in, P_in = _step_like_bench(gp, ITERS)
        assert gp.iterations == ITERS
        u = gp.labels().cpu().numpy()
        q = gp.flows().cpu().numpy()
        E, P = gp.energy()
        du = float(np.abs(u - o["u"]).max())
        dq = float(np.abs(q - o["q"]).max())
        agree = float(np.mean(np.argmax(u, 0) == np.argmax(o["u"], 0)))
        print("PARITY potts3d f32 %d it zc=%d du=%.3e dq=%.3e dE=%.3e dP=%.3e dE499=%.3e agree=%.6f"
              % (ITERS, zc, du, dq, abs(E - o["E"]) / abs(o["E"]), abs(P - o["P"]) / abs(o["P"]),
                 abs(E_in - o["E499"]) / abs(o["E499"]), agree))
        assert du <= TOL_U and dq <= TOL_U
        assert abs(E - o["E"]) <= TOL_E * abs(o["E"]) and abs(P - o["P"]) <= TOL_E * abs(o["P"])
        assert abs(E_in - o["E499"]) <= TOL_E * abs(o["E499"]) and abs(P_in - o["P499"]) <= TOL_E * abs(o["P499"])
        assert agree >= TOL_ARGMAX
        del u, q
        # the workload's stopping rule from here: gap <= 1e-4, checked every 10
        it, gap, ok = gp.run_to_gap(20000)
        print("STOP potts3d f32 after %d + %d iterations rel_gap=%.3e converged=%s" % (ITERS, it, gap, ok))
        assert ok and gap <= 1e-4


@pytest.mark.parametrize("storage", [1, 2], ids=["bf16", "f16"])
def test_fullsize_lowp_after_500_iterations(bench_problem, oracle_500, storage):
    prob, o = bench_problem, oracle_500
    with gpu_problem(prob, storage=storage) as gp:
        assert gp.variant == "fused_tma"
        gp.tune(3)
        _step_like_bench(gp, ITERS)
        u = gp.labels().cpu().numpy()
        E, P = gp.energy()
    d = np.abs(u - o["u"])
    r = dict(max=float(d.max()), p9999=float(np.quantile(d, 0.9999)), frac_gt_1e3=float((d > 1e-3).mean()),
             agree=float(np.mean(np.argmax(u, 0) == np.argmax(o["u"], 0))),
             dE=abs(E - o["E"]) / abs(o["E"]), dP=abs(P - o["P"]) / abs(o["P"]))
    print("PARITY potts3d %s %d it %s" % ("bf16" if storage == 1 else "f16", ITERS,
                                          {k: "%.3e" % v for k, v in r.items()}))
    b = LOWP_BOUNDS[storage]
    assert r["p9999"] <= b["p9999"] and r["dE"] <= b["dE"] and r["dP"] <= b["dE"] and r["agree"] >= b["agree"], r


def test_fullsize_invariants_after_fifty_iterations(bench_problem):
    prob = bench_problem
    with gpu_problem(prob) as gp:
        E_prev = None
        for _ in range(5):
            E, P = gp.iterate_energy(10)
            assert E - P >= -1e-6 * abs(E)
            E_prev = E
        u = gp.labels().cpu().numpy()
        s = u.sum(0)
        assert u.min() >= 0 and np.abs(s - 1).max() <= 1e-5
        del u
        q = gp.flows().cpu().numpy()
        mag = np.sqrt((q.astype(np.float64) ** 2).sum(1))
        assert np.all(mag <= prob.S_field[None].astype(np.float64) * (1 + 1e-5) + 1e-12)
        assert np.all(q[:, 0, :, :, -1] == 0) and np.all(q[:, 1, :, -1, :] == 0) and np.all(q[:, 2, -1] == 0)
        assert E_prev is not None
