"""Parity at the benchmark's full size, in the launch configuration bench.py
times (3-D Potts 256^3 x 8 labels, FP32, TMA-staged fused kernel): every
voxel against the FP64 oracle after a few iterations (the oracle's cost
bounds the count), and properties that hold at any size after many."""
import numpy as np
import pytest

import synth
from helpers import TOL_ARGMAX, TOL_E, TOL_U, gpu_problem, oracle_run

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def bench_problem():
    return synth.potts3d_problem(seed=2000, nl=8, shape=(256, 256, 256))


def test_fullsize_every_voxel_after_three_iterations(bench_problem):
    prob = bench_problem
    with gpu_problem(prob) as gp:
        assert gp.variant == "fused_tma"
        E_in, P_in = gp.iterate_energy(3)       # energy of the state after 2 iterations
        u = gp.labels().cpu().numpy()
        q = gp.flows().cpu().numpy()
        E3, P3 = gp.energy()
    u_o, q_o, E_o, P_o = oracle_run(prob, 3)
    assert np.abs(u - u_o).max() <= TOL_U
    assert np.abs(q - q_o).max() <= TOL_U
    assert abs(E3 - E_o) <= TOL_E * abs(E_o) and abs(P3 - P_o) <= TOL_E * abs(P_o)
    assert np.mean(np.argmax(u, 0) == np.argmax(u_o, 0)) >= TOL_ARGMAX
    del u_o, q_o
    _, _, E2, P2 = oracle_run(prob, 2)
    assert abs(E_in - E2) <= TOL_E * abs(E2) and abs(P_in - P2) <= TOL_E * abs(P2)


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
