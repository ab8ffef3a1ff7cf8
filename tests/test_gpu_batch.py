"""Batched solver (pfm_batch_*): many volumes of uneven sizes and label DAGs
advanced by one persistent kernel per iteration, replayed from CUDA graphs.
Every member must equal the same problem solved on its own, bit for bit,
and match the oracle."""
import numpy as np
import pytest

import synth
from helpers import compare, gpu_problem, oracle_run

pytestmark = pytest.mark.gpu


def as_dict(p):
    return dict(D=p.D, S_field=p.S_field, s_node=p.s_node, n_nodes=p.n_nodes, edges=p.edges)


def dag_volumes(count=5, seed=4500):
    rng = np.random.default_rng(seed)
    out = []
    for v in range(count):
        shape = tuple(int(s) for s in rng.integers(9, 41, size=3))
        out.append(synth.dagmf_problem(seed + 1 + v, shape, iters=30))
    return out


@pytest.mark.parametrize("iters", [7, 20, 47], ids=["direct", "one_graph", "graphs_and_tail"])
def test_batch_members_equal_single_problems(iters):
    import paper_1501_07844_gb300 as pfm
    vols = dag_volumes()
    with pfm.Batch([as_dict(p) for p in vols]) as b:
        b.iterate(iters)
        E_b, P_b = b.energy()
        for k, p in enumerate(vols):
            # the batched kernel runs the register-staged tile body
            with gpu_problem(p, schedule=pfm.FUSED_PLAIN) as single:
                single.iterate(iters)
                m = b.members[k]
                assert np.array_equal(m.labels().cpu().numpy(), single.labels().cpu().numpy())
                assert np.array_equal(m.flows().cpu().numpy(), single.flows().cpu().numpy())
                E, P = single.energy()
                assert E_b[k] == E and P_b[k] == P
                assert m.iterations == iters


def test_batch_matches_oracle_and_mixes_potts_and_dags():
    import paper_1501_07844_gb300 as pfm
    vols = dag_volumes(3, seed=4600) + [synth.potts3d_problem(seed=4610, nl=8, shape=(14, 22, 37))]
    with pfm.Batch([as_dict(p) for p in vols]) as b:
        b.iterate(30)
        for k in (0, 3):
            p = vols[k]
            u_o, q_o, E_o, _ = oracle_run(p, 30)
            u = b.members[k].labels().cpu().numpy()
            assert np.abs(u - u_o).max() <= 1e-3
            assert np.mean(np.argmax(u, 0) == np.argmax(u_o, 0)) >= 0.999


def test_batch_tune_resets_and_keeps_results():
    import paper_1501_07844_gb300 as pfm
    vols = dag_volumes(4, seed=4700)
    with pfm.Batch([as_dict(p) for p in vols]) as b:
        b.iterate(5)
        zc, grid = b.tune(trial_iters=2)
        assert zc in (8, 16, 32, 64) and grid >= 1
        assert all(m.iterations == 0 for m in b.members)
        b.iterate(25)
        with gpu_problem(vols[2], schedule=pfm.FUSED_PLAIN) as single:
            single.iterate(25)
            assert np.array_equal(b.members[2].labels().cpu().numpy(), single.labels().cpu().numpy())


def test_batch_bf16_and_2d():
    import paper_1501_07844_gb300 as pfm
    vols = [synth.random_problem(4800 + k, (30 + 7 * k, 41 - 5 * k), nl=5, s_kind="both") for k in range(4)]
    with pfm.Batch([as_dict(p) for p in vols], storage=pfm.BF16) as b:
        b.iterate(21)
        for k, p in enumerate(vols):
            with gpu_problem(p, storage=pfm.BF16, schedule=pfm.FUSED_PLAIN) as single:
                single.iterate(21)
                assert np.array_equal(b.members[k].labels().cpu().numpy(), single.labels().cpu().numpy())


def test_batch_rejects_bad_members():
    import paper_1501_07844_gb300 as pfm
    good = synth.random_problem(4900, (6, 7, 8), nl=3, s_kind="field")
    with pytest.raises(pfm.PfmError) as ei:
        pfm.Batch([as_dict(good), dict(D=good.D, S_field=good.S_field, n_nodes=2, edges=[(-1, 0, 1.0)])])
    assert ei.value.name in ("PFM_EDAG", "PFM_EINVAL") and "member 1" in str(ei.value)
    flat2d = synth.random_problem(4901, (6, 7), nl=3, s_kind="field")
    with pytest.raises(pfm.PfmError):
        pfm.Batch([as_dict(good), as_dict(flat2d)])
