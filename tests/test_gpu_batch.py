"""Batched solver (pfm_batch_*): many volumes of uneven sizes and label DAGs
advanced by one persistent kernel per iteration, replayed from CUDA graphs.
Every member must equal the same problem solved on its own with the same
kernel body, bit for bit (the TMA-staged DAG batch against the TMA DAG
kernel, the register-staged batch against PFM_SCHEDULE_FUSED_PLAIN), and
match the oracle."""
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


@pytest.mark.parametrize("sched", [0, 2], ids=["tma", "register"])
@pytest.mark.parametrize("iters", [7, 20, 47], ids=["direct", "one_graph", "graphs_and_tail"])
def test_batch_members_equal_single_problems(iters, sched):
    import paper_1501_07844_gb300 as pfm
    vols = dag_volumes()
    with pfm.Batch([as_dict(p) for p in vols], schedule=sched) as b:
        assert b.variant == ("batched_tma_dag4" if sched == pfm.FUSED else "batched")
        b.iterate(iters)
        E_b, P_b = b.energy()
        for k, p in enumerate(vols):
            # the same tile body as the batched kernel
            with gpu_problem(p, schedule=sched) as single:
                if sched == pfm.FUSED:
                    single.select_kernel("fused_tma_dag4")
                assert single.variant == ("fused_tma_dag4" if sched == pfm.FUSED else "fused")
                single.iterate(iters)
                m = b.members[k]
                assert np.array_equal(m.labels().cpu().numpy(), single.labels().cpu().numpy())
                assert np.array_equal(m.flows().cpu().numpy(), single.flows().cpu().numpy())
                E, P = single.energy()
                # the batch reduces every member in one launch at its own
                # chunk length: the same terms, summed in another order
                assert abs(E_b[k] - E) <= 1e-6 * abs(E) and abs(P_b[k] - P) <= 1e-6 * abs(P) + 1e-6
                assert m.iterations == iters


@pytest.mark.parametrize("sched", [0, 2], ids=["tma", "register"])
def test_batch_matches_oracle_and_mixes_potts_and_dags(sched):
    import paper_1501_07844_gb300 as pfm
    vols = dag_volumes(3, seed=4600) + [synth.potts3d_problem(seed=4610, nl=8, shape=(14, 22, 37))]
    with pfm.Batch([as_dict(p) for p in vols], schedule=sched) as b:
        b.iterate(30)
        for k in (0, 3):
            p = vols[k]
            u_o, q_o, E_o, _ = oracle_run(p, 30)
            u = b.members[k].labels().cpu().numpy()
            assert np.abs(u - u_o).max() <= 1e-3
            assert np.mean(np.argmax(u, 0) == np.argmax(u_o, 0)) >= 0.999


@pytest.mark.parametrize("sched", [0, 2], ids=["tma", "register"])
def test_batch_tune_resets_and_keeps_results(sched):
    import paper_1501_07844_gb300 as pfm
    vols = dag_volumes(4, seed=4700)
    with pfm.Batch([as_dict(p) for p in vols], schedule=sched) as b:
        b.iterate(5)
        zc, grid = b.tune(trial_iters=2)
        assert zc in (8, 16, 32, 64) and grid >= 1
        assert all(m.iterations == 0 for m in b.members)
        b.iterate(25)
        with gpu_problem(vols[2], schedule=sched) as single:
            single.iterate(25)
            assert np.array_equal(b.members[2].labels().cpu().numpy(), single.labels().cpu().numpy())


def test_batch_bf16_and_2d():
    import paper_1501_07844_gb300 as pfm
    vols = [synth.random_problem(4800 + k, (30 + 7 * k, 41 - 5 * k), nl=5, s_kind="both") for k in range(4)]
    with pfm.Batch([as_dict(p) for p in vols], storage=pfm.BF16) as b:
        assert b.variant == "batched"  # Potts-only batches keep the register-staged kernel
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


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
def test_tma_dag_batch_2d_bf16_and_hmf(storage):
    """The TMA batch on 2-D DAGMF members and on HMF trees (both have at most
    four inner nodes: the four-inner-node kernel), every storage: bit for bit
    the single-problem kernel with the same tile body."""
    import paper_1501_07844_gb300 as pfm
    vols = [synth.hmf_problem(seed=4950 + k, shape=(19 + 5 * k, 37 - 3 * k, 45 + 2 * k), iters=20) for k in range(2)]
    vols += [synth.dagmf_problem(4960 + k, (53 + 9 * k, 70 - 11 * k), iters=20) for k in range(2)]
    for group in (vols[:2], vols[2:]):
        with pfm.Batch([as_dict(p) for p in group], storage=storage) as b:
            assert b.variant == "batched_tma_dag4"
            b.iterate(23)
            for k, p in enumerate(group):
                with gpu_problem(p, storage=storage) as single:
                    single.select_kernel("fused_tma_dag4")   # the batch's tile body
                    assert single.variant == "fused_tma_dag4"
                    single.iterate(23)
                    assert np.array_equal(b.members[k].labels().cpu().numpy(), single.labels().cpu().numpy())
                    assert np.array_equal(b.members[k].flows().cpu().numpy(), single.flows().cpu().numpy())


def test_tma_dag_batch_mixed_layouts_and_ishikawa():
    """One TMA batch holding members with different shared-memory layouts
    (HMF: 12 end-labels / 15 nodes; DAGMF: 10 / 14; an Ishikawa chain whose
    end-labels carry no flow) and odd widths: every member equals its
    single-problem run bit for bit -- the chain to FP32 rounding, since alone
    it runs the chain-specialised kernel (prefix / suffix sums instead of
    path-weight lists) -- and the chain's end-label flows stay 0."""
    import paper_1501_07844_gb300 as pfm
    vols = [synth.hmf_problem(seed=4970, shape=(17, 23, 29), iters=20),
            synth.dagmf_problem(4971, (21, 19, 35), iters=20),
            synth.ishikawa_problem(4972, (13, 26, 41), nlev=7)]
    with pfm.Batch([as_dict(p) for p in vols]) as b:
        assert b.variant == "batched_tma_dag"
        b.iterate(26)
        for k, p in enumerate(vols):
            with gpu_problem(p) as single:
                if k < 2:
                    single.select_kernel("fused_tma_dag")   # the batch's tile body
                single.iterate(26)
                ub, us = b.members[k].labels().cpu().numpy(), single.labels().cpu().numpy()
                qb, qs = b.members[k].flows().cpu().numpy(), single.flows().cpu().numpy()
                if k == 2:
                    assert single.variant == "fused_tma_ishikawa"
                    assert np.abs(ub - us).max() <= 1e-5 and np.abs(qb - qs).max() <= 1e-5
                else:
                    assert single.variant == "fused_tma_dag"
                    assert np.array_equal(ub, us) and np.array_equal(qb, qs)
        q = b.members[2].flows().cpu().numpy()
        assert np.all(q[7:] == 0)
