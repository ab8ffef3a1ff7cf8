"""GPU parity of the Potts path (Algorithm 1) against the FP64 oracle,
through the C ABI, on seeded phantoms: element by element on small and
ragged grids, every schedule and gradient mode, plus closed forms,
invariants, error handling and checkpoint/resume."""
import numpy as np
import pytest

import synth
from helpers import compare, gpu_problem, oracle_run

pytestmark = pytest.mark.gpu

SCHEDULES = [("fused", 0), ("inplace", 1)]


@pytest.mark.parametrize("sched", SCHEDULES, ids=lambda s: s[0])
@pytest.mark.parametrize("mode", [0, 1], ids=["normalised", "literal"])
def test_potts2d_phantom_128(sched, mode):
    """2-D Potts phantom, 128 x 128, 4 labels, S = 0.1, c = 0.5, tau = 0.11, 200 iterations."""
    prob = synth.potts2d_problem(seed=1000)
    with gpu_problem(prob, schedule=sched[1], grad_source=mode) as gp:
        compare(prob, gp, 200, grad_source=mode)


@pytest.mark.parametrize("sched", SCHEDULES, ids=lambda s: s[0])
def test_potts3d_ragged_tiles(sched):
    """3-D, 8 labels, edge-weighted S, sizes that leave ragged x/y tiles and
    several z-chunks."""
    prob = synth.potts3d_problem(seed=2001, nl=8, shape=(37, 21, 45), iters=60)
    with gpu_problem(prob, schedule=sched[1]) as gp:
        compare(prob, gp, 60)


@pytest.mark.parametrize("nl", [2, 3, 5, 12, 16])
@pytest.mark.parametrize("spatial", [(19, 23, 35), (70, 33)], ids=["3d", "2d"])
def test_label_counts(nl, spatial):
    prob = synth.random_problem(10 + nl, spatial, nl=nl, s_kind="both", s_scale=0.4)
    with gpu_problem(prob, schedule=0) as gp:
        compare(prob, gp, 40)


@pytest.mark.parametrize("sched", SCHEDULES, ids=lambda s: s[0])
def test_anisotropic(sched):
    prob = synth.random_problem(21, (17, 20, 33), nl=4, s_kind="field", s_scale=0.5)
    with gpu_problem(prob, schedule=sched[1], norm=1) as gp:
        compare(prob, gp, 50, norm=1)


@pytest.mark.parametrize("spatial", [(1, 1, 1), (1, 1, 40), (5, 1, 1), (1, 37), (29, 1), (2, 2), (3, 65, 2)])
def test_degenerate_shapes(spatial):
    prob = synth.random_problem(31, spatial, nl=3, s_kind="field", s_scale=0.5)
    for sched in (0, 1):
        with gpu_problem(prob, schedule=sched) as gp:
            compare(prob, gp, 25)


def test_zero_capacity_closed_form():
    """S = 0 pins q = 0 and u_L = softmax(-k D_L / c) after k iterations."""
    prob = synth.random_problem(41, (9, 30, 40), nl=6)
    prob.S_field[:] = 0.0
    k = 13
    z = -k * prob.D.astype(np.float64) / prob.c
    z -= z.max(0)
    ref = np.exp(z) / np.exp(z).sum(0)
    for sched in (0, 1):
        with gpu_problem(prob, schedule=sched) as gp:
            gp.iterate(k)
            u = gp.labels().cpu().numpy()
            assert np.abs(u - ref).max() <= 2e-5
            assert np.all(gp.flows().cpu().numpy() == 0.0)


def test_invariants_after_each_iteration():
    prob = synth.potts3d_problem(seed=2002, nl=8, shape=(24, 40, 36))
    cap = prob.S_field[None, None].astype(np.float64)
    for sched in (0, 1):
        with gpu_problem(prob, schedule=sched) as gp:
            for _ in range(6):
                gp.iterate(5)
                u = gp.labels().cpu().numpy().astype(np.float64)
                q = gp.flows().cpu().numpy().astype(np.float64)
                assert u.min() >= 0 and np.abs(u.sum(0) - 1).max() <= 1e-5
                assert np.all(np.sqrt((q ** 2).sum(1)) <= cap * (1 + 1e-5) + 1e-12)
                assert np.all(q[:, 0, :, :, -1] == 0) and np.all(q[:, 1, :, -1, :] == 0) and np.all(q[:, 2, -1] == 0)
                E, P = gp.energy()
                assert E - P >= -1e-6 * abs(E)


def test_energy_reduction_on_oracle_state():
    """pfm_energy of a state imported from the oracle equals the oracle's
    energy of that state (only the FP32 per-voxel terms differ)."""
    prob = synth.potts3d_problem(seed=2003, nl=8, shape=(30, 31, 50))
    u, q, E_o, P_o = oracle_run(prob, 30)
    with gpu_problem(prob) as gp:
        gp.set_labels(u.astype(np.float32))
        gp.set_flows(q.astype(np.float32))
        E, P = gp.energy()
    assert abs(E - E_o) <= 2e-6 * abs(E_o) and abs(P - P_o) <= 2e-6 * abs(P_o) + 1e-6


@pytest.mark.parametrize("sched", SCHEDULES, ids=lambda s: s[0])
def test_resume_is_bit_exact(sched):
    prob = synth.potts3d_problem(seed=2004, nl=8, shape=(20, 26, 40))
    with gpu_problem(prob, schedule=sched[1]) as a:
        a.iterate(20)
        ref_u, ref_q = a.labels().cpu().numpy(), a.flows().cpu().numpy()
    with gpu_problem(prob, schedule=sched[1]) as b:
        b.iterate(9)
        u_mid, q_mid = b.labels().cpu().numpy(), b.flows().cpu().numpy()
    with gpu_problem(prob, schedule=sched[1]) as c:
        c.set_labels(u_mid)
        c.set_flows(q_mid)
        c.iterate(11)
        assert np.array_equal(c.labels().cpu().numpy(), ref_u)
        assert np.array_equal(c.flows().cpu().numpy(), ref_q)


def test_argmax_ties_go_to_lowest_label():
    prob = synth.random_problem(51, (4, 8), nl=4, s_kind="field")
    prob.D[:] = 0.5
    with gpu_problem(prob) as gp:
        gp.iterate(3)
        assert np.all(gp.argmax().cpu().numpy() == 0)


def test_errors_are_reported_not_trapped():
    import paper_1501_07844_gb300 as pfm
    prob = synth.random_problem(61, (6, 7), nl=3, s_kind="field")
    bad = prob.D.copy()
    bad[1, 2, 3] = np.nan
    with pytest.raises(pfm.PfmError) as ei:
        pfm.Problem(bad, S_field=prob.S_field)
    assert ei.value.name == "PFM_ENONFINITE"
    negS = prob.S_field.copy()
    negS[0, 0] = -1.0
    with pytest.raises(pfm.PfmError) as ei:
        pfm.Problem(prob.D, S_field=negS)
    assert ei.value.name == "PFM_ENONFINITE"
    with gpu_problem(prob) as gp:
        u = np.full((3, 6, 7), 1 / 3, dtype=np.float32)
        u[0, 1, 1] = -0.1
        with pytest.raises(pfm.PfmError) as ei:
            gp.set_labels(u)
        assert ei.value.name == "PFM_EINVAL"
        gp.iterate(2)          # the problem stays usable
        gp.energy()
        with pytest.raises(pfm.PfmError):
            gp.iterate(-1)


def test_run_to_gap_reaches_target():
    prob = synth.potts2d_problem(seed=1001, n=64)
    import paper_1501_07844_gb300 as pfm
    with gpu_problem(prob, tau=0.25, c=1.0, gap_tol=1e-4, check_every=20) as gp:
        it, gap, ok = gp.run_to_gap(5000)
        assert ok and gap <= 1e-4 and it % 20 == 0 and gp.iterations == it
    with gpu_problem(prob, gap_tol=1e-12) as gp:
        it, gap, ok = gp.run_to_gap(30)
        assert not ok and it == 30
    assert pfm.lib().pfm_version() == 1


def test_host_pointer_inputs_and_outputs():
    """pfm_create and the getters accept pinned host memory (cudaMemcpyDefault)."""
    import torch
    import paper_1501_07844_gb300 as pfm
    prob = synth.random_problem(71, (8, 9, 10), nl=4, s_kind="field")
    D = torch.from_numpy(prob.D).pin_memory()
    S = torch.from_numpy(prob.S_field).pin_memory()
    with pfm.Problem(D, S_field=S) as gp, gpu_problem(prob) as ref:
        gp.iterate(7)
        ref.iterate(7)
        out = torch.empty((4, 8, 9, 10), dtype=torch.float32).pin_memory()
        gp.labels(out=out)
        assert torch.equal(out, ref.labels().cpu())
        am = torch.empty((8, 9, 10), dtype=torch.int32).pin_memory()
        gp.argmax(out=am)
        assert torch.equal(am, ref.argmax().cpu())


@pytest.mark.parametrize("shape", [(23, 17, 40), (9, 40, 64), (40, 136)], ids=["3d_ragged_yz", "3d_two_tiles", "2d"])
@pytest.mark.parametrize("nl", [3, 8])
def test_tma_fused_kernel_parity(shape, nl):
    """Row pitch a multiple of 16 bytes selects the TMA-staged fused kernel;
    it must match the oracle and the register-staged fused kernel."""
    import paper_1501_07844_gb300 as pfm
    prob = synth.random_problem(90 + nl, shape, nl=nl, s_kind="both", s_scale=0.4)
    with gpu_problem(prob, schedule=pfm.FUSED) as gp:
        assert gp.variant == "fused_tma"
        compare(prob, gp, 45)
        u_t, q_t = gp.labels().cpu().numpy(), gp.flows().cpu().numpy()
    with gpu_problem(prob, schedule=pfm.FUSED_PLAIN) as gp:
        assert gp.variant == "fused"
        gp.iterate(45)
        assert np.abs(gp.labels().cpu().numpy() - u_t).max() <= 1e-6
        assert np.abs(gp.flows().cpu().numpy() - q_t).max() <= 1e-6


@pytest.mark.parametrize("mode,norm", [(1, 0), (0, 1)], ids=["literal", "aniso"])
def test_tma_fused_modes(mode, norm):
    prob = synth.potts3d_problem(seed=2005, nl=8, shape=(33, 27, 48))
    with gpu_problem(prob, grad_source=mode, norm=norm) as gp:
        assert gp.variant == "fused_tma"
        compare(prob, gp, 40, grad_source=mode, norm=norm)


def test_kernel_variant_selection():
    """Rows are padded to 16 bytes internally, so every width takes the TMA
    kernel; more than 8 labels and FUSED_PLAIN take the register-staged one."""
    import paper_1501_07844_gb300 as pfm
    p8 = synth.random_problem(95, (5, 6, 32), nl=8, s_kind="field")
    p_odd = synth.random_problem(96, (5, 6, 30), nl=8, s_kind="field")
    p12 = synth.random_problem(97, (5, 6, 32), nl=12, s_kind="field")
    with gpu_problem(p8) as a, gpu_problem(p_odd) as b, gpu_problem(p12) as c, \
            gpu_problem(p8, schedule=pfm.INPLACE) as d, gpu_problem(p8, storage=pfm.BF16) as e, \
            gpu_problem(p_odd, storage=pfm.BF16) as f, gpu_problem(p_odd, schedule=pfm.FUSED_PLAIN) as g:
        assert (a.variant, b.variant, c.variant, d.variant, e.variant, f.variant, g.variant) == \
            ("fused_tma", "fused_tma", "fused", "inplace_tma", "fused_tma", "fused_tma", "fused")


@pytest.mark.parametrize("nx", [1, 5, 37, 65])
@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
def test_padded_rows_every_schedule(nx, storage):
    """Widths that are not a multiple of 8: the device rows are padded; every
    schedule matches the oracle (FP32) or the other schedules (BF16), the
    energy matches, and labels / flows / argmax read back dense and import
    back bit for bit."""
    import paper_1501_07844_gb300 as pfm
    prob = synth.random_problem(140 + nx, (6, 11, nx), nl=5, s_kind="both", s_scale=0.4)
    res = {}
    for sched in (pfm.FUSED, pfm.INPLACE, pfm.FUSED_PLAIN):
        with gpu_problem(prob, schedule=sched, storage=storage) as gp:
            if storage == 0:
                compare(prob, gp, 30)
            else:
                gp.iterate(30)
            res[sched] = (gp.labels().cpu().numpy(), gp.flows().cpu().numpy(), gp.energy(), gp.argmax().cpu().numpy())
            u, q = gp.labels(), gp.flows()
            assert tuple(u.shape) == (5, 6, 11, nx) and tuple(q.shape) == (5, 3, 6, 11, nx)
            gp.set_labels(u)
            gp.set_flows(q)
            assert torch_equal(gp.labels(), u) and torch_equal(gp.flows(), q)
    tol = 1e-6 if storage == 0 else 2e-2
    for sched in (pfm.INPLACE, pfm.FUSED_PLAIN):
        assert np.abs(res[sched][0] - res[pfm.FUSED][0]).max() <= tol
        assert np.abs(res[sched][1] - res[pfm.FUSED][1]).max() <= tol
        E0, E1 = res[pfm.FUSED][2][0], res[sched][2][0]
        assert abs(E1 - E0) <= (1e-5 if storage == 0 else 2e-2) * abs(E0)
    for sched in res:
        assert np.array_equal(res[sched][3], np.argmax(res[sched][0], axis=0))


def torch_equal(a, b):
    import torch
    return bool(torch.equal(a, b))


@pytest.mark.parametrize("sched", [0, 1, 2], ids=["fused_tma", "inplace", "fused_plain"])
@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
def test_iterate_energy_reports_input_of_last_iteration(sched, storage):
    """pfm_iterate_energy(n) returns E and P of the state after n-1 iterations
    (reduced inside the last iteration on the TMA path) and leaves the state
    after n iterations, identical to plain iterations."""
    prob = synth.potts3d_problem(seed=2400, nl=8, shape=(19, 27, 40))
    with gpu_problem(prob, schedule=sched, storage=storage) as a, \
            gpu_problem(prob, schedule=sched, storage=storage) as b:
        a.iterate(6)
        E_ref, P_ref = a.energy()
        a.iterate(1)
        E, P = b.iterate_energy(7)
        assert abs(E - E_ref) <= 1e-6 * abs(E_ref) and abs(P - P_ref) <= 1e-6 * abs(P_ref) + 1e-6
        assert np.array_equal(a.labels().cpu().numpy(), b.labels().cpu().numpy())
        assert np.array_equal(a.flows().cpu().numpy(), b.flows().cpu().numpy())
        assert b.iterations == 7
    if storage == 0:
        _, _, E_o, P_o = oracle_run(prob, 6)
        assert abs(E - E_o) <= 1e-5 * abs(E_o) and abs(P - P_o) <= 1e-5 * abs(P_o)


@pytest.mark.parametrize("sched", [0, 1, 2], ids=["fused_tma", "inplace", "fused_plain"])
def test_continuation_schedule_matches_oracle(sched):
    """c lowered between blocks (continuation toward c -> 0): GPU and oracle
    follow the same schedule."""
    import oracle
    prob = synth.potts3d_problem(seed=2500, nl=8, shape=(17, 25, 40))
    D, S = prob.D.astype(np.float64), prob.S_field.astype(np.float64)
    u, q = oracle.potts_init(prob.spatial, 8)
    with gpu_problem(prob, schedule=sched, c=1.0) as gp:
        for c in (1.0, 0.5, 0.25):
            gp.set_step(c, 0.11)
            gp.iterate(15)
            oracle.potts_iterate(D, u, q, 15, c, 0.11, S_field=S)
        assert np.abs(gp.labels().cpu().numpy() - u).max() <= 1e-3
        E, P = gp.energy()
        E_o, _ = oracle.potts_energy(D, u, q, S_field=S)
        assert abs(E - E_o) <= 1e-5 * abs(E_o)


@pytest.mark.parametrize("shape", [(37, 19, 70), (53, 66), (1, 9, 33)], ids=["3d_chunks", "2d", "one_plane"])
@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
def test_inplace_tma_sweeps(shape, storage):
    """The TMA-staged in-place sweeps (z-chunks of 4 planes here, ragged
    tiles) match the oracle (FP32) and the fused TMA schedule; PAPER_LITERAL
    keeps the per-voxel in-place kernels."""
    import paper_1501_07844_gb300 as pfm
    prob = synth.random_problem(150 + len(shape), shape, nl=8, s_kind="both", s_scale=0.4)
    with gpu_problem(prob, schedule=pfm.INPLACE, storage=storage) as gp:
        assert gp.variant == "inplace_tma"
        if storage == 0:
            compare(prob, gp, 35)
        else:
            gp.iterate(35)
        u_i, q_i = gp.labels().cpu().numpy(), gp.flows().cpu().numpy()
    with gpu_problem(prob, schedule=pfm.FUSED, storage=storage) as gp:
        gp.iterate(35)
        tol = 1e-6 if storage == 0 else 2e-2
        assert np.abs(gp.labels().cpu().numpy() - u_i).max() <= tol
        assert np.abs(gp.flows().cpu().numpy() - q_i).max() <= tol
    with gpu_problem(prob, schedule=pfm.INPLACE, grad_source=1) as gp:
        assert gp.variant == "inplace"


def test_prefetch_commit_equals_set_data():
    """pfm_prefetch_data + pfm_commit_data (copy on the library's copy stream,
    overlapping queued iterations) gives the same state as pfm_set_data; a
    second prefetch replaces the first; a commit without a prefetch is
    rejected."""
    import torch
    import paper_1501_07844_gb300 as pfm
    prob = synth.random_problem(170, (12, 21, 45), nl=5, s_kind="field")
    other = synth.random_problem(171, (12, 21, 45), nl=5, s_kind="field")
    hD, hS = torch.from_numpy(other.D).pin_memory(), torch.from_numpy(other.S_field).pin_memory()
    junk = torch.rand_like(hD).pin_memory()
    with gpu_problem(prob) as a, gpu_problem(prob) as b:
        with pytest.raises(pfm.PfmError) as ei:
            a.commit_data()
        assert ei.value.name == "PFM_EINVAL"
        a.iterate(7)
        a.prefetch_data(junk, hS)
        a.prefetch_data(hD, hS)      # replaces the first
        a.iterate(5)                 # still on the old data
        a.commit_data()
        a.iterate(9)
        b.iterate(12)
        b.set_data(hD, hS)
        b.iterate(9)
        assert torch.equal(a.labels(), b.labels()) and torch.equal(a.flows(), b.flows())


def _prefetch_kinds(kind):
    if kind == "hmf":
        return synth.hmf_problem(seed=3310, shape=(11, 19, 40), iters=30), {}
    if kind == "ishikawa":
        return synth.ishikawa_problem(3311, (10, 17, 38), nlev=4), {}
    if kind == "dagmf":
        return synth.dagmf_problem(3312, (9, 18, 37), iters=30), {}
    prob = synth.random_problem(3313, (10, 17, 39), nl=5, s_kind="both")
    if kind == "potts_inplace":
        import paper_1501_07844_gb300 as pfm
        return prob, {"schedule": pfm.INPLACE}
    if kind == "potts_bf16":
        return prob, {"storage": 1}
    return prob, {}


@pytest.mark.parametrize("kind", ["potts", "potts_inplace", "potts_bf16", "hmf", "ishikawa", "dagmf"])
def test_prefetch_commit_rounds_equal_set_data(kind):
    """Several prefetch / commit rounds, in which the data buffers and the
    staging buffers trade places and the kernels' tensor maps follow them,
    give bit for bit the state of the same sequence with pfm_set_data, on
    every kernel family; a staged D with a NaN is reported by the next
    call that checks the problem (the energy)."""
    import torch
    import paper_1501_07844_gb300 as pfm
    prob, kw = _prefetch_kinds(kind)
    rng = np.random.default_rng(77)
    data = []
    for k in range(3):
        D = (prob.D * rng.uniform(0.7, 1.3, size=prob.D.shape)).astype(np.float32)
        S = None if prob.S_field is None else (prob.S_field * rng.uniform(0.5, 1.5, size=prob.S_field.shape)).astype(
            np.float32)
        data.append((torch.from_numpy(D).pin_memory(), None if S is None else torch.from_numpy(S).pin_memory()))
    with gpu_problem(prob, **kw) as a, gpu_problem(prob, **kw) as b:
        a.iterate(5)
        b.iterate(5)
        for k, (iters_before, iters_after) in enumerate([(3, 4), (0, 6), (2, 5)]):
            D, S = data[k % 3] if k < 2 else data[0]
            a.prefetch_data(D, S)
            a.iterate(iters_before)      # still on the previous data
            a.commit_data()
            a.iterate(iters_after)
            b.iterate(iters_before)
            b.set_data(D, S)
            b.iterate(iters_after)
        assert torch.equal(a.labels(), b.labels()) and torch.equal(a.flows(), b.flows())
        assert a.energy() == b.energy()
        bad = data[1][0].clone()
        bad[0].view(-1)[7] = float("nan")
        a.prefetch_data(bad, data[1][1])
        a.commit_data()
        a.iterate(1)
        with pytest.raises(pfm.PfmError) as ei:
            a.energy()
        assert ei.value.name == "PFM_ENONFINITE"


def test_prefetch_commit_on_batch_member():
    """A batch member's prefetch / commit copies the staged data into the
    buffers the batch's kernels read: the batch then iterates on the new data
    exactly as after pfm_set_data on the member."""
    import torch
    import paper_1501_07844_gb300 as pfm
    vols = [synth.dagmf_problem(3320 + k, (8, 13, 35 + 3 * k), iters=30) for k in range(3)]
    new = torch.from_numpy((vols[1].D * 1.25).astype(np.float32)).pin_memory()
    newS = torch.from_numpy(vols[1].S_field).pin_memory()
    states = []
    for mode in ("prefetch", "set"):
        probs = [dict(D=torch.from_numpy(p.D).cuda(), S_field=torch.from_numpy(p.S_field).cuda(), s_node=p.s_node,
                      n_nodes=p.n_nodes, edges=p.edges) for p in vols]
        with pfm.Batch(probs, c=0.5, tau=0.11) as bt:
            bt.iterate(4)
            m = bt.members[1]
            if mode == "prefetch":
                m.prefetch_data(new, newS)
                m.commit_data()
            else:
                m.set_data(new, newS)
            bt.iterate(6)
            states.append([(bm.labels().cpu(), bm.flows().cpu()) for bm in bt.members])
    for (ua, qa), (ub, qb) in zip(*states):
        assert torch.equal(ua, ub) and torch.equal(qa, qb)


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
def test_state_async_equals_readback(storage):
    """pfm_get_state_async (device destinations, stream-ordered, no wait)
    gives the same dense arrays as pfm_get_labels / pfm_get_flows, padded
    rows included; host destinations are rejected."""
    import torch
    import paper_1501_07844_gb300 as pfm
    prob = synth.random_problem(180, (9, 13, 37), nl=5, s_kind="both")
    with gpu_problem(prob, storage=storage) as gp:
        gp.iterate(11)
        u, q = gp.state_async()
        gp.iterate(3)               # queued after the copies
        torch.cuda.synchronize()
        gp2 = None
        with gpu_problem(prob, storage=storage) as ref:
            ref.iterate(11)
            assert torch.equal(u, ref.labels()) and torch.equal(q, ref.flows())
        with pytest.raises(pfm.PfmError) as ei:
            gp.state_async(u_out=torch.empty_like(u.cpu()))
        assert ei.value.name == "PFM_EINVAL"


def test_argmax_async_equals_argmax():
    """pfm_get_argmax_async into pinned host memory, landed after
    pfm_readback_wait, equals pfm_get_argmax; a second read-back reuses the
    buffer only after the first copy."""
    import torch
    prob = synth.random_problem(190, (11, 17, 29), nl=6, s_kind="field")
    with gpu_problem(prob) as gp:
        h1 = torch.empty((11, 17, 29), dtype=torch.int32).pin_memory()
        h2 = torch.empty_like(h1).pin_memory()
        gp.iterate(5)
        gp.argmax_async(out=h1)
        ref1 = gp.argmax().cpu()
        gp.iterate(25)
        gp.argmax_async(out=h2)
        gp.readback_wait()
        assert torch.equal(h1, ref1) and torch.equal(h2, gp.argmax().cpu())


@pytest.mark.parametrize("kind", ["fused_f32", "fused_bf16", "fused_f16", "inplace", "hmf"])
def test_chunk_length_leaves_iterates_unchanged(kind):
    """The z-chunk length (planes per CTA) changes only which CTA runs a
    plane: the iterates are bit-identical for every length, the energy
    agrees up to its summation order; lengths beyond the volume clamp."""
    import paper_1501_07844_gb300 as pfm
    if kind == "hmf":
        prob = synth.hmf_problem(seed=2600, shape=(23, 18, 45))
    else:
        prob = synth.potts3d_problem(seed=2600, nl=8, shape=(23, 18, 45))
    sched = pfm.INPLACE if kind == "inplace" else pfm.FUSED
    storage = {"fused_bf16": pfm.BF16, "fused_f16": pfm.F16}.get(kind, pfm.F32)
    res = []
    for zc in (1, 4, 7, 64):
        with gpu_problem(prob, schedule=sched, storage=storage) as gp:
            gp.chunk_length = zc
            assert gp.chunk_length == min(zc, 23)
            gp.iterate(6)
            E, P = gp.iterate_energy(1)
            res.append((gp.labels().cpu().numpy(), gp.flows().cpu().numpy(), E, P))
    for u, q, E, P in res[1:]:
        assert np.array_equal(u, res[0][0]) and np.array_equal(q, res[0][1])
        # per-thread partials are compensated FP32 sums (about 1e-7 of a
        # thread's share), combined in FP64
        assert abs(E - res[0][2]) <= 1e-6 * abs(res[0][2])
        assert abs(P - res[0][3]) <= 1e-6 * abs(res[0][3]) + 1e-6


def test_tune_picks_a_candidate_and_restarts():
    """pfm_tune keeps one of its candidate lengths, leaves the problem in its
    initial state, and the solver then matches the oracle."""
    prob = synth.potts3d_problem(seed=2601, nl=8, shape=(40, 33, 70), iters=30)
    with gpu_problem(prob) as gp:
        zc = gp.tune(2)
        assert zc == gp.chunk_length and 1 <= zc <= 40
        assert gp.iterations == 0
        assert np.all(gp.labels().cpu().numpy() == np.float32(1.0 / 8))
        assert not np.any(gp.flows().cpu().numpy())
        compare(prob, gp, 30)
    with gpu_problem(prob) as gp:
        with pytest.raises(pfm_error()):
            gp.chunk_length = 0


def pfm_error():
    import paper_1501_07844_gb300 as pfm
    return pfm.PfmError


def test_bounded_wait_gives_up_and_the_context_survives():
    """Failure detection without a fault: a bounded mbarrier wait that
    nothing completes (the wait primitive of every TMA pipeline) gives up,
    the host reads PFM_ETIMEOUT, and the problem then solves correctly."""
    import time
    import paper_1501_07844_gb300 as pfm
    prob = synth.potts3d_problem(seed=2700, nl=8, shape=(12, 20, 40), iters=20)
    with gpu_problem(prob) as gp:
        t0 = time.time()
        st = pfm.lib().pfm_selftest_timeout(gp._h)
        assert st == 6, st  # PFM_ETIMEOUT
        assert b"self-test" in pfm.lib().pfm_last_error()
        assert time.time() - t0 < 60
        compare(prob, gp, 20)
