"""Parity at the full sizes of the other benchmark workloads, in the launch
configurations bench.py times, after each workload's own iteration count:
HMF 192^3 (tree kernel; FP32 voxel by voxel after 100 iterations, every
storage after the workload's 400 within the bounds FP32 storage itself
costs there), Ishikawa 256^3 with 8 labels (200 iterations, chain-specialised
kernel at the tuned chunk length), the 32-volume DAGMF batch (300
iterations, the batched four-inner-node kernel; every member bit for bit
against its single-problem run, three members against the oracle at every
voxel within bounds set by the rounding amplification measured there) and
the differentiable Potts 128^3 x 6 (100 unrolled iterations,
checkpoint every 10; the adjoint at 64 uniformly drawn entries against
central differences of the oracle's forward run)."""
import numpy as np
import pytest

import synth
from helpers import TOL_ARGMAX, TOL_E, TOL_U, gpu_problem, oracle_run

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def compare_state(name, u, q, E, P, o, tol_u, tol_e, margin=0.0, tol_p9999=None):
    u_o, q_o, E_o, P_o = o
    du = float(np.abs(u - u_o).max())
    if tol_p9999 is not None:
        p9999 = float(np.quantile(np.abs(u - u_o), 0.9999))
        print("PARITY %s p99.99 |du| %.3e" % (name, p9999))
        assert p9999 <= tol_p9999
    dq = float(np.abs(q - q_o).max())
    dE, dP = abs(E - E_o) / abs(E_o), abs(P - P_o) / max(abs(P_o), 1e-30)
    same = np.argmax(u, 0) == np.argmax(u_o, 0)
    decided = np.ones(same.shape, dtype=bool)
    if margin > 0:
        top2 = np.sort(u_o, axis=0)[-2:]
        decided = (top2[1] - top2[0]) >= margin
    agree = float(np.mean(same[decided]))
    print("PARITY %s du=%.3e dq=%.3e dE=%.3e dP=%.3e agree=%.6f decided=%.4f"
          % (name, du, dq, dE, dP, agree, float(decided.mean())))
    assert du <= tol_u and dq <= tol_u
    assert dE <= tol_e
    assert abs(P - P_o) <= tol_e * abs(P_o) + 1e-6
    assert decided.mean() >= 0.5 and agree >= TOL_ARGMAX


HMF_ITERS = 400
HMF_STRICT_ITERS = 100
# After its 400 iterations the HMF volume is still far from the optimum
# (relative gap 0.13) and amplifies rounding: the FP64 iteration whose only
# change is rounding its stored state (u, q) to FP32 after every iteration
# already differs from the oracle by max |du| 1.0 (labels agree on 99.855 %
# of voxels, relative E 1.07e-3), while a 2^-24 relative perturbation of D
# alone gives max |du| 0.18.  No FP32-storage implementation can meet the
# voxel-wise FP32 bounds there; the GPU's FP32 kernels land where that
# FP32-stored FP64 iteration lands (agreement 99.855 %, E 1.1e-3).  The
# voxel-wise bounds are asserted after 100 iterations; after 400 the bounds
# below, a little above what FP32 storage itself costs.
HMF400_BOUNDS = {0: dict(agree=0.998, dE=2e-3, dP=2e-3, p999=5e-2),
                 1: dict(agree=0.997, dE=3e-3, dP=3e-3, p999=8e-2),
                 2: dict(agree=0.99, dE=2e-2, dP=2e-2, p999=2e-1)}


@pytest.fixture(scope="module")
def hmf_case():
    prob = synth.hmf_problem(seed=2000, shape=(192, 192, 192))
    u, q, E, P = oracle_run(prob, HMF_STRICT_ITERS)
    early = (u.copy(), q.copy(), E, P)
    late = oracle_run(prob, HMF_ITERS - HMF_STRICT_ITERS, state=(u, q))
    return prob, early, late


@pytest.mark.parametrize("storage", [0, 1, 2], ids=["f32", "bf16", "f16"])
def test_hmf_192_every_voxel(hmf_case, storage):
    prob, early, late = hmf_case
    with gpu_problem(prob, storage=storage) as gp:
        assert gp.variant == "fused_tma_tree"
        gp.tune(3)
        gp.iterate(HMF_STRICT_ITERS)
        u1, q1, (E1, P1) = gp.labels().cpu().numpy(), gp.flows().cpu().numpy(), gp.energy()
        gp.iterate(HMF_ITERS - HMF_STRICT_ITERS)
        u, q, (E, P) = gp.labels().cpu().numpy(), gp.flows().cpu().numpy(), gp.energy()
    name = ("f32", "bf16", "f16")[storage]
    if storage == 0:
        compare_state("hmf192 f32 %d it" % HMF_STRICT_ITERS, u1, q1, E1, P1, early, TOL_U, TOL_E)
    del u1, q1
    u_o, q_o, E_o, P_o = late
    d = np.abs(u - u_o)
    r = dict(max=float(d.max()), p999=float(np.quantile(d, 0.999)),
             agree=float(np.mean(np.argmax(u, 0) == np.argmax(u_o, 0))),
             dE=abs(E - E_o) / abs(E_o), dP=abs(P - P_o) / abs(P_o))
    print("PARITY hmf192 %s %d it %s" % (name, HMF_ITERS, {k: "%.3e" % v for k, v in r.items()}))
    b = HMF400_BOUNDS[storage]
    assert r["agree"] >= b["agree"] and r["dE"] <= b["dE"] and r["dP"] <= b["dP"] and r["p999"] <= b["p999"], r


# The DAGMF volumes after 300 iterations have a few voxels (label
# boundaries where two end-labels share the voxel, e.g. 0.175 / 0.825) that
# amplify rounding: in the FP64 iteration, a 2^-24 relative perturbation of
# D alone moves u there by 1.1e-4 after 300 iterations, and perturbing the
# stored state by up to 4 FP32 ulps (uniform, independent) after every
# iteration moves it by 7.7e-4 (99.99th percentile 3.0e-5, flows 9.9e-5).
# The FP32 kernels, whose approximate exponential, reciprocal and summation
# orders err by a few ulps per step, land there: max |du| 8.0e-4 (general
# DAG kernel), 9.5e-4 (register-staged), 2.0e-3 (four-inner-node kernel),
# 99.99th percentile 2.5-2.8e-5.  Max |du| is bounded a little above that,
# the 99.99th percentile and the energies as everywhere else.
DAGMF300_TOL_U = 5e-3
DAGMF300_TOL_P9999 = 1e-4


def test_dagmf_batch_32_volumes_300_iterations():
    """The bench's 32 volumes (46.8 M voxels) after 300 batched iterations
    (graph-replayed, tuned z-chunk and grid): every member equals its
    single-problem TMA run bit for bit; three members (the smallest, the
    largest and one in between) match the oracle at every voxel within the
    bounds above."""
    import torch
    import paper_1501_07844_gb300 as pfm
    iters = 300
    vols = synth.dagmf_batch(seed=4000, count=32)
    stream = torch.cuda.Stream()
    probs = [dict(D=torch.from_numpy(p.D).cuda(), S_field=torch.from_numpy(p.S_field).cuda(), s_node=p.s_node,
                  n_nodes=p.n_nodes, edges=p.edges) for p in vols]
    sizes = [int(np.prod(p.spatial)) for p in vols]
    order = np.argsort(sizes)
    sampled = {int(order[0]), int(order[len(order) // 2]), int(order[-1])}
    with pfm.Batch(probs, c=0.5, tau=0.11, stream=stream.cuda_stream) as b:
        assert b.variant == "batched_tma_dag4"
        b.tune(trial_iters=3)
        b.iterate(iters)
        for k, p in enumerate(vols):
            u_b = b.members[k].labels().cpu().numpy()
            q_b = b.members[k].flows().cpu().numpy()
            with gpu_problem(p) as single:
                single.select_kernel("fused_tma_dag4")   # the batch's tile body
                single.iterate(iters)
                assert np.array_equal(u_b, single.labels().cpu().numpy())
                assert np.array_equal(q_b, single.flows().cpu().numpy())
                E, P = single.energy()
            if k in sampled:
                compare_state("dagmf member %d %s %d it" % (k, p.spatial, iters), u_b, q_b, E, P,
                              oracle_run(p, iters), DAGMF300_TOL_U, TOL_E, tol_p9999=DAGMF300_TOL_P9999)
            del u_b, q_b
    del probs
    torch.cuda.empty_cache()


def test_diff_128_gradients_at_64_random_entries():
    """dL/dD and dL/dS of L = -sum log u_target after 100 iterations
    (checkpoint every 10) against central differences of the FP64 oracle's
    forward run at 64 entries drawn uniformly (32 of D, 32 of S).  The loss
    is piecewise smooth (the capacity projection has a kink at |y| = S);
    an entry whose one-sided difference quotients on the oracle's runs
    disagree (a kink within the step) is replaced by a new draw."""
    import torch
    import oracle
    from paper_1501_07844_gb300.autograd import potts_solve
    prob = synth.diff_problem(seed=5000)
    iters = 100
    D = torch.tensor(prob.D, device="cuda", requires_grad=True)
    S = torch.tensor(prob.S_field, device="cuda", requires_grad=True)
    target = prob.truth.astype(np.int64)
    tgt = torch.from_numpy(target).cuda().unsqueeze(0)
    u = potts_solve(D, S, iters=iters, c=prob.c, tau=prob.tau, checkpoint_every=10)
    L = -torch.log(torch.gather(u.double(), 0, tgt)).sum()
    L.backward()
    gD = D.grad.double().cpu().numpy()
    gS = S.grad.double().cpu().numpy()
    D0, S0 = prob.D.astype(np.float64), prob.S_field.astype(np.float64)

    def loss(Dv, Sv):
        uo, qo = oracle.potts_init(prob.spatial, prob.n_leaf)
        oracle.potts_iterate(Dv, uo, qo, iters, prob.c, prob.tau, S_field=Sv)
        return float(-np.log(np.take_along_axis(uo, target[None], 0)).sum())

    L_o = loss(D0, S0)
    assert abs(float(L) - L_o) <= 1e-4 * abs(L_o)
    rng = np.random.default_rng(5001)
    h = 1e-5
    gscale = max(np.abs(gD).max(), np.abs(gS).max())
    rows, kinks = [], 0
    for which, count, shape in (("D", 32, D0.shape), ("S", 32, S0.shape)):
        got = 0
        while got < count:
            idx = tuple(int(rng.integers(0, s)) for s in shape)
            Dp, Dm, Sp, Sm = D0, D0, S0, S0
            if which == "D":
                Dp, Dm = D0.copy(), D0.copy()
                Dp[idx] += h
                Dm[idx] -= h
                g = gD[idx]
            else:
                if S0[idx] < 2 * h:
                    continue
                Sp, Sm = S0.copy(), S0.copy()
                Sp[idx] += h
                Sm[idx] -= h
                g = gS[idx]
            Lp, Lm = loss(Dp, Sp), loss(Dm, Sm)
            fwd, bwd = (Lp - L_o) / h, (L_o - Lm) / h
            if abs(fwd - bwd) > 2e-2 * max(abs(fwd), abs(bwd)) + 1e-5 * gscale:
                kinks += 1                        # a kink within the step: draw again
                continue
            rows.append((which, idx, g, (Lp - Lm) / (2 * h)))
            got += 1
    err = [abs(g - fd) / (abs(fd) + 1e-6 * gscale) for _, _, g, fd in rows]
    worst = int(np.argmax(err))
    print("ADJOINT diff128 64 entries: worst rel err %.3e at %s (g=%.6e fd=%.6e), |g|max=%.3e, redrawn %d"
          % (err[worst], rows[worst][:2], rows[worst][2], rows[worst][3], gscale, kinks))
    for which, idx, g, fd in rows:
        assert abs(g - fd) <= 1e-3 * abs(fd) + 1e-6 * gscale, (which, idx, g, fd)


def test_ishikawa_256_every_voxel_after_200_iterations():
    """The bench's Ishikawa volume (256^3, 7 levels / 8 labels) on the
    chain-specialised kernel at the tuned chunk length, against the oracle's
    literal Algorithm 3 at every voxel after 200 iterations."""
    import oracle
    nlev, iters = 7, 200
    prob = synth.ishikawa_problem(seed=2000, spatial=(256, 256, 256), nlev=nlev)
    with gpu_problem(prob) as gp:
        assert gp.variant == "fused_tma_ishikawa"
        gp.tune(3)
        gp.iterate(iters)
        u = gp.labels().cpu().numpy()
        q = gp.flows().cpu().numpy()
        E, P = gp.energy()
    D = prob.D.astype(np.float64)
    u3, q3 = oracle.ishikawa_init(prob.spatial, nlev)
    oracle.ishikawa_iterate(D, u3, q3, iters, prob.c, prob.tau, s_level=prob.s_node[:nlev].astype(np.float64))
    # energy of the Ishikawa model: the chain's DAG energy (Section 3.4), the
    # labels carrying no flow
    qd = np.concatenate([q3, np.zeros((prob.n_nodes - nlev,) + q3.shape[1:])])
    E3, P3 = oracle.dag_energy(oracle.Dag(prob.n_nodes, prob.edges), D, u3, qd,
                               s_node=prob.s_node.astype(np.float64))
    del qd
    du = float(np.abs(u - u3).max())
    dq = float(np.abs(q[:nlev] - q3).max())
    agree = float(np.mean(np.argmax(u, 0) == np.argmax(u3, 0)))
    print("PARITY ishikawa256 %d it du=%.3e dq=%.3e dE=%.3e dP=%.3e agree=%.6f"
          % (iters, du, dq, abs(E - E3) / abs(E3), abs(P - P3) / abs(P3), agree))
    assert du <= TOL_U and dq <= TOL_U and not np.any(q[nlev:])
    assert abs(E - E3) <= TOL_E * abs(E3) and abs(P - P3) <= TOL_E * abs(P3)
    assert agree >= TOL_ARGMAX
