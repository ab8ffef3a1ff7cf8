"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a
hand-computed value, a closed form, an invariant, an independent algorithm
(explicit-flow ALM, linear programming, exhaustive search) or the paper's
own definitions (path weights W, flow excess d).
"""
import math

import numpy as np
import pytest

import synth


def softmax_closed_form(D, k, c):
    """S = 0 (or spatially constant D): q stays 0, so after k iterations of
    Algorithm 1 u_L = exp(-k D_L / c) / sum_L' exp(-k D_L' / c)."""
    z = -k * D.astype(np.float64) / c
    z -= z.max(axis=0, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=0, keepdims=True)


# ---------------------------------------------------------------- operators

def test_grad_hand_values(orc):
    u = np.array([[1.0, 4.0, 2.0],
                  [0.5, 0.0, 7.0]])          # (ny=2, nx=3)
    g = orc.grad(u)
    gx = np.array([[3.0, -2.0, 0.0], [-0.5, 7.0, 0.0]])
    gy = np.array([[-0.5, -4.0, 5.0], [0.0, 0.0, 0.0]])
    assert np.array_equal(g[0], gx) and np.array_equal(g[1], gy)


def test_div_hand_values(orc):
    qx = np.array([[1.0, 2.0, 9.0]])          # last x entry is ignored
    qy = np.array([[5.0, 5.0, 5.0]])          # ny = 1: y flow never enters
    d = orc.div(np.stack([qx, qy]))
    assert np.array_equal(d, np.array([[1.0, 1.0, -2.0]]))


@pytest.mark.parametrize("spatial", [(7, 5), (4, 6, 5), (1, 9), (3, 1, 4)])
def test_div_is_negative_adjoint_of_grad(orc, spatial):
    rng = np.random.default_rng(1)
    u = rng.standard_normal(spatial)
    q = rng.standard_normal((len(spatial),) + spatial)
    lhs = np.sum(orc.grad(u) * q)
    rhs = -np.sum(u * orc.div(q))
    assert abs(lhs - rhs) <= 1e-12 * (1 + abs(lhs))


def test_projection_iso_and_aniso(orc):
    rng = np.random.default_rng(2)
    for _ in range(200):
        y = rng.standard_normal(3) * rng.uniform(0.01, 3)
        s = rng.uniform(0, 2)
        p = orc.project(y, s, orc.ISO)
        r = np.linalg.norm(y)
        if r <= s:
            assert np.array_equal(p, y)
        else:
            assert abs(np.linalg.norm(p) - s) <= 1e-12 and np.allclose(p * r, y * s)
        # nearest point of the ball: no sampled ball point is closer
        pts = rng.standard_normal((64, 3))
        pts *= (s * rng.random((64, 1)) ** (1 / 3)) / np.maximum(np.linalg.norm(pts, axis=1, keepdims=True), 1e-300)
        assert np.linalg.norm(y - p) <= np.min(np.linalg.norm(pts - y, axis=1)) + 1e-12
        pa = orc.project(y, s, orc.ANISO)
        assert np.array_equal(pa, np.clip(y, -s, s))
    assert np.array_equal(orc.project([0.3, -0.4], 0.0, orc.ISO), np.zeros(2))


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("spatial", [(9, 11), (3, 4, 5)])
def test_potts_zero_capacity_closed_form(orc, mode, spatial):
    p = synth.random_problem(3, spatial, nl=4)
    D = p.D.astype(np.float64)
    S = np.zeros(spatial)
    u, q = orc.potts_init(spatial, 4)
    done = 0
    for k in (1, 7, 20):
        orc.potts_iterate(D, u, q, k - done, 0.5, 0.11, S_field=S, grad_source=mode)
        done = k
        assert np.abs(u - softmax_closed_form(D, k, 0.5)).max() <= 1e-13
        assert np.all(q == 0.0)


@pytest.mark.parametrize("mode", [0, 1])
def test_potts_constant_data_any_capacity(orc, mode):
    rng = np.random.default_rng(4)
    spatial = (6, 5)
    D = np.broadcast_to(rng.random((3, 1, 1)), (3,) + spatial).copy()
    S = rng.random(spatial)
    u, q = orc.potts_init(spatial, 3)
    orc.potts_iterate(D, u, q, 15, 0.5, 0.11, S_field=S, grad_source=mode)
    assert np.abs(u - softmax_closed_form(D, 15, 0.5)).max() <= 1e-13
    assert np.all(q == 0.0)


def test_dag_zero_capacity_closed_form(orc):
    """With q = 0 the excess of an end-label is its own data term (d_S = 0,
    inner nodes carry no data), so the Potts closed form holds on leaves."""
    rng = np.random.default_rng(5)
    nn, edges = synth.random_dag(rng, 3, 5, 2)
    dag = orc.Dag(nn, edges)
    spatial = (4, 5, 3)
    D = rng.random((5,) + spatial)
    u, q = orc.dag_init(spatial, dag)
    orc.dag_iterate(dag, D, u, q, 12, 0.5, 0.11, S_field=np.zeros(spatial))
    assert np.abs(u - softmax_closed_form(D, 12, 0.5)).max() <= 1e-13


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("norm", [0, 1])
def test_potts_invariants_every_iteration(orc, mode, norm):
    p = synth.random_problem(6, (5, 7, 6), nl=4, s_kind="both")
    D, S, sn = p.D.astype(np.float64), p.S_field.astype(np.float64), p.s_node.astype(np.float64)
    u, q = orc.potts_init(p.spatial, 4)
    cap = sn[:, None, None, None] * S[None]
    for _ in range(25):
        orc.potts_iterate(D, u, q, 1, 0.5, 0.11, S_field=S, s_node=sn, norm=norm, grad_source=mode)
        assert np.all(u >= 0) and np.abs(u.sum(0) - 1).max() <= 1e-12
        mag = np.sqrt((q ** 2).sum(1)) if norm == 0 else np.abs(q).max(1)
        assert np.all(mag <= cap * (1 + 1e-12) + 1e-300)
        # zero normal flux at the far boundary of every axis
        assert np.all(q[:, 0, :, :, -1] == 0) and np.all(q[:, 1, :, -1, :] == 0) and np.all(q[:, 2, -1] == 0)
        E, P = orc.potts_energy(D, u, q, S_field=S, s_node=sn, norm=norm)
        assert E - P >= -1e-12 * abs(E)


@pytest.mark.parametrize("mode", [0, 1])
def test_dag_invariants_every_iteration(orc, mode):
    rng = np.random.default_rng(7)
    nn, edges = synth.random_dag(rng, 3, 6, 2)
    dag = orc.Dag(nn, edges)
    spatial = (6, 5)
    D = rng.random((6,) + spatial)
    sn = rng.uniform(0.05, 0.5, nn)
    u, q = orc.dag_init(spatial, dag)
    for _ in range(20):
        orc.dag_iterate(dag, D, u, q, 1, 0.5, 0.11, s_node=sn, grad_source=mode)
        assert np.all(u >= 0) and np.abs(u.sum(0) - 1).max() <= 1e-12
        assert np.all(np.sqrt((q ** 2).sum(1)) <= sn[:, None, None] * (1 + 1e-12))
        E, P = orc.dag_energy(dag, D, u, q, s_node=sn)
        assert E - P >= -1e-12 * abs(E)


@pytest.mark.parametrize("norm", [0, 1])
def test_weak_duality_random_feasible_pairs(orc, norm):
    """P(q) <= E(u) for ANY simplex u and ANY capacity-feasible q."""
    rng = np.random.default_rng(8)
    nn, edges = synth.hmf_tree(2, 3)
    dag = orc.Dag(nn, edges)
    spatial = (4, 5, 6)
    for trial in range(10):
        D = rng.random((6,) + spatial)
        u = rng.random((6,) + spatial) ** 3
        u /= u.sum(0)
        sn = rng.uniform(0, 0.6, nn)
        q = rng.standard_normal((nn, 3) + spatial)
        for A in range(nn):
            for idx in np.ndindex(spatial):
                q[(A, slice(None)) + idx] = orc.project(q[(A, slice(None)) + idx], sn[A], norm)
        E, P = orc.dag_energy(dag, D, u, q, s_node=sn, norm=norm)
        assert P <= E + 1e-12
        E2, P2 = orc.potts_energy(D, u, q[:6], s_node=sn[:6], norm=norm)
        assert P2 <= E2 + 1e-12


# ---------------------------------------------------------------- the paper's own definitions

def test_path_weights_definition(orc):
    # S -> 0 (w 1), S -> 1 (w 1); 0 -> 2 (0.5), 1 -> 2 (0.5), 0 -> 3 (0.5), 1 -> 3 (0.25), 1 -> 4 (0.25)
    edges = [(-1, 0, 1.0), (-1, 1, 1.0), (0, 2, 0.5), (1, 2, 0.5), (0, 3, 0.5), (1, 3, 0.25), (1, 4, 0.25)]
    W = orc.Dag(5, edges).path_weights()
    expect = np.eye(5)
    expect[0, 2], expect[1, 2], expect[0, 3], expect[1, 3], expect[1, 4] = 0.5, 0.5, 0.5, 0.25, 0.25
    assert np.array_equal(W, expect)
    # two-level paths multiply and add
    edges2 = [(-1, 0, 1.0), (0, 1, 0.5), (0, 2, 0.5), (1, 3, 1.0), (2, 3, 1.0)]
    W2 = orc.Dag(4, edges2).path_weights()
    assert W2[0, 3] == 1.0 and W2[1, 3] == 1.0 and W2[0, 1] == 0.5


def test_generated_dags_have_unit_source_weight(orc):
    rng = np.random.default_rng(9)
    for _ in range(20):
        nn, edges = synth.random_dag(rng, 4, 10, 2)
        dag = orc.Dag(nn, edges)
        W = dag.path_weights()
        roots = [b for a, b, _ in edges if a == -1]
        w_s = {b: w for a, b, w in edges if a == -1}
        for leaf in dag.leaves():
            assert abs(sum(w_s[r] * W[r, leaf] for r in roots) - 1.0) <= 1e-12


def test_dag_excess_equals_path_weight_form(orc):
    """The top-down pass of Algorithm 2 equals the definition of d_L in
    Section 3.3 unrolled with the path weights: d_leaf = sum_A W_(A,leaf) e_A,
    e_A = div q_A (+ D_A on end-labels).  Checked through P(q) = sum min d."""
    rng = np.random.default_rng(10)
    nn, edges = synth.random_dag(rng, 3, 5, 2)
    dag = orc.Dag(nn, edges)
    W = dag.path_weights()
    leaves = dag.leaves()
    spatial = (5, 4, 3)
    D = rng.random((5,) + spatial)
    q = 0.3 * rng.standard_normal((nn, 3) + spatial)
    u = np.full((5,) + spatial, 0.2)
    _, P = orc.dag_energy(dag, D, u, q)
    e = np.stack([orc.div(q[A]) for A in range(nn)])
    for j, leaf in enumerate(leaves):
        e[leaf] += D[j]
    d = np.stack([sum(W[A, leaf] * e[A] for A in range(nn)) for leaf in leaves])
    assert abs(P - d.min(0).sum()) <= 1e-12 * (1 + abs(P))


def test_flat_dag_is_potts_bitwise(orc):
    for mode in (0, 1):
        p = synth.random_problem(11, (6, 7), nl=4, s_kind="both")
        D, S, sn = (a.astype(np.float64) for a in (p.D, p.S_field, p.s_node))
        u1, q1 = orc.potts_init(p.spatial, 4)
        orc.potts_iterate(D, u1, q1, 30, 0.5, 0.11, S_field=S, s_node=sn, grad_source=mode)
        dag = orc.Dag.flat(4)
        u2, q2 = orc.dag_init(p.spatial, dag)
        orc.dag_iterate(dag, D, u2, q2, 30, 0.5, 0.11, S_field=S, s_node=sn, grad_source=mode)
        assert np.array_equal(u1, u2) and np.array_equal(q1, q2)
        assert orc.potts_energy(D, u1, q1, S, sn) == orc.dag_energy(dag, D, u2, q2, S, sn)


def test_malformed_dags_rejected(orc):
    for n, edges in [(2, [(-1, 0, 1.0), (0, 1, 1.0), (1, 0, 1.0)]),      # cycle
                     (2, [(-1, 0, 1.0)]),                                  # orphan node 1
                     (2, [(-1, 0, 1.0), (0, 5, 1.0)]),                     # bad index
                     (1, [(-1, 0, 1.0), (0, 0, 1.0)])]:                   # self loop
        assert orc.Dag(n, edges).n_leaves() == -1


# ---------------------------------------------------------------- optimum pins

def _lp_optimum(D, W, leaves, S_field, s_node, norm_aniso=True):
    """Relaxed optimum of Eq. dagmf_original (Potts: W = I) with the l1
    (anisotropic) TV, solved as a linear program by HiGHS.  The difference
    operators are built here from scratch, independently of the oracle."""
    from scipy.optimize import linprog
    from scipy import sparse
    nl = D.shape[0]
    spatial = D.shape[1:]
    n = int(np.prod(spatial))
    nd = len(spatial)
    idx = np.arange(n).reshape(spatial)
    Gs = []
    for comp in range(nd):
        ax = nd - 1 - comp                    # component 0 = x = last numpy axis
        rows, cols, vals = [], [], []
        for pos in np.ndindex(spatial):
            if pos[ax] + 1 < spatial[ax]:
                nxt = list(pos)
                nxt[ax] += 1
                i, j = idx[pos], idx[tuple(nxt)]
                rows += [i, i]
                cols += [j, i]
                vals += [1.0, -1.0]
        Gs.append(sparse.csr_matrix((vals, (rows, cols)), shape=(n, n)))
    nn = W.shape[0]
    nu, nt = nl * n, nn * nd * n
    cost = np.concatenate([D.reshape(-1)])
    capv = []
    for A in range(nn):
        s = s_node[A] if s_node is not None else 1.0
        f = S_field.reshape(-1) if S_field is not None else np.ones(n)
        for _ in range(nd):
            capv.append(s * f)
    cost = np.concatenate([D.reshape(-1), np.concatenate(capv)])
    A_ub_blocks = []
    for A in range(nn):
        # u_A = sum_leaf W[A, leaf] u_leaf
        Wrow = sparse.hstack([W[A, leaf] * sparse.identity(n) for leaf in leaves])
        for comp in range(nd):
            GA = Gs[comp] @ Wrow
            sel = sparse.lil_matrix((n, nt))
            base = (A * nd + comp) * n
            sel[np.arange(n), base + np.arange(n)] = -1.0
            A_ub_blocks.append(sparse.hstack([GA, sel.tocsr()]))
            A_ub_blocks.append(sparse.hstack([-GA, sel.tocsr()]))
    A_ub = sparse.vstack(A_ub_blocks).tocsr()
    A_eq = sparse.hstack([sparse.hstack([sparse.identity(n)] * nl), sparse.csr_matrix((n, nt))])
    res = linprog(cost, A_ub=A_ub, b_ub=np.zeros(A_ub.shape[0]), A_eq=A_eq, b_eq=np.ones(n),
                  bounds=(0, None), method="highs")
    assert res.status == 0
    return res.fun


def _converge_potts(orc, D, S, sn, norm, iters=20000, c=1.0, tau=0.25):
    u, q = orc.potts_init(D.shape[1:], D.shape[0])
    orc.potts_iterate(D, u, q, iters, c, tau, S_field=S, s_node=sn, norm=norm)
    return u, q, orc.potts_energy(D, u, q, S_field=S, s_node=sn, norm=norm)


@pytest.mark.parametrize("spatial", [(5, 4), (3, 3, 3)])
def test_potts_converges_to_lp_optimum_aniso(orc, spatial):
    rng = np.random.default_rng(12)
    D = rng.random((3,) + spatial)
    S = 0.4 * rng.random(spatial)
    tau = 0.25 if len(spatial) == 2 else 0.16
    u, q, (E, P) = _converge_potts(orc, D, S, None, orc.ANISO, tau=tau)
    lp = _lp_optimum(D, np.eye(3), [0, 1, 2], S, None)
    assert abs(E - lp) <= 1e-8 * abs(lp) and abs(P - lp) <= 1e-8 * abs(lp)


@pytest.mark.parametrize("kind", ["hmf", "dag"])
def test_dag_converges_to_lp_optimum_aniso(orc, kind):
    rng = np.random.default_rng(13)
    if kind == "hmf":
        nn, edges = synth.hmf_tree(2, 2)
    else:
        nn, edges = synth.random_dag(rng, 2, 4, 2)
    dag = orc.Dag(nn, edges)
    leaves = dag.leaves()
    spatial = (4, 5)
    D = rng.random((len(leaves),) + spatial)
    sn = rng.uniform(0.05, 0.5, nn)
    u, q = orc.dag_init(spatial, dag)
    orc.dag_iterate(dag, D, u, q, 30000, 1.0, 0.15, s_node=sn, norm=orc.ANISO)
    E, P = orc.dag_energy(dag, D, u, q, s_node=sn, norm=orc.ANISO)
    lp = _lp_optimum(D, dag.path_weights(), leaves, None, sn)
    assert abs(E - lp) <= 1e-7 * abs(lp) and abs(P - lp) <= 1e-7 * abs(lp)


def test_potts_iso_matches_explicit_flow_alm(orc):
    """The pseudo-flow optimum equals the full-flow continuous max-flow
    optimum (the equivalence chain of Section 3.2)."""
    rng = np.random.default_rng(14)
    spatial = (12, 10)
    D = rng.random((3,) + spatial)
    S = 0.3 * np.ones(spatial)
    u, q, (E, P) = _converge_potts(orc, D, S, None, orc.ISO, iters=30000)
    flow, _ = orc.alm_potts(D, 40000, 0.3, 0.25, S_field=S)
    assert (E - P) <= 1e-10 * abs(E)
    assert abs(E - flow) <= 1e-9 * abs(flow)


@pytest.mark.parametrize("seed", range(6))
def test_two_label_threshold_equals_bruteforce(orc, seed):
    rng = np.random.default_rng(100 + seed)
    spatial = (4, 4)
    D = rng.random((2,) + spatial)
    sn = np.array([0.15, 0.15]) * rng.uniform(0.5, 2)
    u, q, (E, P) = _converge_potts(orc, D, None, sn, orc.ANISO, iters=20000)
    best, second, lab0 = orc.bruteforce_binary(D, s_node=sn, norm=orc.ANISO)
    thr = (u[0] > 0.5).astype(np.float64)
    ub = np.stack([thr, 1 - thr])
    Eb, _ = orc.potts_energy(D, ub, np.zeros((2, 2) + spatial), s_node=sn, norm=orc.ANISO)
    assert abs(E - best) <= 1e-8 and abs(Eb - best) <= 1e-9
    if second - best > 1e-6:
        assert np.array_equal(thr.astype(np.uint8), lab0)


def test_two_label_1d_iso_equals_bruteforce(orc):
    rng = np.random.default_rng(120)
    spatial = (1, 16)                       # ISO and ANISO coincide on a line
    D = rng.random((2,) + spatial)
    sn = np.array([0.1, 0.1])
    u, q, (E, P) = _converge_potts(orc, D, None, sn, orc.ISO, iters=20000)
    best, _, _ = orc.bruteforce_binary(D, s_node=sn, norm=orc.ISO)
    assert abs(E - best) <= 1e-8


def test_chain_reduction_to_potts(orc):
    """A leaf whose only parent is an inner node with that single child:
    u_inner = u_leaf, so at the optimum the DAG energy equals Potts with the
    two capacities added on that label (Eq. dagmf_original)."""
    rng = np.random.default_rng(15)
    spatial = (6, 6)
    D = rng.random((3,) + spatial)
    # nodes: 0 inner (under S), leaves 1, 2, 3; 1 under 0, 2 and 3 under S
    edges = [(-1, 0, 1.0), (0, 1, 1.0), (-1, 2, 1.0), (-1, 3, 1.0)]
    dag = orc.Dag(4, edges)
    sn = np.array([0.2, 0.1, 0.25, 0.15])
    u, q = orc.dag_init(spatial, dag)
    orc.dag_iterate(dag, D, u, q, 30000, 1.0, 0.2, s_node=sn)
    E, P = orc.dag_energy(dag, D, u, q, s_node=sn)
    _, _, (E2, P2) = _converge_potts(orc, D, None, np.array([0.3, 0.25, 0.15]), orc.ISO, iters=30000)
    assert abs(E - E2) <= 1e-8 * abs(E2) and (E - P) <= 1e-8 * abs(E)


@pytest.mark.parametrize("mode", [0, 1])
def test_algorithm3_equals_algorithm2_on_the_ishikawa_chain(orc, mode):
    """Section 3.4: Ishikawa is the DAGMF model on a chain (Alg. 3 is Alg. 2
    specialised): the level flows are the inner-node flows, the labels carry
    none."""
    N = 4
    prob = synth.ishikawa_problem(5400, (6, 7, 9), nlev=N)
    D = prob.D.astype(np.float64)
    s_level = prob.s_node[:N].astype(np.float64)
    u3, q3 = orc.ishikawa_init(prob.spatial, N)
    orc.ishikawa_iterate(D, u3, q3, 25, 0.5, 0.11, s_level=s_level, grad_source=mode)
    dag = orc.Dag(prob.n_nodes, prob.edges)
    u2, q2 = orc.dag_init(prob.spatial, dag)
    orc.dag_iterate(dag, D, u2, q2, 25, 0.5, 0.11, s_node=prob.s_node.astype(np.float64), grad_source=mode)
    assert np.abs(u3 - u2).max() <= 1e-12
    assert np.abs(q3 - q2[:N]).max() <= 1e-12 and np.all(q2[N:] == 0)


def test_ishikawa_converges_to_lp_optimum(orc):
    """Ishikawa energy (Section 1): data on the labels, TV on the cumulative
    labels u_{A_i} = sum_{j >= i} u_{L_j}; relaxed optimum by LP (ANISO)."""
    N = 3
    prob = synth.ishikawa_problem(5500, (5, 6), nlev=N)
    D = prob.D.astype(np.float64)
    dag = orc.Dag(prob.n_nodes, prob.edges)
    s_level = prob.s_node[:N].astype(np.float64)
    u, q = orc.ishikawa_init(prob.spatial, N)
    orc.ishikawa_iterate(D, u, q, 30000, 1.0, 0.15, s_level=s_level, norm=orc.ANISO)
    qd = np.concatenate([q, np.zeros((N + 1,) + q.shape[1:])])
    E, P = orc.dag_energy(dag, D, u, qd, s_node=prob.s_node.astype(np.float64), norm=orc.ANISO)
    lp = _lp_optimum(D, dag.path_weights(), dag.leaves(), None, prob.s_node.astype(np.float64))
    assert abs(E - lp) <= 1e-7 * abs(lp) and abs(P - lp) <= 1e-7 * abs(lp)


# ---------------------------------------------------------------- PAPER_LITERAL worked by hand
#
# The flow step as Algorithms 1, 2 and 3 print it differentiates the
# UNNORMALISED product u exp(-d/c), formed before the normaliser a(x)
# divides it out.  These two-voxel examples (grid nx = 2, ny = 1, so only the
# x flow at x = 0 can be nonzero: the forward difference is zero at the last
# index and along y) are worked by hand from the algorithms' lines, two
# iterations each so that the second divergence uses the literal flow.  The
# data terms are multiples of ln 2 with c = 1, so the first iteration's
# numbers are exact binary fractions; the applied step is c tau = 1/4.
# Divergence on this grid: div q = (q(0), -q(0)).

LN2 = math.log(2.0)
C_HAND, TAU_HAND = 1.0, 0.25
STEP_HAND = C_HAND * TAU_HAND


def _clip(y, s):
    """Proj onto |y| <= s for a one-component (x-only) flow; also returns
    whether the capacity was active."""
    return (max(-s, min(s, y)), abs(y) > s)


def test_potts_paper_literal_worked_by_hand(orc):
    """Algorithm 1 with the flow step on u exp(-(D + div q)/c), two labels."""
    D = np.array([[[0.0, 2 * LN2]], [[LN2, 0.0]]])      # [label][y][x]
    s = np.array([0.2, 1.0])                             # capacity per label
    # iteration 1: q = 0, div q = 0, u = 1/2
    ut0 = [0.5, 0.125]                                   # 0.5 * 2^0, 0.5 * 2^-2
    ut1 = [0.25, 0.5]                                    # 0.5 * 2^-1, 0.5 * 2^0
    q0, act0 = _clip(0.0 - STEP_HAND * (ut0[1] - ut0[0]), s[0])   # 0.09375
    q1, act1 = _clip(0.0 - STEP_HAND * (ut1[1] - ut1[0]), s[1])   # -0.0625
    assert (q0, q1, act0, act1) == (0.09375, -0.0625, False, False)
    a = [ut0[0] + ut1[0], ut0[1] + ut1[1]]               # 3/4, 5/8
    u0 = [ut0[0] / a[0], ut0[1] / a[1]]                  # 2/3, 1/5
    u1 = [ut1[0] / a[0], ut1[1] / a[1]]                  # 1/3, 4/5
    u, q = orc.potts_init((1, 2), 2)
    orc.potts_iterate(D, u, q, 1, C_HAND, TAU_HAND, s_node=s, grad_source=orc.PAPER_LITERAL)
    assert np.abs(u[:, 0] - [u0, u1]).max() <= 1e-15
    assert np.array_equal(q[:, 0, 0], [[q0, 0.0], [q1, 0.0]]) and not np.any(q[:, 1])
    # iteration 2: d_L = D_L + div q_L with the literal flows
    ut0 = [u0[0] * math.exp(-(0.0 + q0)), u0[1] * math.exp(-(2 * LN2 - q0))]
    ut1 = [u1[0] * math.exp(-(LN2 + q1)), u1[1] * math.exp(-(0.0 - q1))]
    q0, act0 = _clip(q0 - STEP_HAND * (ut0[1] - ut0[0]), s[0])
    q1, act1 = _clip(q1 - STEP_HAND * (ut1[1] - ut1[0]), s[1])
    assert act0 and not act1 and q0 == 0.2               # the capacity bites on label 0 now
    a = [ut0[0] + ut1[0], ut0[1] + ut1[1]]
    u_hand = np.array([[ut0[0] / a[0], ut0[1] / a[1]], [ut1[0] / a[0], ut1[1] / a[1]]])
    orc.potts_iterate(D, u, q, 1, C_HAND, TAU_HAND, s_node=s, grad_source=orc.PAPER_LITERAL)
    assert np.abs(u[:, 0] - u_hand).max() <= 1e-15
    assert np.abs(q[:, 0, 0] - [[q0, 0.0], [q1, 0.0]]).max() <= 1e-15 and not np.any(q[:, 1])
    # the flow step on the normalised labelling gives different numbers
    un, qn = orc.potts_init((1, 2), 2)
    orc.potts_iterate(D, un, qn, 2, C_HAND, TAU_HAND, s_node=s, grad_source=orc.NORMALISED)
    assert np.abs(qn[1, 0, 0, 0] - q1) > 1e-2 and np.abs(un - u).max() > 1e-3


def test_potts_normalised_first_iteration_by_hand(orc):
    """Algorithm 1 with the flow step on the normalised labelling (the
    gradient of Eq. potts_bregmanopt), first iteration of the same example."""
    D = np.array([[[0.0, 2 * LN2]], [[LN2, 0.0]]])
    s = np.array([0.2, 1.0])
    u, q = orc.potts_init((1, 2), 2)
    orc.potts_iterate(D, u, q, 1, C_HAND, TAU_HAND, s_node=s, grad_source=orc.NORMALISED)
    # u = (2/3, 1/5) and (1/3, 4/5); y_L = -1/4 (u_L(1) - u_L(0))
    assert np.abs(u[:, 0] - [[2 / 3, 0.2], [1 / 3, 0.8]]).max() <= 1e-15
    assert np.abs(q[:, 0, 0, 0] - [0.25 * (2 / 3 - 0.2), -0.25 * (0.8 - 1 / 3)]).max() <= 1e-15


def test_dag_paper_literal_worked_by_hand(orc):
    """Algorithm 2 on S -> A -> {L0, L1} (w = 1): the inner node's flow is
    driven by g_A = sum of its end-labels' UNNORMALISED products, which is
    the normaliser a(x) -- not 1, as it would be on the normalised labels
    (where q_A stays zero)."""
    dag = orc.Dag(3, [(-1, 0, 1.0), (0, 1, 1.0), (0, 2, 1.0)])
    D = np.array([[[0.0, 2 * LN2]], [[LN2, 0.0]]])      # leaves L0 (node 1), L1 (node 2)
    s = np.array([0.05, 0.2, 1.0])                       # A, L0, L1
    # iteration 1: q = 0, d = D on the leaves, u = 1/2
    ut0, ut1 = [0.5, 0.125], [0.25, 0.5]
    qL0, _ = _clip(-STEP_HAND * (ut0[1] - ut0[0]), s[1])           # 0.09375
    qL1, _ = _clip(-STEP_HAND * (ut1[1] - ut1[0]), s[2])           # -0.0625
    gA = [ut0[0] + ut1[0], ut0[1] + ut1[1]]                        # 3/4, 5/8
    qA, actA = _clip(-STEP_HAND * (gA[1] - gA[0]), s[0])           # 1/32
    assert (qL0, qL1, qA, actA) == (0.09375, -0.0625, 0.03125, False)
    u0, u1 = [ut0[0] / gA[0], ut0[1] / gA[1]], [ut1[0] / gA[0], ut1[1] / gA[1]]
    u, q = orc.dag_init((1, 2), dag)
    orc.dag_iterate(dag, D, u, q, 1, C_HAND, TAU_HAND, s_node=s, grad_source=orc.PAPER_LITERAL)
    assert np.abs(u[:, 0] - [u0, u1]).max() <= 1e-15
    assert np.array_equal(q[:, 0, 0], [[qA, 0.0], [qL0, 0.0], [qL1, 0.0]]) and not np.any(q[:, 1])
    # iteration 2: top-down excess d_L = D_L + div q_L + d_A, d_A = div q_A
    dA = [qA, -qA]
    d0 = [0.0 + qL0 + dA[0], 2 * LN2 - qL0 + dA[1]]
    d1 = [LN2 + qL1 + dA[0], 0.0 - qL1 + dA[1]]
    ut0 = [u0[k] * math.exp(-d0[k]) for k in range(2)]
    ut1 = [u1[k] * math.exp(-d1[k]) for k in range(2)]
    qL0, _ = _clip(qL0 - STEP_HAND * (ut0[1] - ut0[0]), s[1])
    qL1, _ = _clip(qL1 - STEP_HAND * (ut1[1] - ut1[0]), s[2])
    gA = [ut0[0] + ut1[0], ut0[1] + ut1[1]]
    qA, actA = _clip(qA - STEP_HAND * (gA[1] - gA[0]), s[0])
    assert not actA and abs(qA) > 1e-3
    u_hand = np.array([[ut0[0] / gA[0], ut0[1] / gA[1]], [ut1[0] / gA[0], ut1[1] / gA[1]]])
    orc.dag_iterate(dag, D, u, q, 1, C_HAND, TAU_HAND, s_node=s, grad_source=orc.PAPER_LITERAL)
    assert np.abs(u[:, 0] - u_hand).max() <= 1e-15
    assert np.abs(q[:, 0, 0] - [[qA, 0.0], [qL0, 0.0], [qL1, 0.0]]).max() <= 1e-15 and not np.any(q[:, 1])
    # on the normalised labels the inner flow never moves
    un, qn = orc.dag_init((1, 2), dag)
    orc.dag_iterate(dag, D, un, qn, 2, C_HAND, TAU_HAND, s_node=s, grad_source=orc.NORMALISED)
    assert not np.any(qn[0])


def test_ishikawa_paper_literal_worked_by_hand(orc):
    """Algorithm 3 with N = 2 levels (labels L0, L1, L2): the cumulative
    excess d_{L_i} = D_{L_i} + div q_1 + ... + div q_i, and the level flows
    driven by the bottom-up sums g_1 = u~_1 + u~_2, g_2 = u~_2 of the
    UNNORMALISED products."""
    D = np.array([[[0.0, 2 * LN2]], [[LN2, LN2]], [[2 * LN2, 0.0]]])
    s = np.array([0.2, 0.05])                            # levels 1, 2
    # iteration 1: q = 0, u = 1/3
    ut = [[1 / 3, 1 / 12], [1 / 6, 1 / 6], [1 / 12, 1 / 3]]
    g1 = [ut[1][0] + ut[2][0], ut[1][1] + ut[2][1]]                 # 1/4, 1/2
    g2 = ut[2]
    q1, act1 = _clip(-STEP_HAND * (g1[1] - g1[0]), s[0])           # -1/16
    q2, act2 = _clip(-STEP_HAND * (g2[1] - g2[0]), s[1])           # -1/16 -> -0.05
    assert (q1, act1, q2, act2) == (-0.0625, False, -0.05, True)
    a = [sum(ut[L][k] for L in range(3)) for k in range(2)]        # 7/12, 7/12
    un = [[ut[L][k] / a[k] for k in range(2)] for L in range(3)]   # 4/7 1/7, 2/7 2/7, 1/7 4/7
    u, q = orc.ishikawa_init((1, 2), 2)
    orc.ishikawa_iterate(D, u, q, 1, C_HAND, TAU_HAND, s_level=s, grad_source=orc.PAPER_LITERAL)
    assert np.abs(u[:, 0] - un).max() <= 1e-15
    assert np.array_equal(q[:, 0, 0], [[q1, 0.0], [q2, 0.0]]) and not np.any(q[:, 1])
    # iteration 2
    e1, e2 = [q1, -q1], [q2, -q2]                        # div q_1, div q_2
    d = [[D[0, 0, k] for k in range(2)],
         [D[1, 0, k] + e1[k] for k in range(2)],
         [D[2, 0, k] + e1[k] + e2[k] for k in range(2)]]
    ut = [[un[L][k] * math.exp(-d[L][k]) for k in range(2)] for L in range(3)]
    g1 = [ut[1][k] + ut[2][k] for k in range(2)]
    g2 = ut[2]
    q1, _ = _clip(q1 - STEP_HAND * (g1[1] - g1[0]), s[0])
    q2, _ = _clip(q2 - STEP_HAND * (g2[1] - g2[0]), s[1])
    a = [sum(ut[L][k] for L in range(3)) for k in range(2)]
    u_hand = np.array([[ut[L][k] / a[k] for k in range(2)] for L in range(3)])
    orc.ishikawa_iterate(D, u, q, 1, C_HAND, TAU_HAND, s_level=s, grad_source=orc.PAPER_LITERAL)
    assert np.abs(u[:, 0] - u_hand).max() <= 1e-15
    assert np.abs(q[:, 0, 0] - [[q1, 0.0], [q2, 0.0]]).max() <= 1e-15 and not np.any(q[:, 1])
    un2, qn2 = orc.ishikawa_init((1, 2), 2)
    orc.ishikawa_iterate(D, un2, qn2, 2, C_HAND, TAU_HAND, s_level=s, grad_source=orc.NORMALISED)
    assert np.abs(qn2[0, 0, 0, 0] - q1) > 1e-2
