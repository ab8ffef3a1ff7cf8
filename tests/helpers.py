"""Shared test helpers: run the FP64 oracle and the CUDA solver on the same
seeded problem and compare them element by element."""
import numpy as np

import oracle

TOL_U = 1e-3        # max |u_gpu - u_oracle| (FP32 storage)
TOL_E = 1e-5        # relative primal energy difference
TOL_ARGMAX = 0.999  # fraction of voxels with the same thresholded label


def is_flat(prob):
    return prob.n_nodes == prob.n_leaf and all(a == -1 and w == 1.0 for a, _, w in prob.edges) \
        and len(prob.edges) == prob.n_nodes


def f64(a):
    return None if a is None else np.asarray(a, dtype=np.float64)


def oracle_run(prob, iters, grad_source=0, norm=0, state=None):
    """FP64 oracle: Algorithm 1 for flat DAGs, Algorithm 2 otherwise, on the
    FP32 inputs widened to FP64.  Returns (u, q, E, P)."""
    D, S, sn = f64(prob.D), f64(prob.S_field), f64(prob.s_node)
    if is_flat(prob):
        u, q = state if state is not None else oracle.potts_init(prob.spatial, prob.n_leaf)
        oracle.potts_iterate(D, u, q, iters, prob.c, prob.tau, S_field=S, s_node=sn, norm=norm,
                             grad_source=grad_source)
        E, P = oracle.potts_energy(D, u, q, S_field=S, s_node=sn, norm=norm)
    else:
        dag = oracle.Dag(prob.n_nodes, prob.edges)
        u, q = state if state is not None else oracle.dag_init(prob.spatial, dag)
        oracle.dag_iterate(dag, D, u, q, iters, prob.c, prob.tau, S_field=S, s_node=sn, norm=norm,
                           grad_source=grad_source)
        E, P = oracle.dag_energy(dag, D, u, q, S_field=S, s_node=sn, norm=norm)
    return u, q, E, P


def oracle_energy(prob, u, q, norm=0):
    D, S, sn = f64(prob.D), f64(prob.S_field), f64(prob.s_node)
    if is_flat(prob):
        return oracle.potts_energy(D, f64(u), f64(q), S_field=S, s_node=sn, norm=norm)
    return oracle.dag_energy(oracle.Dag(prob.n_nodes, prob.edges), D, f64(u), f64(q), S_field=S, s_node=sn,
                             norm=norm)


def gpu_problem(prob, **kw):
    import torch
    import paper_1501_07844_gb300 as pfm
    D = torch.from_numpy(np.ascontiguousarray(prob.D)).cuda()
    S = None if prob.S_field is None else torch.from_numpy(np.ascontiguousarray(prob.S_field)).cuda()
    kw.setdefault("c", prob.c)
    kw.setdefault("tau", prob.tau)
    return pfm.Problem(D, S_field=S, s_node=prob.s_node, n_nodes=prob.n_nodes, edges=prob.edges, **kw)


def argmax_lowest(u):
    """Index of the largest label, ties to the lowest index."""
    return np.argmax(u, axis=0)


def compare(prob, gp, iters, grad_source=0, norm=0, tol_u=TOL_U, tol_e=TOL_E, tol_argmax=TOL_ARGMAX, tol_q=None):
    """Run both sides for `iters` iterations from the initial state and assert
    parity.  Returns a dict of the measured differences."""
    u_o, q_o, E_o, P_o = oracle_run(prob, iters, grad_source, norm)
    gp.iterate(iters)
    E_g, P_g = gp.energy()
    u_g = gp.labels().cpu().numpy().astype(np.float64)
    q_g = gp.flows().cpu().numpy().astype(np.float64)
    am_g = gp.argmax().cpu().numpy()
    du = float(np.abs(u_g - u_o).max())
    dq = float(np.abs(q_g - q_o).max())
    agree = float(np.mean(am_g == argmax_lowest(u_o)))
    # energy of the GPU state evaluated by the oracle: isolates the iteration from the reduction
    E_go, P_go = oracle_energy(prob, u_g, q_g, norm)
    res = dict(du=du, dq=dq, agree=agree, dE=abs(E_g - E_o) / abs(E_o), dP=abs(P_g - P_o) / max(abs(P_o), 1e-30),
               dE_red=abs(E_g - E_go) / abs(E_go), E=E_o, P=P_o)
    assert du <= tol_u, res
    assert res["dE"] <= tol_e, res
    assert agree >= tol_argmax, res
    assert res["dE_red"] <= 1e-6, res
    if tol_q is not None:
        assert dq <= tol_q, res
    return res
