"""FP64 CPU oracle for the pseudo-flow continuous max-flow method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA solver in ``paper_1501_07844_gb300``.

Array conventions (numpy, float64, C order):
  spatial shape ``(ny, nx)`` (2-D) or ``(nz, ny, nx)`` (3-D), x fastest;
  labelling ``u[leaf, *spatial]``, data term ``D[leaf, *spatial]``,
  flows ``q[node, component, *spatial]`` with component 0 = x, 1 = y, 2 = z;
  capacity of node A at x: ``s_node[A] * S_field[x]`` (either may be None).

Each wrapper names the passage of the paper its C function follows; the C
source holds the arithmetic.
"""
import ctypes as C

import numpy as np

from . import build as _build_mod

ISO, ANISO = 0, 1
NORMALISED, PAPER_LITERAL = 0, 1

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class _Grid(C.Structure):
    _fields_ = [("ndim", C.c_int), ("nx", C.c_long), ("ny", C.c_long), ("nz", C.c_long)]


class _Params(C.Structure):
    _fields_ = [("c", C.c_double), ("tau", C.c_double), ("norm", C.c_int), ("grad_source", C.c_int)]


class _Dag(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("n_edges", C.c_int), ("parent", _ip), ("child", _ip), ("w", _dp)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build_mod.build())
        for name in ("orc_potts_iterate", "orc_potts_energy", "orc_potts_init", "orc_grad", "orc_div",
                     "orc_alm_potts_init", "orc_alm_potts_iterate", "orc_ishikawa_init", "orc_ishikawa_iterate"):
            getattr(_lib, name).restype = None
        for name in ("orc_dag_iterate", "orc_dag_energy", "orc_dag_init", "orc_dag_n_leaves",
                     "orc_dag_path_weights", "orc_bruteforce_binary"):
            getattr(_lib, name).restype = C.c_int
        _lib.orc_project.restype = None
        _lib.orc_threads.restype = C.c_int
    return _lib


def threads():
    """OpenMP threads the oracle's sweeps use."""
    return lib().orc_threads()


def _grid(spatial):
    spatial = tuple(int(s) for s in spatial)
    if len(spatial) == 2:
        return _Grid(2, spatial[1], spatial[0], 1)
    if len(spatial) == 3:
        return _Grid(3, spatial[2], spatial[1], spatial[0])
    raise ValueError("spatial shape must be 2-D or 3-D")


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class Dag:
    """Label DAG (Section 3.3): nodes 0..n_nodes-1, edges (parent, child, w); parent -1 is S."""

    def __init__(self, n_nodes, edges):
        self.n_nodes = int(n_nodes)
        self.edges = [(int(a), int(b), float(w)) for a, b, w in edges]
        self._parent = np.array([e[0] for e in self.edges], dtype=np.int32)
        self._child = np.array([e[1] for e in self.edges], dtype=np.int32)
        self._w = np.array([e[2] for e in self.edges], dtype=np.float64)
        self.c = _Dag(self.n_nodes, len(self.edges), self._parent.ctypes.data_as(_ip),
                      self._child.ctypes.data_as(_ip), self._w.ctypes.data_as(_dp))

    @staticmethod
    def flat(nl):
        """Potts as a DAG: every label is a child of the source with weight 1."""
        return Dag(nl, [(-1, L, 1.0) for L in range(nl)])

    def n_leaves(self):
        return lib().orc_dag_n_leaves(C.byref(self.c))

    def path_weights(self):
        W = np.zeros((self.n_nodes, self.n_nodes))
        if lib().orc_dag_path_weights(C.byref(self.c), _p(W)) != 0:
            raise ValueError("malformed DAG")
        return W

    def leaves(self):
        has_child = {a for a, _, _ in self.edges if a >= 0}
        return [v for v in range(self.n_nodes) if v not in has_child]


def grad(u):
    """Forward-difference gradient (zero at the last index); returns [ndim, *spatial]."""
    u = _f64(u)
    g = _grid(u.shape)
    out = np.empty((g.ndim,) + u.shape)
    lib().orc_grad(C.byref(g), _p(u), _p(out))
    return out


def div(q):
    """Divergence, the negative adjoint of grad; q is [ndim, *spatial]."""
    q = _f64(q)
    g = _grid(q.shape[1:])
    out = np.empty(q.shape[1:])
    lib().orc_div(C.byref(g), _p(q), _p(out))
    return out


def project(y, s, norm=ISO):
    """Projection of one vector onto {|y| <= s} (ball for ISO, box for ANISO)."""
    y = np.array(y, dtype=np.float64)
    lib().orc_project(C.c_int(y.size), C.c_int(norm), C.c_double(s), _p(y))
    return y


def _params(c, tau, norm, grad_source):
    return _Params(float(c), float(tau), int(norm), int(grad_source))


def potts_init(spatial, nl):
    """Algorithm 1, first line: u = 1/#L; q = 0."""
    g = _grid(spatial)
    u = np.empty((nl,) + tuple(spatial))
    q = np.empty((nl, g.ndim) + tuple(spatial))
    lib().orc_potts_init(C.byref(g), C.c_int(nl), _p(u), _p(q))
    return u, q


def potts_iterate(D, u, q, iters, c, tau, S_field=None, s_node=None, norm=ISO, grad_source=NORMALISED):
    """Algorithm 1 loop body, ``iters`` times, in place on (u, q)."""
    D = _f64(D)
    assert u.dtype == np.float64 and q.dtype == np.float64 and u.flags.c_contiguous and q.flags.c_contiguous
    g = _grid(D.shape[1:])
    prm = _params(c, tau, norm, grad_source)
    lib().orc_potts_iterate(C.byref(g), C.c_int(D.shape[0]), _p(D), _p(_f64(S_field)), _p(_f64(s_node)),
                            C.byref(prm), C.c_int(iters), _p(u), _p(q))
    return u, q


def potts_energy(D, u, q, S_field=None, s_node=None, norm=ISO):
    """(E(u) of Eq. potts_original, P(q) of Eq. potts_pseudo)."""
    D, u, q = _f64(D), _f64(u), _f64(q)
    g = _grid(D.shape[1:])
    E, P = C.c_double(), C.c_double()
    lib().orc_potts_energy(C.byref(g), C.c_int(D.shape[0]), _p(D), _p(_f64(S_field)), _p(_f64(s_node)),
                           C.c_int(norm), _p(u), _p(q), C.byref(E), C.byref(P))
    return E.value, P.value


def dag_init(spatial, dag):
    """Algorithm 2, first line: u = 1/|L| on end-labels; q = 0."""
    g = _grid(spatial)
    nleaf = dag.n_leaves()
    if nleaf < 0:
        raise ValueError("malformed DAG")
    u = np.empty((nleaf,) + tuple(spatial))
    q = np.empty((dag.n_nodes, g.ndim) + tuple(spatial))
    lib().orc_dag_init(C.byref(g), C.byref(dag.c), _p(u), _p(q))
    return u, q


def dag_iterate(dag, D, u, q, iters, c, tau, S_field=None, s_node=None, norm=ISO, grad_source=NORMALISED):
    """Algorithm 2 loop body, ``iters`` times, in place on (u, q)."""
    D = _f64(D)
    assert u.dtype == np.float64 and q.dtype == np.float64 and u.flags.c_contiguous and q.flags.c_contiguous
    g = _grid(D.shape[1:])
    prm = _params(c, tau, norm, grad_source)
    r = lib().orc_dag_iterate(C.byref(g), C.byref(dag.c), _p(D), _p(_f64(S_field)), _p(_f64(s_node)),
                              C.byref(prm), C.c_int(iters), _p(u), _p(q))
    if r != 0:
        raise ValueError("malformed DAG")
    return u, q


def dag_energy(dag, D, u, q, S_field=None, s_node=None, norm=ISO):
    """(E(u) of Eq. dagmf_original, P(q) of Eq. dagmf_pseudo)."""
    D, u, q = _f64(D), _f64(u), _f64(q)
    g = _grid(D.shape[1:])
    E, P = C.c_double(), C.c_double()
    r = lib().orc_dag_energy(C.byref(g), C.byref(dag.c), _p(D), _p(_f64(S_field)), _p(_f64(s_node)),
                             C.c_int(norm), _p(u), _p(q), C.byref(E), C.byref(P))
    if r != 0:
        raise ValueError("malformed DAG")
    return E.value, P.value


def ishikawa_init(spatial, nlev):
    """Algorithm 3, first line: u = 1/(N+1) over the N+1 labels; N flow fields = 0."""
    g = _grid(spatial)
    u = np.empty((nlev + 1,) + tuple(spatial))
    q = np.empty((nlev, g.ndim) + tuple(spatial))
    lib().orc_ishikawa_init(C.byref(g), C.c_int(nlev), _p(u), _p(q))
    return u, q


def ishikawa_iterate(D, u, q, iters, c, tau, S_field=None, s_level=None, norm=ISO, grad_source=NORMALISED):
    """Algorithm 3 loop body, ``iters`` times, in place on (u, q); D is [N+1, *spatial]."""
    D = _f64(D)
    g = _grid(D.shape[1:])
    prm = _params(c, tau, norm, grad_source)
    lib().orc_ishikawa_iterate(C.byref(g), C.c_int(D.shape[0] - 1), _p(D), _p(_f64(S_field)), _p(_f64(s_level)),
                               C.byref(prm), C.c_int(iters), _p(u), _p(q))
    return u, q


def alm_potts(D, iters, gamma, step, S_field=None, s_node=None, norm=ISO, state=None):
    """Explicit-flow augmented-Lagrangian max-flow (primal Eq. potts_primal).

    Returns (flow_value, state) where state = (u, q, pS, pL) can be passed back
    to continue."""
    D = _f64(D)
    nl, spatial = D.shape[0], D.shape[1:]
    g = _grid(spatial)
    if state is None:
        u = np.empty(D.shape)
        q = np.empty((nl, g.ndim) + spatial)
        pS = np.empty(spatial)
        pL = np.empty(D.shape)
        lib().orc_alm_potts_init(C.byref(g), C.c_int(nl), _p(D), _p(u), _p(q), _p(pS), _p(pL))
    else:
        u, q, pS, pL = state
    fv = C.c_double()
    lib().orc_alm_potts_iterate(C.byref(g), C.c_int(nl), _p(D), _p(_f64(S_field)), _p(_f64(s_node)),
                                C.c_int(norm), C.c_double(gamma), C.c_double(step), C.c_int(iters),
                                _p(u), _p(q), _p(pS), _p(pL), C.byref(fv))
    return fv.value, (u, q, pS, pL)


def bruteforce_binary(D, S_field=None, s_node=None, norm=ANISO):
    """Exhaustive minimum of the 2-label Potts energy: (best, second_best, label0_map)."""
    D = _f64(D)
    g = _grid(D.shape[1:])
    best, second = C.c_double(), C.c_double()
    lab = np.zeros(D.shape[1:], dtype=np.uint8)
    r = lib().orc_bruteforce_binary(C.byref(g), _p(D), _p(_f64(S_field)), _p(_f64(s_node)), C.c_int(norm),
                                    C.byref(best), C.byref(second), lab.ctypes.data_as(C.POINTER(C.c_ubyte)))
    if r != 0:
        raise ValueError("too many voxels for exhaustive search")
    return best.value, second.value, lab
