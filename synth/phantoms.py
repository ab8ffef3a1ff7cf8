"""Seeded phantom generators for the workloads the solver is measured on.

The paper has no datasets; these stand in for the segmentation volumes it
targets.  Every generator uses numpy's PCG64 with an explicit seed and
returns float32 data terms (what the GPU consumes; the oracle receives the
same values widened to float64).

Layouts: D[leaf, *spatial], S field [*spatial], spatial = (ny, nx) or
(nz, ny, nx), x fastest.  A DAG is (n_nodes, [(parent, child, w), ...]) with
parent -1 for the source.
"""
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np


@dataclass
class Problem:
    D: np.ndarray                       # float32 [n_leaf, *spatial]
    S_field: Optional[np.ndarray]       # float32 [*spatial] or None
    s_node: Optional[np.ndarray]        # float32 [n_nodes] or None
    n_nodes: int
    edges: List[Tuple[int, int, float]]
    c: float = 0.5
    tau: float = 0.11
    iters: int = 100
    truth: Optional[np.ndarray] = None  # int region map [*spatial] (phantom ground truth)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def spatial(self):
        return self.D.shape[1:]

    @property
    def n_leaf(self):
        return self.D.shape[0]


def flat_edges(nl):
    return [(-1, L, 1.0) for L in range(nl)]


def _edge_capacity(I, scale=0.2, beta=0.01):
    """S(x) = scale * exp(-|grad I|^2 / beta), forward differences (last index 0)."""
    g2 = np.zeros_like(I)
    for ax in range(I.ndim):
        d = np.zeros_like(I)
        sl_hi = [slice(None)] * I.ndim
        sl_lo = [slice(None)] * I.ndim
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        d[tuple(sl_lo)] = I[tuple(sl_hi)] - I[tuple(sl_lo)]
        g2 += d * d
    return scale * np.exp(-g2 / beta)


def _paint_spheres(rng, shape, n_spheres, rmin=0.08, rmax=0.25):
    """Label map: background 0, then spheres with labels 1..n painted in order."""
    lab = np.zeros(shape, dtype=np.int32)
    n = min(shape)
    coords = np.meshgrid(*[np.arange(s, dtype=np.float32) for s in shape], indexing="ij")
    for k in range(1, n_spheres + 1):
        centre = [rng.uniform(0, s) for s in shape]
        r = rng.uniform(rmin, rmax) * n
        d2 = np.zeros(shape, dtype=np.float32)
        for ax in range(len(shape)):
            d2 += (coords[ax] - np.float32(centre[ax])) ** 2
        lab[d2 <= r * r] = k
    return lab


def potts2d_problem(seed=1000, n=128, iters=200):
    """2-D Potts: n x n image, 4 labels from 3 random ellipses painted over a
    background; intensities c = {0.1, 0.4, 0.7, 0.9} plus N(0, 0.08^2);
    D_L = |I - c_L|; S = 0.1 constant; c = 0.5, tau = 0.11."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    lab = np.zeros((n, n), dtype=np.int32)
    for k in (1, 2, 3):
        cy, cx = rng.uniform(0, n), rng.uniform(0, n)
        a, b = rng.uniform(0.1, 0.35) * n, rng.uniform(0.1, 0.35) * n
        th = rng.uniform(0, np.pi)
        dx, dy = xx - cx, yy - cy
        xr = dx * np.cos(th) + dy * np.sin(th)
        yr = -dx * np.sin(th) + dy * np.cos(th)
        lab[(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] = k
    cl = np.array([0.1, 0.4, 0.7, 0.9])
    I = cl[lab] + rng.normal(0.0, 0.08, size=(n, n))
    D = np.abs(I[None] - cl[:, None, None]).astype(np.float32)
    S = np.full((n, n), 0.1, dtype=np.float32)
    return Problem(D, S, None, 4, flat_edges(4), c=0.5, tau=0.11, iters=iters, truth=lab, name="potts2d")


def potts3d_problem(seed=2000, n=256, nl=8, sigma=0.05, iters=500, shape=None):
    """3-D Potts: n^3 volume, nl labels (background + nl-1 random spheres),
    intensities c_L = L/(nl-1), noise sigma; D_L = (I - c_L)^2;
    S(x) = 0.2 exp(-|grad I|^2 / 0.01)."""
    rng = np.random.default_rng(seed)
    shape = tuple(shape) if shape is not None else (n, n, n)
    lab = _paint_spheres(rng, shape, nl - 1)
    cl = (np.arange(nl) / (nl - 1)).astype(np.float32)
    I = cl[lab] + rng.normal(0.0, sigma, size=shape).astype(np.float32)
    D = np.empty((nl,) + shape, dtype=np.float32)
    for L in range(nl):
        np.square(I - cl[L], out=D[L])
    S = _edge_capacity(I, 0.2, 0.01).astype(np.float32)
    return Problem(D, S, None, nl, flat_edges(nl), c=0.5, tau=0.11, iters=iters, truth=lab, name="potts3d")


def hmf_tree(n_inner=3, per_inner=4):
    """Tree: S -> n_inner inner nodes -> per_inner leaves each, all weights 1.
    Node ids: inner nodes 0..n_inner-1, leaves after them, so that leaf k
    (k-th leaf in ascending node id) sits under inner node k // per_inner."""
    edges = [(-1, a, 1.0) for a in range(n_inner)]
    for a in range(n_inner):
        for j in range(per_inner):
            edges.append((a, n_inner + a * per_inner + j, 1.0))
    return n_inner + n_inner * per_inner, edges


def hmf_problem(seed=3000, n=192, sigma=0.05, iters=400, shape=None):
    """HMF: n^3 volume, depth-3 tree (S -> 3 inner -> 4 leaves each = 12
    leaves); 12-region sphere phantom, c_L = L/11; leaf D_L = |I - c_L|,
    inner D = 0; per-node capacities uniform in [0.05, 0.5]."""
    rng = np.random.default_rng(seed)
    shape = tuple(shape) if shape is not None else (n, n, n)
    nn, edges = hmf_tree(3, 4)
    lab = _paint_spheres(rng, shape, 11)
    cl = (np.arange(12) / 11).astype(np.float32)
    I = cl[lab] + rng.normal(0.0, sigma, size=shape).astype(np.float32)
    D = np.empty((12,) + shape, dtype=np.float32)
    for L in range(12):
        np.abs(I - cl[L], out=D[L])
    s_node = rng.uniform(0.05, 0.5, size=nn).astype(np.float32)
    return Problem(D, None, s_node, nn, edges, c=0.5, tau=0.11, iters=iters, truth=lab, name="hmf")


def random_dag(rng, n_inner=4, n_leaf=10, max_parents=2):
    """DAG with n_inner inner nodes under S (w = 1) and n_leaf leaves, each
    with 1..max_parents inner parents of weight 1/#parents; every inner node
    gets at least one child.  Path weight S -> leaf is 1 for every leaf."""
    assert n_leaf >= n_inner
    nn = n_inner + n_leaf
    edges = [(-1, a, 1.0) for a in range(n_inner)]
    parents = []
    for j in range(n_leaf):
        ps = {j} if j < n_inner else {int(rng.integers(n_inner))}
        while len(ps) < max_parents and rng.random() < 0.5:
            ps.add(int(rng.integers(n_inner)))
        parents.append(sorted(ps))
    for j, ps in enumerate(parents):
        for a in ps:
            edges.append((a, n_inner + j, 1.0 / len(ps)))
    return nn, edges


def dagmf_problem(seed, shape, sigma=0.1, iters=300):
    """One DAGMF volume: 10 leaves, 4 inner nodes, leaves with up to 2
    parents; c_L = L/9, D_L = |I - c_L|, S = 0.15 constant."""
    rng = np.random.default_rng(seed)
    shape = tuple(shape)
    nn, edges = random_dag(rng, 4, 10, 2)
    lab = _paint_spheres(rng, shape, 9)
    cl = (np.arange(10) / 9).astype(np.float32)
    I = cl[lab] + rng.normal(0.0, sigma, size=shape).astype(np.float32)
    D = np.empty((10,) + shape, dtype=np.float32)
    for L in range(10):
        np.abs(I - cl[L], out=D[L])
    S = np.full(shape, 0.15, dtype=np.float32)
    return Problem(D, S, None, nn, edges, c=0.5, tau=0.11, iters=iters, truth=lab, name="dagmf")


def dagmf_batch(seed=4000, count=32, lo=64, hi=160, scale=1.0):
    """count volumes with per-axis sizes drawn from U{lo..hi} (times scale)."""
    rng = np.random.default_rng(seed)
    out = []
    for v in range(count):
        shape = tuple(max(2, int(round(int(rng.integers(lo, hi + 1)) * scale))) for _ in range(3))
        out.append(dagmf_problem(seed + 1 + v, shape))
    return out


def diff_problem(seed=5000, n=128, nl=6, iters=100):
    """Differentiable Potts: n^3, 6 labels (background + 5 spheres),
    D_L = (I - c_L)^2, S as in the 3-D Potts volume."""
    p = potts3d_problem(seed, n=n, nl=nl, sigma=0.05, iters=iters)
    p.name = "diff"
    return p


def random_problem(seed, spatial, nl=3, s_scale=0.3, s_kind="field", c=0.5, tau=0.11, iters=50,
                   n_nodes=None, edges=None):
    """Small random problem for tests: D ~ U[0,1), capacities either a random
    field in [0, s_scale], per-node scalars, or both."""
    rng = np.random.default_rng(seed)
    spatial = tuple(spatial)
    D = rng.random((nl,) + spatial).astype(np.float32)
    nn = nl if n_nodes is None else n_nodes
    e = flat_edges(nl) if edges is None else edges
    S = s_node = None
    if s_kind in ("field", "both"):
        S = (s_scale * rng.random(spatial)).astype(np.float32)
    if s_kind in ("node", "both"):
        s_node = rng.uniform(0.05, 1.0, size=nn).astype(np.float32)
        if s_kind == "node":
            s_node *= s_scale
    return Problem(D, S, s_node, nn, e, c=c, tau=tau, iters=iters, name="random")


def ishikawa_chain(nlev):
    """The Ishikawa model (N levels, N+1 ordered labels) as a label DAG:
    chain S -> A_1 -> ... -> A_N of inner nodes, label L_0 under S and
    label L_i under A_i.  Node ids: A_i = i - 1 (i = 1..N), L_i = N + i.
    The labels carry no flow of their own (capacity 0); A_i's flow is the
    flow of level i."""
    N = int(nlev)
    edges = [(-1, 0, 1.0), (-1, N, 1.0)]
    for i in range(1, N):
        edges.append((i - 1, i, 1.0))          # A_i -> A_{i+1}
    for i in range(1, N + 1):
        edges.append((i - 1, N + i, 1.0))      # A_i -> L_i
    return 2 * N + 1, edges


def ishikawa_problem(seed, spatial, nlev=4, sigma=0.08, iters=50):
    """Ordered labels c_i = i/N on a noisy staircase image; per-level
    capacities U[0.1, 0.4] (leaves 0)."""
    rng = np.random.default_rng(seed)
    spatial = tuple(spatial)
    lab = np.zeros(spatial, dtype=np.int32)
    coords = np.meshgrid(*[np.arange(s) for s in spatial], indexing="ij")
    lab = np.minimum((coords[-1] * (nlev + 1)) // spatial[-1], nlev).astype(np.int32)
    cl = np.arange(nlev + 1) / nlev
    I = cl[lab] + rng.normal(0.0, sigma, size=spatial)
    D = np.abs(I[None] - cl.reshape((-1,) + (1,) * len(spatial))).astype(np.float32)
    nn, edges = ishikawa_chain(nlev)
    s_node = np.zeros(nn, dtype=np.float32)
    s_node[:nlev] = rng.uniform(0.1, 0.4, size=nlev)
    return Problem(D, None, s_node, nn, edges, c=0.5, tau=0.11, iters=iters, truth=lab, name="ishikawa")
