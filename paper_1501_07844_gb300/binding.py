"""ctypes binding of libpfm: argument marshalling only.

``lib()`` returns the loaded library with argument and result types set for
every function declared in ``include/pfm.h``; ``Problem`` wraps one
``pfm_problem`` and accepts torch tensors (CUDA or pinned/CPU) or numpy
arrays for inputs and outputs.  Layouts are those of ``pfm.h``:
D / labels ``[n_leaf, *spatial]``, flows ``[n_nodes, ndim, *spatial]``,
spatial ``(ny, nx)`` or ``(nz, ny, nx)`` with x fastest.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

ISO, ANISO = 0, 1
NORMALISED, PAPER_LITERAL = 0, 1
F32, BF16, F16 = 0, 1, 2
FUSED, INPLACE, FUSED_PLAIN = 0, 1, 2

_STATUS = {0: "PFM_OK", 1: "PFM_EINVAL", 2: "PFM_EDAG", 3: "PFM_ENOMEM", 4: "PFM_ECUDA", 5: "PFM_ENONFINITE",
           6: "PFM_ETIMEOUT", 7: "PFM_ENOTCONVERGED", 8: "PFM_EUNSUPPORTED"}


class PfmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status
        self.name = _STATUS.get(status, str(status))


class pfm_params(C.Structure):
    _fields_ = [("c", C.c_double), ("tau", C.c_double), ("norm", C.c_int), ("grad_source", C.c_int),
                ("storage", C.c_int), ("schedule", C.c_int), ("check_every", C.c_int), ("gap_tol", C.c_double)]


class pfm_desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("dims", C.c_int64 * 3), ("n_nodes", C.c_int), ("n_edges", C.c_int),
                ("edge_parent", C.POINTER(C.c_int32)), ("edge_child", C.POINTER(C.c_int32)),
                ("edge_w", C.POINTER(C.c_double)), ("D", C.c_void_p), ("S_field", C.c_void_p),
                ("s_node", C.POINTER(C.c_float))]


_P = C.c_void_p
_SIGS = {
    "pfm_version": (C.c_int, []),
    "pfm_last_error": (C.c_char_p, []),
    "pfm_params_default": (None, [C.POINTER(pfm_params)]),
    "pfm_footprint": (C.c_int, [C.POINTER(pfm_desc), C.POINTER(pfm_params), C.POINTER(C.c_size_t),
                                C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "pfm_create": (C.c_int, [C.POINTER(pfm_desc), C.POINTER(pfm_params), _P, C.POINTER(_P)]),
    "pfm_destroy": (None, [_P]),
    "pfm_set_data": (C.c_int, [_P, _P, _P]),
    "pfm_prefetch_data": (C.c_int, [_P, _P, _P]),
    "pfm_commit_data": (C.c_int, [_P]),
    "pfm_get_state_async": (C.c_int, [_P, _P, _P]),
    "pfm_get_state": (C.c_int, [_P, _P, C.POINTER(C.c_size_t)]),
    "pfm_set_state": (C.c_int, [_P, _P, C.c_size_t]),
    "pfm_get_argmax_async": (C.c_int, [_P, _P]),
    "pfm_readback_wait": (C.c_int, [_P]),
    "pfm_reset": (C.c_int, [_P]),
    "pfm_iterate": (C.c_int, [_P, C.c_int]),
    "pfm_set_step": (C.c_int, [_P, C.c_double, C.c_double]),
    "pfm_energy": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pfm_run_to_gap": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "pfm_iterate_energy": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pfm_get_labels": (C.c_int, [_P, _P]),
    "pfm_get_argmax": (C.c_int, [_P, _P]),
    "pfm_get_flows": (C.c_int, [_P, _P]),
    "pfm_set_labels": (C.c_int, [_P, _P]),
    "pfm_set_flows": (C.c_int, [_P, _P]),
    "pfm_shape": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int),
                            C.POINTER(C.c_int)]),
    "pfm_kernel_variant": (C.c_char_p, [_P]),
    "pfm_iterations_done": (C.c_int64, [_P]),
    "pfm_launch_count": (C.c_int64, [_P]),
    "pfm_tune": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int)]),
    "pfm_selftest_timeout": (C.c_int, [_P]),
    "pfm_set_chunk_length": (C.c_int, [_P, C.c_int]),
    "pfm_chunk_length": (C.c_int, [_P]),
    "pfm_select_kernel": (C.c_int, [_P, C.c_char_p]),
    "pfm_adjoint_step": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "pfm_adjoint_steps": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "pfm_batch_create": (C.c_int, [C.c_int, C.c_void_p, C.POINTER(pfm_params), _P, C.POINTER(_P)]),
    "pfm_batch_destroy": (None, [_P]),
    "pfm_batch_size": (C.c_int, [_P]),
    "pfm_batch_kernel_variant": (C.c_char_p, [_P]),
    "pfm_batch_member": (C.c_int, [_P, C.c_int, C.POINTER(_P)]),
    "pfm_batch_iterate": (C.c_int, [_P, C.c_int]),
    "pfm_batch_energy": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pfm_batch_tune": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pfm_batch_launch_count": (C.c_int64, [_P]),
    "pfm_alm_footprint": (C.c_int, [C.POINTER(pfm_desc), C.POINTER(C.c_size_t), C.POINTER(C.c_int64)]),
    "pfm_alm_create": (C.c_int, [C.POINTER(pfm_desc), C.c_double, C.c_double, C.c_int, _P, C.POINTER(_P)]),
    "pfm_alm_destroy": (None, [_P]),
    "pfm_alm_iterate": (C.c_int, [_P, C.c_int]),
    "pfm_alm_energy": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pfm_alm_get_labels": (C.c_int, [_P, _P]),
    "pfm_alm_iterations_done": (C.c_int64, [_P]),
    "pfm_potts_energy_noalloc": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.c_int, _P, _P, _P, _P,
                                           C.POINTER(C.c_float), C.c_int, _P, _P]),
}

_lib = None


def library_path():
    return _build.LIB


def lib():
    """Build (if stale) and load libpfm.so; raises if it cannot be loaded."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libpfm.so is missing at %s" % path)
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status):
    if status != 0:
        raise PfmError(status, lib().pfm_last_error().decode(errors="replace"))
    return status


def _ptr(a):
    """Address of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _as_f32(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float32)
    import torch
    return a.to(torch.float32).contiguous()


def _stream_handle(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch absent
        pass
    return None


def params(c=0.5, tau=0.11, norm=ISO, grad_source=NORMALISED, storage=F32, schedule=FUSED, check_every=10,
           gap_tol=1e-4):
    p = pfm_params()
    lib().pfm_params_default(C.byref(p))
    p.c, p.tau, p.norm, p.grad_source = float(c), float(tau), int(norm), int(grad_source)
    p.storage, p.schedule, p.check_every, p.gap_tol = int(storage), int(schedule), int(check_every), float(gap_tol)
    return p


class _Desc:
    """Keeps the host arrays a pfm_desc points at alive."""

    def __init__(self, spatial, n_nodes, edges, D_ptr, S_ptr, s_node):
        spatial = tuple(int(s) for s in spatial)
        self.ndim = len(spatial)
        if self.ndim not in (2, 3):
            raise ValueError("spatial shape must be 2-D or 3-D")
        nx, ny, nz = spatial[-1], spatial[-2], (spatial[0] if self.ndim == 3 else 1)
        self.parent = np.array([e[0] for e in edges], dtype=np.int32)
        self.child = np.array([e[1] for e in edges], dtype=np.int32)
        self.w = np.array([e[2] for e in edges], dtype=np.float64)
        self.s_node = None if s_node is None else np.ascontiguousarray(np.asarray(s_node, dtype=np.float32))
        d = pfm_desc()
        d.ndim = self.ndim
        d.dims[0], d.dims[1], d.dims[2] = nx, ny, nz
        d.n_nodes = int(n_nodes)
        d.n_edges = len(edges)
        d.edge_parent = self.parent.ctypes.data_as(C.POINTER(C.c_int32))
        d.edge_child = self.child.ctypes.data_as(C.POINTER(C.c_int32))
        d.edge_w = self.w.ctypes.data_as(C.POINTER(C.c_double))
        d.D = D_ptr
        d.S_field = S_ptr
        d.s_node = None if self.s_node is None else self.s_node.ctypes.data_as(C.POINTER(C.c_float))
        self.c = d


def footprint(spatial, n_nodes, edges, has_S_field=False, s_node=None, **kw):
    """(device bytes, number of full-grid buffers, n_leaf) pfm_create would allocate (host-only)."""
    dummy = C.c_void_p(1)  # D / S pointers are not dereferenced by pfm_footprint
    d = _Desc(spatial, n_nodes, edges, dummy, dummy if has_S_field else None, s_node)
    p = params(**kw)
    nb, nbuf, nl = C.c_size_t(), C.c_int64(), C.c_int()
    check(lib().pfm_footprint(C.byref(d.c), C.byref(p), C.byref(nb), C.byref(nbuf), C.byref(nl)))
    return nb.value, nbuf.value, nl.value


class Problem:
    """One solver instance (``pfm_create`` ... ``pfm_destroy``).

    D: [n_leaf, *spatial] float32 (torch CUDA/CPU tensor or numpy array);
    S_field: [*spatial] or None; s_node: [n_nodes] or None;
    edges: [(parent, child, w)], parent -1 = source; default = Potts (flat).
    """

    def __init__(self, D, S_field=None, s_node=None, n_nodes=None, edges=None, stream=None, **kw):
        D = _as_f32(D)
        S_field = _as_f32(S_field)
        nl = D.shape[0]
        if edges is None:
            n_nodes, edges = nl, [(-1, L, 1.0) for L in range(nl)]
        self.spatial = tuple(D.shape[1:])
        self.n_nodes = int(n_nodes)
        self.stream = _stream_handle(stream)
        self._desc = _Desc(self.spatial, n_nodes, edges, _ptr(D), _ptr(S_field), s_node)
        self._params = params(**kw)
        h = C.c_void_p()
        check(lib().pfm_create(C.byref(self._desc.c), C.byref(self._params), self.stream, C.byref(h)))
        self._h = h
        nd, dims, nleaf, nnod = C.c_int(), (C.c_int64 * 3)(), C.c_int(), C.c_int()
        check(lib().pfm_shape(self._h, C.byref(nd), dims, C.byref(nleaf), C.byref(nnod)))
        self.ndim, self.n_leaf = nd.value, nleaf.value
        self.has_S_field = S_field is not None

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None):
            lib().pfm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- solver calls
    def reset(self):
        check(lib().pfm_reset(self._h))

    def set_data(self, D, S_field=None):
        D, S_field = _as_f32(D), _as_f32(S_field)
        check(lib().pfm_set_data(self._h, _ptr(D), _ptr(S_field)))

    def prefetch_data(self, D, S_field=None):
        """Start copying new D (and S) into the staging buffer on the library's
        copy stream (pfm_prefetch_data); the sources are kept until commit."""
        D, S_field = _as_f32(D), _as_f32(S_field)
        check(lib().pfm_prefetch_data(self._h, _ptr(D), _ptr(S_field)))
        # a copy may still be reading the previous sources: keep the last two
        kept = getattr(self, "_prefetched", [])
        self._prefetched = (kept + [(D, S_field)])[-2:]

    def commit_data(self):
        """Make the prefetched data current (pfm_commit_data)."""
        check(lib().pfm_commit_data(self._h))

    def iterate(self, n):
        check(lib().pfm_iterate(self._h, int(n)))

    def set_step(self, c, tau):
        """Entropic weight c and step tau for the following iterations."""
        check(lib().pfm_set_step(self._h, float(c), float(tau)))

    def energy(self):
        E, P = C.c_double(), C.c_double()
        check(lib().pfm_energy(self._h, C.byref(E), C.byref(P)))
        return E.value, P.value

    def iterate_energy(self, n):
        """n iterations; returns (E, P) of the state the last one started from."""
        E, P = C.c_double(), C.c_double()
        check(lib().pfm_iterate_energy(self._h, int(n), C.byref(E), C.byref(P)))
        return E.value, P.value

    def tune(self, trial_iters=3):
        """Times the z-chunk lengths and keeps the fastest; resets the state
        to the initial one.  Returns the chunk length."""
        zc = C.c_int()
        check(lib().pfm_tune(self._h, int(trial_iters), C.byref(zc)))
        return zc.value

    @property
    def chunk_length(self):
        return lib().pfm_chunk_length(self._h)

    @chunk_length.setter
    def chunk_length(self, zc):
        check(lib().pfm_set_chunk_length(self._h, int(zc)))

    def select_kernel(self, family):
        """pfm_select_kernel: force the fused schedule's kernel family."""
        check(lib().pfm_select_kernel(self._h, family.encode()))

    def run_to_gap(self, max_iters):
        it, gap = C.c_int(), C.c_double()
        st = lib().pfm_run_to_gap(self._h, int(max_iters), C.byref(it), C.byref(gap))
        if st not in (0, 7):
            check(st)
        return it.value, gap.value, st == 0

    @property
    def iterations(self):
        return lib().pfm_iterations_done(self._h)

    @property
    def variant(self):
        return lib().pfm_kernel_variant(self._h).decode()

    @property
    def launches(self):
        return lib().pfm_launch_count(self._h)

    # -- state in / out (dst / src: torch CUDA tensor, pinned CPU tensor or numpy)
    def _out(self, shape, dtype, out):
        if out is not None:
            return out
        import torch
        return torch.empty(shape, dtype=dtype, device="cuda")

    def labels(self, out=None):
        import torch
        out = self._out((self.n_leaf,) + self.spatial, torch.float32, out)
        check(lib().pfm_get_labels(self._h, _ptr(out)))
        return out

    def argmax(self, out=None):
        import torch
        out = self._out(self.spatial, torch.int32, out)
        check(lib().pfm_get_argmax(self._h, _ptr(out)))
        return out

    def argmax_async(self, out):
        """pfm_get_argmax_async into `out` (int32, pinned host or device);
        complete after readback_wait()."""
        self._readback = out
        check(lib().pfm_get_argmax_async(self._h, _ptr(out)))
        return out

    def readback_wait(self):
        check(lib().pfm_readback_wait(self._h))

    def flows(self, out=None):
        import torch
        out = self._out((self.n_nodes, self.ndim) + self.spatial, torch.float32, out)
        check(lib().pfm_get_flows(self._h, _ptr(out)))
        return out

    def state_async(self, u_out=None, q_out=None):
        """pfm_get_state_async: device copies of u and q ordered on the
        problem's stream, not waited for."""
        import torch
        u_out = u_out if u_out is not None else torch.empty((self.n_leaf,) + self.spatial, dtype=torch.float32,
                                                            device="cuda")
        q_out = q_out if q_out is not None else torch.empty((self.n_nodes, self.ndim) + self.spatial,
                                                            dtype=torch.float32, device="cuda")
        check(lib().pfm_get_state_async(self._h, _ptr(u_out), _ptr(q_out)))
        return u_out, q_out

    def state_size(self):
        """Bytes of the checkpoint blob (pfm_get_state with no destination)."""
        n = C.c_size_t(0)
        check(lib().pfm_get_state(self._h, None, C.byref(n)))
        return n.value

    def get_state(self, out=None):
        """pfm_get_state: the solver state (iteration counter, c, tau, u, q in
        the storage type) as one blob; a host uint8 numpy array unless `out`
        (a uint8 numpy array or torch tensor, host or device) is given."""
        size = self.state_size()
        if out is None:
            out = np.empty(size, dtype=np.uint8)
        n = C.c_size_t(out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size())
        check(lib().pfm_get_state(self._h, _ptr(out), C.byref(n)))
        return out

    def set_state(self, blob):
        """pfm_set_state from a blob written by get_state (host or device)."""
        n = blob.nbytes if isinstance(blob, np.ndarray) else blob.numel() * blob.element_size()
        check(lib().pfm_set_state(self._h, _ptr(blob), C.c_size_t(n)))

    def set_labels(self, u):
        u = _as_f32(u)
        check(lib().pfm_set_labels(self._h, _ptr(u)))

    def adjoint_step(self, u_k, q_k, u_k1, ubar_k1, qbar_k1, ubar_k, qbar_k, Dbar, Sbar, work):
        """pfm_adjoint_step on FP32 CUDA tensors (see pfm.h)."""
        check(lib().pfm_adjoint_step(self._h, _ptr(u_k), _ptr(q_k), _ptr(u_k1), _ptr(ubar_k1), _ptr(qbar_k1),
                                     _ptr(ubar_k), _ptr(qbar_k), _ptr(Dbar), _ptr(Sbar), _ptr(work)))

    def adjoint_steps(self, us, qs, ubar, qbar, Dbar, Sbar, work):
        """pfm_adjoint_steps over a segment: us = [u_0, ..., u_n], qs = [q_0, ...,
        q_{n-1}] (FP32 CUDA tensors); ubar / qbar in place (see pfm.h)."""
        n = len(qs)
        if len(us) != n + 1:
            raise ValueError("need one more labelling than flows")
        U = (C.c_void_p * (n + 1))(*[_ptr(u) for u in us])
        Q = (C.c_void_p * n)(*[_ptr(q) for q in qs])
        check(lib().pfm_adjoint_steps(self._h, n, U, Q, _ptr(ubar), _ptr(qbar), _ptr(Dbar), _ptr(Sbar),
                                      _ptr(work)))

    def set_flows(self, q):
        q = _as_f32(q)
        check(lib().pfm_set_flows(self._h, _ptr(q)))


class _Member(Problem):
    """A batch member: a pfm_problem owned by its batch (read-only use)."""

    def __init__(self, handle, spatial, n_nodes):
        self._h = handle
        self.spatial = tuple(spatial)
        self.n_nodes = int(n_nodes)
        nd, dims, nleaf, nnod = C.c_int(), (C.c_int64 * 3)(), C.c_int(), C.c_int()
        check(lib().pfm_shape(self._h, C.byref(nd), dims, C.byref(nleaf), C.byref(nnod)))
        self.ndim, self.n_leaf = nd.value, nleaf.value

    def close(self):  # owned by the batch
        self._h = None

    def iterate(self, n):
        raise RuntimeError("batch members advance only through Batch.iterate")


class Batch:
    """Many independent problems advanced together (pfm_batch_*).

    problems: list of dicts with keys D, S_field, s_node, n_nodes, edges
    (as for Problem); every member shares the keyword parameters."""

    def __init__(self, problems, stream=None, **kw):
        kw.setdefault("schedule", FUSED)
        self._keep = []
        descs = (pfm_desc * len(problems))()
        self._shapes = []
        for k, p in enumerate(problems):
            D = _as_f32(p["D"])
            S = _as_f32(p.get("S_field"))
            edges = p.get("edges")
            nn = p.get("n_nodes")
            if edges is None:
                nn, edges = D.shape[0], [(-1, L, 1.0) for L in range(D.shape[0])]
            d = _Desc(tuple(D.shape[1:]), nn, edges, _ptr(D), _ptr(S), p.get("s_node"))
            self._keep += [D, S, d]
            descs[k] = d.c
            self._shapes.append((tuple(D.shape[1:]), nn))
        self._params = params(**kw)
        h = C.c_void_p()
        check(lib().pfm_batch_create(len(problems), C.cast(descs, C.c_void_p), C.byref(self._params),
                                     stream if stream is not None else _stream_handle(None), C.byref(h)))
        self._h = h
        self.members = []
        for k, (spatial, nn) in enumerate(self._shapes):
            m = C.c_void_p()
            check(lib().pfm_batch_member(self._h, k, C.byref(m)))
            self.members.append(_Member(m, spatial, nn))

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m.close()
            lib().pfm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def iterate(self, n):
        check(lib().pfm_batch_iterate(self._h, int(n)))

    def energy(self):
        n = len(self.members)
        E, P = (C.c_double * n)(), (C.c_double * n)()
        check(lib().pfm_batch_energy(self._h, E, P))
        return list(E), list(P)

    def tune(self, trial_iters=3):
        zc, grid = C.c_int(), C.c_int()
        check(lib().pfm_batch_tune(self._h, int(trial_iters), C.byref(zc), C.byref(grid)))
        return zc.value, grid.value

    @property
    def launches(self):
        return lib().pfm_batch_launch_count(self._h)

    @property
    def variant(self):
        """Kernel family of iterate(): "batched_tma_dag" or "batched"."""
        return lib().pfm_batch_kernel_variant(self._h).decode()


def alm_footprint(spatial, nl, has_S_field=True):
    """(device bytes, full-grid buffers) of the explicit-flow solver (host-only)."""
    dummy = C.c_void_p(1)
    d = _Desc(spatial, nl, [(-1, L, 1.0) for L in range(nl)], dummy, dummy if has_S_field else None, None)
    nb, nbuf = C.c_size_t(), C.c_int64()
    check(lib().pfm_alm_footprint(C.byref(d.c), C.byref(nb), C.byref(nbuf)))
    return nb.value, nbuf.value


class AlmProblem:
    """Explicit-flow augmented-Lagrangian max-flow of a Potts problem (pfm_alm_*)."""

    def __init__(self, D, S_field=None, s_node=None, gamma=0.3, step=0.2, norm=ISO, stream=None):
        D = _as_f32(D)
        S_field = _as_f32(S_field)
        nl = D.shape[0]
        self.spatial = tuple(D.shape[1:])
        self.n_leaf = nl
        self._desc = _Desc(self.spatial, nl, [(-1, L, 1.0) for L in range(nl)], _ptr(D), _ptr(S_field), s_node)
        h = C.c_void_p()
        check(lib().pfm_alm_create(C.byref(self._desc.c), float(gamma), float(step), int(norm),
                                   _stream_handle(stream), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().pfm_alm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def iterate(self, n):
        check(lib().pfm_alm_iterate(self._h, int(n)))

    def energy(self):
        """(E(u), P(q), sum p_S)."""
        E, P, F = C.c_double(), C.c_double(), C.c_double()
        st = lib().pfm_alm_energy(self._h, C.byref(E), C.byref(P), C.byref(F))
        if st not in (0, 5):
            check(st)
        return E.value, P.value, F.value

    def labels(self, out=None):
        import torch
        out = out if out is not None else torch.empty((self.n_leaf,) + self.spatial, dtype=torch.float32,
                                                      device="cuda")
        check(lib().pfm_alm_get_labels(self._h, _ptr(out)))
        return out
