"""Benchmark: pseudo-flow continuous max-flow, 3-D Potts, 256^3 voxels x 8 labels, FP32.

One step = 10 iterations of the fused pseudo-flow update (label prox +
flow step, Algorithm 1), the last of which also reduces the FP64 primal
energy and pseudo-flow dual of its input state (the gap check that drives
the stopping test), on a seeded 8-region sphere phantom.
Metric: voxel-label updates per second (VLU/s, one VLU = one (voxel, label)
pair advanced by one iteration).  Inputs (4.9 GB of state per iteration)
are larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (under torchrun): every rank solves its own independent volume
(weak scaling, no collective on the data path).  --impl reference times the
FP64 CPU oracle on the host cores doing the same steps on the same full
volume (rank 0 only).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ITERS_PER_STEP = 10
CONFIGS = {
    # name: (shape, labels, generator, schedule, storage)
    "potts3d": ((256, 256, 256), 8, "potts3d", 0, 0),
    "potts3d_inplace": ((256, 256, 256), 8, "potts3d", 1, 0),
    "potts3d_bf16": ((256, 256, 256), 8, "potts3d", 0, 1),
    "potts3d_f16": ((256, 256, 256), 8, "potts3d", 0, 2),
    "hmf": ((192, 192, 192), 12, "hmf", 0, 0),
    "hmf_bf16": ((192, 192, 192), 12, "hmf", 0, 1),
    "hmf_f16": ((192, 192, 192), 12, "hmf", 0, 2),
    "dagmf_batched": (None, 10, "dagmf_batch", 0, 0),
    "ishikawa": ((256, 256, 256), 8, "ishikawa", 0, 0),
    "continuation": ((128, 128, 128), 8, "potts3d", 0, 0),
    "potts3d_solve": ((256, 256, 256), 8, "potts3d", 0, 0),
    "fullflow": ((256, 256, 256), 8, "potts3d", 1, 0),
    "diff": ((128, 128, 128), 6, "potts3d", 0, 0),
    "capacity": ((512, 512, 512), 8, "potts3d", 1, 0),
}
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1501_07844_gb300", "csrc", f) for f in ("pfm_device.cuh", "pfm_tma.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pfm", choices=["pfm", "reference"])
    ap.add_argument("--config", default="potts3d", choices=sorted(CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dims", type=int, default=0, help="cube edge override (profiling of small cases)")
    ap.add_argument("--volumes", type=int, default=32, help="volumes of the batched workload (profiling of small cases)")
    ap.add_argument("--zc", type=int, default=0, help="z-chunk length instead of the tuned one (profiling of small cases)")
    ap.add_argument("--kernel", default="", help="kernel family instead of the most specialised one (comparisons)")
    return ap.parse_args()


def rank_seed(rank):
    """Each rank solves its own seeded volume (weak scaling, no exchange)."""
    return 2000 + rank


def reduce_max(value, dist, device):
    """Max of a per-rank scalar over all ranks (the slowest rank's time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(world, steps, units_per_step, seconds):
    """Whole-job units per second: every rank processed steps * units_per_step."""
    return world * steps * units_per_step / seconds


def make_problem(cfg, seed, shape=None):
    import synth
    shape0, nl, gen, _, _ = CONFIGS[cfg]
    shape = shape or shape0
    if gen == "potts3d":
        return synth.potts3d_problem(seed=seed, nl=nl, shape=shape)
    if gen == "ishikawa":
        return synth.ishikawa_problem(seed=seed, spatial=shape, nlev=nl - 1)
    return synth.hmf_problem(seed=seed, shape=shape)


def algorithmic_bytes_per_iter(prob, storage, schedule):
    """Minimum bytes one iteration of the schedule must move: fused, read u,
    D, q and write u, q (d and the normaliser stay on chip), plus the S field
    once per voxel; in-place, the two sweeps' reads and writes.
    Only nodes with nonzero capacity carry flow (a zero-capacity node's flow
    is identically zero: the Ishikawa chain's end-labels)."""
    n = int(np.prod(prob.spatial))
    ts = 4 if storage == 0 else 2
    ndim = len(prob.spatial)
    n_flow = prob.n_nodes if prob.s_node is None else int(np.count_nonzero(np.asarray(prob.s_node) > 0))
    if schedule == 1:
        # in-place schedule: the prox sweep reads u, D, q and writes u; the
        # flow sweep reads u, q and writes q (u and q cross HBM twice)
        b = n * (prob.n_leaf * (3 * ts + 4 + ndim * ts) + n_flow * ndim * 2 * ts)
    else:
        b = n * (prob.n_leaf * (2 * ts + 4) + n_flow * ndim * 2 * ts)
    if prob.S_field is not None:
        b += 4 * n
    return b


def kernel_sha(sources=None):
    h = hashlib.sha256()
    for f in sources or KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def load_traffic(cfg):
    """DRAM bytes per launch of the dominant kernel from a committed ncu
    capture, valid only while the kernel source is unchanged."""
    try:
        t = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    e = t.get(cfg)
    if not e:
        return None
    src = [os.path.join(ROOT, "paper_1501_07844_gb300", "csrc", f) for f in e.get("sources", [])]
    if e.get("kernel_source_sha") != kernel_sha(src or None):
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(cfg, min_seconds=10.0, max_iters=1000, zslab=64, seed=2000):
    """The FP64 oracle, as it stands, on a z-slab of the same phantom (same
    x-y extent, labels and parameters): iterations until min_seconds passed."""
    import oracle
    import synth
    shape, nl, gen, _, _ = CONFIGS[cfg]
    slab = (min(zslab, shape[0]),) + tuple(shape[1:])
    if gen == "potts3d":
        p = synth.potts3d_problem(seed=seed, nl=nl, shape=slab)
    else:
        p = synth.hmf_problem(seed=seed, shape=slab)
    D = p.D.astype(np.float64)
    S = None if p.S_field is None else p.S_field.astype(np.float64)
    sn = None if p.s_node is None else p.s_node.astype(np.float64)
    flat = gen == "potts3d"
    if flat:
        u, q = oracle.potts_init(p.spatial, p.n_leaf)
    else:
        dag = oracle.Dag(p.n_nodes, p.edges)
        u, q = oracle.dag_init(p.spatial, dag)
    its, t0 = 0, time.perf_counter()
    while its < max_iters:
        if flat:
            oracle.potts_iterate(D, u, q, 1, p.c, p.tau, S_field=S, s_node=sn)
        else:
            oracle.dag_iterate(dag, D, u, q, 1, p.c, p.tau, S_field=S, s_node=sn)
        its += 1
        if time.perf_counter() - t0 >= min_seconds and its >= 2:
            break
    dt = time.perf_counter() - t0
    vlu = its * int(np.prod(slab)) * p.n_nodes
    return {"value": vlu / dt, "unit": "VLU/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d FP64 iterations of Algorithm %s on a %dx%dx%d slab (%d labels) of the same phantom, %.1f s"
                      % (its, "1" if flat else "2", slab[0], slab[1], slab[2], p.n_nodes, dt)}


def metric_name(cfg):
    """The metric string of a workload, shared by both arms."""
    return ("voxel-label updates/s, 3-D Potts 256^3 x 8 labels" if cfg == "potts3d" else
            "voxel-label updates/s (%s)" % cfg)


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, as it stands, doing exactly the work
    of one GPU step per step: ITERS_PER_STEP iterations of Algorithm 1 / 2 on
    the full volume of the same workload, the last preceded by E and P of its
    input (the gap check).  ms_per_step is the measured wall time of that
    work; rank 0 only (other ranks exit without work)."""
    if rank != 0:
        return
    import oracle
    cfg = args.config
    if cfg not in ("potts3d", "potts3d_inplace", "potts3d_bf16", "hmf", "hmf_bf16", "ishikawa"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the single-volume workloads only"}))
        return
    shape, nl, gen, _, _ = CONFIGS[cfg]
    if args.dims:
        shape = (args.dims,) * 3
    prob = make_problem(cfg, seed=rank_seed(0), shape=shape)
    D = prob.D.astype(np.float64)
    S = None if prob.S_field is None else prob.S_field.astype(np.float64)
    sn = None if prob.s_node is None else prob.s_node.astype(np.float64)
    flat = gen == "potts3d"
    if flat:
        u, q = oracle.potts_init(prob.spatial, prob.n_leaf)
    else:
        dag = oracle.Dag(prob.n_nodes, prob.edges)
        u, q = oracle.dag_init(prob.spatial, dag)

    def step():
        if flat:
            oracle.potts_iterate(D, u, q, ITERS_PER_STEP - 1, prob.c, prob.tau, S_field=S, s_node=sn)
            oracle.potts_energy(D, u, q, S_field=S, s_node=sn)
            oracle.potts_iterate(D, u, q, 1, prob.c, prob.tau, S_field=S, s_node=sn)
        else:
            oracle.dag_iterate(dag, D, u, q, ITERS_PER_STEP - 1, prob.c, prob.tau, S_field=S, s_node=sn)
            oracle.dag_energy(dag, D, u, q, S_field=S, s_node=sn)
            oracle.dag_iterate(dag, D, u, q, 1, prob.c, prob.tau, S_field=S, s_node=sn)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    elapsed = time.perf_counter() - t0
    vlu_step = ITERS_PER_STEP * int(np.prod(shape)) * prob.n_nodes
    v = args.steps * vlu_step / elapsed
    sample = ("each step: %d FP64 iterations of Algorithm %s on the full %s volume (%d nodes), the last preceded "
              "by E and P of its input" % (ITERS_PER_STEP, "1" if flat else "2", "x".join(map(str, shape)),
                                           prob.n_nodes))
    line = {"impl": "reference", "metric": metric_name(cfg), "value": v, "unit": "VLU/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded sphere phantom)",
            "config": {"workload": cfg, "dims": list(shape), "labels": prob.n_leaf, "nodes": prob.n_nodes,
                       "iters_per_step": ITERS_PER_STEP, "c": prob.c, "tau": prob.tau},
            "cpu_baseline": {"value": v, "unit": "VLU/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "VLU/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args, rank, world):
    """32 DAGMF volumes of seeded uneven sizes (64..160 per axis), 10
    end-labels and 4 inner nodes each, advanced together by the batched
    persistent kernel (tuned z-chunk and grid, graph-replayed).  One step =
    10 iterations of every volume + their FP64 energies."""
    import torch
    import paper_1501_07844_gb300 as pfm
    import synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    vols = synth.dagmf_batch(seed=4000 + 100 * rank, count=args.volumes)
    stream = torch.cuda.Stream()  # a capturable (non-default) stream shared with the events
    torch.cuda.set_stream(stream)
    probs = [dict(D=torch.from_numpy(p.D).cuda(), S_field=torch.from_numpy(p.S_field).cuda(), s_node=p.s_node,
                  n_nodes=p.n_nodes, edges=p.edges) for p in vols]
    b = pfm.Batch(probs, c=0.5, tau=0.11, stream=stream.cuda_stream)
    zc, grid = b.tune(trial_iters=3)
    vox = sum(int(np.prod(p.spatial)) for p in vols)
    vlu_step = ITERS_PER_STEP * sum(int(np.prod(p.spatial)) * p.n_nodes for p in vols)
    alg = sum(algorithmic_bytes_per_iter(p, 0, 0) for p in vols)
    for _ in range(args.warmup):
        b.iterate(ITERS_PER_STEP)
        b.energy()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = b.launches
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t0.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            b.iterate(ITERS_PER_STEP)
            ev[k][1].record(stream)
            b.energy()
        t1.record(stream)
        torch.cuda.synchronize()
    elapsed = t0.elapsed_time(t1) / 1e3
    it_ms = sum(a.elapsed_time(c) for a, c in ev) / (args.steps * ITERS_PER_STEP)
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)
    achieved = alg / (it_ms / 1e3) / 1e9
    launches = int(b.launches - l0)
    variant = b.variant
    b.close()
    del b
    torch.cuda.empty_cache()
    # the plain FP32 form on the same volumes: one single-problem solver per
    # volume (each on its most specialised fused kernel), stepped one after
    # another on the stream
    singles = [pfm.Problem(p["D"], S_field=p["S_field"], s_node=p["s_node"], n_nodes=p["n_nodes"],
                           edges=p["edges"], c=0.5, tau=0.11, stream=stream.cuda_stream) for p in probs]
    for _ in range(args.warmup):
        for sp in singles:
            sp.iterate(ITERS_PER_STEP)
            sp.energy()
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for k in range(args.steps):
        for sp in singles:
            sp.iterate(ITERS_PER_STEP)
            sp.energy()
    s1.record(stream)
    torch.cuda.synchronize()
    single_elapsed = s0.elapsed_time(s1) / 1e3
    single_kernels = sorted({sp.variant for sp in singles})
    for sp in singles:
        sp.close()
    singles_line = {"value": args.steps * vlu_step / single_elapsed, "unit": "VLU/s",
                    "ms_per_step": 1e3 * single_elapsed / args.steps,
                    "kernel": "%s, one problem per volume" % "/".join(single_kernels),
                    "batched_over_singles": single_elapsed / elapsed}
    line = {"metric": "voxel-label updates/s (dagmf_batched)", "value": args.steps * vlu_step / elapsed, "unit": "VLU/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "dagmf_batched", "volumes": len(vols), "voxels": vox, "labels": 10, "nodes": 14,
                       "iters_per_step": ITERS_PER_STEP, "tuned_zc": zc, "tuned_grid": grid,
                       "kernel_variant": variant,
                       "shapes": [list(p.spatial) for p in vols]},
            "roofline": {"bound": "hbm", "kernel": {"batched_tma_dag": "batched_dag_tma_kernel",
                                                    "batched_tma_dag4": "batched_dag4_tma_kernel"}.get(variant, "batched_step_kernel"),
                         "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": "measured",
                         "traffic": load_traffic("dagmf_batched") if len(vols) == 32 else None,
                         "algorithmic_bytes_per_launch": alg,
                         "kernel_ms_per_launch": it_ms},
            "gpu_launches": launches, "clocks": clk.summary(), "plain_fp32_singles": singles_line}
    print(json.dumps(line), flush=True)


def run_continuation(args):
    """Iterations to a relative primal-dual gap of 1e-4 on the 3-D Potts
    phantom (128^3 x 8): fixed c = 0.5 against schedules that lower c by
    half every 100 iterations down to a floor (continuation toward the
    c -> 0 limit), and against a larger fixed c."""
    import torch
    import paper_1501_07844_gb300 as pfm
    prob = make_problem("continuation", seed=2000)
    D = torch.from_numpy(prob.D).cuda()
    S = torch.from_numpy(prob.S_field).cuda()
    out = {}
    for name, c0, floor in (("fixed_c0.5", 0.5, 0.5), ("fixed_c1.0", 1.0, 1.0), ("cont_1.0_to_0.25", 1.0, 0.25),
                            ("cont_2.0_to_0.5", 2.0, 0.5)):
        gp = pfm.Problem(D, S_field=S, c=c0, tau=0.11, check_every=10)
        c, done, gap = c0, 0, float("inf")
        t0 = time.perf_counter()
        while done < 20000 and gap > 1e-4:
            if done and done % 100 == 0 and c > floor:
                c = max(floor, c / 2)
                gp.set_step(c, 0.11)
            E, P = gp.iterate_energy(10)
            done += 10
            gap = (E - P) / abs(E)
        torch.cuda.synchronize()
        out[name] = {"iters_to_gap_1e-4": done, "final_gap": gap, "seconds": time.perf_counter() - t0, "final_c": c}
        gp.close()
    print(json.dumps({"metric": "iterations to relative gap 1e-4 (continuation)", "config": {"workload": "potts3d 128^3 x 8"},
                      "results": out}), flush=True)


def run_solve(args):
    """The 3-D Potts workload's stopping rule end to end: 500 fixed
    iterations, then the relative primal-dual gap (E - P)/|E| checked every
    10 iterations until it is <= 1e-4 (pfm_run_to_gap), from the initial
    state; reports the iteration count and the device time (CUDA events),
    median of three solves."""
    import torch
    import paper_1501_07844_gb300 as pfm
    prob = make_problem("potts3d_solve", seed=2000)
    D = torch.from_numpy(prob.D).cuda()
    S = torch.from_numpy(prob.S_field).cuda()
    stream = torch.cuda.current_stream()
    gp = pfm.Problem(D, S_field=S, c=prob.c, tau=prob.tau, check_every=10, gap_tol=1e-4, stream=stream.cuda_stream)
    zc = gp.tune(3)
    runs = []
    for rep in range(3):
        gp.reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gp.iterate(500)
        it, gap, ok = gp.run_to_gap(20000)
        e1.record(stream)
        torch.cuda.synchronize()
        runs.append({"iterations": 500 + it, "rel_gap": gap, "converged": ok, "ms": e0.elapsed_time(e1)})
    E, P = gp.energy()
    gp.close()
    ms = sorted(r["ms"] for r in runs)[1]
    print(json.dumps({"metric": "time to the stopping rule (500 iterations, then gap <= 1e-4 every 10)",
                      "config": {"workload": "potts3d 256^3 x 8", "tuned_zc": zc},
                      "results": {"iterations": runs[0]["iterations"], "rel_gap": runs[0]["rel_gap"],
                                  "converged": runs[0]["converged"], "ms_median": ms, "runs": runs,
                                  "E": E, "P": P}}), flush=True)


def run_fullflow(args):
    """Pseudo-flow (in-place and fused schedules) against the explicit-flow
    augmented-Lagrangian solver on the 3-D Potts volume (256^3 x 8): device
    memory, time and bytes per iteration, and iterations / time until the
    primal objective is within 1e-4 of the optimum estimate E* (pseudo-flow
    run to a relative gap of 1e-6)."""
    import torch
    import paper_1501_07844_gb300 as pfm
    from paper_1501_07844_gb300.binding import alm_footprint, footprint
    prob = make_problem("fullflow", seed=2000)
    D = torch.from_numpy(prob.D).cuda()
    S = torch.from_numpy(prob.S_field).cuda()
    nl, n = prob.n_leaf, int(np.prod(prob.spatial))
    edges = [(-1, L, 1.0) for L in range(nl)]

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        fn(reps)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    ref = pfm.Problem(D, S_field=S, gap_tol=1e-6, check_every=50)
    it_ref, gap_ref, _ = ref.run_to_gap(20000)
    E_star, _ = ref.energy()
    ref.close()
    out["E_star"] = {"value": E_star, "iters": it_ref, "rel_gap": gap_ref}
    for name, sched in (("pseudo_flow_inplace", pfm.INPLACE), ("pseudo_flow_fused", pfm.FUSED)):
        nbytes, nbuf, _ = footprint(prob.spatial, nl, edges, has_S_field=True, schedule=sched)
        gp = pfm.Problem(D, S_field=S, schedule=sched)
        ms = timed(gp.iterate, 20)
        gp.reset()
        done, t_used, reached = 0, 0.0, None
        while done < 5000:
            t_used += 50 * timed(gp.iterate, 50)
            done += 50
            E, _ = gp.energy()
            if abs(E - E_star) <= 1e-4 * abs(E_star):
                reached = done
                break
        out[name] = {"device_bytes": nbytes, "grid_buffers": nbuf, "ms_per_iter": ms,
                     "iters_to_1e-4": reached, "ms_to_1e-4": t_used if reached else None}
        gp.close()
    nbytes, nbuf = alm_footprint(prob.spatial, nl)
    a = pfm.AlmProblem(D, S_field=S, gamma=0.3, step=0.2)
    ms = timed(a.iterate, 20)
    a.close()
    a = pfm.AlmProblem(D, S_field=S, gamma=0.3, step=0.2)
    done, t_used, reached = 0, 0.0, None
    while done < 5000:
        t_used += 50 * timed(a.iterate, 50)
        done += 50
        _, _, flow = a.energy()
        if abs(flow - E_star) <= 1e-4 * abs(E_star):
            reached = done
            break
    out["explicit_flow_alm"] = {"device_bytes": nbytes, "grid_buffers": nbuf, "ms_per_iter": ms,
                                "iters_to_1e-4": reached, "ms_to_1e-4": t_used if reached else None,
                                "last_flow": flow}
    a.close()
    print(json.dumps({"metric": "pseudo-flow vs explicit-flow (memory, time, iterations to 1e-4 of E*)",
                      "config": {"workload": "potts3d 256^3 x 8", "voxels": n}, "results": out}), flush=True)


def run_diff(args):
    """Differentiable Potts: 128^3 x 6 labels, 100 unrolled iterations,
    checkpoint every 10; loss = -sum log u_target.  Times the plain forward
    (100 iterations), the differentiable forward (with checkpoints) and the
    backward (segment recomputation + adjoint kernels)."""
    import torch
    import synth
    import paper_1501_07844_gb300 as pfm
    from paper_1501_07844_gb300.autograd import potts_solve
    prob = synth.diff_problem(seed=5000)
    D = torch.tensor(prob.D, device="cuda", requires_grad=True)
    S = torch.tensor(prob.S_field, device="cuda", requires_grad=True)
    tgt = torch.from_numpy(prob.truth.astype(np.int64)).cuda().unsqueeze(0)

    def ev():
        return torch.cuda.Event(enable_timing=True)
    res = {}
    for rep in range(2):  # first round warms up
        gp = pfm.Problem(D.detach(), S_field=S.detach())
        e0, e1 = ev(), ev()
        e0.record()
        gp.iterate(100)
        e1.record()
        torch.cuda.synchronize()
        plain = e0.elapsed_time(e1)
        gp.close()
        e0, e1, e2 = ev(), ev(), ev()
        e0.record()
        u = potts_solve(D, S, iters=100, checkpoint_every=10)
        L = -torch.log(torch.gather(u.double(), 0, tgt)).sum()
        e1.record()
        D.grad = None
        S.grad = None
        L.backward()
        e2.record()
        torch.cuda.synchronize()
        res = {"plain_forward_ms": plain, "diff_forward_ms": e0.elapsed_time(e1), "backward_ms": e1.elapsed_time(e2),
               "loss": float(L), "grad_D_norm": float(D.grad.norm()), "grad_S_norm": float(S.grad.norm())}
    print(json.dumps({"metric": "differentiable Potts 128^3 x 6, 100 iterations, checkpoint 10 (ms)",
                      "config": {"workload": "diff"}, "results": res}), flush=True)


def run_capacity(args):
    """Largest cube per model and storage that fits the GPU (from the
    library's own footprint), and one measured in-place iteration on a
    512^3 x 8 Potts volume (21 GB in place)."""
    import torch
    import paper_1501_07844_gb300 as pfm
    from paper_1501_07844_gb300.binding import footprint
    import synth
    free, total = torch.cuda.mem_get_info()
    budget = free * 0.95
    out = {"device_bytes_free": free}
    models = {"potts8": (8, [(-1, L, 1.0) for L in range(8)], True), "hmf12": (15, synth.hmf_tree(3, 4)[1], False)}
    for mname, (nn, edges, field) in models.items():
        for sname, sched, stor in (("inplace_f32", pfm.INPLACE, pfm.F32), ("inplace_bf16", pfm.INPLACE, pfm.BF16),
                                   ("fused_f32", pfm.FUSED, pfm.F32), ("fused_bf16", pfm.FUSED, pfm.BF16)):
            b, nbuf, _ = footprint((64, 64, 64), nn, edges, has_S_field=field, schedule=sched, storage=stor)
            per_voxel = b / 64 ** 3
            edge = int((budget / per_voxel) ** (1 / 3))
            out["%s_%s" % (mname, sname)] = {"bytes_per_voxel": per_voxel, "max_cube_edge": edge}
    prob = synth.potts3d_problem(seed=2000, nl=8, shape=(512, 512, 512))
    gp = pfm.Problem(prob.D, S_field=prob.S_field, schedule=pfm.INPLACE)
    del prob
    gp.iterate(2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    gp.iterate(5)
    e1.record()
    torch.cuda.synchronize()
    E, P = gp.energy()
    out["run_512_inplace_f32"] = {"ms_per_iter": e0.elapsed_time(e1) / 5, "E": E, "P": P,
                                  "device_bytes": footprint((512, 512, 512), 8, [(-1, L, 1.0) for L in range(8)],
                                                            has_S_field=True, schedule=pfm.INPLACE)[0]}
    gp.close()
    print(json.dumps({"metric": "largest volume per model in HBM (from pfm_footprint) + 512^3 in-place run",
                      "config": {"workload": "capacity"}, "results": out}), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.config == "dagmf_batched":
        run_batched(args, rank, world)
        return
    if args.config == "continuation":
        run_continuation(args)
        return
    if args.config == "fullflow":
        run_fullflow(args)
        return
    if args.config == "potts3d_solve":
        run_solve(args)
        return
    if args.config == "diff":
        run_diff(args)
        return
    if args.config == "capacity":
        run_capacity(args)
        return

    import torch
    import paper_1501_07844_gb300 as pfm
    assert torch.cuda.is_available(), "bench.py needs a CUDA GPU"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    cfg = args.config
    shape, nl, gen, schedule, storage = CONFIGS[cfg]
    if args.dims:
        shape = (args.dims,) * 3
    prob = make_problem(cfg, seed=rank_seed(rank), shape=shape)
    D = torch.from_numpy(prob.D).cuda()
    S = None if prob.S_field is None else torch.from_numpy(prob.S_field).cuda()
    stream = torch.cuda.current_stream()
    gp = pfm.Problem(D, S_field=S, s_node=prob.s_node, n_nodes=prob.n_nodes, edges=prob.edges,
                     c=prob.c, tau=prob.tau, schedule=schedule, storage=storage,
                     stream=stream.cuda_stream)
    if args.kernel:
        gp.select_kernel(args.kernel)
    # z-chunk length of the plane-marching kernels picked by the autotuner
    # (the trials are discarded: the state starts from the initial one)
    zc = gp.tune(3)
    if args.zc:
        gp.chunk_length = args.zc
        zc = gp.chunk_length
    n = int(np.prod(shape))
    vlu_step = ITERS_PER_STEP * n * prob.n_nodes
    alg_bytes = algorithmic_bytes_per_iter(prob, storage, schedule)

    def step():
        # ITERS_PER_STEP iterations; the last also reduces its input state to
        # (E, P), the gap check (inside the iteration kernel on the TMA path)
        return gp.iterate_energy(ITERS_PER_STEP)

    for _ in range(args.warmup):
        step()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = gp.launches
    barrier()
    with ClockSampler(local) as clk:
        t_start.record(stream)
        for k in range(args.steps):
            ev[k][0].record(stream)
            gp.iterate(ITERS_PER_STEP - 1)      # the dominant kernel, plain launches
            ev[k][1].record(stream)
            gp.iterate_energy(1)                 # last iteration + FP64 energy / dual of its input
        t_end.record(stream)
        barrier()
    launches = gp.launches - launches0
    elapsed = t_start.elapsed_time(t_end) / 1e3
    kern_ms = sum(a.elapsed_time(b) for a, b in ev) / (args.steps * (ITERS_PER_STEP - 1))  # per iteration
    elapsed = reduce_max(elapsed, dist, "cuda")
    value = throughput(world, args.steps, vlu_step, elapsed)

    # end to end through the C ABI with pinned host buffers, every step: make
    # the step's D and S current (uploaded by the library's copy stream while
    # the previous step ran: pfm_prefetch_data / pfm_commit_data), start the
    # next step's upload, iterate with the gap check, read the thresholded
    # labelling back (pfm_get_argmax_async: the copy overlaps the next step;
    # every read-back has landed before the timed region closes)
    e2e = None
    if not args.no_e2e:
        hD = torch.from_numpy(prob.D).pin_memory()
        hS = None if prob.S_field is None else torch.from_numpy(prob.S_field).pin_memory()
        hL = torch.empty(prob.spatial, dtype=torch.int32).pin_memory()
        h2d = hD.numel() * 4 + (0 if hS is None else hS.numel() * 4)
        d2h = hL.numel() * 4 + 16

        def e2e_steps(k_steps):
            gp.prefetch_data(hD, hS)
            for k in range(k_steps):
                gp.commit_data()
                if k + 1 < k_steps:
                    gp.prefetch_data(hD, hS)
                step()
                gp.argmax_async(out=hL)   # lands while the next step runs
            gp.readback_wait()
        e2e_steps(max(1, args.warmup))
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_steps(args.steps)
        e1.record(stream)
        barrier()
        te = e0.elapsed_time(e1) / 1e3
        te = reduce_max(te, dist, "cuda")
        e2e = {"value": throughput(world, args.steps, vlu_step, te), "unit": "VLU/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = alg_bytes / (kern_ms / 1e3) / 1e9
    traffic = load_traffic(cfg)
    # 3-D Potts iterations with BF16 storage run the voxel-pair kernel
    kname = {"fused_tma": "fused_tma_x2_kernel" if (len(shape) == 3 and storage != 0) else "fused_tma_kernel",
             "fused_tma_dag": "fused_dag_tma_kernel", "fused_tma_ishikawa": "ishikawa_tma_kernel",
             "fused_tma_tree": "tree_tma_kernel", "fused_tma_dag4": "dag4_tma_kernel",
             "fused": "fused_step_kernel",
             "inplace": "prox_inplace_kernel+flow_inplace_kernel",
             "inplace_tma": "prox_inplace_tma_kernel+flow_inplace_tma_kernel"}.get(gp.variant, gp.variant)
    gp_variant = gp.variant

    gp.close()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(cfg)
    line = {
        "metric": metric_name(cfg),
        "value": value, "unit": "VLU/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": ("f32", "f32 math, bf16 u/q storage", "f32 math, f16 u/q storage")[storage],
        "data": "synthetic (seeded sphere phantom)",
        "config": {"workload": cfg, "dims": list(shape), "labels": prob.n_leaf, "nodes": prob.n_nodes,
                   "iters_per_step": ITERS_PER_STEP, "schedule": "fused" if schedule == 0 else "in-place",
                   "tuned_zc": zc, "kernel_family": gp_variant,
                   "c": prob.c, "tau": prob.tau, "norm": "iso", "grad_source": "normalised",
                   "l2": "inputs larger than L2 (%.2f GB moved per iteration)" % (alg_bytes / 1e9),
                   "parallelism": "independent volume per GPU" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src, "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms_per_launch": kern_ms},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
