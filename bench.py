"""Benchmark: layered-media FMM apply throughput (targets/s) on GB300.

Workload: the 1M-point wide strip in the k2 = 8 medium (x in [0,20],
y in [-0.95,-0.05], interfaces y = 0 and y = -1, k = (1, 8, 2)), 16 complex
density vectors.  One step = one lm_apply of all 16 vectors (every FMM phase:
permute, S2M, M2M, M2L, L2L, L2T + S2T).  Inputs are resident in HBM when the
timed region starts; they are larger than L2 (256 MB of densities), so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   # the CPU oracle, timed on a sample

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica (the method is not sharded here); value = all ranks' targets / max
rank time.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "targets/s, layered FMM apply at N=1M, rel-err≤1e-6: mixed vs FP64 on GPU"
UNIT = "targets/s"
N_POINTS = 1_000_000
NVEC = 16
PHASES = ["permute", "s2m", "m2m", "m2l", "l2l", "l2t_s2t", "refine"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "mixed", "fp64"])
    ap.add_argument("--n", type=int, default=N_POINTS)
    ap.add_argument("--xmax", type=float, default=20.0,
                    help="strip workload: x in [0, xmax] (20 for the headline; e.g. 400k points on [0, 8] keep its "
                         "49 points per leaf at depth 5 for a smaller profiling case)")
    ap.add_argument("--p", type=int, default=0)
    ap.add_argument("--depth", type=int, default=-2, help="tree depth (-1 automatic; default per precision)")
    ap.add_argument("--tree", default="adaptive", choices=["adaptive", "uniform"],
                    help="clustered workload: adaptive tree (boxes refined where the points are) or uniform depth")
    ap.add_argument("--leaf-target", type=int, default=0, help="points per leaf (0: library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the summaries of the batched, clustered and adjoint workloads that the "
                         "default run adds to its line (each timed on its own, after the headline)")
    ap.add_argument("--workload", default="strip", choices=["strip", "batched", "adjoint", "clustered"],
                    help="strip: the 1M-point headline apply; batched: 48 independent instances in one graph; "
                         "adjoint: J = sum |u - u_obs|^2 and its gradients in q, x, y, d at N = 200k (FP64); "
                         "clustered: N = 100k, half within 0.01 of y = 0, on the adaptive tree (FP64, or "
                         "--precision mixed)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    # 10 ms: about 75 samples per second on GB300 (nvidia-smi returns one line per query), so a
    # 0.1 s region of 20 applies still holds several samples
    PERIOD_MS = 10

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.skip = 0
        # raw samples: $LM_CLOCKS_DIR if set, else the temporary directory
        d = os.environ.get("LM_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"lmfmm_clocks_rank{index}_{os.getpid()}.csv")

    def start(self):
        """Start sampling and wait (up to 3 s) for the sampler's first line, so that
        the region that follows is covered; lines written before it is entered are
        left out of the summary."""
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            with open(self.path) as f:
                n = sum(1 for _ in f)
            if n:
                self.skip = n
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        out = self.summary()
        if not os.environ.get("LM_CLOCKS_DIR"):  # kept only where asked for
            try:
                os.remove(self.path)
            except OSError:
                pass
        return out

    def summary(self):
        """Median SM clock, the maximum, and the throttle reasons seen in the samples
        taken inside the region."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln, line in enumerate(open(self.path)):
            if ln < self.skip:
                continue
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def kernel_hash():
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_1902_08250_gb300", "csrc"))):
        h.update(open(os.path.join(ROOT, "paper_1902_08250_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the
    kernel sources are unchanged since it was captured."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except Exception:
        return None
    ent = rec.get(kernel)
    if not ent or ent.get("source_hash") != kernel_hash():
        return None
    return ent.get("bytes_per_launch")


# ---------------------------------------------------------------------------
def cpu_baseline(x, y, q, medium, budget_s=12.0, ntgt=None, nsrc=None, seed=1):
    """Time the oracle's direct sum (Eq. (direct_sum)) on a bounded sample: a
    few targets summed over a random subset of sources; extrapolated to full
    source sums."""
    import oracle

    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    n = x.size
    ntgt = ntgt or max(2, cores)
    # calibrate: ntgt targets (one per thread) over 300 sources
    src = rng.choice(n, size=min(n, 300), replace=False)
    t0 = time.time()
    oracle.direct_apply(medium, x[src], y[src], q[:1, src], targets=np.arange(min(ntgt, src.size)))
    wall_per_pair = (time.time() - t0) / (min(ntgt, src.size) * src.size)
    nsrc = nsrc or int(min(n, max(500, budget_s / (wall_per_pair * ntgt))))
    src = np.sort(rng.choice(n, size=nsrc, replace=False))
    tg = np.arange(ntgt)
    t0 = time.time()
    oracle.direct_apply(medium, x[src], y[src], q[:1, src], targets=tg, nthreads=cores)
    dt = time.time() - t0
    per_target_full = dt / ntgt * (n / nsrc)
    # the same oracle on one core: one target over a tenth of the sampled sources
    src1 = src[: max(50, nsrc // 10)]
    t0 = time.time()
    oracle.direct_apply(medium, x[src1], y[src1], q[:1, src1], targets=np.arange(1), nthreads=1)
    dt1 = time.time() - t0
    oracle.direct_apply(medium, x[src1[:2]], y[src1[:2]], q[:1, src1[:2]], targets=np.arange(1), nthreads=cores)
    return {"value": 1.0 / per_target_full, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_core_value": 1.0 / (dt1 * (n / src1.size)),
            "sample": f"{ntgt} targets x {nsrc} of {n} sources (1 density vector), "
                      f"{dt:.1f} s wall on {cores} threads, extrapolated to full source sums; single core: "
                      f"1 target x {src1.size} sources, {dt1:.2f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads

    x, y, q = workloads.wide_uniform(args.n, 1)
    med = workloads.MEDIUM_B
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_baseline(x, y, q, med, budget_s=1.0, ntgt=cores)
    vals = []
    # each step is a bounded sample: at most 6 s, and about 3 minutes over all steps
    budget = min(6.0, 180.0 / max(1, args.steps))
    t0 = time.time()
    for _ in range(args.steps):
        vals.append(cpu_baseline(x, y, q, med, budget_s=budget, ntgt=cores))
    wall = time.time() - t0
    v = float(np.mean([c["value"] for c in vals]))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "wide-strip N=1M k=(1,8,2) d=1, 16 vectors",
                                        "n": args.n, "reference": "CPU oracle direct sum (sampled)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": vals[-1]["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def max_over_ranks(times, world, device):
    """Each rank's timings -> their maximum over all ranks (the replicas run concurrently, so
    the job takes as long as its slowest rank); a no-op for one rank."""
    if world <= 1:
        return list(times)
    import torch

    tt = torch.tensor(list(times), dtype=torch.float64, device=device)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return tt.tolist()


def whole_job_value(n_per_rank, world, ms):
    """Targets per second of the whole job: all ranks' targets over the slowest rank's time."""
    return world * n_per_rank / (ms * 1e-3)


def run_batched(args):
    """48 independent instances (own medium, N log-uniform in [10k, 500k], 4
    complex64 vectors), mixed precision, captured into one CUDA graph with one
    tile-form M2L launch over every instance; one step = one launch of the whole
    batch."""
    import torch

    import paper_1902_08250_gb300 as lm
    import workloads

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    inst = workloads.batched_instances(48, seed=0)
    t0 = time.time()
    trees, qs, us = [], [], []
    for med, x, y, q in inst:
        m = lm.create_medium(*med, p=14, precision="mixed")
        t = lm.build_tree(m, torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
        qd = torch.from_numpy(q).to(dev)
        ud = torch.empty_like(qd)
        trees.append(t)
        qs.append(qd)
        us.append(ud)
    torch.cuda.synchronize(dev)
    setup_s = time.time() - t0
    batch = lm.Batch(trees, qs, us)
    launches, joint_m2l = batch.info()   # kernel nodes of the captured graph
    for _ in range(args.warmup):
        batch.launch()
    torch.cuda.synchronize(dev)
    clocks = Clocks(0)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        batch.launch()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ntot = sum(x.size for _, x, _, _ in inst)
    # end to end: pinned host buffers copied in and out around each launch
    qh = [torch.from_numpy(q).pin_memory() for *_, q in inst]
    uh = [torch.empty_like(a).pin_memory() for a in qh]
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        for a, b in zip(qs, qh):
            a.copy_(b, non_blocking=True)
        batch.launch()
        for a, b in zip(uh, us):
            a.copy_(b, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize(dev)
    ms_e2e = e2.elapsed_time(e3) / args.steps
    nbytes = sum(a.numel() * a.element_size() for a in qh)
    # accuracy: each of 8 instances against its FP64 GPU apply
    errs = []
    if not args.no_fp64_compare:
        for i in range(0, 48, 6):
            med, x, y, q = inst[i]
            m = lm.create_medium(*med, p=20)
            t = lm.build_tree(m, torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
            ref = lm.apply(t, qs[i].to(torch.complex128))
            errs.append(float(torch.linalg.norm(us[i].to(torch.complex128) - ref) / torch.linalg.norm(ref)))
            del t, ref
    line = {
        "metric": "targets/s, batched layered FMM apply (48 independent instances, one graph launch)",
        "value": ntot / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "48 instances, N log-uniform in [10k, 500k], k1,k2,k3 ~ U[0.5,4], d ~ U[0.5,2], "
                               "x ~ U[0,10], y ~ U[-0.9d,-0.1d]; 4 complex64 N(0,1) vectors each",
                   "instances": 48, "points": ntot, "nvec": 4, "precision": "mixed", "p": 14,
                   "io": "complex64", "joint_m2l": joint_m2l,
                   "setup_s": setup_s, "parallelism": "replicas x1",
                   "target_vector_evals_per_s": ntot * 4 / (ms * 1e-3)},
        "clocks": ck,
        "e2e": {"value": ntot / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches * args.steps,
        "rel_err_vs_fp64_gpu_max": max(errs) if errs else None,
        "rel_err_instances_checked": len(errs),
    }
    return line


def run_adjoint(args):
    """One step = the forward apply and the backward pass of J = sum |G q - u_obs|^2 with respect
    to the densities, the coordinates and the thickness (FP64, N = 200k, medium k = (1, 1.5, 2))."""
    import torch

    import paper_1902_08250_gb300 as lm
    import workloads

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    n = 200_000
    med = workloads.MEDIUM_A
    x, y, q = workloads.uniform_strip(n, 0.0, 40.0, -0.9, -0.1, nvec=1, seed=0)
    _, _, qref = workloads.uniform_strip(n, 0.0, 40.0, -0.9, -0.1, nvec=1, seed=1)
    p = args.p or 20
    t0 = time.time()
    m = lm.create_medium(*med, p=p)
    tree = lm.build_tree(m, torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
    tree.d_tree()
    torch.cuda.synchronize(dev)
    setup_s = time.time() - t0
    uobs = lm.apply(tree, torch.from_numpy(qref[0]).to(dev))
    q0 = torch.from_numpy(q[0]).to(dev)

    def step():
        qd = q0.clone().requires_grad_(True)
        xd = tree._x.clone().requires_grad_(True)
        yd = tree._y.clone().requires_grad_(True)
        dd = torch.tensor(med[3], dtype=torch.float64, requires_grad=True)
        u = lm.green_apply(tree, qd, xd, yd, dd)
        J = torch.sum(torch.abs(u - uobs) ** 2)
        return torch.autograd.grad(J, (qd, xd, yd, dd))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = Clocks(0)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g = step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    line = {
        "metric": "targets/s, loss + gradients (densities, coordinates, thickness) through the FMM, FP64",
        "value": n / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "N=200k uniform x in [0,40], y in [-0.9,-0.1]; medium k=(1,1.5,2), d=1; "
                               "J = sum |u - u_obs|^2, u_obs from a seed-1 density",
                   "n": n, "p": p, "depth": tree.info["depth"], "setup_s": setup_s,
                   "calls_per_step": "apply + apply_adjoint + apply_grad (2 vectors) + dG/dd apply",
                   "parallelism": "replicas x1"},
        "clocks": ck,
        "gradient_norms": {"q": float(torch.linalg.norm(g[0])), "x": float(torch.linalg.norm(g[1])),
                           "y": float(torch.linalg.norm(g[2])), "d": float(g[3])},
    }
    return line


def run_clustered(args):
    """N = 100k: half the points uniform in the middle layer, half within 0.01 of y = 0 (x spread
    10), one complex128 vector, FP64 (or --precision mixed, p = 14), on the adaptive tree (--tree
    adaptive, default: 16 points per leaf, p = 22) or the uniform tree of automatic
    (occupancy-driven) depth (p = 24); the error is measured against the oracle's direct sum on 16
    targets x all sources."""
    import torch

    import oracle
    import paper_1902_08250_gb300 as lm
    import workloads

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    n = 100_000
    med = workloads.MEDIUM_A
    x, y, q = workloads.clustered(n, 1, seed=0)
    # the least order that meets 1e-10 on this workload: adaptive p = 22 (1.7e-11; p = 20 gives
    # 1.35e-10), uniform p = 24 (4.5e-12; p = 20 gives 1.4e-10); the mixed form's bar is 1e-6 (p = 14)
    mixed = args.precision == "mixed"
    p = args.p or (14 if mixed else (22 if args.tree == "adaptive" else 24))
    t0 = time.time()
    opt = dict(p=p, adaptive=args.tree == "adaptive", precision="mixed" if mixed else "fp64")
    if args.leaf_target > 0:
        opt["leaf_target"] = args.leaf_target
    elif args.tree == "adaptive":
        opt["leaf_target"] = 16  # fastest of 8, 12, 16, 24, 32, 64, 128
    if args.depth >= -1:
        opt["depth"] = args.depth
    m = lm.create_medium(*med, **opt)
    tree = lm.build_tree(m, torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev))
    torch.cuda.synchronize(dev)
    setup_s = time.time() - t0
    qd = torch.from_numpy(q).to(dev)
    ud = torch.empty_like(qd)
    for _ in range(args.warmup):
        lm.apply(tree, qd, ud)
    torch.cuda.synchronize(dev)
    clocks = Clocks(0)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lm.apply(tree, qd, ud)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # phase times from two further applies with per-phase events (outside the timed region)
    lib = lm._lib
    lib.lm_profile_begin(tree._h, 2)
    for _ in range(2):
        lm.apply(tree, qd, ud)
    torch.cuda.synchronize(dev)
    ph_ms = (ctypes.c_double * len(PHASES))()
    ph_n = (ctypes.c_int64 * len(PHASES))()
    napp = ctypes.c_int()
    lib.lm_profile_end(tree._h, ph_ms, ph_n, len(PHASES), ctypes.byref(napp))
    phase_ms = {PHASES[i]: ph_ms[i] / max(1, napp.value) for i in range(len(PHASES))}
    sub = np.sort(np.random.default_rng(0).choice(n, 16, replace=False))
    err = None
    if not args.no_fp64_compare:
        ref = oracle.direct_apply(med, x, y, q, targets=sub)
        err = float(np.linalg.norm(ud.cpu().numpy()[:, sub] - ref) / np.linalg.norm(ref))
    line = {
        "metric": "targets/s, layered FMM apply, clustered N=100k (half within 0.01 of y=0), "
                  + ("mixed precision" if mixed else "FP64"),
        "value": n / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if mixed else "f64",
        "data": "synthetic",
        "config": {"workload": "N=100k: 50k x in [0,10], y in [-0.9,-0.1]; 50k x in [0,10], y in [-0.01,0); "
                               "medium k=(1,1.5,2), d=1; 1 complex N(0,1) vector",
                   "n": n, "p": p, "tree": args.tree, "depth": tree.info["depth"], "nbox": tree.info["nbox"],
                   "nleaf": tree.info["nleaf"], "leaf_target": m.options["leaf_target"], "setup_s": setup_s,
                   "parallelism": "replicas x1"},
        "clocks": ck,
        "phase_ms": phase_ms,
        "rel_err_vs_oracle_direct": err,
        "rel_err_sample": "16 random targets x all 100k sources (oracle direct sum, FP64 adaptive quadrature)",
    }
    return line


def extra_workloads(args):
    """The other workloads of the build, each timed as its own --workload run does (CUDA events over
    10 steps after 3 warm-up steps, clocks sampled), summarised in the headline line."""
    import copy

    keep = ("metric", "value", "unit", "ms_per_step", "dtype", "e2e", "clocks", "rel_err_vs_fp64_gpu_max",
            "rel_err_instances_checked", "rel_err_vs_oracle_direct", "gradient_norms", "gpu_launches")
    out = {}
    for name, fn, extra in (("batched", run_batched, {}), ("clustered_mixed", run_clustered, {"precision": "mixed"}),
                            ("clustered_fp64", run_clustered, {"precision": "fp64"}), ("adjoint", run_adjoint, {})):
        a = copy.copy(args)
        a.steps, a.warmup, a.p, a.depth, a.tree, a.leaf_target = 10, 3, 0, -2, "adaptive", 0
        for k, v in extra.items():
            setattr(a, k, v)
        try:
            ln = fn(a)
            out[name] = {k: ln[k] for k in keep if k in ln}
            out[name]["config"] = ln.get("config", {}).get("workload")
        except Exception as e:  # one workload failing leaves the others and the headline intact
            out[name] = {"error": f"{type(e).__name__}: {e}"}
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batched", "adjoint", "clustered"):
        fn = {"batched": run_batched, "adjoint": run_adjoint, "clustered": run_clustered}[args.workload]
        print(json.dumps(fn(args)), flush=True)
        return
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_1902_08250_gb300 as lm
    import workloads

    precision = args.precision
    if precision == "auto":
        precision = "mixed" if getattr(lm, "HAS_MIXED", False) else "fp64"
    p = args.p or (14 if precision == "mixed" else 20)
    depth = args.depth if args.depth != -2 else (5 if precision == "mixed" else 6)
    if args.xmax == 20.0:
        x, y, q = workloads.wide_uniform(args.n, NVEC, seed=0)
    else:
        x, y, q = workloads.uniform_strip(args.n, 0.0, args.xmax, -0.95, -0.05, NVEC, seed=0)
    med = workloads.MEDIUM_B
    xd = torch.from_numpy(x).to(dev)
    yd = torch.from_numpy(y).to(dev)
    qd = torch.from_numpy(q).to(dev)
    ud = torch.empty_like(qd)
    stream = torch.cuda.current_stream(dev)

    def make(prec, pp=None, dd=None):
        m = lm.create_medium(*med, p=pp or p, precision=prec, depth=depth if dd is None else dd)
        t0 = time.time()
        tr = lm.build_tree(m, xd, yd)
        torch.cuda.synchronize(dev)
        return tr, time.time() - t0

    tree, setup_s = make(precision)
    for _ in range(args.warmup):
        lm.apply(tree, qd, ud)
    torch.cuda.synchronize(dev)

    # --- timed region (device time, CUDA events on the launching stream; no per-phase events) ---
    clocks = Clocks(dev.index if dev.index is not None else 0)
    lib = lm._lib
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lm.apply(tree, qd, ud)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1) / args.steps

    # --- phase times: a second pass of K applies with the library's per-phase CUDA events on
    # the launching stream (kept out of the timed region above) ---
    ph_ms = (ctypes.c_double * len(PHASES))()
    ph_n = (ctypes.c_int64 * len(PHASES))()
    napp = ctypes.c_int()
    lib.lm_profile_begin(tree._h, args.steps)
    for _ in range(args.steps):
        lm.apply(tree, qd, ud)
    torch.cuda.synchronize(dev)
    lib.lm_profile_end(tree._h, ph_ms, ph_n, len(PHASES), ctypes.byref(napp))
    phase_ms = {PHASES[i]: ph_ms[i] / max(1, napp.value) for i in range(len(PHASES))}
    launches = int(sum(ph_n[i] for i in range(len(PHASES))))  # per profiled apply x steps
    launches = launches // max(1, napp.value) * args.steps

    # --- end to end: host (pinned) buffers through the C ABI ---
    # Every step copies its densities in from pinned host memory and its potentials
    # out.  Serial form: copy in, apply, copy out on one stream.  Pipelined form (the
    # reported e2e): two device buffer pairs; step i's copy in runs on a copy stream
    # while step i-1 computes, and its copy out on a second copy stream while step
    # i+1 computes (events order each buffer's reuse).
    qh = torch.from_numpy(q).pin_memory()
    uh = torch.empty_like(qh).pin_memory()
    for _ in range(2):
        qd.copy_(qh, non_blocking=True)
        lm.apply(tree, qd, ud)
        uh.copy_(ud, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        qd.copy_(qh, non_blocking=True)
        lm.apply(tree, qd, ud)
        uh.copy_(ud, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize(dev)
    ms_e2e_serial = e2.elapsed_time(e3) / args.steps
    qb, ub = [qd, torch.empty_like(qd)], [ud, torch.empty_like(ud)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    ev_start = torch.cuda.Event()
    torch.cuda.synchronize(dev)
    e2.record(stream)
    ev_start.record(stream)
    for i in range(args.steps):
        b = i % 2
        s_in.wait_event(ev_start)
        if i >= 2:
            s_in.wait_event(ev_done[b])  # qb[b] is free once step i-2 has computed
        with torch.cuda.stream(s_in):
            qb[b].copy_(qh, non_blocking=True)
        ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        if i >= 2:
            stream.wait_event(ev_out[b])  # ub[b] is free once step i-2's result is out
        lm.apply(tree, qb[b], ub[b], stream=stream)
        ev_done[b].record(stream)
        s_out.wait_event(ev_done[b])
        with torch.cuda.stream(s_out):
            uh.copy_(ub[b], non_blocking=True)
        ev_out[b].record(s_out)
    stream.wait_event(ev_out[(args.steps - 1) % 2])
    e3.record(stream)
    torch.cuda.synchronize(dev)
    ms_e2e = e2.elapsed_time(e3) / args.steps
    bytes_q = q.nbytes

    ms, ms_e2e, ms_e2e_serial = max_over_ranks([ms, ms_e2e, ms_e2e_serial], world, dev)

    # --- accuracy of this precision against the FP64 GPU form (sampled) ---
    rel_err = None
    fp64_val = None
    if precision == "mixed" and not args.no_fp64_compare:
        ref_tree, _ = make("fp64", 20, 6)
        uref = lm.apply(ref_tree, qd)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lm.apply(ref_tree, qd, uref)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        fp64_val = args.n / (ev0.elapsed_time(ev1) * 1e-3)
        rel_err = float(torch.linalg.norm(ud - uref) / torch.linalg.norm(uref))
        del ref_tree, uref

    # --- roofline of the dominant phase ---
    info = tree.info
    P = info["p"]
    npc = 2 * P + 1
    peaks = measured_peaks()
    dom = max(phase_ms, key=phase_ms.get)
    mhz = ck.get("sm_mhz") if isinstance(ck, dict) else None
    roof = roofline(lm, tree, dom, phase_ms[dom], npc, precision, dev, peaks, mhz)
    roof_m2l = roofline(lm, tree, "m2l", phase_ms["m2l"], npc, precision, dev, peaks, mhz) if dom != "m2l" else None

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(x, y, q, med)
        except Exception as e:  # the oracle build needs gcc; report why if absent
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"unavailable: {e}"}
    value = whole_job_value(args.n, world, ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": (f"wide-strip N={args.n / 1e6:g}M uniform x in [0,{args.xmax:g}], y in [-0.95,-0.05]; "
                                "medium k=(1,8,2), d=1; 16 complex N(0,1) density vectors"),
                   "n": args.n, "nvec": NVEC, "precision": precision, "p": P, "depth": info["depth"],
                   "roots": info["R"], "leaves": info["nleaf"],
                   "l2": f"inputs ({q.nbytes / 1e6:.0f} MB of densities) larger than L2 (129 MB)"
                         if q.nbytes > 129e6 else "inputs smaller than L2",
                   "parallelism": f"replicas x{world}", "setup_s": setup_s,
                   "target_vector_evals_per_s": value * NVEC},
        "clocks": ck,
        "e2e": {"value": whole_job_value(args.n, world, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": bytes_q,
                "d2h_bytes_per_step": bytes_q, "form": "two-deep pipeline: copy in / apply / copy out on three "
                "streams", "serial_value": whole_job_value(args.n, world, ms_e2e_serial)},
        "gpu_launches": launches,
        "phase_ms": phase_ms,
        "roofline": roof,
        "roofline_m2l": roof_m2l,
        "cpu_baseline": cpu,
    }
    if rel_err is not None:
        line["rel_err_vs_fp64_gpu"] = rel_err
        line["fp64_value"] = fp64_val
    if world == 1 and not args.no_extras:
        line["workloads"] = extra_workloads(args)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def _probe(lm, kind, dev):
    import torch

    rate = ctypes.c_double()
    lm._lib.lm_peak_probe(kind, 20000, ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream),
                          ctypes.byref(rate))
    return rate.value / 1e12


FP32_LANES_PER_SM = 128      # FP32 FMA lanes per SM: 4 partitions x 32
FP64_DENSE_TFLOPS = 1.25     # GB300 dense FP64, nominal
SM_MAX_MHZ = 2070.0          # GB300 maximum SM clock


def alu_peak(precision, n_sm, mhz=None):
    """The ALU roofline denominator in TFLOP/s, from unit counts and clocks: FP32 FMA
    lanes x 2 flop x SMs x SM clock (the clock sampled during the timed region, else the
    maximum); FP64 at the part's nominal dense rate."""
    if precision == "fp64":
        return FP64_DENSE_TFLOPS, "nominal GB300 dense FP64"
    mhz = float(mhz) if mhz else SM_MAX_MHZ
    peak = n_sm * FP32_LANES_PER_SM * 2.0 * mhz * 1e6 / 1e12
    return peak, f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {mhz:.0f} MHz"


H0_FLOPS = 60        # flops per free-space (i/4) H0 evaluation (series or far form)
TAIL_NODE_FLOPS = 35 # flops per tail quadrature node of a reflected pair (about 4 transcendentals)
BESSEL_FLOPS = 20    # flops per order of the per-target Bessel recurrence of L2T


def leaf_work(tree, npc, nvec):
    """Algorithmic flops of the leaf phase (L2T + S2T) per apply, counted per unit of
    work: a free direct pair is one H0 evaluation plus nvec complex multiply-adds; a
    reflected direct pair is its tail quadrature (tail_order nodes) plus nvec complex
    multiply-adds; L2T is (2p+1) Bessel recurrence steps plus nvec (2p+1) complex
    multiply-adds per target.  The MAC-only count leaves out the kernel evaluations."""
    perm, ls = tree.export()
    cnt = np.diff(ls)
    U = tree.list_export(1)
    pp = cnt[U[:, 0]] * cnt[U[:, 2]]
    free = int(np.sum(pp[U[:, 1] == 0])) - tree.n
    refl = int(np.sum(pp[U[:, 1] != 0]))
    o = tree.medium.options
    q_tail = o.get("tail_order") or (24 if o.get("precision") == 1 else 48)  # the library's defaults
    mac = 8.0 * nvec
    flops = (free * (H0_FLOPS + mac) + refl * (q_tail * TAIL_NODE_FLOPS + mac)
             + tree.n * npc * (BESSEL_FLOPS + mac))
    mac_flops = mac * (free + refl) + mac * npc * tree.n
    desc = (f"{free} free pairs x ({H0_FLOPS} flop H0 + 8x{nvec} MAC) + {refl} reflected pairs x "
            f"({q_tail} tail nodes x {TAIL_NODE_FLOPS} + 8x{nvec}) + {tree.n} targets x {npc} orders x "
            f"({BESSEL_FLOPS} + 8x{nvec})")
    # MMA work the tensor-core leaf step issues: per pass of up to 64 targets of a leaf, one chunk
    # per 64 U-list sources plus the L2T chunk, each M=128 x N=64 x K=128
    tsrc = np.zeros(cnt.size, np.int64)
    np.add.at(tsrc, U[:, 0], cnt[U[:, 2]])
    chunks = int(np.sum(((cnt + 63) // 64) * ((tsrc + 63) // 64 + 1)))
    mma_flops = chunks * 2.0 * 128 * 64 * 128
    return {"flops": flops, "mac_flops": mac_flops, "free_pairs": free, "refl_pairs": refl, "desc": desc,
            "mma_flops": mma_flops}


def roofline(lm, tree, phase, ms, npc, precision, dev, peaks, mhz=None):
    """Algorithmic work of the dominant phase per apply over its measured time
    (CUDA events the library records on the launching stream)."""
    info = tree.info
    L = info["depth"]
    if phase == "m2l":
        entries = sum(tree.list_export(0, l).shape[0] for l in range(L + 1))
        flops = 8.0 * npc * npc * entries * NVEC
        if precision == "fp64":
            peak, src = _probe(lm, 0, dev), "lm_peak_probe FP64 FMA chains on all SMs (measured live)"
        else:
            # the 16-vector tile form runs tcgen05 kind::f16 (FP16 hi/lo operands): the measured bf16
            # dense peak (fp16 has the same dense rate)
            bf = (peaks or {}).get("bf16_tflops")
            peak = bf if bf else 1900.0
            src = "MEASURED_PEAKS bf16_tflops (fp16 has the same dense rate)" if bf else "fallback 1.9 PF bf16"
        ach = flops / (ms * 1e-3) / 1e12
        return {"bound": "tensor" if precision != "fp64" else "alu", "kernel": "m2l", "achieved": ach,
                "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": recorded_traffic("m2l"),
                "work": f"8 (2p+1)^2 flop per V-list entry per vector; {entries} entries", "peak_source": src}
    if phase == "l2t_s2t":
        w = leaf_work(tree, npc, NVEC)
        import torch

        peak, src = alu_peak(precision, torch.cuda.get_device_properties(dev).multi_processor_count, mhz)
        probe = _probe(lm, 0 if precision == "fp64" else 1, dev)
        ach = w["flops"] / (ms * 1e-3) / 1e12
        ach_mac = w["mac_flops"] / (ms * 1e-3) / 1e12
        tl = precision != "fp64" and bool(info.get("tensor_leaf"))
        out = {"bound": "alu",
               "kernel": "k_leaf64" if precision == "fp64" else ("k_leaf_tt" if tl else "k_leaf32") + " + k_near_pw32",
               "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
               "traffic": recorded_traffic("l2t_s2t"),
               "work": w["desc"],
               "achieved_mac_only": ach_mac, "frac_mac_only": ach_mac / peak,
               "peak_source": src + ("" if mhz else " (no clock samples: maximum clock assumed)"),
               "peak_probe": probe,
               "peak_probe_source": "lm_peak_probe %s FMA chains on all SMs (measured live)" %
                                    ("FP64" if precision == "fp64" else "FP32")}
        if tl:
            # the kernel values (H0 series, tails, L2T basis) run on the CUDA cores, the multiply-adds
            # over the vectors on tcgen05 kind::f16: report each side against its own peak
            kv = w["flops"] - w["mac_flops"]
            ach_kv = kv / (ms * 1e-3) / 1e12
            mma = w["mma_flops"]
            bf = (peaks or {}).get("bf16_tflops")
            tpk = bf if bf else 1900.0
            ach_t = mma / (ms * 1e-3) / 1e12
            out["note"] = ("achieved counts the per-unit work of the leaf step (kernel values + 8 nvec MAC per pair) "
                           "against the FP32 pipes; the MACs run on the tensor cores")
            out["kernel_values"] = {"achieved": ach_kv, "peak": peak, "frac": ach_kv / peak, "unit": "TFLOP/s"}
            out["tensor"] = {"mma_flops_per_launch": mma, "achieved": ach_t, "peak": tpk, "frac": ach_t / tpk,
                             "unit": "TFLOP/s",
                             "peak_source": ("MEASURED_PEAKS bf16_tflops (fp16 has the same dense rate)" if bf
                                             else "fallback 1.9 PF bf16"),
                             "work": "per chunk of 64 sources (or the L2T orders) and 64 target slots: "
                                     "M=128 (hi/lo rows) x N=64 (hi/lo, re/im, 16 vectors) x K=128, 2 flop per MAC"}
        return out
    return {"bound": "alu", "kernel": phase, "achieved": None, "peak": None, "unit": "TFLOP/s",
            "frac": None, "traffic": recorded_traffic(phase), "phase_ms": ms}


if __name__ == "__main__":
    main()
