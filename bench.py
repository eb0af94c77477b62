"""Benchmark of the PIT/PIDT particle step on one GB300 (or N replicas).

Metric: particle updates per second of the hot path -- deposit of the current
positions, fused gather + leapfrog push + re-location + key, stable re-bin --
with the field held fixed (the Poisson solve is auxiliary and timed apart).

Default workload: the 3D uniform Langmuir plasma, tripartition depth 5 (243^3
leaves), 8 particles per cell (114,791,256 particles), FP32 split precision
(int32 leaf + 3 x FP32 offset + 3 x FP32 velocity), PIT buckets.

One JSON line on rank 0.  `--impl reference` times the CPU oracle instead, on a
bounded sample of the same workload.  Under torchrun every rank runs its own
replica (the path has no exchange step on one instance per GPU).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1508_02435_gb300 import workloads as W  # noqa: E402

METRIC = "particle-updates/sec (push+rebin+deposit+gather)"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")

# Algorithmic bytes per particle-step of the whole hot path (deposit read,
# state read, state write, amortised grid terms), 3D split / FP64, 2D split /
# FP64 at 16 particles per cell.
STEP_BYTES = {(3, 1): 70.0, (3, 0): 132.0, (2, 1): 48.5, (2, 0): 89.0}

# DRAM traffic that ncu measured per launch of each brick kernel, stored in
# profiles/ as CSV by `bench.py --ingest-ncu` together with the digest of the
# kernel sources at capture time; a row whose digest differs from the current
# sources is stale and reads as unmeasured.
TRAFFIC_CSV = os.path.join(ROOT, "profiles", "dram_traffic_langmuir3d_243cubed_8ppc.csv")
_BRICK_SOURCES = ("paper_1508_02435_gb300/csrc/brick.cu", "paper_1508_02435_gb300/csrc/dev.cuh",
                  "paper_1508_02435_gb300/csrc/segsort.cuh", "paper_1508_02435_gb300/csrc/launch.hpp")
# the sources each measured kernel is compiled from
KERNEL_SOURCES = {"k_brick_push_st": _BRICK_SOURCES, "k_brick_pull_st": _BRICK_SOURCES,
                  "k_vertex_charge": ("paper_1508_02435_gb300/csrc/kernels.cu", "paper_1508_02435_gb300/csrc/dev.cuh",
                                      "paper_1508_02435_gb300/csrc/launch.hpp")}
PHASE_KERNEL = {"push": "k_brick_push_st", "rebin": "k_brick_pull_st", "deposit": "k_vertex_charge"}


def kernel_digest(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, kernel: str):
    """(bytes per launch, row) of the kernel from the committed CSV when it
    was captured from the current sources, else (None, row or None)."""
    import csv
    try:
        rows = [r for r in csv.DictReader(ln for ln in open(TRAFFIC_CSV) if not ln.startswith("#"))]
    except OSError:
        return None, None
    for r in rows:
        if r["workload"] == workload and r["kernel"] == kernel:
            if r["sources_digest"] != kernel_digest(kernel):
                return None, r
            return (float(r["read_bytes"]) + float(r["write_bytes"])) / float(r["launches"]), r
    return None, None


def ingest_ncu(path: str, workload: str, particles: int) -> str:
    """CSV rows (one per brick kernel) from an ncu --csv log of the metrics
    dram__bytes_read.sum, dram__bytes_write.sum and gpu__time_duration.sum,
    stamped with the digest of the current kernel sources."""
    import csv
    acc = {}
    lines = [ln for ln in open(path) if ln.startswith('"')]
    for r in csv.DictReader(lines):
        name = r.get("Kernel Name", "")
        for k in PHASE_KERNEL.values():
            if name.startswith("void pic::" + k + "<") or name.startswith(k + "<") or name.startswith("void " + k) \
                    or ("::" + k + "<") in name or name.startswith(k + "("):
                d = acc.setdefault(k, {"ids": set(), "read": 0.0, "write": 0.0, "ns": 0.0})
                d["ids"].add(r["ID"])
                v = float(r["Metric Value"].replace(",", ""))
                unit = r.get("Metric Unit", "")
                scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1, "usecond": 1e3,
                         "msecond": 1e6}.get(unit, 1)
                if r["Metric Name"] == "dram__bytes_read.sum":
                    d["read"] += v * scale
                elif r["Metric Name"] == "dram__bytes_write.sum":
                    d["write"] += v * scale
                elif r["Metric Name"] == "gpu__time_duration.sum":
                    d["ns"] += v * scale
    out = ["# DRAM bytes of the brick kernels per ncu capture (dram__bytes_read.sum + dram__bytes_write.sum,",
           "# --clock-control none); written by bench.py --ingest-ncu from the capture's CSV log",
           "workload,kernel,launches,read_bytes,write_bytes,duration_ns,particles,sources_digest"]
    for k, d in acc.items():
        out.append(f"{workload},{k},{len(d['ids'])},{d['read']:.0f},{d['write']:.0f},{d['ns']:.0f},{particles},"
                   f"{kernel_digest(k)}")
    return "\n".join(out) + "\n"


def brick_bytes(d: int, ppc: float, track_ids: bool) -> dict:
    """Compulsory bytes per particle of each phase of the brick path (uniform
    tree, PIT, FP32 split), bricks of 9^d leaves: what each kernel must read
    and write given its inputs and outputs.
      push   (k_brick_push_st): offsets + velocities (+ id) in, the brick's
             staged field ((9+1)^d vertices x d x 4 B) and leaf offsets, the
             pushed offsets + velocities (+ id), a 2-byte leaf code and a
             4-byte canonical key out to the destination's staging area;
      rebin  (k_brick_pull_st + helpers): the staged arrivals in, the
             bucket-ordered state (+ id), leaf offsets and 2^d corner partials
             per leaf out;
      deposit (k_vertex_charge): corner partials in, vertex charge out."""
    s0 = 2 * d * 4
    idb = 4 if track_ids else 0
    staged = s0 + idb + 2 + 4
    field = (10 ** d) * d * 4 / ((9 ** d) * ppc)
    nc = 1 << d
    return {
        "push": s0 + idb + field + 4 / ppc + staged,
        "rebin": staged + s0 + idb + 4 / ppc + nc * 4 / ppc,
        "deposit": nc * 4 / ppc + 4 / ppc,
        "permute": 0.0,
    }


def step_shares(d: int, split: bool, ppc: float, brick: bool) -> dict:
    """Each phase's share of the algorithmic bytes of one particle-step (the
    STEP_BYTES of the method: deposit read of the positions, state read,
    state write, grid terms amortised over ppc), by which phase moves them.
      brick path: push reads the state and the field (K1), rebin writes the
        state and sums the deposit partials of the new positions from shared
        memory (K2: the deposit's read of the positions happens there),
        deposit sums the partials into vertex charges;
      generic path: deposit reads the positions, push reads the state and
        the field, permute writes the state; the re-bin bookkeeping moves no
        algorithmic bytes."""
    f = 4 if split else 8
    pos = d * f                                   # positions (split: cell offsets; leaf implicit)
    state = 2 * d * f + 4                         # positions + velocities + leaf
    field = d * f / ppc                           # vertex field, read once
    charge = f / ppc                              # vertex charge, written once
    if brick:
        return {"push": state + field, "rebin": state + pos, "deposit": charge, "permute": 0.0}
    return {"deposit": pos + charge, "push": state + field, "rebin": 0.0, "permute": state}


def max_over_ranks(x: float, dist, device: str) -> float:
    """The largest of every rank's x (the job's time is its slowest rank's);
    x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, n_per_rank: int, steps: int, t_max_ms: float) -> float:
    """Particle updates per second of the whole job: every rank advances its
    own n_per_rank particles `steps` times (weak scaling, replicas)."""
    return world * n_per_rank * steps / (t_max_ms / 1e3)


def load_peaks():
    try:
        return json.load(open(PEAKS)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:  # sampling runs before the timed region starts
                time.sleep(0.01)
            self.lines.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                mx = float(parts[2].split()[0])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload_config(name: str) -> dict:
    n3 = {"langmuir3d": 243 ** 3 * 8, "langmuir3d-small": 81 ** 3 * 8}
    if name == "langmuir3d":
        return {"workload": "3D uniform Langmuir, depth 5 (243^3 leaves), 8 ppc, "
                            f"{n3[name]} particles, vth=0.05, omega_p dt=0.1",
                "precision": "fp32_split", "scheme": "PIT", "d": 3, "ppc": 8}
    if name == "langmuir3d-small":
        return {"workload": "3D uniform Langmuir, depth 4 (81^3 leaves), 8 ppc, "
                            f"{n3[name]} particles (profiling case)",
                "precision": "fp32_split", "scheme": "PIT", "d": 3, "ppc": 8}
    if name == "langmuir2d":
        return {"workload": "2D uniform Langmuir, depth 3 (27^2 leaves), 16 ppc, 11664 particles",
                "precision": "fp64", "scheme": "PIT", "d": 2, "ppc": 16}
    raise SystemExit(f"unknown workload {name}")


def build_workload(name: str):
    if name == "langmuir3d":
        return W.langmuir(3, 5, 8, vth=0.05, dt=0.1, steps=200), workload_config(name)
    if name == "langmuir3d-small":
        return W.langmuir(3, 4, 8, vth=0.05, dt=0.1, steps=200), workload_config(name)
    if name == "langmuir2d":
        return W.langmuir(2, 3, 16), workload_config(name)
    raise SystemExit(f"unknown workload {name}")


_ORACLE = {}


def _oracle_init(d, depth, split, scheme):
    """Per host process: the CPU oracle, as it stands, on its own copy of the
    sample (the 3D Langmuir plasma on a depth-4 tree, 8 particles per cell),
    with the field of the start positions held fixed."""
    import oracle
    w = W.langmuir(d, depth, 8 if d == 3 else 16, vth=0.05, dt=0.1)
    tree = oracle.Tree(d, w.flags)
    prm = oracle.Params(scheme=scheme, q=w.q, qm=w.qm, ion=w.ion, sweeps=10, omega=0.8)
    st = oracle.State32(tree, w.x, w.v, prm) if split else oracle.State64(tree, w.x, w.v, prm)
    Q, tot, res, E = st.field()
    _ORACLE.update(w=w, tree=tree, st=st, E=E, split=split, scheme=scheme)


def _oracle_steps(budget_s):
    """Oracle steps (deposit + gather/push + re-bin) for at least one step and
    about budget_s seconds; returns (particle-updates, seconds, steps, n)."""
    o = _ORACLE
    w, tree, st, E = o["w"], o["tree"], o["st"], o["E"]
    steps, t0 = 0, time.perf_counter()
    while True:
        if o["split"]:
            tree.deposit32(o["scheme"], st.leaf, st.o, np.float32(w.q), np.float32(w.ion))
            tree.push32(st.leaf, st.o, st.v, E, w.qm, w.dt)
        else:
            tree.deposit64(o["scheme"], st.x, w.q, w.ion)
            tree.push64(st.x, st.v, E, w.qm, w.dt)
        st.rebin()
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return w.n * steps, el, steps, w.n


class OraclePool:
    """The CPU oracle on every host core at once: one spawned process per core,
    each stepping its own copy of a bounded sample of the bench workload."""

    def __init__(self, d: int, split: bool, scheme: int = 0, cores: int | None = None):
        import multiprocessing as mp

        import oracle
        oracle.build()
        self.cores = cores or (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())
        self.d, self.depth = d, (4 if d == 3 else 5)
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_oracle_init,
                                                  initargs=(d, self.depth, split, scheme))

    def run(self, budget_s: float):
        """(particle-updates/s of all cores together, wall seconds, steps, n)."""
        res = self.pool.map(_oracle_steps, [budget_s] * self.cores, chunksize=1)
        secs = max(r[1] for r in res)
        return sum(r[0] for r in res) / secs, secs, min(r[2] for r in res), res[0][3]

    def info(self, steps: int, n: int) -> dict:
        return {"kind": "oracle", "cores": self.cores,
                "sample": f"{self.cores} processes, one per host core, each stepping ({steps}+ steps) its own "
                          f"depth-{self.depth} {self.d}D Langmuir sample ({n} particles, 8 ppc: the bench "
                          "workload's density and velocities on a coarser tree) with the single-threaded C "
                          "oracle, field fixed"}

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_rate(d: int, split: bool, scheme: int, budget_s: float, cores: int | None = None):
    """The CPU oracle as it stands, timed on every host core at once for about
    budget_s seconds (OraclePool); returns (rate, cpu_baseline info)."""
    pool = OraclePool(d, split, scheme, cores)
    try:
        rate, _, steps, n = pool.run(budget_s)
        return rate, pool.info(steps, n)
    finally:
        pool.close()


def run_reference(args):
    """The reference arm: the CPU oracle, as it stands, on every host core,
    each timed step one oracle step of every core's own sample of the bench
    workload (OraclePool)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w_name = args.workload
    d = 3 if w_name.startswith("langmuir3d") else 2
    split = d == 3
    pool = OraclePool(d, split)
    try:
        for _ in range(args.warmup):
            pool.run(0.0)
        rates, secs = [], []
        steps, n = 0, 0
        for _ in range(args.steps):
            r, sec, steps, n = pool.run(0.0)
            rates.append(r)
            secs.append(sec)
        info = pool.info(args.steps, n)
    finally:
        pool.close()
    value = sum(r * t for r, t in zip(rates, secs)) / sum(secs)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-updates/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if split else "f64", "data": "synthetic",
           "config": {**workload_config(w_name), "field": "held fixed (solve timed apart)",
                      "parallelism": "1 GPU"},
           "cpu_baseline": {"value": value, "unit": "particle-updates/s", **info},
           "e2e": {"value": value, "unit": "particle-updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_batch(args):
    """256 independent 2D Langmuir instances of uneven size (particle counts
    log-uniform 1e3..1e6, depths 3..5) in one handle: one launch per phase over
    all instances, the fixed-field step captured in a CUDA graph after the
    autotuner picked the block shapes; FP32 split, and FP64 for comparison."""
    import torch
    from paper_1508_02435_gb300 import pic

    insts = W.batched_langmuir(256, 1000, 1_000_000)
    n = sum(w.n for w in insts)
    out = {"metric": METRIC, "unit": "particle-updates/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "data": "synthetic",
           "config": {"workload": f"batch of 256 2D Langmuir instances, {n} particles, depths 3-5, "
                                  "particle counts log-uniform 1e3..1e6",
                      "scheme": "PIT", "d": 2, "parallelism": "1 GPU",
                      "l2": "inputs larger than L2 (state > 1 GB)", "field": "held fixed (solve timed apart)"}}
    res = {}
    for prec, name in ((pic.FP32_SPLIT, "fp32_split"), (pic.FP64, "fp64")):
        stream = torch.cuda.Stream()
        g = pic.Pic.batch(2, [w.flags for w in insts], [w.x for w in insts], [w.v for w in insts],
                          qs=[w.q for w in insts], scheme=pic.PIT, precision=prec, sweeps=10, omega=0.8,
                          track_ids=False, stream=stream)
        g.init_leapfrog(0.1)
        tuned = g.autotune(0.1, trials=2)
        g.graph_capture(0.1)
        g.graph_launch(max(args.warmup, 3))
        g.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.graph_launch(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        if g.stats().error:
            raise SystemExit("device reported non-finite particle state")
        res[name] = {"value": n / (ms / 1e3), "ms_per_step": ms, "tuning": tuned,
                     "step_roofline_frac": STEP_BYTES[(2, 1 if prec == pic.FP32_SPLIT else 0)] * n
                     / (ms / 1e3) / 1e9 / float(load_peaks()[0]["hbm_gbs"])}
        g.close()
    out.update(value=res["fp32_split"]["value"], ms_per_step=res["fp32_split"]["ms_per_step"], dtype="f32",
               fp64=res["fp64"], tuning=res["fp32_split"]["tuning"],
               step_roofline={"bytes_per_particle": STEP_BYTES[(2, 1)],
                              "frac": res["fp32_split"]["step_roofline_frac"]})
    return out


def run_twostream(args):
    """The 3D adaptive two-stream configuration: 2e8 particles (two beams at
    +-8 cells per step plus a thermal background), PIDT, FP32 split, the tree
    refined above 32 particles per leaf between depths 4 and 6 by the device's
    ppc criterion (pic_adapt).  The fixed-field step is timed on the adapted
    tree (generic kernels: the brick path is PIT on uniform trees only); one
    re-refinement is timed apart and amortised over the 5 steps between
    re-refinements."""
    import torch
    from paper_1508_02435_gb300 import pic

    w = W.two_stream(n=getattr(args, "twostream_particles", 200_000_000))
    n = w.n
    stream = torch.cuda.Stream()
    g = pic.Pic(3, w.flags, w.x, w.v, scheme=pic.PIDT, precision=pic.FP32_SPLIT, q=w.q, qm=w.qm, ion=w.ion,
                sweeps=10, omega=0.8, track_ids=False, stream=stream)
    del w.x, w.v
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.adapt(32, 4, 6)
    g.sync()
    retree_ms = (time.perf_counter() - t0) * 1e3
    info = g.info()
    g.init_leapfrog(w.dt)
    for _ in range(max(args.warmup, 3)):
        g.step_fixed_field(w.dt)
    g.sync()
    g.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if getattr(args, "profile_range", False):
        torch.cuda.profiler.start()
    e0.record(stream)
    for _ in range(args.steps):
        g.step_fixed_field(w.dt)
    e1.record(stream)
    torch.cuda.synchronize()
    if getattr(args, "profile_range", False):
        torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    phases = g.phase_times()
    if g.stats().error:
        raise SystemExit("device reported non-finite particle state")
    hbm = float(load_peaks()[0]["hbm_gbs"])
    out = {"metric": METRIC, "value": n / (ms / 1e3), "unit": "particle-updates/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"3D adaptive two-stream, {n} particles, PIDT, depth 4-6 refined above 32 "
                                  "particles per leaf", "precision": "fp32_split", "scheme": "PIDT", "d": 3,
                      "leaves": int(info.n_leaves), "depth": int(info.depth), "field": "held fixed (solve timed apart)",
                      "l2": "inputs larger than L2", "parallelism": "1 GPU"},
           "retree": {"ms": retree_ms, "every": 5,
                      "value_with_retree": n / ((ms + retree_ms / 5) / 1e3)},
           "step_roofline": {"bytes_per_particle": STEP_BYTES[(3, 1)],
                             "frac": STEP_BYTES[(3, 1)] * n / (ms / 1e3) / 1e9 / hbm},
           "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()}}
    g.close()
    return out


def run_particles(args):
    """The particle-handling benchmark of the paper's experiments (Section 6):
    no field, velocities of uniform speed 0 <= |v| <= 1 in random directions,
    reflecting walls, the tree re-refined by the ppc criterion before every
    step (pic_adapt: refine above ppc, coarsen sibling sets whose union stays
    within ppc).  2D, 1e7 particles, ppc = 1000, homogeneous and (0, 0.1)^2
    ("breaking dam") starts, PIT and PIDT, dt in {1e-4, 1e-3, 1e-2}, FP32
    split.  Throughput = particle updates per second over 50 steps including
    the re-refinements (set-up excluded); lifts, drops and tunnellers per
    particle and step from a second, counting run of the first 50 steps; the
    artificial flops per move (0 ... 4096) on the homogeneous PIT case."""
    import torch
    from paper_1508_02435_gb300 import pic

    d, n, ppc, dmin, dmax, steps = 2, 10_000_000, 1000, 1, 8, 50
    hbm = float(load_peaks()[0]["hbm_gbs"])
    state_b = 4 + 2 * d * 4          # leaf id + FP32 offsets + FP32 velocities
    rows = []

    def run(dam, scheme, dt, flops, precision=pic.FP32_SPLIT, count=False):
        w = W.particle_handling(d, n, dam=dam, seed=7)
        stream = torch.cuda.Stream()
        g = pic.Pic(d, w.flags, w.x, w.v, scheme=scheme, precision=precision, q=0.0, qm=0.0, ion=0.0,
                    sweeps=0, track_ids=count, stream=stream)
        del w
        g.adapt(ppc, dmin, dmax)                       # set-up, not timed
        if count:
            g.count_lifts(True)
        else:
            for _ in range(3):
                g.adapt(ppc, dmin, dmax)
                g.step_particles(dt, reflect=True, flops=flops)
        g.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.adapt(ppc, dmin, dmax)
            g.step_particles(dt, reflect=True, flops=flops)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        info = g.info()
        if g.stats().error:
            raise SystemExit("device reported non-finite particle state")
        res = {"ms_per_step": ms, "value": n / (ms / 1e3), "leaves": int(info.n_leaves),
               "depth": int(info.depth)}
        if count:
            li, dr, tu, st = g.lift_counts()
            res = {"lifts_per_particle_step": li / (n * st), "drops_per_particle_step": dr / (n * st),
                   "tunnellers_per_particle_step": tu / (n * st)}
        g.close()
        torch.cuda.empty_cache()
        return res

    for dam in (False, True):
        for scheme in (pic.PIT, pic.PIDT):
            for dt in (1e-4, 1e-3, 1e-2):
                r = run(dam, scheme, dt, 0)
                r.update(run(dam, scheme, dt, 0, count=True))
                rows.append({"start": "dam" if dam else "homogeneous",
                             "scheme": "PIT" if scheme == pic.PIT else "PIDT", "dt": dt, **r})
    flops_rows = []
    for fl in (128, 1024, 4096):
        r = run(False, pic.PIT, 1e-4, fl)
        flops_rows.append({"flops": fl, **r, "flop_rate_tflops": fl * n / (r["ms_per_step"] / 1e3) / 1e12})
    fp64 = run(False, pic.PIT, 1e-4, 0, precision=pic.FP64)
    head = rows[0]
    return {"metric": "particle-updates/s (particle handling: move + re-bin + re-refinement)",
            "value": head["value"], "unit": "particle-updates/s", "n_gpus": 1, "steps": steps, "warmup": 3,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"2D particle handling, {n} particles, ppc {ppc}, depth {dmin}-{dmax}, "
                                   "reflecting walls, re-refined before every step; headline: homogeneous "
                                   "start, PIT, dt 1e-4",
                       "precision": "fp32_split", "d": d, "parallelism": "1 GPU",
                       "l2": "inputs larger than L2 (state 200 MB per buffer)"},
            "step_roofline": {"bytes_per_particle": 2 * state_b,
                              "frac": 2 * state_b * n / (head["ms_per_step"] / 1e3) / 1e9 / hbm},
            "sweep": rows, "flops": flops_rows, "fp64": fp64}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="langmuir3d",
                    choices=["langmuir3d", "langmuir3d-small", "langmuir2d", "batch256", "twostream3d"])
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--twostream-particles", type=int, default=200_000_000,
                    help="particles of the 3D two-stream configuration (smaller for profiling)")
    ap.add_argument("--profile-range", action="store_true",
                    help="start and stop the CUDA profiler around the timed steps (for ncu --profile-from-start off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--oracle-seconds", type=float, default=15.0)
    ap.add_argument("--only-main", action="store_true",
                    help="skip the other configurations (3D adaptive two-stream PIDT, batch of 256)")
    ap.add_argument("--ingest-ncu", default=None,
                    help="write the DRAM-traffic CSV of the brick kernels from an ncu --csv log and exit")
    ap.add_argument("--particles", type=int, default=243 ** 3 * 8,
                    help="particles of the captured workload (with --ingest-ncu)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch256":
        print(json.dumps(run_batch(args)))
        return
    if args.workload == "twostream3d":
        print(json.dumps(run_twostream(args)))
        return
    if args.ingest_ncu:
        sys.stdout.write(ingest_ncu(args.ingest_ncu, args.workload, args.particles))
        return

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1508_02435_gb300 import pic

    w, cfg = build_workload(args.workload)
    d = cfg["d"]
    split = cfg["precision"] == "fp32_split"
    stream = torch.cuda.Stream()
    g = pic.Pic(d, w.flags, w.x, w.v, scheme=pic.PIT, precision=pic.FP32_SPLIT if split else pic.FP64,
                q=w.q, qm=w.qm, ion=w.ion, sweeps=10, omega=0.8, track_ids=False, stream=stream)
    n = g.n
    g.init_leapfrog(w.dt)
    # a second, independent handle for the pipelined end-to-end measurement
    stream2 = torch.cuda.Stream()
    g2 = pic.Pic(d, w.flags, w.x, w.v, scheme=pic.PIT, precision=pic.FP32_SPLIT if split else pic.FP64,
                 q=w.q, qm=w.qm, ion=w.ion, sweeps=10, omega=0.8, track_ids=False, stream=stream2)
    g2.init_leapfrog(w.dt)
    fp64 = None
    if split and not args.no_fp64 and world == 1:
        # the same workload in FP64 (generic kernels), timed apart: the metric
        # compares FP32 split with FP64
        g64 = pic.Pic(d, w.flags, w.x, w.v, scheme=pic.PIT, precision=pic.FP64, q=w.q, qm=w.qm, ion=w.ion,
                      sweeps=10, omega=0.8, track_ids=False, stream=stream)
        g64.init_leapfrog(w.dt)
        for _ in range(3):
            g64.step_fixed_field(w.dt)
        g64.sync()
        k64 = max(5, min(args.steps, 20))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k64):
            g64.step_fixed_field(w.dt)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / k64
        fp64 = {"value": n / (ms64 / 1e3), "unit": "particle-updates/s", "ms_per_step": ms64, "steps": k64,
                "path": "generic kernels (FP64 positions and velocities, 132 B per particle-step)",
                "step_roofline_frac": STEP_BYTES[(d, 0)] * n / (ms64 / 1e3) / 1e9 / float(load_peaks()[0]["hbm_gbs"])}
        g64.close()
    del w.x, w.v
    for _ in range(max(args.warmup, 3)):
        g.step_fixed_field(w.dt)
    g.sync()

    # ---- timed region: device-resident state --------------------------
    g.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        if args.profile_range:   # the profiler captures exactly the timed steps (ncu --profile-from-start off)
            torch.cuda.profiler.start()
        ev0.record(stream)
        for _ in range(args.steps):
            g.step_fixed_field(w.dt)
        ev1.record(stream)
        torch.cuda.synchronize()
        if args.profile_range:
            torch.cuda.profiler.stop()
        barrier()
    ms = ev0.elapsed_time(ev1)
    phases = g.phase_times()
    g.profile(False)
    st = g.stats()
    if st.error:
        raise SystemExit("device reported non-finite particle state")
    t_max = max_over_ranks(ms, dist, "cuda")
    ms_step = t_max / args.steps
    value = whole_job_rate(world, n, args.steps, t_max)

    # ---- end to end through the C ABI with host buffers ------------------
    fs = 4 if split else 8
    leaf_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
    pos_h = torch.empty((d, n), dtype=torch.float32 if split else torch.float64, pin_memory=True)
    vel_h = torch.empty_like(pos_h, pin_memory=True)
    g.get_state(leaf_h, pos_h, vel_h)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        g.set_state(leaf_h, pos_h, vel_h)
        g.step_fixed_field(w.dt)
        g.get_state(leaf_h, pos_h, vel_h)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    state_bytes = n * (4 + 2 * d * fs)
    e2e_serial = world * n * args.e2e_steps / e2e_s

    # pipelined: two independent handles, each on its own stream and host
    # thread, each step still uploading its input and downloading its result;
    # one handle's upload overlaps the other's download (the link is full duplex)
    import threading
    bufs = (leaf_h, pos_h, vel_h)
    bufs2 = (torch.empty_like(leaf_h, pin_memory=True), torch.empty_like(pos_h, pin_memory=True),
             torch.empty_like(vel_h, pin_memory=True))
    g2.get_state(*bufs2)
    errors = []

    def drive(gg, bb, k):
        try:
            for _ in range(k):
                gg.set_state(*bb)
                gg.step_fixed_field(w.dt)
                gg.get_state(*bb)
        except Exception as exc:  # re-raised below
            errors.append(exc)

    drive(g2, bufs2, 1)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    threads = [threading.Thread(target=drive, args=(gg, bb, args.e2e_steps)) for gg, bb in ((g, bufs), (g2, bufs2))]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    torch.cuda.synchronize()
    e2e_pipe_s = time.perf_counter() - t0
    barrier()
    if errors:
        raise errors[0]
    e2e_value = world * 2 * n * args.e2e_steps / e2e_pipe_s
    g2.close()

    # ---- calibration: the paper's stream-like particle update ------------
    # (explicit Euler + wall reflection, no grid, no reordering) on arrays of
    # the same particle count: the ceiling of any particle step here
    calib = {}
    for name, dt_ in (("fp32", torch.float32), ("fp64", torch.float64)):
        xs = torch.rand((d, n), dtype=dt_, device="cuda")
        vs = (torch.rand((d, n), dtype=dt_, device="cuda") - 0.5) * 0.1
        pic.stream_step(xs, vs, w.dt, steps=3, stream=stream)
        k = 10
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pic.stream_step(xs, vs, w.dt, steps=k, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / k
        bpp = 3 * d * xs.element_size()   # x and v read, x written
        calib["stream_" + name] = {"particles_per_s": n / sec, "gbs": bpp * n / sec / 1e9, "bytes_per_particle": bpp,
                                   "ms_per_pass": sec * 1e3}
        del xs, vs
    calib["paper"] = ("the same update on SuperMUC (16 Sandy Bridge cores, 1e8 particles): 2.84e8 (d=2) and "
                      "1.92e8 (d=3) particles/s")

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    info = g.info()
    shares = step_shares(d, split, cfg["ppc"], bool(info.brick))
    names = {"push": "k_brick_push_st (gather + kick + drift + re-location + append to the destination's staging area)",
             "rebin": "k_brick_pull_st (+ overflow and unit-offset helpers): canonical re-bin + corner partials",
             "deposit": "k_vertex_charge (vertex sums of the corner partials)"} if info.brick else {}
    dom = max(("deposit", "push", "rebin", "permute"), key=lambda k: phases[k][0])
    dom_ms = phases[dom][0] / args.steps
    achieved = shares[dom] * n / (dom_ms / 1e3) / 1e9
    step_bytes = STEP_BYTES[(d, 1 if split else 0)]
    traffic, trow = (measured_traffic(args.workload, PHASE_KERNEL[dom]) if info.brick and dom in PHASE_KERNEL
                     else (None, None))
    staged = brick_bytes(d, cfg["ppc"], track_ids=False) if info.brick else None
    launches = sum(k for _, k in phases.values())
    out = {
        "metric": METRIC, "value": value, "unit": "particle-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if split else "f64", "data": "synthetic",
        "config": {**cfg, "n_particles": n, "field": "held fixed (solve timed apart)",
                   "l2": "inputs larger than L2 (state > 3 GB)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": {"bound": "hbm", "kernel": names.get(dom, dom), "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind, "traffic": traffic,
                     "algorithmic_bytes_per_particle": shares[dom],
                     "algorithmic_bytes": f"the kernel's share of the {step_bytes:g} B particle-step "
                                          "(state read + field read, grid terms over ppc)" if dom == "push" else
                                          f"the kernel's share of the {step_bytes:g} B particle-step",
                     "traffic_source": (f"ncu capture of these sources ({trow['launches']} launches), "
                                        "profiles/dram_traffic_langmuir3d_243cubed_8ppc.csv") if traffic else
                                       ("stale: the kernel changed since the committed capture" if trow else None),
                     "design_bytes_per_particle": staged[dom] if staged else None,
                     "launch_ms": dom_ms},
        "phase_roofline": {k: {"algorithmic_bytes_per_particle": shares[k],
                               "achieved_gbs": shares[k] * n / (phases[k][0] / args.steps / 1e3) / 1e9
                               if phases[k][0] > 0 else None,
                               "frac": shares[k] * n / (phases[k][0] / args.steps / 1e3) / 1e9 / hbm
                               if phases[k][0] > 0 else None,
                               "ms": phases[k][0] / args.steps}
                           for k in ("deposit", "push", "rebin", "permute") if shares[k] > 0},
        "step_roofline": {"bytes_per_particle": step_bytes,
                          "achieved_gbs": step_bytes * n / (ms_step / 1e3) / 1e9,
                          "frac": step_bytes * n / (ms_step / 1e3) / 1e9 / hbm},
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": "particle-updates/s", "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes, "steps": args.e2e_steps,
                "mode": "two independent handles, each driven by its own host thread and stream: every step "
                        "uploads its state from pinned host memory (pic_set_state), steps, and downloads the "
                        "result (pic_get_state); one handle's upload overlaps the other's download",
                "serial": {"value": e2e_serial, "steps": args.e2e_steps,
                           "mode": "one handle, upload / step / download in sequence"}},
    }
    out["calibration"] = calib
    if fp64 is not None:
        out["fp64"] = fp64
    if world == 1 and not args.only_main and args.workload == "langmuir3d":
        # the other configurations, each timed on its own (their handles are
        # created after the main handles are closed)
        g.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        out["workloads"] = {"twostream3d": run_twostream(args), "batch256": run_batch(args),
                            "particle_handling2d": run_particles(args)}
    if world == 1 and not args.no_cpu_baseline:
        rate, info = oracle_rate(d, split, 0, args.oracle_seconds)
        out["cpu_baseline"] = {"value": rate, "unit": "particle-updates/s", **info}
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
