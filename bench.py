"""Benchmark: forward window + discrete adjoint of the windowed LBM-LES.

One step = one pass of the whole hot path on the largest single-GPU workload,
the D3Q19 U-bend duct 384x192x192 (14.2 M nodes, Re 3000, Cs 0.15,
|W| = 2000, FP32 populations, BF16 checkpoints every 50 steps): a forward
window of 2000 fused collide-stream steps with sampling and checkpoints, the
window-end reduction and the consecutive-window test, the discrete adjoint
over that window (40 segments recomputed from their checkpoints, 2000 adjoint
steps) and the design gradient.

value = (forward + adjoint) lattice updates / second over all ranks, in MLUPS.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

``--impl reference`` times the FP64 CPU oracle instead, on this host's cores,
on a bounded sample of the same workload (for the U-bends, the same duct
scaled down so that the oracle's per-node Jacobians fit in host memory).
Under torchrun each rank runs an independent replica (the path is one GPU per
problem).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# Each CPU oracle process runs on one thread: pin every BLAS / OpenMP pool to
# one thread before numpy loads (spawned workers inherit it), so that the
# reported core count is exact.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

METRIC = "forward & adjoint MLUPS and % HBM roofline, FP32/mixed vs FP64 at stated error"
WORKLOAD = "ubend384x192x192"
CKPT_NAMES = ["fp32", "fp16", "bf16", "moment"]   # lbm_config.ckpt_format
KERNEL_SRC = os.path.join(ROOT, "paper_2608_19617_b300", "csrc", "kernels.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
FP64_OPS_FILE = os.path.join(ROOT, "profiles", "fp64_ops.json")
# FP64 thread-instructions an SM issues per clock on B300: the nominal 1.25
# TFLOP/s over 148 SMs at 2032 MHz is 2.08 flops per SM per clock, one FMA pair.
FP64_INST_PER_SM_CLK = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-check", action="store_true")
    ap.add_argument("--window-len", type=int, default=0, help="override |W| (profiling runs)")
    ap.add_argument("--ckpt-every", type=int, default=0, help="override K (profiling runs)")
    ap.add_argument("--spinup-windows", type=int, default=20,
                    help="spin-up: windows of Alg. 1 until Eq. 26 holds, at most this many")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--ckpt-format", default="", choices=[""] + CKPT_NAMES,
                    help="override the workload's checkpoint format")
    ap.add_argument("--graphs", type=int, default=1, help="replay windows / sweeps as CUDA graphs")
    ap.add_argument("--pipeline", type=int, default=1,
                    help="recompute the next segment while the adjoint sweeps the current one")
    ap.add_argument("--pdl", type=int, default=1, help="programmatic dependent launch of the step kernels")
    ap.add_argument("--quick", action="store_true",
                    help="profiling run: no CPU baseline, no FP64 check, no e2e pass")
    ap.add_argument("--full-time", action="store_true",
                    help="Sec. 4.2.3 comparison instead of the throughput line: one design gradient by the "
                         "consecutive-window framework against the full-time adjoint (default workload "
                         "cylinder200x100)")
    ap.add_argument("--optimize", type=int, default=0,
                    help="run this many iterations of the optimization loop (Alg. 2: windows until Eq. 26, "
                         "adjoint, filter chain rule, MMA) on the cylinder drag case and print their timing")
    ap.add_argument("--fd-protocol", action="store_true",
                    help="the sensitivity validation of Sec. 4.2.1 on the cylinder case: finite differences "
                         "(perturbations 1e-3 and 1e-4, FP64 batches of independent slices) against the adjoint "
                         "at 60 points in the downstream half of the cylinder")
    ap.add_argument("--ckpt-sweep", action="store_true",
                    help="checkpoint-storage sweep: FP32, FP16 and BF16 checkpoints of the FP32 adjoint against "
                         "the FP64 GPU adjoint along the same trajectory (gradient cosine, J error, sweep time, "
                         "workspace)")
    ap.add_argument("--full-time-k", type=int, default=1,
                    help="checkpoint interval of the full-time run (1: the complete history)")
    ap.add_argument("--full-time-cap-gb", type=float, default=96.0,
                    help="largest device workspace the full-time run may take")
    a = ap.parse_args()
    if a.quick:
        a.no_cpu_baseline = a.no_fp64_check = True
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def clocks_rejected(c):
    """A clock record the timing rules reject: hw_slowdown, hw_thermal_slowdown
    or sw_thermal_slowdown active, or a median SM clock below 85% of the
    maximum with no reason active (sw_power_cap is kept and noted)."""
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(c.get("reasons", [])):
        return True
    sm, mx = c.get("sm_mhz"), c.get("sm_max_mhz")
    return bool(sm and mx and sm < 0.85 * mx and not c.get("reasons"))


# --------------------------------------------------------------- roofline --

def bytes_per_lu(case, phase, rs=4):
    """Algorithmic DRAM bytes per lattice update of one launch (FP32 unless rs=8).

    forward / recompute: read Q populations, write Q, read g: (2Q+1) rs.
    adjoint: read Q adjoints, Q populations, g; write Q adjoints: (3Q+1) rs;
    plus the per-segment sensitivity partial (rs read + rs write) per
    design-box node and the objective weight (4 B) per objective-box node at
    sampling steps.
    """
    q, n = case.lattice, case.n
    if phase in ("forward", "recompute"):
        return (2 * q + 1) * rs
    x0, x1, y0, y1, z0, z1 = case.design_box
    nd = (x1 - x0) * (y1 - y0) * (z1 - z0)
    x0, x1, y0, y1, z0, z1 = case.obj_box
    no = (x1 - x0) * (y1 - y0) * (z1 - z0)
    return (3 * q + 1) * rs + 2.0 * rs * nd / n + 4.0 * no / n / case.sample_every


def scope_bytes_per_lu(case, unit, rs=4):
    """The scope table's algorithmic bytes per lattice update of a unit of
    work: forward (2Q + 1) 4 B (D2Q9 76, D3Q19 156; FP64 148 / 308); adjoint
    sweep step = adjoint kernel (12Q + 4 + 32 B: two population reads, one
    write, g, an FP64 (sum, comp) accumulator read and written per step) plus
    a recompute step and a segment store (D2Q9 256, D3Q19 496), twice that in
    FP64.  This count is an upper bound for this design, which folds an FP32
    per-segment partial (8 B per design node per step, not 32) and whose
    recompute writes each state once (no separate store); bytes_per_lu() is
    the design's own count."""
    q = case.lattice
    fwd = {9: 76, 19: 156}[q] if rs == 4 else {9: 148, 19: 308}[q]
    if unit == "forward step":
        return fwd
    return {9: 256, 19: 496}[q] * (rs // 4)


def kernel_hash():
    return hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]


def measured_traffic(kernel, case, precision="fp32"):
    """DRAM bytes per launch of kernel on this workload from profiles/traffic.json:
    an ncu capture of the workload itself, or of a smaller lattice of the same
    family listed as scaling to it (bytes per node x this lattice's nodes;
    DRAM traffic of a step grows with the node count).  None without a
    capture of the current kernel source in this precision."""
    try:
        t = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    for e in t.get("entries", []):
        if e.get("kernel") != kernel or e.get("source_hash") != kernel_hash():
            continue
        if e.get("precision", "fp32") != precision:
            continue
        if e.get("workload") == case.name:
            return e.get("bytes_per_launch")
        if case.name in e.get("scales_to", []):
            return e["bytes_per_launch"] / e["nodes"] * case.n
    return None


def fp64_check_window(case, cap_bytes=150e9):
    """Window and checkpoint interval of the FP64 cross-check: the longest of
    |W|, |W|/2, 1000, 500, 250, 200 steps whose FP64 workspace stays under
    cap_bytes.  K is the workload's own interval where it divides the window
    (the FP64 run follows the FP32 run's checkpoints), else the interval
    minimising |W|/K + K slots."""
    slot = case.lattice * case.n * 8
    W = case.window_len
    for Wc in [W, W // 2, 1000, 500, 250, 200]:
        if Wc > W or Wc < 1:
            continue
        if Wc % case.ckpt_every == 0:
            K = case.ckpt_every
        else:
            K = min((d for d in range(1, Wc + 1) if Wc % d == 0), key=lambda d: Wc // d + d)
        if (Wc // K + K + 6) * slot <= cap_bytes:
            return Wc, K
    return 200, 10


def reduce_max(value, world, device="cuda"):
    """Max of a per-rank scalar over all ranks (the slowest rank's time)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(lus_per_step_per_rank, steps, world, ms_max):
    """Lattice updates of all ranks over the slowest rank's time, in MLUPS."""
    return world * steps * lus_per_step_per_rank / (ms_max / 1e3) / 1e6


FWD_KERNELS = ("fwd_row_kernel", "fwd_facerow_kernel")
ADJ_KERNELS = ("adj_step_kernel",)


def unit_traffic(unit, case, precision="fp32"):
    """ncu DRAM bytes of one launch of a step (forward: its two kernels;
    adjoint: its kernel), None if a kernel has no capture for the current
    source in this precision."""
    ks = FWD_KERNELS if unit == "forward step" else ADJ_KERNELS
    v = [measured_traffic(k, case, precision) for k in ks]
    return None if None in v else sum(v)


def fp64_inst_per_lu(unit, case):
    """FP64 thread-instructions (DADD + DMUL + DFMA) per lattice update of one
    launch of a step in FP64, from the ncu counts in profiles/fp64_ops.json
    (forward: its two kernels; adjoint: its kernel); None without a capture of
    the current kernel source."""
    try:
        t = json.load(open(FP64_OPS_FILE))
    except (OSError, ValueError):
        return None
    lat = f"D{2 if case.lattice == 9 else 3}Q{case.lattice}"
    ks = FWD_KERNELS if unit == "forward step" else ADJ_KERNELS
    v = {e["kernel"]: e["inst_per_lu"] for e in t.get("entries", [])
         if e.get("lattice") == lat and e.get("source_hash") == kernel_hash()}
    return sum(v[k] for k in ks) if all(k in v for k in ks) else None


def fp64_alu_roofline(roof, kernels, dom, n, clocks):
    """The roofline of an FP64 run: B300 issues FP64 arithmetic at
    FP64_INST_PER_SM_CLK thread-instructions per SM per clock, about 1/64 of
    its FP32 rate, so an FP64 step is bound by that pipe, not by HBM.  achieved
    = the dominant step's FP64 instructions per launch (ncu counts per node x
    nodes) over its event-timed duration; peak = SMs x 2 x the maximum SM
    clock.  The HBM figures stay beside it under "hbm"."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2032.0
    peak = sms * FP64_INST_PER_SM_CLK * mhz / 1e3          # G instructions / s
    case = kernels[dom]["case"]
    ipl = fp64_inst_per_lu(dom, case)
    hbm = {k_: roof[k_] for k_ in ("achieved", "peak", "unit", "frac", "traffic", "peak_kind")}
    out = dict(roof)
    out.update({"bound": "alu", "unit": "G FP64 inst/s", "peak": peak,
                "peak_kind": f"derived: {sms} SMs x {FP64_INST_PER_SM_CLK} FP64 thread-instructions per clock x "
                             f"{mhz:.0f} MHz (maximum SM clock)",
                "inst_per_lu": ipl, "hbm": hbm})
    if ipl is None:
        out.update({"achieved": None, "frac": None})
    else:
        ach = ipl * n / (kernels[dom]["us"] / 1e6) / 1e9
        out.update({"achieved": ach, "frac": ach / peak})
        for k_, v in kernels.items():
            i_ = fp64_inst_per_lu(k_, case)
            if i_ is not None:
                out["kernels"][k_]["fp64_ginst_s"] = i_ * n / (v["us"] / 1e6) / 1e9
                out["kernels"][k_]["fp64_frac"] = out["kernels"][k_]["fp64_ginst_s"] / peak
    return out


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0}, "fallback"


# ------------------------------------------------------------ CPU oracle --

# Largest lattice the oracle times in one process: its adjoint assembles the
# literal Q x Q Jacobian of every node (Q^2 N doubles, plus temporaries).
ORACLE_MAX_JAC_BYTES = 0.1e9


def oracle_case(case):
    """The bounded sample of a workload that the oracle is timed on: the
    workload itself when its per-node Jacobians fit in ORACLE_MAX_JAC_BYTES,
    otherwise (the 3D U-bends) the same duct scaled down by the smallest
    integer factor that fits, with the same tau, Cs, inlet speed and objective."""
    from paper_2608_19617_b300 import inputs as I
    if case.lattice ** 2 * case.n * 8 <= ORACLE_MAX_JAC_BYTES:
        return case, 1
    if case.lattice == 9 and case.nz == 1:
        return crop_2d(case, max(8, int(ORACLE_MAX_JAC_BYTES / (81 * 8 * case.ny)))), 1
    if not case.name.startswith("ubend"):
        raise SystemExit(f"no bounded oracle sample for {case.name}")
    lf = int(case.monitor_l)
    for f in range(2, lf + 1):
        if lf % f or case.nx % f or case.ny % f or case.nz % f:
            continue
        c = I.ubend_case(case.nx // f, case.ny // f, case.nz // f, lf // f, tau=case.tau, cs_smag=case.cs_smag,
                         window_len=case.window_len, ckpt_every=case.ckpt_every, ckpt_format=case.ckpt_format,
                         name=f"{case.name}/{f}")
        if case.lattice ** 2 * c.n * 8 <= ORACLE_MAX_JAC_BYTES:
            return c, f
    raise SystemExit(f"no bounded oracle sample for {case.name}")


def crop_2d(case, nxc):
    """The first nxc columns of a 2D workload, a zero-gradient outlet on the
    new last column (walls kept): the same rows, inlet and design near the
    inlet, a lattice the oracle's Jacobians fit."""
    from paper_2608_19617_b300 import inputs as I
    cls = case.node_class[:, :, :nxc].copy()
    last = cls[:, :, nxc - 1]
    last[(last != I.WALL)] = I.OUTLET_ZG
    x0, x1, y0, y1, z0, z1 = case.design_box
    box = (min(x0, nxc - 1), min(x1, nxc - 1), y0, y1, z0, z1)
    return case.replace(name=f"{case.name}[:{nxc}]", nx=nxc, node_class=cls, gamma=case.gamma[:, :, :nxc].copy(),
                        obj_weights=case.obj_weights[:, :, :nxc].copy(), design_box=box)


def oracle_sample(case, fwd_steps):
    """Time the FP64 oracle, as it stands, on one thread: a window of
    ``fwd_steps`` steps from rest, then its adjoint.  Returns MLUPS over both."""
    from oracle import lbm as O
    c = case.replace(window_len=fwd_steps, ckpt_every=fwd_steps, sample_every=1, sample_from=0)
    pr = O.Problem(c)
    p0 = pr.initial_state()
    t0 = time.perf_counter()
    _, J, M, traj = pr.run_window(p0)
    t1 = time.perf_counter()
    pr.adjoint_window(traj)
    t2 = time.perf_counter()
    lus = 2 * fwd_steps * c.n
    return {"value": lus / (t2 - t0) / 1e6, "fwd_s": t1 - t0, "adj_s": t2 - t1, "seconds": t2 - t0,
            "lattice_updates": lus}


def _oracle_worker(args):
    """One spawned process: build the sample case and time it (args = workload
    name, step count, repeats)."""
    name, fwd_steps, reps = args
    from paper_2608_19617_b300 import inputs as I
    c, _ = oracle_case(I.WORKLOADS[name]())
    return [oracle_sample(c, fwd_steps) for _ in range(reps)]


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_processes(case_sample):
    """Processes for the all-core oracle timing: one per host core, fewer if
    the host's available memory would not hold that many oracle working sets
    (about 40 Q^2 N bytes each, the Jacobian and its temporaries, plus 0.3 GB)."""
    per = 40 * case_sample.lattice ** 2 * case_sample.n + 0.3e9
    avail = None
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                avail = float(ln.split()[1]) * 1024
    except OSError:
        pass
    n = host_cores()
    if avail:
        n = max(1, min(n, int(0.5 * avail // per)))
    return n


class OraclePool:
    """The FP64 oracle on every host core: P spawned single-thread processes,
    each timing its own replica of the sample (the oracle is a serial numpy
    program; replicas are how it uses a many-core host).  Throughput = all
    processes' lattice updates over the wall time of the batch."""

    def __init__(self, workload, procs):
        import multiprocessing as mp
        self.workload = workload
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs)

    def run(self, fwd_steps, reps=1):
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(self.workload, fwd_steps, reps)] * self.procs)
        wall = time.perf_counter() - t0
        lus = sum(r["lattice_updates"] for rr in res for r in rr)
        return {"value": lus / wall / 1e6, "seconds": wall, "lattice_updates": lus,
                "per_process_mlups": statistics.median(r["value"] for rr in res for r in rr)}

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def sample_text(case, c_s, f, fwd_steps, procs):
    scaled = (f"the {case.name} duct scaled by 1/{f} ({c_s.nx}x{c_s.ny}x{c_s.nz}, same tau, Cs and inlet speed)"
              if f > 1 else f"the first {c_s.nx} columns of {case.name} (zero-gradient outlet on the cut)"
              if c_s.nx < case.nx else f"the full {case.name} lattice")
    return (f"FP64 numpy oracle: a {fwd_steps}-step window from rest of {scaled} plus its adjoint, "
            f"{2 * fwd_steps * c_s.n} lattice updates per process, {procs} single-thread process(es) in parallel")


def cpu_baseline_legs(case, fwd_steps=2):
    """The oracle timed on one thread and on every host core (both bounded:
    a few seconds each), for the GPU arm's cpu_baseline."""
    c_s, f = oracle_case(case)
    one = oracle_sample(c_s, fwd_steps)
    procs = oracle_processes(c_s)
    pool = OraclePool(case.name, procs)
    try:
        pool.run(1)                       # workers import numpy / scipy and build their problem once
        allc = pool.run(fwd_steps)
    finally:
        pool.close()
    return {"value": allc["value"], "unit": "MLUPS", "cores": procs, "kind": "oracle",
            "sample": sample_text(case, c_s, f, fwd_steps, procs), "cpu": cpu_model(),
            "host_cores": host_cores(), "seconds": allc["seconds"],
            "single_thread": {"value": one["value"], "unit": "MLUPS", "cores": 1, "seconds": one["seconds"]}}


def run_reference(args, case, rank, world):
    """The reference arm: the FP64 oracle as it stands on this host's cores
    (rank 0 only).  Each step is one bounded sample per process: a 2-step
    window of the sample lattice plus its adjoint."""
    if rank != 0:
        return 0
    fwd_steps = 2
    c_s, f = oracle_case(case)
    procs = oracle_processes(c_s)
    pool = OraclePool(case.name, procs)
    try:
        pool.run(1)
        for _ in range(args.warmup):
            pool.run(fwd_steps)
        secs, lus = 0.0, 0
        for _ in range(args.steps):
            r = pool.run(fwd_steps)
            secs += r["seconds"]
            lus += r["lattice_updates"]
    finally:
        pool.close()
    value = lus / secs / 1e6
    sample = sample_text(case, c_s, f, fwd_steps, procs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": f"synthetic (seeded inputs shaped like the paper's {'U-bend' if case.lattice == 19 else '2D'} case)",
        "config": {"workload": case.name, "nx": case.nx, "ny": case.ny, "nz": case.nz,
                   "window_len": case.window_len, "ckpt_every": case.ckpt_every,
                   "oracle_sample": f"{c_s.nx}x{c_s.ny}x{c_s.nz}"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": procs, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model(), "host_cores": host_cores()},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- GPU path --

def run_ours(args, case, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2608_19617_b300 import binding as B
    from paper_2608_19617_b300 import build as bld

    torch.cuda.set_device(local)
    if rank == 0:
        bld.build()
    if world > 1:
        dist.barrier()
    bld.build()
    B.lib()

    stream = torch.cuda.Stream()
    prec = B.LBM_FP64 if args.precision == "fp64" else B.LBM_FP32
    with torch.cuda.stream(stream):
        sol = B.Solver(case, prec, stream=stream, pipeline=int(args.pipeline))
    sol.set_graphs(bool(args.graphs))
    sol.set_pdl(bool(args.pdl))
    n = case.n
    W, K = case.window_len, case.ckpt_every
    grad_dev = torch.empty(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > L2 (126 MB)

    sweep_ev = []     # CUDA events around each timed adjoint sweep (library stream)

    def one_step(timed=False):
        sol.step_window()
        sol.window_converged()
        if timed:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        sol.adjoint_window()
        if timed:
            b.record(stream)
            sweep_ev.append((a, b))
        sol.design_gradient(grad_dev)

    # Spin-up: Alg. 1 from rest, consecutive windows until the test of Eq. 26
    # holds (or the cap), so that the timed windows see the developed flow.
    t0 = time.perf_counter()
    rec = sol.run_until_converged(max_windows=max(1, args.spinup_windows)) if args.spinup_windows > 0 else []
    protocol = {"windows": len(rec), "steps": len(rec) * W, "converged": bool(rec and rec[-1]["converged"]),
                "ratios": [r["ratio"] for r in rec[1:]],
                "last_ratio": rec[-1]["ratio"] if rec else None, "J_eff": rec[-1]["J"] if rec else None,
                "conv_tol": case.conv_tol, "seconds": time.perf_counter() - t0}
    # Phase timing is on from the first warm-up step: the graphs that carry its
    # event nodes are captured and instantiated there, outside the timed region.
    sol.set_timing(True)
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    def timed_pass():
        """The timed region: K steps, the L2 flushed before each, CUDA events
        on the library stream, nvidia-smi clocks sampled throughout."""
        sol.get_timing()          # reset the phase counters
        sweep_ev.clear()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            for k in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.fill_(k & 0xff)
                    ev[k][0].record(stream)
                    one_step(timed=True)
                    ev[k][1].record(stream)
            torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev), clk.summary()

    ms, clocks = timed_pass()
    # A pass that saw a hardware or thermal slowdown, or SM clocks far below
    # their maximum with no reason given (a leftover clock lock), is measured
    # once more; every rank takes part if any rank saw one.
    if reduce_max(float(clocks_rejected(clocks)), world) > 0:
        first = clocks
        if world > 1:
            dist.barrier()
        ms, clocks = timed_pass()
        clocks["remeasured_after"] = first
    timing = sol.get_timing()
    sched = sol.schedule()
    ms = reduce_max(ms, world)
    if world > 1:
        dist.barrier()
    lus_step = 2 * W * n
    value = whole_job_mlups(lus_step, args.steps, world, ms)

    # e2e: host design in, host gradient out, through the C ABI, per step.
    e2e_value = None
    if not args.quick:
        gam_host = torch.from_numpy(case.gamma.reshape(-1).astype(np.float32)).pin_memory()
        grad_host = torch.empty(n, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sol.set_design(gam_host)
            sol.step_window()
            sol.window_converged()
            sol.adjoint_window()
            sol.design_gradient(grad_host)
        torch.cuda.synchronize()
        e2e_s = reduce_max(time.perf_counter() - t0, world)
        e2e_value = whole_job_mlups(lus_step, args.steps, world, 1e3 * e2e_s)

    if rank != 0:
        return 0

    pk, pk_kind = peaks()
    hbm = float(pk["hbm_gbs"])
    rs = 8 if prec == B.LBM_FP64 else 4
    phase_rows = {}
    for ph in ("forward", "recompute", "adjoint"):
        t = timing[ph]
        if t["launches"]:
            avg_ms = t["ms"] / t["launches"]
            bpl = bytes_per_lu(case, ph, rs=rs) * n
            phase_rows[ph] = {"steps": t["launches"], "ms": t["ms"], "avg_step_us": 1e3 * avg_ms,
                              "bytes_per_step": bpl, "gbs": bpl / (avg_ms / 1e3) / 1e9}
    # Units of the roofline: a forward step, and an adjoint-sweep
    # step = one adjoint step plus its share (K-1)/K of a recompute step.  The
    # sweep is timed whole (events around lbm_adjoint_window), since recompute
    # and adjoint steps may run concurrently.
    sweep_ms = sum(a.elapsed_time(b) for a, b in sweep_ev) / len(sweep_ev)
    sweep_b = (bytes_per_lu(case, "adjoint", rs=rs) + bytes_per_lu(case, "recompute", rs=rs) * (K - 1) / K) * n
    fk = "fwd_row_kernel+fwd_facerow_kernel"
    ak = "adj_step_kernel"
    # Kernels of a bench step: the forward-step pair (inner rows + face rows)
    # runs W times in the window and S (K - 1) times in the recompute, the
    # adjoint-step kernel W times.  Forward steps are timed in the window phase
    # (nothing runs beside them); a serial sweep (--pipeline 0) times the
    # recompute and adjoint phases apart, a pipelined one overlaps them, and
    # then the adjoint step's time is the sweep step less its recompute share.
    S = W // K
    fwd_us = phase_rows["forward"]["avg_step_us"]
    sweep_us = 1e3 * sweep_ms / W
    serial = not args.pipeline
    adj_us = phase_rows["adjoint"]["avg_step_us"] if serial else sweep_us - fwd_us * (K - 1) / K
    kernels = {
        "forward step": {"kernel": fk, "us": fwd_us, "launches": W + S * (K - 1),
                         "bytes": bytes_per_lu(case, "forward", rs=rs) * n,
                         "scope_bytes_per_lu": scope_bytes_per_lu(case, "forward step", rs=rs)},
        "adjoint step": {"kernel": ak, "us": adj_us, "launches": W, "bytes": bytes_per_lu(case, "adjoint", rs=rs) * n,
                         "scope_bytes_per_lu": (12 * case.lattice + 4 + 32) * rs // 4,
                         "timing": "adjoint phase events (serial sweep)" if serial
                                   else "sweep step less its recompute share (pipelined sweep)"},
    }
    for v in kernels.values():
        v["ms_per_bench_step"] = v["us"] * v["launches"] / 1e3
    dom = max(kernels, key=lambda k_: kernels[k_]["ms_per_bench_step"])
    u = kernels[dom]
    sv = u["scope_bytes_per_lu"] * n      # the scope table's count for one launch
    ach = sv / (u["us"] / 1e6) / 1e9
    ach_design = u["bytes"] / (u["us"] / 1e6) / 1e9
    sweep_sv = scope_bytes_per_lu(case, "adjoint sweep step", rs=rs) * n
    roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": unit_traffic(dom, case, "fp64" if rs == 8 else "fp32"),
            "dominant": dom, "kernel": u["kernel"], "bytes_per_launch": sv, "bytes_per_lu": u["scope_bytes_per_lu"],
            "us_per_launch": u["us"], "launches_per_bench_step": u["launches"],
            "design_count": {"bytes_per_launch": u["bytes"], "bytes_per_lu": u["bytes"] / n,
                             "achieved": ach_design, "frac": ach_design / hbm},
            "peak_kind": f"{pk_kind} hbm_gbs (copy)",
            "timing": "CUDA events on the library stream inside the timed region: per forward-window phase, and "
                      "around each whole adjoint sweep",
            "kernels": {k_: {"us": v["us"], "launches": v["launches"], "ms_per_bench_step": v["ms_per_bench_step"],
                             "gbs": v["scope_bytes_per_lu"] * n / (v["us"] / 1e6) / 1e9,
                             "gbs_design_count": v["bytes"] / (v["us"] / 1e6) / 1e9} for k_, v in kernels.items()},
            "adjoint_sweep_step": {"us": sweep_us, "scope_bytes_per_lu": scope_bytes_per_lu(case, "adjoint sweep step", rs=rs),
                                   "gbs": sweep_sv / (sweep_us / 1e6) / 1e9, "frac": sweep_sv / (sweep_us / 1e6) / 1e9 / hbm,
                                   "design_bytes_per_lu": sweep_b / n, "gbs_design_count": sweep_b / (sweep_us / 1e6) / 1e9,
                                   "frac_design_count": sweep_b / (sweep_us / 1e6) / 1e9 / hbm},
            "phases": phase_rows}
    if rs == 8:
        for v in kernels.values():
            v["case"] = case
        roof = fp64_alu_roofline(roof, kernels, dom, n, clocks)

    # Accuracy beside the number: the FP32 (or mixed-precision) window and
    # adjoint against the FP64 GPU path on the same trajectory.  The FP64
    # window runs along the FP32 one (lbm_step_window_along): every
    # checkpoint segment starts from the FP32 run's checkpoint, so the two
    # adjoints differentiate the same primal trajectory; the flow is chaotic,
    # and independent FP32 and FP64 runs over a long window drift apart.
    # That independent run is reported too.  The window is shortened when the
    # FP64 workspace would exceed ~150 GB (said in the output).
    def _cmp(g, J, g64, J64):
        n, n64 = float(np.linalg.norm(g)), float(np.linalg.norm(g64))
        return {"J_rel_err": abs(J - J64) / abs(J64),
                "grad_cosine": float(g @ g64 / (n * n64)) if n > 0 and n64 > 0 else None,
                "grad_rel_err": float(np.linalg.norm(g - g64) / n64) if n64 > 0 else None}

    err = None
    if not args.no_fp64_check and prec == B.LBM_FP32:
        W_err, K_err = fp64_check_window(case)
        c32 = case.replace(window_len=W_err, ckpt_every=K_err)
        c64 = case.replace(window_len=W_err, ckpt_every=K_err, ckpt_format=0)
        p = sol.get_state()
        if W_err != W or K_err != case.ckpt_every:   # free the timed solver's workspace first
            sol.close()
            sol.workspace = None
            torch.cuda.empty_cache()
        with torch.cuda.stream(stream):
            s32 = B.Solver(c32, B.LBM_FP32, stream=stream) if sol.ctx is None else sol
            ref = B.Solver(c64, B.LBM_FP64, stream=stream)
        s32.set_state(p)
        J32, _ = s32.step_window()
        s32.adjoint_window()
        g32 = s32.design_gradient()
        J64, _ = ref.step_window_along(s32)
        ref.adjoint_window()
        g64 = ref.design_gradient()
        same = _cmp(g32, J32, g64, J64)
        ref.set_state(p)            # an independent FP64 run from the same start field
        J64i, _ = ref.step_window()
        ref.adjoint_window()
        indep = _cmp(g32, J32, ref.design_gradient(), J64i)
        err = {"J_rel_err_fp32_vs_fp64": same["J_rel_err"], "grad_cosine_fp32_vs_fp64": same["grad_cosine"],
               "grad_rel_err_fp32_vs_fp64": same["grad_rel_err"], "grad_norm_fp64": float(np.linalg.norm(g64)),
               "reference": "FP64 along the FP32 trajectory (each segment restarts from the FP32 checkpoint)",
               "independent_fp64_run": indep,
               "window_len": W_err, "ckpt_every": K_err, "fp32_ckpt": CKPT_NAMES[c32.ckpt_format]}
        ref.close()
        if s32 is not sol:
            s32.close()

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_legs(case)

    # kernels the library enqueued for the last window and sweep, plus the gradient kernel
    launches_per_step = sched["kernels_window"] + sched["kernels_adjoint"] + 1
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == B.LBM_FP64 else "f32",
        "data": ("synthetic (seeded inputs shaped like the paper's U-bend, extruded to 3D)" if case.lattice == 19
                 else "synthetic (seeded inputs shaped like the paper's 2D cases)"),
        "config": {"workload": case.name, "lattice": f"D{2 if case.lattice == 9 else 3}Q{case.lattice}",
                   "nx": case.nx, "ny": case.ny, "nz": case.nz,
                   "window_len": W, "sample_every": case.sample_every, "ckpt_every": K,
                   "ckpt_format": CKPT_NAMES[case.ckpt_format], "tau": case.tau,
                   "cs_smag": case.cs_smag, "parallelism": f"replicas x{world}",
                   "cuda_graphs": bool(args.graphs), "pipeline": bool(args.pipeline),
                   "pdl": bool(args.pdl),
                   "l2": (f"flushed (256 MB write) before every timed step; each population field is "
                          f"{case.lattice * n * rs / 1e6:.0f} MB against a 126 MB L2")},
        "fwd_mlups": 1e-6 * timing["forward"]["lattice_updates"] / (timing["forward"]["ms"] / 1e3),
        "adj_mlups_incl_recompute": 1e-6 * W * n / (sweep_ms / 1e3),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": (None if e2e_value is None else
                {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 8 * n}),
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "error": err,
        "protocol": protocol,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_full_time(args, case):
    """The comparison of Sec. 4.2.3 (its table of time per iteration and
    storage), for one design gradient from the initial field:

    * window framework: windows of |W| steps until the consecutive-window test
      of Eq. 26 holds (at most case.max_windows), then the adjoint of the last
      window only (checkpoints of that window, K = case.ckpt_every);
    * full-time adjoint: the same n |W| steps as one window whose samples are
      the last |W| steps (lbm_set_sample_start), every state kept
      (K = --full-time-k, 1 = the complete history), the adjoint traced back to
      the initial time.

    Both start from the same field, so the objectives agree bit for bit; the
    gradients differ by the sensitivity carried through the transient.  Times
    are host wall clock around the synchronised calls (the window arm after one
    warm-up iteration that captures its graphs; the full-time arm launches
    directly, since its window would make a graph of some 10^5 nodes).
    Storage is the device workspace each context takes."""
    import numpy as np
    import torch
    from paper_2608_19617_b300 import binding as B
    B.lib()
    prec = B.LBM_FP64 if args.precision == "fp64" else B.LBM_FP32
    W = case.window_len
    win = B.Solver(case, prec, pipeline=args.pipeline)
    win.set_graphs(bool(args.graphs))
    p_init = win.get_state()

    def window_iteration():
        win.set_state(p_init)
        n, conv, ratio, J = 0, False, float("inf"), None
        while n < case.max_windows:
            J, _ = win.step_window()
            n += 1
            conv, ratio = win.window_converged()
            if conv:
                break
        win.adjoint_window()
        return n, conv, ratio, J, win.design_gradient()

    window_iteration()                       # warm-up: graph capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n, conv, ratio, J_win, g_win = window_iteration()
    torch.cuda.synchronize()
    t_win = time.perf_counter() - t0
    ws_win = int(win.workspace.numel())
    win.close()

    T = n * W
    K = args.full_time_k
    if T % K:
        raise SystemExit(f"--full-time-k {K} must divide the run length {T}")
    ft = case.replace(window_len=T, ckpt_every=K, sample_from=T - W)
    ws_full = B.workspace_size(B.config_from_case(ft, prec, pipeline=args.pipeline))
    out = {"metric": "time per design gradient and storage: consecutive-window framework vs full-time adjoint "
                     "(Sec. 4.2.3)",
           "impl": "ours", "dtype": "f64" if prec == B.LBM_FP64 else "f32", "data": "synthetic",
           "config": {"workload": case.name, "window_len": W, "sample_every": case.sample_every,
                      "ckpt_every_window": case.ckpt_every, "ckpt_every_full_time": K,
                      "pipeline": bool(args.pipeline), "graphs_window": bool(args.graphs)},
           "window": {"windows": n, "converged": bool(conv), "ratio": ratio, "steps_forward": T,
                      "steps_adjoint": W, "seconds": t_win, "workspace_bytes": ws_win, "J": J_win},
           "paper": {"minutes_per_iteration": {"full_time": 1.63, "window": 0.663},
                     "storage": {"full_time": "558 GB", "window": "217 MB"}}}
    if ws_full > args.full_time_cap_gb * 1e9:
        out["full_time"] = {"skipped": f"workspace {ws_full / 1e9:.1f} GB above --full-time-cap-gb"}
        print(json.dumps(out))
        return 0
    full = B.Solver(ft, prec, pipeline=args.pipeline)
    full.set_graphs(False)
    full.set_state(p_init)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J_full, _ = full.step_window()
    full.adjoint_window()
    g_full = full.design_gradient()
    torch.cuda.synchronize()
    t_full = time.perf_counter() - t0
    full.close()
    m = np.abs(g_win) + np.abs(g_full) > 0
    cos = float(g_win[m] @ g_full[m] / (np.linalg.norm(g_win[m]) * np.linalg.norm(g_full[m])))
    out["full_time"] = {"steps_forward": T, "steps_adjoint": T, "seconds": t_full, "workspace_bytes": ws_full,
                        "J": J_full}
    out.update({"time_ratio": t_full / t_win, "storage_ratio": ws_full / ws_win,
                "J_bitwise_equal": J_full == J_win, "grad_cosine": cos,
                "grad_rel_diff": float(np.linalg.norm(g_full - g_win) / np.linalg.norm(g_full))})
    print(json.dumps(out))
    return 0


def run_optimize(args, case):
    """Iterations of the optimization loop on the cylinder drag case with the
    paper's settings (Sec. 3.3 and the cylinder case of Sec. 4): filter radius
    4, projection eta = 0.5 with beta 2 doubling every 10 iterations up to 16,
    MMA under a volume band.  The paper bounds V to [0.014, 0.016] of its
    design domain; here the design domain is the 32x32 square around the
    cylinder, so the band is scaled to the same amount of solid on the
    200x100 lattice: [0.014, 0.016] x 20000 / 1024."""
    import torch
    from paper_2608_19617_b300 import optimize as OPT
    n_d = (case.design_box[1] - case.design_box[0]) * (case.design_box[3] - case.design_box[2])
    scale = case.nx * case.ny / n_d
    vmin, vmax = 0.014 * scale, 0.016 * scale
    t = []
    last = [time.perf_counter()]

    def log(row):
        torch.cuda.synchronize()
        now = time.perf_counter()
        t.append(now - last[0])
        last[0] = now

    hist, _ = OPT.optimize(case, n_max=args.optimize, eps_o=0.0, vmin=vmin, vmax=vmax, log=log)
    out = {"metric": "seconds per optimization iteration (Alg. 2 on the cylinder drag case)", "impl": "ours",
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": case.name, "window_len": case.window_len, "sample_every": case.sample_every,
                      "max_windows": case.max_windows, "vmin": vmin, "vmax": vmax, "filter_radius": 4.0},
           "iterations": len(hist),
           "seconds_per_iteration": statistics.median(t[1:]) if len(t) > 1 else t[0],
           "first_iteration_seconds": t[0],
           "history": [{k: h[k] for k in ("iteration", "beta", "J", "volume", "windows", "converged")} for h in hist],
           "paper": {"minutes_per_iteration": 0.663}}
    print(json.dumps(out))
    return 0


def run_ckpt_sweep(args, case):
    """Mixed-precision checkpoints against the plain FP64 GPU adjoint.

    After a spin-up of the workload (FP32, its own window length), one window
    of W_c steps with K_c-step segments (fp64_check_window: the longest window
    whose FP64 context fits in ~150 GB next to the FP32 one) is run from the
    same start field with FP32 populations and each checkpoint format (FP32
    native, FP16, BF16, lossless moment planes).  The forward pass does not
    depend on the format, so every run follows the same primal trajectory; the
    FP64 reference runs its window along the FP32-native run's checkpoints
    (lbm_step_window_along) and its adjoint over that trajectory.  Reported
    per format: gradient cosine and relative error against FP64, J relative
    error, adjoint-sweep time (CUDA events on the library stream, the second
    of two sweeps) and the context's workspace bytes."""
    import numpy as np
    import torch
    from paper_2608_19617_b300 import binding as B
    B.lib()
    stream = torch.cuda.Stream()
    W_c, K_c = fp64_check_window(case)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        spin = B.Solver(case, B.LBM_FP32, stream=stream)
    rec = spin.run_until_converged(max_windows=max(1, args.spinup_windows))
    p0 = spin.get_state()
    spin.close()
    del spin
    torch.cuda.empty_cache()

    def timed_sweep(sol):
        ms = []
        for _ in range(2):
            sol.set_state(p0)
            J, _ = sol.step_window()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sol.adjoint_window()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return J, sol.design_gradient(), ms[-1]

    def cmp(g, J, g64, J64):
        m = np.abs(g64) > 0
        n1, n2 = float(np.linalg.norm(g[m])), float(np.linalg.norm(g64[m]))
        return {"grad_cosine": float(g[m] @ g64[m] / (n1 * n2)), "grad_rel_err": float(np.linalg.norm(g - g64) / n2),
                "J_rel_err": abs(J - J64) / abs(J64)}

    rows = {}
    base = case.replace(window_len=W_c, ckpt_every=K_c)
    with torch.cuda.stream(stream):
        nat = B.Solver(base.replace(ckpt_format=0), B.LBM_FP32, stream=stream, pipeline=0)
    J32, g32, ms32 = timed_sweep(nat)
    with torch.cuda.stream(stream):
        ref = B.Solver(base.replace(ckpt_format=0), B.LBM_FP64, stream=stream, pipeline=0)
    ref.set_state(p0)
    t1 = time.perf_counter()
    J64, _ = ref.step_window_along(nat)
    torch.cuda.synchronize()
    t_fwd64 = time.perf_counter() - t1
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    ref.adjoint_window()
    b.record(stream)
    torch.cuda.synchronize()
    ms64 = a.elapsed_time(b)
    g64 = ref.design_gradient()
    fp64 = {"workspace_bytes": int(ref.workspace.numel()), "adjoint_sweep_ms": ms64,
            "adjoint_mlups_incl_recompute": W_c * case.n / (ms64 / 1e3) / 1e6,
            "forward_window_s_host": t_fwd64, "grad_norm": float(np.linalg.norm(g64))}
    ref.close()
    rows["fp32"] = dict(cmp(g32, J32, g64, J64), workspace_bytes=int(nat.workspace.numel()), adjoint_sweep_ms=ms32,
                        adjoint_mlups_incl_recompute=W_c * case.n / (ms32 / 1e3) / 1e6)
    nat.close()
    del nat, ref
    torch.cuda.empty_cache()
    for name, fmt in (("fp16", 1), ("bf16", 2), ("moment", 3)):
        with torch.cuda.stream(stream):
            sol = B.Solver(base.replace(ckpt_format=fmt), B.LBM_FP32, stream=stream, pipeline=0)
        J, g, ms = timed_sweep(sol)
        rows[name] = dict(cmp(g, J, g64, J64), workspace_bytes=int(sol.workspace.numel()), adjoint_sweep_ms=ms,
                          adjoint_mlups_incl_recompute=W_c * case.n / (ms / 1e3) / 1e6, J_equals_fp32=J == J32)
        sol.close()
        del sol
        torch.cuda.empty_cache()
    out = {"metric": "checkpoint-storage sweep: FP32 adjoint with FP32/FP16/BF16/moment checkpoints against the FP64 "
                     "GPU adjoint on the same trajectory",
           "impl": "ours", "data": "synthetic",
           "config": {"workload": case.name, "window_len": W_c, "ckpt_every": K_c,
                      "workload_window_len": case.window_len, "spinup_windows": len(rec),
                      "spinup_converged": bool(rec[-1]["converged"]), "pipeline": False},
           "J_fp64": J64, "fp64": fp64, "formats": rows, "seconds": time.perf_counter() - t0}
    print(json.dumps(out))
    return 0


def run_fd_protocol(args, case):
    """Sec. 4.2.1: single-point perturbations of the design against the
    adjoint sensitivity, with the same representative window and sampling
    instants (|W| = 5000, Delta W = 50), in FP64.  The start field is the
    flow once the consecutive-window test holds.  The 60 points are spread
    over the downstream half of the cylinder, where phi = 0.5 (gamma = 0.5)
    takes central differences of +-1e-3 and +-1e-4; the perturbed designs run
    as D2Q9 batches of independent slices, forward only."""
    import numpy as np
    import torch
    from paper_2608_19617_b300 import binding as B
    from paper_2608_19617_b300 import inputs as I
    B.lib()
    t0 = time.perf_counter()
    base = case.replace(ckpt_every=100)
    sol = B.Solver(base, B.LBM_FP64)
    rec = sol.run_until_converged()
    p0 = sol.get_state()
    sol.set_state(p0)
    J0, _ = sol.step_window()
    sol.adjoint_window()
    grad = sol.design_gradient().reshape(base.ny, base.nx)
    sol.close()
    gam = base.gamma[0].astype(np.float32)
    cand = [(y, x) for y in range(base.ny) for x in range(101, base.nx)
            if (x - 100) ** 2 + (y - 50) ** 2 <= 49 and gam[y, x] == np.float32(0.5)]
    pick = [cand[int(k)] for k in np.linspace(0, len(cand) - 1, 60).round().astype(int)]
    steps = (1e-3, 1e-4)
    jobs = []                                  # (point, h, sign, design)
    for (y, x) in pick:
        for h in steps:
            for sgn in (1, -1):
                g2 = gam.copy()
                g2[y, x] += np.float32(sgn * h)
                jobs.append(((y, x), h, sgn, float(g2[y, x]), g2))
    fwd_case = base.replace(ckpt_every=50)
    J = {}
    per = 40
    for b0 in range(0, len(jobs), per):
        chunk = jobs[b0:b0 + per]
        batch = I.stack_cases([fwd_case.replace(gamma=j[4][None].astype(np.float64)) for j in chunk])
        bs = B.Solver(batch, B.LBM_FP64)
        bs.set_state(np.concatenate([p0] * len(chunk), axis=1))
        bs.step_window()
        Js, _ = bs.window_objectives()
        bs.close()
        for j, v in zip(chunk, Js):
            J[(j[0], j[1], j[2])] = (v, j[3])
    torch.cuda.synchronize()
    rows, err = [], {h: [] for h in steps}
    for (y, x) in pick:
        row = {"x": x, "y": y, "adjoint": float(grad[y, x])}
        for h in steps:
            (jp, vp), (jm, vm) = J[((y, x), h, 1)], J[((y, x), h, -1)]
            fd = (jp - jm) / (vp - vm)
            row[f"fd_{h:g}"] = fd
            e = abs(fd - grad[y, x]) / abs(grad[y, x])
            row[f"rel_err_{h:g}"] = e
            err[h].append(e)
        rows.append(row)
    out = {"metric": "finite differences vs adjoint sensitivity (Sec. 4.2.1 protocol, cylinder, FP64)",
           "impl": "ours", "dtype": "f64", "data": "synthetic",
           "config": {"workload": case.name, "window_len": base.window_len, "sample_every": base.sample_every,
                      "spinup_windows": len(rec), "converged": bool(rec[-1]["converged"]), "points": len(pick),
                      "perturbations": list(steps), "fd_slices": len(jobs)},
           "J": J0,
           "rel_err": {f"{h:g}": {"median": float(np.median(err[h])), "max": float(np.max(err[h])),
                                  "below_1pct": int(np.sum(np.array(err[h]) < 0.01))} for h in steps},
           "seconds": time.perf_counter() - t0, "points": rows}
    print(json.dumps(out))
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    from paper_2608_19617_b300 import inputs as I
    if (args.full_time or args.optimize or args.fd_protocol) and args.workload == WORKLOAD:
        args.workload = "cylinder200x100"
    case = I.WORKLOADS[args.workload]()
    if args.window_len or args.ckpt_every:
        wl = args.window_len or case.window_len
        case = case.replace(window_len=wl, ckpt_every=args.ckpt_every or wl)
    if args.ckpt_format:
        case = case.replace(ckpt_format=CKPT_NAMES.index(args.ckpt_format))
    if args.precision == "fp64" and case.ckpt_format in (1, 2):
        case = case.replace(ckpt_format=0)    # 16-bit checkpoints exist for the FP32 solver only
    if args.impl == "reference":
        rc = run_reference(args, case, rank, world)
        return rc
    if args.full_time:
        return run_full_time(args, case) if rank == 0 else 0
    if args.optimize:
        return run_optimize(args, case) if rank == 0 else 0
    if args.fd_protocol:
        return run_fd_protocol(args, case) if rank == 0 else 0
    if args.ckpt_sweep:
        return run_ckpt_sweep(args, case) if rank == 0 else 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        return run_ours(args, case, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
