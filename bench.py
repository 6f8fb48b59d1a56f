"""Throughput benchmark of the lattice update (MLUPS) on the pool-boiling workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]
                    [--kernel auto|two_pass|fused] [--precision fp32|bf16|fp16]
                    [--workload pool_boiling|evaporation|static_droplet|nucleate_boiling|batch]

A "step" is one lattice time step of the whole update (psi/EOS, interaction and buoyancy
forces, D3Q19 MRT collision, local div u and grad T, phase-change source, D3Q7 MRT collision,
streaming with the wall / outflow boundaries) over the 200 x 200 x 300 pool-boiling lattice
(12.0M nodes).  Prints one JSON line (rank 0).

N > 1 (torchrun): every rank runs an independent replica of the lattice (the update has no
data-path exchange in this build); a barrier brackets the timed region and the time is the
max over ranks; value = node updates of all ranks / that time ("scaling": "weak").

--workload batch runs the 256-instance ensemble (periodic droplets and slabs, edges 24..96)
as one batched persistent launch per step (plan autotuned), beside the same instances advanced
one after another through single-lattice contexts (the sequential FP32 loop).

--impl reference times the FP64 CPU oracle (the plain restatement of the paper's equations)
on the host cores, on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

BYTES_PER_NODE = {"fp32": 216, "bf16": 112, "fp16": 112}   # algorithmic bytes of one node update
PREC_CODE = {"fp32": 0, "bf16": 1, "fp16": 2}
KERNEL_CODE = {"auto": 0, "two_pass": 1, "fused": 2, "fused_generic": 2}


def workload(name, nx=None, ny=None, nz=None):
    if name == "pool_boiling" and (nx or ny or nz):
        nx, ny, nz = nx or 200, ny or 200, nz or 300
        scale = nz / 300.0
        return W.pool_boiling(nx, ny, nz, height=100.0 * scale, hot_sigma=10.0 * min(nx, ny) / 200.0)
    if name == "pool_boiling":
        return W.pool_boiling()
    if name == "evaporation":
        return W.evaporation()
    if name == "static_droplet":
        return W.static_droplet()
    if name == "nucleate_boiling":
        return W.nucleate_boiling()
    raise ValueError(name)


def job_time_ms(ms_local, world, device="cuda"):
    """The job's time: the maximum of the ranks' times (every rank gets it)."""
    if world <= 1:
        return float(ms_local)
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank, steps, world, ms):
    """Node updates of all ranks divided by the job's time (replicas: weak scaling)."""
    return nodes_per_rank * steps * world / (ms * 1e-3) / 1e6


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = ("lbm_fused.cu", "lbm_device.cuh", "lbm_launch.h")   # sources of the timed kernels


def kernel_source_sha():
    """Hash of the sources the timed kernels are built from (stale ncu counters are not reported)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2201_06039_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel_name, precision, nodes):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d[f"{kernel_name}/{precision}"]
        if e.get("source_sha") != kernel_source_sha():
            return None
        return float(e["dram_bytes_per_node"]) * nodes
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def init_fields(case):
    from paper_2201_06039_gb300 import thermo
    s = case["setup"]
    Tc = thermo.critical_temperature(s.a, s.b, s.R)
    Tr = case.get("Tr_drop", case.get("Tr_liquid", 0.86))
    rl, rv, _ = thermo.coexistence(Tr * Tc, s.a, s.b, s.R, s.acentric)
    rho, T, u = W.build_fields(case, Tc, rl, rv)
    return rho.astype(np.float32), T.astype(np.float32)


def cpu_baseline_run(case, budget_s=20.0, steps=None, warm=1, one_thread=True):
    """Time the FP64 oracle on a bounded sample: a z-slab of the same workload sized so that one
    step takes about budget_s / steps seconds (all host cores through OpenMP), then (one_thread)
    the same slab on one thread."""
    import oracle
    s = case["setup"]
    probe_nodes = 200 * 200 * 10
    nz_probe = max(2, probe_nodes // (s.nx * s.ny))
    sub = dict(case)
    sub_setup = W.LatticeSetup(**{**s.__dict__, "nz": nz_probe})
    sub["setup"] = sub_setup
    if "height" in sub:
        sub["height"] = min(case["height"], nz_probe / 2)
    Tc = oracle.Tc_of(sub_setup)
    rl, rv, _ = oracle.maxwell(sub_setup, 0.86 * Tc)
    rho, T, _ = W.build_fields(sub, Tc, rl, rv)
    o = oracle.Oracle(sub_setup)
    o.init(rho, T)
    o.step(warm)
    t0 = time.perf_counter()
    o.step(1)
    per_step = time.perf_counter() - t0
    mlups = sub_setup.n_nodes / per_step / 1e6
    n = steps if steps is not None else max(1, int(budget_s / max(per_step, 1e-3)))
    n = min(n, 50)
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    mlups = sub_setup.n_nodes * n / dt / 1e6
    cores = oracle.num_threads()
    if not one_thread:
        o.close()
        return dict(value=mlups, unit="MLUPS", cores=cores, kind="oracle", sample="sizing probe", seconds=dt)
    # the same slab on one thread (a few steps, bounded to about budget_s / 2 seconds)
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        o.step(1)
        one = time.perf_counter() - t0
        n1 = max(1, min(10, int(0.5 * budget_s / max(one, 1e-3))))
        t0 = time.perf_counter()
        o.step(n1)
        mlups_1 = sub_setup.n_nodes * n1 / (time.perf_counter() - t0) / 1e6
    finally:
        oracle.set_num_threads(cores)
    o.close()
    return dict(value=mlups, unit="MLUPS", cores=cores, kind="oracle",
                sample=f"{n} steps of a {s.nx}x{s.ny}x{nz_probe} z-slab of the same workload (same "
                       f"boundaries and parameters), FP64, after {warm + 1} warm-up steps",
                value_1_thread=mlups_1, steps_1_thread=n1, cpu_model=cpu_model(), seconds=dt)


def cpu_model():
    """The host CPU as lscpu names it (model name, or vendor and part on Arm), and its core count."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        f = {}
        for line in out.splitlines():
            if ":" in line:
                k, v = line.split(":", 1)
                f.setdefault(k.strip(), v.strip())
        name = f.get("Model name") or f.get("Vendor ID") or "unknown"
        return f"{name}, {os.cpu_count()} logical CPUs"
    except Exception:
        return f"unknown, {os.cpu_count()} logical CPUs"


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    case = workload(args.workload, args.nx, args.ny, args.nz)
    import oracle
    s = case["setup"]
    total_budget = 150.0
    per_step_budget = total_budget / max(1, args.steps + args.warmup)
    # size a z-slab of the workload so that one oracle step fits the per-step budget
    probe = cpu_baseline_run(case, steps=1, warm=0, one_thread=False)
    nodes = max(s.nx * s.ny * 2, int(probe["value"] * 1e6 * per_step_budget))
    nz = max(2, min(s.nz, nodes // (s.nx * s.ny)))
    sub = dict(case)
    sub_setup = W.LatticeSetup(**{**s.__dict__, "nz": nz})
    sub["setup"] = sub_setup
    if "height" in sub:
        sub["height"] = min(case["height"], nz / 2)
    Tc = oracle.Tc_of(sub_setup)
    rl, rv, _ = oracle.maxwell(sub_setup, 0.86 * Tc)
    rho, T, _ = W.build_fields(sub, Tc, rl, rv)
    o = oracle.Oracle(sub_setup)
    o.init(rho, T)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = sub_setup.n_nodes * args.steps / dt / 1e6
    sample = f"each step: one FP64 oracle step of a {s.nx}x{s.ny}x{nz} z-slab of the {case['name']} workload"
    line = {
        "impl": "reference", "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": case["name"], "nodes": case["setup"].n_nodes, "sample_nodes": sub_setup.n_nodes,
                   "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_fields(cases):
    rho, T = [], []
    for c in cases:
        r, t = init_fields(c)
        rho.append(r.ravel())
        T.append(t.ravel())
    return np.concatenate(rho), np.concatenate(T)


def run_batch(args):
    """Batched ensemble: one persistent launch per step over all instances vs a sequential loop."""
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2201_06039_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2201_06039_gb300 import lbm
    cases = W.batch_instances()
    dims = [(c["setup"].nx, c["setup"].ny, c["setup"].nz) for c in cases]
    rho, T = batch_fields(cases)
    N = rho.size
    stream = torch.cuda.current_stream()
    common = lbm.params_from_setup(cases[0]["setup"], use_graph=1, check_nonfinite=0)
    bt = lbm.Batch(common, dims, stream=stream)
    bt.init(torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
    bt.step(args.warmup)
    tuned_ms = bt.autotune(3)
    plan = bt.plan
    # tile rows 0: the TMA mode (a TMA-kernel launch per instance); else the persistent batched kernel
    batch_kernel = "fused_tma_per_instance" if plan["tile_rows"] == 0 else "fused_batch"
    launches_per_step = lbm.lbm_batch_launches_per_step(bt.b)
    bt.step(args.steps)             # captures the K-step graph outside the timed region
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0.record(stream)
    bt.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = job_time_ms(e0.elapsed_time(e1), world)
    finite = bool(np.all(np.isfinite(bt.totals())))
    mlups = whole_job_mlups(N, args.steps, world, ms)
    peak, peak_kind = measured_peaks()
    k_ms = ms / args.steps          # the step's launches (one batched launch, or the TMA mode's fan-out)
    achieved = BYTES_PER_NODE["fp32"] * N / (k_ms * 1e-3) / 1e9

    # end to end: host fields in, K steps, host moments out (pinned buffers)
    h_rho = torch.from_numpy(rho).pin_memory()
    h_T = torch.from_numpy(T).pin_memory()
    outs = [torch.empty(N, dtype=torch.float32).pin_memory() for _ in range(5)]

    def e2e_once():
        lbm.lbm_batch_init_fields(bt.b, h_rho, h_T, None)
        lbm.lbm_batch_step(bt.b, args.steps)
        lbm.lbm_batch_get_moments(bt.b, *outs)

    e2e_once()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_once()
    e2e_s = job_time_ms((time.perf_counter() - t0) * 1e3, world) * 1e-3
    bt.close()

    # the same instances one after another through single-lattice contexts (FP32, own graphs)
    seq_steps = min(args.steps, 100)
    lats, off = [], 0
    for c, (nx, ny, nz) in zip(cases, dims):
        n = nx * ny * nz
        lat = lbm.Lattice(lbm.params_from_setup(c["setup"], use_graph=1, check_nonfinite=0), stream=stream)
        lat.init(torch.from_numpy(rho[off:off + n]).cuda(), torch.from_numpy(T[off:off + n]).cuda())
        lat.step(seq_steps)
        lat.step(seq_steps)         # captures the seq_steps graph
        lats.append(lat)
        off += n
    torch.cuda.synchronize()
    e0.record(stream)
    for lat in lats:
        lat.step(seq_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    kernels = sorted({lat.kernel for lat in lats})
    for lat in lats:
        lat.close()
    seq_mlups = N * seq_steps / (seq_ms * 1e-3) / 1e6

    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch_{len(cases)}_droplets_and_slabs_edges_24_96", "nodes": N,
                   "instances": len(cases), "kernel": batch_kernel, "precision": "fp32", "plan": plan,
                   "l2": "no flush: working set > 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": batch_kernel, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes_per_node": BYTES_PER_NODE["fp32"], "kernel_avg_ms": k_ms},
        "sequential": {"value": seq_mlups, "unit": "MLUPS", "steps": seq_steps,
                       "kernels": kernels, "what": "each instance alone through its own context"},
        "autotune_ms_per_step": tuned_ms,
        "e2e": {"value": whole_job_mlups(N, args.steps, world, e2e_s * 1e3), "unit": "MLUPS",
                "h2d_bytes_per_step": 2 * 4 * N / args.steps, "d2h_bytes_per_step": 5 * 4 * N / args.steps},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "finite": finite,
    }
    if args.cpu_baseline and rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline_batch(cases)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def cpu_baseline_batch(cases, budget_s=15.0):
    """FP64 oracle over the first instances of the ensemble, one after another."""
    import oracle
    nodes = steps_done = 0
    t_all = 0.0
    k = 0
    while t_all < budget_s and k < len(cases):
        c = cases[k]
        s = c["setup"]
        Tc = oracle.Tc_of(s)
        rl, rv, _ = oracle.maxwell(s, c["Tr_drop"] * Tc)
        rho, T, _ = W.build_fields(c, Tc, rl, rv)
        o = oracle.Oracle(s)
        o.init(rho, T)
        o.step(1)
        t0 = time.perf_counter()
        o.step(3)
        t_all += time.perf_counter() - t0
        o.close()
        nodes += s.n_nodes * 3
        k += 1
    return dict(value=nodes / t_all / 1e6, unit="MLUPS", cores=oracle.num_threads(), kind="oracle",
                sample=f"3 FP64 oracle steps of each of the first {k} ensemble instances, one after another")


def rel_err(a, b):
    """max |a - b| / max |b| (u as a vector: the largest component error over the largest |u_k|)."""
    out = {}
    for k in ("rho", "T"):
        out[k] = float(np.max(np.abs(a[k].astype(np.float64) - b[k]))) / float(np.max(np.abs(b[k])))
    den = max(float(np.max(np.abs(b[k]))) for k in ("ux", "uy", "uz"))
    out["u"] = max(float(np.max(np.abs(a[k].astype(np.float64) - b[k]))) for k in ("ux", "uy", "uz")) / den
    return out


def compare_16bit(lbm, case, rho, T, stream, steps):
    """Shifted BF16 / FP16 storage beside FP32: throughput on the benchmark lattice, and the field
    error against FP32 storage on the 64 x 64 x 96 copy of the workload after 300 steps (the FP64
    oracle comparison of the same case is a GPU test)."""
    import torch
    out = {"error_case": "64x64x96 pool boiling, 300 steps, max-norm relative to FP32 storage"}
    s = case["setup"]
    small = W.pool_boiling_downscaled()
    r_s, t_s = init_fields(small)
    Tc_small = lbm.lbm_eos_critical(lbm.params_from_setup(small["setup"]))[0]
    ref = None
    res = {}
    for prec in ("fp32", "bf16", "fp16"):
        over = {} if prec == "fp32" else dict(precision=PREC_CODE[prec], rho_ref=float(r_s.mean()),
                                              T_ref=0.86 * Tc_small)
        lat = lbm.Lattice(lbm.params_from_setup(small["setup"], check_nonfinite=0, **over), stream=stream)
        lat.init(r_s, t_s)
        lat.step(300)
        m = lat.moments()
        lat.close()
        if prec == "fp32":
            ref = {k: v.astype(np.float64) for k, v in m.items()}
        else:
            res[prec] = rel_err(m, ref)
    for prec in ("bf16", "fp16"):
        p = lbm.params_from_setup(s, check_nonfinite=0, precision=PREC_CODE[prec], rho_ref=float(rho.mean()))
        p.T_ref = 0.86 * lbm.lbm_eos_critical(p)[0]
        lat = lbm.Lattice(p, stream=stream)
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
        lat.autotune(steps=20)
        lat.step(10)
        lat.step(steps)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[prec] = {"value": s.n_nodes / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms,
                     "algorithmic_bytes_per_node": BYTES_PER_NODE[prec], "steps": steps,
                     "err_vs_fp32": res[prec]}
        lat.close()
    return out


def run_mine(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2201_06039_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2201_06039_gb300 import lbm

    case = workload(args.workload, args.nx, args.ny, args.nz)
    s = case["setup"]
    N = s.n_nodes
    rho, T = init_fields(case)
    stream = torch.cuda.current_stream()
    p = lbm.params_from_setup(s, kernel=KERNEL_CODE[args.kernel], precision=PREC_CODE[args.precision],
                              use_graph=1, check_nonfinite=0, use_tma=0 if args.kernel == "fused_generic" else 1,
                              thermal_q=args.thermal_q)
    if args.precision != "fp32":
        p.rho_ref = float(rho.mean())
        p.T_ref = 0.86 * lbm.lbm_eos_critical(p)[0]
    lat = lbm.Lattice(p, stream=stream)
    kernel_name = {lbm.LBM_KERNEL_FUSED: "fused", lbm.LBM_KERNEL_FUSED_TMA: "fused_tma"}.get(lat.kernel, "collide")

    # ---- device-resident timing
    lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
    tuned = None
    if lat.kernel == lbm.LBM_KERNEL_FUSED_TMA:
        if args.plan:   # pinned tile shape and z-chunk (profiling runs of one plan)
            shape, zchunk = (int(v) for v in args.plan.split(","))
            lat.select_plan(shape, zchunk)
            tuned = {"shape": lat.plan[0], "zchunk": lat.plan[1]}
        else:
            tuned = lat.autotune(steps=20)   # plan by timing
    lat.step(args.warmup)
    lat.step(args.steps)            # captures the K-step graph outside the timed region
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = job_time_ms(e0.elapsed_time(e1), world)
    mass, Tsum, _ = lat.totals()
    finite = math.isfinite(mass) and math.isfinite(Tsum)
    mlups = whole_job_mlups(N, args.steps, world, ms)

    # ---- per-kernel durations (CUDA events on the lattice's stream) for the roofline
    kms, kn = lbm.lbm_step_profiled(lat.ctx, max(3, min(50, args.steps)))
    k_idx = 1 if kernel_name == "collide" else 0
    k_avg_ms = kms[k_idx] / max(1, kn[k_idx])
    peak, peak_kind = measured_peaks()
    bpn = BYTES_PER_NODE[args.precision] if args.thermal_q == 7 else (19 + 19) * 4 * 2 + 8   # D3Q19 g: 312 B
    achieved = bpn * N / (k_avg_ms * 1e-3) / 1e9
    traffic = committed_traffic(kernel_name, args.precision, N)

    # ---- end to end through the C-ABI with pinned host buffers (copies inside the timed region)
    h_rho = torch.from_numpy(rho).pin_memory()
    h_T = torch.from_numpy(T).pin_memory()
    outs = [torch.empty(s.shape, dtype=torch.float32).pin_memory() for _ in range(5)]

    def e2e_once():
        lbm.lbm_init_fields(lat.ctx, h_rho, h_T, None)
        lbm.lbm_step(lat.ctx, args.steps)
        lbm.lbm_get_moments(lat.ctx, *outs)

    e2e_once()                      # graph capture for the post-init step count
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_once()
    e2e_s = job_time_ms((time.perf_counter() - t0) * 1e3, world) * 1e-3
    e2e_mlups = whole_job_mlups(N, args.steps, world, e2e_s * 1e3)

    # kernels per step as counted by the profiled steps (fused or psi + collide, ghost refresh)
    launches_per_step = sum(kn) / max(3, min(50, args.steps))
    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else f"f32 compute, {args.precision} storage",
        "data": "synthetic",
        "config": {"workload": case["name"], "nodes": N, "kernel": kernel_name, "precision": args.precision,
                   "thermal_lattice": f"D3Q{args.thermal_q}",
                   "plan": None if tuned is None else {"tile": list(lbm.lbm_plan_shapes()[tuned["shape"]]),
                                                       "zchunk": tuned["zchunk"]},
                   "l2": "no flush: working set %.2f GB > 129 MB L2" % (lbm.lbm_workspace_bytes(p) / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "hbm_gbs_step": bpn * N * args.steps / (ms * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "kernel": kernel_name, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_node": bpn, "kernel_avg_ms": k_avg_ms},
        "e2e": {"value": e2e_mlups, "unit": "MLUPS", "h2d_bytes_per_step": 2 * 4 * N / args.steps,
                "d2h_bytes_per_step": 5 * 4 * N / args.steps},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "finite": finite,
    }
    lat.close()
    if args.precision == "fp32" and args.compare_16bit and args.workload == "pool_boiling" and not args.nx \
            and args.thermal_q == 7:
        line["storage_16bit"] = compare_16bit(lbm, case, rho, T, stream, min(args.steps, 500))
    if args.cpu_baseline and rank == 0 and world == 1:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline_run(case).items() if k != "seconds"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--kernel", default="auto", choices=list(KERNEL_CODE))
    ap.add_argument("--precision", default="fp32", choices=list(PREC_CODE))
    ap.add_argument("--thermal-q", dest="thermal_q", type=int, default=7, choices=[7, 19],
                    help="temperature lattice: D3Q7 (MRT, default) or D3Q19 (Eq. 19 BGK; generic kernels)")
    ap.add_argument("--workload", default="pool_boiling")
    ap.add_argument("--nx", type=int, default=None, help="override the lattice size (profiling runs)")
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--nz", type=int, default=None)
    ap.add_argument("--plan", default=None, help="SHAPE,ZCHUNK: pin the TMA kernel's plan instead of autotuning")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-16bit", dest="compare_16bit", action="store_false",
                    help="skip the BF16 / FP16 storage comparison of the default run")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    return run_mine(args)


if __name__ == "__main__":
    sys.exit(main())
