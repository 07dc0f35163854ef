#!/usr/bin/env python
"""Throughput of the full moving-boundary electrokinetics step (S1-S5) on GB300.

Workload (default, the headline): many moving colloids in the large box --
512^3 periodic lattice, D3Q19 BGK tau = 1, 1000 spheres R = 6, Z = -200 at
seeded non-overlapping positions, free to move, 2 ion species (z = +1/-1,
D = 0.3, bulk 5e-4, neutralised), Bjerrum length 0.7, E = 0.002 along x, in
the FP32-storage form (float populations, int32 fixed-point species, FP64
particle sums and integrator).  A step is one full time step: Poisson, fused
flux + LB, advection, particle forces and integration, re-flagging and
transitions.  Beside it: the single-sphere 128^3 box in both storage forms
(the plain FP64 form is the parity reference), the 256^3 box with 64 spheres
and three species, the batched ensemble of 256 small boxes, and the
multigrid Poisson solve.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  `value` is MLUPS (million lattice-node updates
per second, boundary nodes included) over all ranks; with N > 1 every rank
runs its own replica of the box (weak scaling, no collective on the data path).
`--impl reference` times the FP64 CPU oracle on all host cores instead (a
bounded sub-box sample of the same workload, one oracle replica per core).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS per full EK step and % of HBM roofline, FP32/batched vs plain FP64 at 1e-3 mobility"
HEADLINE = "large"
SAMPLE_EDGE = 128  # edge of the sub-box the CPU oracle is timed on


def l2_note(w, fp32):
    n = w["shape"][0] * w["shape"][1] * w["shape"][2]
    mb = 2 * 19 * (4 if fp32 else 8) * n / 1e6
    return (f"state > L2 (populations 2 x 19 x {4 if fp32 else 8} B x N = {mb:.0f} MB; "
            f"L2 129 MB), no flush needed")


def describe(w):
    P = len(w["particles"])
    R = sorted({p["radius"] for p in w["particles"]})
    Z = [p["charge"] for p in w["particles"]]
    zs = f"{Z[0]:g}" if len(set(Z)) == 1 else f"U[{min(Z):.0f},{max(Z):.0f}]"
    nx, ny, nz = w["shape"]
    return (f"{w['name']}: {nx}x{ny}x{nz}, {P} sphere(s) R={','.join(f'{r:g}' for r in R)}, "
            f"Z={zs}, {len(w['valence'])} species z={list(w['valence'])} bulk {w['bulk'][0]:g}, "
            f"E={w['E'][0]:g} along x, BGK tau=1")


# Algorithmic bytes per lattice node of the fused flux + LB kernel: what the
# stage must read and write once per step by the method's own state (the items
# of the step's per-node byte budget that S2 touches): populations read +
# written, species read and written after the flux divergence, Psi and the
# node class, Phi.  The u,
# internal-force and sign-byte writes it also makes (for S3 and S4) are
# implementation overhead and count against the fraction.
def lb_bytes_per_node(fp32, K):
    if fp32:
        return 2 * 19 * 4 + 2 * K * 4 + 5 + 4        # 177 for K = 2
    return 2 * 19 * 8 + 2 * K * 8 + 9 + 8            # 353 for K = 2


LB_FP64_FLOP_PER_NODE = 950


# Algorithmic bytes per node of a whole step (S1-S5), the state read once and
# written once with every intermediate fused: populations read + written,
# species read + written, Psi and the node class read, Phi written (S1) and read
# (S2), the charge written and read, one round trip of the half spectrum.  The
# stored u, the extra FFT passes and the particle boxes count against it.
def step_bytes_per_node(fp32, K):
    if fp32:
        return 2 * 19 * 4 + 2 * K * 4 + 5 + 8 + 8 + 8      # 197 for K = 2
    return 2 * 19 * 8 + 2 * K * 8 + 9 + 16 + 16 + 16       # 393 for K = 2


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def step_roofline(mlups, bytes_per_node, hbm_peak):
    gbs = mlups * 1e6 * bytes_per_node / 1e9
    return {"bytes_per_node": bytes_per_node, "achieved": round(gbs, 1), "unit": "GB/s",
            "peak": hbm_peak, "frac": round(gbs / hbm_peak, 4), "nominal_peak": NOMINAL_HBM_GBS,
            "frac_nominal": round(gbs / NOMINAL_HBM_GBS, 4)}


# FP64 peak derived from the unit counts: 152 SMs x 2.07 GHz x 4 flop/clk/SM
# (2 DFMA per clock per SM); a DFMA probe on this pool measured 1.19 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per lattice node
# of one launch of the kernel, from an ncu capture, valid only for the kernel
# source it was taken on (otherwise the traffic is reported as null).
TRAFFIC = {"k_lb32": {"bytes_per_node": (202409472 + 178517504) / 128 ** 3,
                      "source_sha": "b124e8565c46b3fd", "file": "ek_lattice32.cu"}}


def src_sha(name: str) -> str:
    p = os.path.join(ROOT, "paper_1607_04572_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def traffic(kernel, nodes):
    t = TRAFFIC.get(kernel)
    if t is None:
        return None
    if t["source_sha"] != src_sha(t["file"]):
        return None
    return int(round(t["bytes_per_node"] * nodes))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock samples around the timed region: started (and waited
    for) before it, stopped a little after it; the samples whose timestamps
    fall within MARGIN seconds of the region are kept (a short region can lie
    between two samples)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    MARGIN = 0.25

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            deadline = time.time() + 5.0
            while time.time() < deadline and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(self.MARGIN)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        import datetime
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            if self.t0 is None or self.t0 - self.MARGIN <= ts <= self.t1 + self.MARGIN:
                rows.append(f[1:])
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "window_s": round(self.t1 - self.t0 + 2 * self.MARGIN, 3) if self.t0 else None}


def build_system(ek, w, fp32=True):
    flags = ek.EK_PV | ek.EK_NEUTRALIZE | (ek.EK_FP32 if fp32 else 0)
    s = ek.EKSystem(w["shape"], nu=w["nu"], rho0=w["rho0"], bjerrum=w["bjerrum"],
                    valence=w["valence"], D=w["D"], bulk=w["bulk"], flags=flags)
    for p in w["particles"]:
        s.add_particle(p["pos"], radius=p["radius"], charge=p["charge"], rho_p=w["rho_p"])
    import numpy as np
    s.set_field(ek.FIELD_E_EXT, np.array(w["E"], dtype=np.float64))
    return s


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores (the CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_replica(job, start, out):
    """One oracle replica of the sample in its own process (single-threaded
    numpy): `warmup` untimed steps, a barrier with the other replicas, then
    steps until `steps` are done or the budget is spent.  Puts (steps done,
    wall-clock start and end) on `out`."""
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    name, edge, steps, warmup, budget_s = job
    import numpy as np
    import workloads
    from oracle.ek_oracle import EKOracle, NEUTRALIZE, PV
    w = workloads.sub_box(name, edge)
    o = EKOracle(*w["shape"], nu=w["nu"], rho0=w["rho0"], bjerrum=w["bjerrum"],
                 valence=w["valence"], D=w["D"], bulk=w["bulk"], flags=PV | NEUTRALIZE)
    for p in w["particles"]:
        o.add_particle(p["pos"], radius=p["radius"], charge=p["charge"], rho_p=w["rho_p"])
    o.E = np.array(w["E"], dtype=np.float64)
    for _ in range(warmup):
        o.step()
    start.wait(timeout=600)  # all replicas start their timed steps together
    t0 = time.time()
    done = 0
    while done < steps:
        o.step()
        done += 1
        if time.time() - t0 > budget_s:
            break
    out.put((done, t0, time.time()))


def oracle_procs(edge):
    """Replicas to run at once: one per host core, as far as the host memory
    holds them (an oracle of n^3 nodes peaks near 1.8 kB per node)."""
    cores = os.cpu_count() or 1
    try:
        avail = [int(l.split()[1]) * 1024 for l in open("/proc/meminfo") if l.startswith("MemAvailable")][0]
    except Exception:
        avail = 8 << 30
    per = 1800 * edge ** 3
    return max(1, min(cores, int(0.6 * avail // per)))


def time_oracle_all_cores(name, edge, steps, warmup, budget_s):
    """Oracle MLUPS on the host: one replica of the sub-box sample per core,
    spawned processes (no fork of a CUDA process), timed steps aligned;
    throughput = all replicas' node updates over the span of their timed
    steps."""
    import multiprocessing as mp
    procs = oracle_procs(edge)
    ctx = mp.get_context("spawn")
    start = ctx.Barrier(procs)
    out = ctx.Queue()
    ps = [ctx.Process(target=_oracle_replica, args=((name, edge, steps, warmup, budget_s), start, out))
          for _ in range(procs)]
    for p in ps:
        p.start()
    res = [out.get(timeout=1200) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    done = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    nodes = edge ** 3
    return {"value": nodes * done / span / 1e6, "procs": procs, "steps": min(r[0] for r in res),
            "span_s": span}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks_of(x, ws, device):
    """The largest of the ranks' values, on every rank (a replica job takes as
    long as its slowest rank)."""
    if ws == 1:
        return x
    import torch
    t = torch.tensor([float(x)], device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_mlups(nodes, steps, ws, ms):
    """Whole-job MLUPS of ws replicas (weak scaling): every rank advanced its
    own box of `nodes` nodes `steps` times; ms is the slowest rank's time."""
    return nodes * steps * ws / (ms / 1e3) / 1e6


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    warm = min(args.warmup, 1)
    import workloads
    edge = min(SAMPLE_EDGE, w["shape"][0])
    r = time_oracle_all_cores(w["name"], edge, args.steps, warm, budget_s=150.0)
    sample = (f"{edge}^3 periodic sub-box of the {describe(w)} workload "
              f"({len(workloads.sub_box(w['name'], edge)['particles'])} "
              f"sphere(s) wholly inside); {r['procs']} single-threaded numpy FP64 oracle "
              f"replicas in parallel, {r['steps']} timed of {args.steps} requested steps each "
              f"after {warm} warm-up step(s)")
    line = {"impl": "reference", "metric": METRIC, "value": round(r["value"], 4), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": r["steps"], "warmup": warm,
            "ms_per_step": round(r["span_s"] / max(r["steps"], 1) * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": describe(w), "nodes": edge ** 3,
                       "parallelism": "replicas", "l2": "host run"},
            "cpu_baseline": {"value": round(r["value"], 4), "unit": "MLUPS", "cores": r["procs"],
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(r["value"], 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure(ek, torch, w, fp32, args, stream, barrier, max_over_ranks, ws, stage_steps=None):
    """Warm-up, then K steps timed with CUDA events on the context's stream
    (inputs resident in HBM); then a per-stage split of more steps."""
    s = build_system(ek, w, fp32)
    s.set_stream(stream)
    s.step(max(args.warmup, 3))
    nodes = w["shape"][0] * w["shape"][1] * w["shape"][2]
    clk = ClockSampler(dist_env()[2])
    barrier()
    clk.start()
    launches0 = s.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clk.mark(True)
    ev0.record(stream)
    s.step_async(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    clk.mark(False)
    barrier()
    clocks = clk.stop()
    launches = s.kernel_launches() - launches0
    s.sync()
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    kst = stage_steps or max(10, min(args.steps, 50))
    stage = s.step_timed(kst)
    return dict(system=s, ms=ms, value=job_mlups(nodes, args.steps, ws, ms), nodes=nodes,
                launches=launches, clocks=clocks,
                stages={k: round(v / kst, 4) for k, v in
                        zip(["S1_poisson", "S2_flux_lb", "S3_advection", "S4_particles",
                             "S5_reflag", "total"], stage)},
                lb_ms=stage[1] / kst)


def end_to_end(ek, torch, w, s, stream, steps, barrier, max_over_ranks, ws):
    """The same metric through the public API with host buffers: every step the
    field E is read from pinned host memory into the step's launch, the step
    runs, and the particle records (the mobility observable) are copied into
    pinned host memory and decoded on the host; two record buffers let step
    t + 1 run while step t's records are read."""
    nodes = w["shape"][0] * w["shape"][1] * w["shape"][2]
    e_host = torch.tensor(w["E"], dtype=torch.float64).pin_memory()
    npart = s.num_particles()
    recbytes = npart * ctypes_sizeof_particle(ek)
    bufs = [torch.zeros(max(recbytes, 1), dtype=torch.uint8).pin_memory() for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    barrier()
    t0 = time.perf_counter()
    parts = []
    for t in range(steps):
        s.set_field(ek.FIELD_E_EXT, e_host)
        s.step_async(1)
        s.get_particles_async(bufs[t % 2])
        evs[t % 2].record(stream)
        if t > 0:
            evs[(t - 1) % 2].synchronize()
            parts = ek.particles_from_buffer(bufs[(t - 1) % 2], npart)
    evs[(steps - 1) % 2].synchronize()
    parts = ek.particles_from_buffer(bufs[(steps - 1) % 2], npart)
    s.sync()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    return {"value": round(job_mlups(nodes, steps, ws, e2e_s * 1e3), 3), "unit": "MLUPS",
            "h2d_bytes_per_step": 3 * 8, "d2h_bytes_per_step": len(parts) * ctypes_sizeof_particle(ek),
            "steps": steps}


def form_line(r, w, fp32, hbm_peak, peak_kind):
    """Throughput, stages and rooflines of one measured system."""
    K = len(w["valence"])
    n = r["nodes"]
    d = {"value": round(r["value"], 3), "unit": "MLUPS", "ms_per_step": None,
         "stages_ms_per_step": r["stages"], "gpu_launches": r["launches"], "clocks": r["clocks"],
         "step_roofline": step_roofline(r["value"], step_bytes_per_node(fp32, K), hbm_peak)}
    lb_alg = lb_bytes_per_node(fp32, K) * n
    gbs = lb_alg / (r["lb_ms"] / 1e3) / 1e9
    if fp32:
        d["roofline"] = {"bound": "hbm", "kernel": "k_lb32_tiled", "achieved": round(gbs, 1),
                         "peak": hbm_peak, "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
                         "peak_kind": peak_kind, "traffic": traffic("k_lb32", n),
                         "algorithmic_bytes": lb_alg, "kernel_ms": round(r["lb_ms"], 4)}
    else:
        tflops = LB_FP64_FLOP_PER_NODE * n / (r["lb_ms"] / 1e3) / 1e12
        d["roofline"] = {"bound": "alu", "kernel": "k_lb_fused", "achieved": round(tflops, 4),
                         "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s (FP64)",
                         "frac": round(tflops / FP64_PEAK_TFLOPS, 4),
                         "traffic": traffic("k_lb_fused", n), "algorithmic_bytes": lb_alg,
                         "hbm": {"achieved": round(gbs, 1), "frac": round(gbs / hbm_peak, 4)},
                         "kernel_ms": round(r["lb_ms"], 4)}
    return d


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline workload only (no 128^3 / 256^3 / FP64 / batched / multigrid / CG lines)")
    ap.add_argument("--workload", default=HEADLINE, choices=["large", "many", "single", "small"],
                    help="the measured workload (the headline is the large box; the others are "
                         "for profiling smaller cases)")
    ap.add_argument("--batch-only", action="store_true",
                    help="only the batched ensemble (its line; for profiling the batched step)")
    ap.add_argument("--no-tune", action="store_true",
                    help="batched ensemble: the fused form with 8-plane S2 segments and the "
                         "particle chain beside S3 instead of the autotuner's choice")
    args = ap.parse_args()
    import workloads
    w = workloads.workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, w)

    ws, rank, local = dist_env()
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the host baseline before any CUDA call: its processes are spawned,
        # and the GPU is not yet busy
        cpu = time_oracle_all_cores(w["name"], min(SAMPLE_EDGE, w["shape"][0]), 2, 1, budget_s=30.0)
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU path)")
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1607_04572_gb300 import ek

    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return max_over_ranks_of(x, ws, "cuda")

    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs"))
    if args.batch_only:
        rb = measure_batch(ek, torch, args, barrier, max_over_ranks)
        rb["step_roofline"] = step_roofline(rb["value"], step_bytes_per_node(True, 2), hbm_peak)
        if rank == 0:
            print(json.dumps({"metric": "MLUPS of the batched ensemble", **rb}), flush=True)
        return 0

    # ---- the headline: the large box, FP32-storage form -----------------------
    r = measure(ek, torch, w, True, args, stream, barrier, max_over_ranks, ws, stage_steps=10)
    e2e = end_to_end(ek, torch, w, r["system"], stream, max(5, min(args.steps, 20)), barrier,
                     max_over_ranks, ws)
    head = form_line(r, w, True, hbm_peak, peak_kind)
    r["system"].close()
    line = {
        "metric": METRIC, "value": head["value"], "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(r["ms"] / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (int32 species, f64 particle sums)", "data": "synthetic",
        "config": {"workload": describe(w) + "; FP32-storage form", "nodes": r["nodes"],
                   "particles": len(w["particles"]),
                   "parallelism": "replicas" if ws > 1 else "single", "l2": l2_note(w, True)},
        "roofline": head["roofline"],
        "step_roofline": head["step_roofline"],
        "stages_ms_per_step": head["stages_ms_per_step"],
        "e2e": e2e,
        "gpu_launches": r["launches"],
        "clocks": r["clocks"],
    }
    if not args.no_extra:
        extra_args = argparse.Namespace(**vars(args))
        extra_args.steps = min(args.steps, 50)
        # the single-sphere box in both storage forms (FP64: the parity form)
        ws1 = workloads.workload("single")
        r32 = measure(ek, torch, ws1, True, extra_args, stream, barrier, max_over_ranks, ws)
        r64 = measure(ek, torch, ws1, False, extra_args, stream, barrier, max_over_ranks, ws)
        l32 = form_line(r32, ws1, True, hbm_peak, peak_kind)
        l32["ms_per_step"] = round(r32["ms"] / extra_args.steps, 4)
        l32["workload"] = describe(ws1)
        l32["e2e"] = end_to_end(ek, torch, ws1, r32["system"], stream, max(5, min(args.steps, 50)),
                                barrier, max_over_ranks, ws)
        l64 = form_line(r64, ws1, False, hbm_peak, peak_kind)
        l64["ms_per_step"] = round(r64["ms"] / extra_args.steps, 4)
        l64["workload"] = describe(ws1)
        r32["system"].close()
        r64["system"].close()
        line["single_128"] = l32
        line["fp64_form"] = l64
        line["speedup_fp32_vs_fp64_128"] = round(r32["value"] / r64["value"], 2)
        # the 256^3 box with 64 spheres and three species
        wm = workloads.workload("many")
        rm = measure(ek, torch, wm, True, extra_args, stream, barrier, max_over_ranks, ws)
        lm = form_line(rm, wm, True, hbm_peak, peak_kind)
        lm["ms_per_step"] = round(rm["ms"] / extra_args.steps, 4)
        lm["workload"] = describe(wm)
        rm["system"].close()
        line["many_256"] = lm
        if rank == 0 and ws == 1:
            line["poisson_mg"] = measure_poisson_mg(ek, torch)
            line["poisson_cg"] = measure_poisson_cg(ek, torch)
        rb = measure_batch(ek, torch, args, barrier, max_over_ranks)
        rb["step_roofline"] = step_roofline(rb["value"], step_bytes_per_node(True, 2), hbm_peak)
        line["batched_form"] = rb
    if cpu is not None:
        edge = min(SAMPLE_EDGE, w["shape"][0])
        nsp = len(workloads.sub_box(w["name"], edge)["particles"])
        line["cpu_baseline"] = {
            "value": round(cpu["value"], 4), "unit": "MLUPS", "cores": cpu["procs"],
            "kind": "oracle",
            "sample": (f"{edge}^3 periodic sub-box of the measured workload ({nsp} "
                       f"sphere(s) wholly inside), {cpu['procs']} single-threaded numpy FP64 "
                       f"oracle replicas in parallel, {cpu['steps']} timed step(s) each after "
                       f"1 warm-up, {cpu['span_s']:.1f} s")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# Multigrid V-cycle traffic at the finest level, per node (an estimate of the
# bytes that must cross HBM, intermediates in L2 not subtracted): 8 red-black
# half-sweeps (read phi and the colour's b, write the colour's phi: 16 B),
# residual 24, restriction 8, prolongation 17, the residual and its norm
# after the cycle 32; the coarser levels add an eighth per level.
MG_BYTES_PER_NODE_CYCLE = round((8 * 16 + 24 + 8 + 17 + 32) * 8 / 7)   # 239


def measure_poisson_mg(ek, torch, shape=(128, 128, 128), reps=3):
    """The periodic Poisson solve of S1 (FP64) by multigrid V-cycles against
    the FFT solve, on the same seeded charge: time per solve (CUDA events on
    the solvers' stream, after a warm-up solve), cycles, residual, and the
    largest difference between the two solutions."""
    import numpy as np
    nx, ny, nz = shape
    n = nx * ny * nz
    rng = np.random.default_rng(1607)
    q = torch.tensor(rng.random(n) - 0.5, device="cuda", dtype=torch.float64)
    phi_mg = torch.empty_like(q)
    phi_fft = torch.empty_like(q)
    scratch = torch.empty(ek.poisson_mg_scratch_bytes(shape), dtype=torch.uint8, device="cuda")
    spectrum = torch.empty(ek.load_library().ek_poisson_scratch_bytes(nx, ny, nz), dtype=torch.uint8,
                           device="cuda")
    st = torch.cuda.Stream()
    times = {}
    for name in ("mg", "fft"):
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            if name == "mg":
                cycles, res = ek.poisson_solve_mg(q, phi_mg, shape, 0.7, scratch, tol=1e-12,
                                                  max_cycles=50, stream=st)
            else:
                ek.poisson_solve(q, phi_fft, shape, 0.7, spectrum, stream=st)
            e1.record(st)
            e1.synchronize()
            if r > 0:
                times.setdefault(name, []).append(e0.elapsed_time(e1))
    ms = min(times["mg"])
    diff = (phi_mg - phi_fft).abs().max().item() / phi_fft.abs().max().item()
    gbs = MG_BYTES_PER_NODE_CYCLE * n * cycles / (ms / 1e3) / 1e9
    return {"shape": list(shape), "ms": round(ms, 4), "cycles": cycles, "residual": res,
            "ms_per_cycle": round(ms / max(cycles, 1), 4), "fft_ms": round(min(times["fft"]), 4),
            "max_rel_diff_vs_fft": diff,
            "bytes_per_node_cycle": MG_BYTES_PER_NODE_CYCLE, "achieved_gbs": round(gbs, 1),
            "note": "FP64; every V-cycle's residual norm is read on the host to test convergence"}


# Conjugate-gradient traffic per node and iteration (FP64): the operator
# reads p, D^-1 and the node's three face permittivities and writes Ap (48);
# the update reads D^-1, p, Ap and reads and writes x and r (56); the new
# direction reads D^-1 and reads and writes r and p (40).
CG_BYTES_PER_NODE_ITER = 48 + 56 + 40   # 144


def measure_poisson_cg(ek, torch, shape=(128, 128, 128), tol=1e-10):
    """The Poisson solve with an inhomogeneous permittivity and fixed
    potentials (FP64 preconditioned conjugate gradients): a low-permittivity sphere (eps 2,
    R = 20) in water (eps 80) with a charged shell, between planes held at
    +-1: time per solve (CUDA events, after a warm-up solve), iterations and
    achieved bandwidth on the CG's bytes per node and iteration."""
    import numpy as np
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((x - nx / 2 + 0.3) ** 2 + (y - ny / 2 - 0.2) ** 2 + (z - nz / 2 + 0.1) ** 2)
    dev = "cuda"
    eps = torch.tensor(np.where(r < 20.0, 2.0, 80.0), device=dev, dtype=torch.float64)
    q = torch.tensor(np.where((r >= 20.0) & (r < 22.0), -0.01, 0.0), device=dev, dtype=torch.float64)
    fixed = torch.tensor(((z == 0) | (z == nz - 1)).astype(np.uint8), device=dev)
    pf = torch.tensor(np.where(z == 0, 1.0, -1.0), device=dev, dtype=torch.float64)
    phi = torch.empty_like(q)
    scratch = torch.empty(ek.poisson_cg_scratch_bytes(shape), dtype=torch.uint8, device=dev)
    st = torch.cuda.Stream()
    best = None
    for rep in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        it, res = ek.poisson_solve_cg(q, phi, shape, 0.7, scratch, eps=eps, fixed=fixed, phi_fixed=pf,
                                      tol=tol, max_iter=20000, stream=st)
        e1.record(st)
        e1.synchronize()
        if rep > 0:
            best = e0.elapsed_time(e1)
    n = nx * ny * nz
    gbs = CG_BYTES_PER_NODE_ITER * n * it / (best / 1e3) / 1e9
    return {"shape": list(shape), "ms": round(best, 3), "iterations": it, "residual": res,
            "ms_per_iteration": round(best / max(it, 1), 4),
            "bytes_per_node_iteration": CG_BYTES_PER_NODE_ITER, "achieved_gbs": round(gbs, 1),
            "note": "FP64 CG preconditioned by a multigrid V-cycle, tol 1e-10; eps 2 sphere R=20 "
                    "in eps 80 with a charged shell, planes z=0 and z=nz-1 held at +1 and -1; the "
                    "bytes are the CG's own (the V-cycle's are not counted)"}


def measure_batch(ek, torch, args, barrier, max_over_ranks):
    """The batched ensemble (256 boxes with edges from {32, 48, 64}, one sphere
    each, FP32 form): autotuned, then timed with CUDA events on the batch
    stream; beside it the same systems stepped one after another."""
    import workloads
    ws_ = workloads.batch_ensemble(256)
    nodes = sum(w["shape"][0] * w["shape"][1] * w["shape"][2] for w in ws_)
    systems = [build_system(ek, w, True) for w in ws_]
    stream = torch.cuda.Stream()
    b = ek.EKBatch(systems)
    b.set_stream(stream)
    if getattr(args, "no_tune", False):
        b.set_config(fused=1, planes_per_block=8, particle_chain_beside_s3=1)
        cfg, tuned_ms = b.config(), 0.0
    else:
        cfg, tuned_ms = b.tune(2)
    b.step(2)
    steps = max(3, min(args.steps, 20))
    barrier()
    launches0 = sum(s.kernel_launches() for s in systems)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b.step_async(steps)
    ev1.record(stream)
    ev1.synchronize()
    b.sync()
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    launches = sum(s.kernel_launches() for s in systems) - launches0
    # the same systems, one ek_step after another on one stream (no batching)
    for sy in systems:
        sy.set_stream(stream)
    seq_steps = 3
    ev0.record(stream)
    for _ in range(seq_steps):
        for sy in systems:
            sy.step_async(1)
    ev1.record(stream)
    ev1.synchronize()
    ms_seq = max_over_ranks(ev0.elapsed_time(ev1))
    b.close()
    for sy in systems:
        sy.close()
    return {"value": round(nodes * steps / (ms / 1e3) / 1e6, 3), "unit": "MLUPS",
            "ms_per_step": round(ms / steps, 4), "steps": steps, "systems": len(ws_),
            "nodes": nodes, "gpu_launches": launches, "tuned": cfg,
            "tuner_ms_per_step": round(tuned_ms, 4),
            "one_by_one": {"value": round(nodes * seq_steps / (ms_seq / 1e3) / 1e6, 3),
                           "ms_per_step": round(ms_seq / seq_steps, 4)},
            "config": "256 boxes, edges {32,48,64} per axis, one sphere R U[3,6], Z U[-min(100,12R),-20], "
                      "salt log-U[1e-4,1e-2], E log-U[1e-3,1e-2], FP32 form, one graph launch per step"}


def ctypes_sizeof_particle(ek):
    import ctypes
    return ctypes.sizeof(ek.ParticleRec)


if __name__ == "__main__":
    sys.exit(main())
