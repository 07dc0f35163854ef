#!/usr/bin/env python
"""Throughput of the full moving-boundary electrokinetics step (S1-S5) on GB300.

Workload (default): the single-sphere electrophoresis box -- 128^3 periodic
lattice, D3Q19 BGK tau = 1, 2 ion species (z = +1/-1, D = 0.3, bulk 1e-3,
neutralised), Bjerrum length 0.7, one sphere R = 8, Z = -300 at a seeded
off-centre position, free to move, E = 0.005 along x.  A step is one full time
step: Poisson, fused flux + LB, advection, particle forces and integration,
re-flagging and transitions.  `value` is the FP32-storage form (float
populations, int32 fixed-point species, FP64 particle sums and integrator);
the plain FP64 form is measured beside it under "fp64_form".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  `value` is MLUPS (million lattice-node updates
per second, boundary nodes included) over all ranks; with N > 1 every rank
runs its own replica of the box (weak scaling, no collective on the data path).
`--impl reference` times the FP64 CPU oracle on the same workload instead.
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
FLUSH_NOTE = ("state > L2 (populations 2 x 19 x 4 B x N = 319 MB in the FP32 form, 637 MB in "
              "FP64, at 128^3; L2 129 MB), no flush needed")

# Algorithmic work of the fused flux + LB kernel, per fluid node, two species,
# partial volumes on, bulk node (all 18 links fluid): bytes that must cross
# HBM once per step (populations read + written, species read + written after
# the flux divergence, Psi, Phi and the node class read, u and the internal
# solute force written for S3 / S4, one sign byte) and FP64 operations of the
# formulas.
LB_BYTES_PER_NODE = 2 * 19 * 8 + 2 * 2 * 8 + 8 + 8 + 4 + 3 * 8 + 3 * 8 + 1   # 405 (k_lb_fused)
LB_FP64_FLOP_PER_NODE = 950
# the same for the FP32-storage kernel (k_lb32_tiled): float populations,
# int32 species, float Psi / Phi / u / internal force
LB32_BYTES_PER_NODE = 2 * 19 * 4 + 2 * 2 * 4 + 4 + 4 + 4 + 3 * 4 + 3 * 4 + 1  # 205
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

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch
# from an ncu capture of the 128^3 workload (profiles/), valid only for the
# kernel source it was taken on.
TRAFFIC = {"k_lb_fused": {"bytes_per_launch": 755997696,  # profiles/fp64_k_lb_fused_k_advect_single128.md
                           "source_sha": "85d705496daa5794", "file": "ek_lattice.cu"},
           "k_lb32": {"bytes_per_launch": 202392832 + 179882240,  # profiles/fp32_kernels_single128.md
                      "source_sha": "8e4ea3cf1efc08bf", "file": "ek_lattice32.cu"}}


def src_sha(name: str) -> str:
    p = os.path.join(ROOT, "paper_1607_04572_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


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


def build_oracle(w):
    import numpy as np
    from oracle.ek_oracle import EKOracle, NEUTRALIZE, PV
    o = EKOracle(*w["shape"], nu=w["nu"], rho0=w["rho0"], bjerrum=w["bjerrum"],
                 valence=w["valence"], D=w["D"], bulk=w["bulk"], flags=PV | NEUTRALIZE)
    for p in w["particles"]:
        o.add_particle(p["pos"], radius=p["radius"], charge=p["charge"], rho_p=w["rho_p"])
    o.E = np.array(w["E"], dtype=np.float64)
    return o


def time_oracle(w, max_steps, budget_s, warmup=1):
    """Oracle MLUPS on the host: `warmup` untimed steps, then up to max_steps
    timed steps or until budget_s seconds are spent."""
    o = build_oracle(w)
    for _ in range(warmup):
        o.step()
    nodes = w["shape"][0] * w["shape"][1] * w["shape"][2]
    t0 = time.perf_counter()
    done = 0
    while done < max_steps:
        o.step()
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return nodes * done / dt / 1e6, done, dt


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
    nodes = w["shape"][0] * w["shape"][1] * w["shape"][2]
    # each oracle step of the 128^3 box takes seconds: time a bounded sample
    value, done, dt = time_oracle(w, args.steps, budget_s=120.0, warmup=min(args.warmup, 1))
    sample = (f"{done} timed of {args.steps} requested steps of the {w['shape'][0]}^3 workload "
              f"after {min(args.warmup, 1)} warm-up step(s); numpy FP64 oracle, single thread")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": done, "warmup": min(args.warmup, 1),
            "ms_per_step": round(dt / done * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "single-sphere electrophoresis 128^3, R=8, Z=-300, 2 species, "
                                   "E=0.005, FP64", "nodes": nodes, "parallelism": "replicas",
                       "l2": FLUSH_NOTE},
            "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": 1,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-ensemble measurement")
    args = ap.parse_args()
    import workloads
    w = workloads.workload("single")
    if args.impl == "reference":
        return run_reference(args, w)

    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU path)")
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1607_04572_gb300 import ek

    nodes = w["shape"][0] * w["shape"][1] * w["shape"][2]
    stream = torch.cuda.Stream()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return max_over_ranks_of(x, ws, "cuda")

    def measure(fp32):
        """Warm-up, then K steps timed with CUDA events on the context's stream
        (inputs resident in HBM); then a per-stage split of more steps."""
        s = build_system(ek, w, fp32)
        s.set_stream(stream)
        s.step(max(args.warmup, 3))
        clk = ClockSampler(local)
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
        kst = max(10, min(args.steps, 50))
        stage = s.step_timed(kst)
        return dict(system=s, ms=ms, value=job_mlups(nodes, args.steps, ws, ms),
                    launches=launches, clocks=clocks,
                    stages={k: round(v / kst, 4) for k, v in
                            zip(["S1_poisson", "S2_flux_lb", "S3_advection", "S4_particles",
                                 "S5_reflag", "total"], stage)},
                    lb_ms=stage[1] / kst)

    r32 = measure(True)
    r64 = measure(False)
    s = r32["system"]
    rb = None if args.no_batch else measure_batch(ek, torch, args, barrier, max_over_ranks)

    # ---- end to end through the public API with host buffers (FP32 form) ----
    # every step: the field E is read from pinned host memory into the step's
    # launch, the step runs, and the particle records (the mobility
    # observable) are copied into pinned host memory and decoded on the host;
    # two record buffers let step t + 1 run while step t's records are read
    e_host = torch.tensor(w["E"], dtype=torch.float64).pin_memory()
    e2e_steps = max(5, min(args.steps, 50))
    npart = s.num_particles()
    recbytes = npart * ctypes_sizeof_particle(ek)
    bufs = [torch.zeros(max(recbytes, 1), dtype=torch.uint8).pin_memory() for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    barrier()
    t0 = time.perf_counter()
    parts = []
    for t in range(e2e_steps):
        s.set_field(ek.FIELD_E_EXT, e_host)
        s.step_async(1)
        s.get_particles_async(bufs[t % 2])
        evs[t % 2].record(stream)
        if t > 0:
            evs[(t - 1) % 2].synchronize()
            parts = ek.particles_from_buffer(bufs[(t - 1) % 2], npart)
    evs[(e2e_steps - 1) % 2].synchronize()
    parts = ek.particles_from_buffer(bufs[(e2e_steps - 1) % 2], npart)
    s.sync()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = job_mlups(nodes, e2e_steps, ws, e2e_s * 1e3)
    h2d = 3 * 8
    d2h = len(parts) * ctypes_sizeof_particle(ek)

    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs"))

    def traffic(kernel):
        t = TRAFFIC[kernel]
        return t["bytes_per_launch"] if t["source_sha"] == src_sha(t["file"]) else None

    gbs32 = LB32_BYTES_PER_NODE * nodes / (r32["lb_ms"] / 1e3) / 1e9
    tflops64 = LB_FP64_FLOP_PER_NODE * nodes / (r64["lb_ms"] / 1e3) / 1e12
    gbs64 = LB_BYTES_PER_NODE * nodes / (r64["lb_ms"] / 1e3) / 1e9

    line = {
        "metric": METRIC, "value": round(r32["value"], 3), "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(r32["ms"] / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (int32 species, f64 particle sums)", "data": "synthetic",
        "config": {"workload": "single-sphere electrophoresis 128^3, R=8, Z=-300, 2 species, "
                               "E=0.005; FP32-storage form (FP64 form beside it)",
                   "nodes": nodes, "particles": len(w["particles"]),
                   "parallelism": "replicas" if ws > 1 else "single", "l2": FLUSH_NOTE},
        "roofline": {"bound": "hbm", "kernel": "k_lb32", "achieved": round(gbs32, 1),
                     "peak": hbm_peak, "unit": "GB/s", "frac": round(gbs32 / hbm_peak, 4),
                     "peak_kind": peak_kind, "traffic": traffic("k_lb32"),
                     "algorithmic_bytes": LB32_BYTES_PER_NODE * nodes,
                     "kernel_ms": round(r32["lb_ms"], 4)},
        "step_roofline": step_roofline(r32["value"], step_bytes_per_node(True, len(w["valence"])),
                                       hbm_peak),
        "stages_ms_per_step": r32["stages"],
        "fp64_form": {
            "value": round(r64["value"], 3), "unit": "MLUPS",
            "ms_per_step": round(r64["ms"] / args.steps, 4), "stages_ms_per_step": r64["stages"],
            "gpu_launches": r64["launches"], "clocks": r64["clocks"],
            "step_roofline": step_roofline(r64["value"], step_bytes_per_node(False, len(w["valence"])),
                                           hbm_peak),
            "roofline": {"bound": "alu", "kernel": "k_lb_fused", "achieved": round(tflops64, 4),
                         "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s (FP64)",
                         "frac": round(tflops64 / FP64_PEAK_TFLOPS, 4),
                         "traffic": traffic("k_lb_fused"),
                         "algorithmic_bytes": LB_BYTES_PER_NODE * nodes,
                         "hbm": {"achieved": round(gbs64, 1), "frac": round(gbs64 / hbm_peak, 4)},
                         "kernel_ms": round(r64["lb_ms"], 4)}},
        "speedup_vs_fp64": round(r32["value"] / r64["value"], 2),
        "e2e": {"value": round(e2e_value, 3), "unit": "MLUPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": r32["launches"],
        "clocks": r32["clocks"],
    }
    if rank == 0 and ws == 1 and not args.no_batch:
        line["poisson_mg"] = measure_poisson_mg(ek, torch)
    if rb is not None:
        rb["step_roofline"] = step_roofline(rb["value"], step_bytes_per_node(True, 2), hbm_peak)
        line["batched_form"] = rb
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, done, dt = time_oracle(w, 3, budget_s=20.0, warmup=0)
        line["cpu_baseline"] = {"value": round(v, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
                                "sample": f"{done} steps of the {w['shape'][0]}^3 workload, "
                                          f"{dt:.1f} s, numpy FP64 oracle, single thread"}
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
