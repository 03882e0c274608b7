#!/usr/bin/env python3
"""Throughput of the MSM velocity-Verlet step on GB300.

One step = one velocity-Verlet step of the rigid-water workload through the
whole hot path: bit-exact binning and sort, short-range g* sum (+ O-O LJ of the
water completion), anterpolation, restriction and lattice cutoff on every
level, FP64 top level, prolongation, interpolation, exclusions, FP64 energy
reductions, half kicks and SHAKE/RATTLE.

Workload: 1,000,000 atoms (333,333 rigid 3-site water-like molecules + 1
filler site) in a 21.5 nm cube (+1 nm margin with a flat-bottom wall), a =
1.2 nm, h = 0.25 nm, 5 levels, dt = 2 fs, 1000 NVE steps by default.  Inputs are resident in HBM when the timed region
starts; the working set (~0.3 GB) is larger than L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own replica
of the workload (the path does not shard; "replicas only").  Besides the timed
1M-atom run the line carries the FP64 GPU path, the force error against the
oracle, an end-to-end run through host buffers, the uneven 7-box batch and the
10,000-atom parareal run.
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
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "MSM atom-steps/s @1M atoms, FP32 batched vs plain FP64 GPU at force err ≤1e-4"
UNIT = "atom-steps/s"
A, H, DT = 1.2, 0.25, 0.002
WALL = dict(wall_k=1.0e4, wall_width=0.8)     # flat-bottom wall of the water completion (1 nm margin)
FLOPS_PER_PAIR = 29          # algorithmic FP32 flops per ordered in-cutoff pair (FMA = 2)
FP32_LANES_PER_SM = 128


def args_parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="water1M")
    p.add_argument("--fp64-steps", type=int, default=3)
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--no-oracle", action="store_true", help="skip the oracle force error and CPU baseline")
    p.add_argument("--profile-steps", type=int, default=30, help="eager profiled steps after the timed region")
    p.add_argument("--batch-steps", type=int, default=100, help="steps of the uneven 7-box batch (0: skip)")
    p.add_argument("--parareal", type=int, default=1, help="run the 10,000-atom parareal leg (0: skip)")
    p.add_argument("--paper-scale", type=int, default=0,
                   help="run the 12.7 M-atom leg: one evaluation plus an 8-slice parareal run (1: run)")
    return p.parse_args()


def workload_config(name):
    from paper_1309_1889_gb300 import inputs
    cfg = dict(inputs.WORKLOADS[name])
    region = cfg["region"]
    return cfg, {
        "workload": f"{name}: {cfg['n_atoms']:,} atoms of rigid 3-site water-like molecules "
                    f"(O -0.834 e, H +0.417 e) in a {region} nm box + 1 nm margin, open boundaries",
        "a_nm": A, "h_nm": H, "levels": cfg["levels"], "dt_ps": DT, "ensemble": "NVE",
        "precision": "FP32 pair/grid/stencil arithmetic, FP64 state, top level and reductions",
        "l2": "no flush: working set (~0.3 GB) larger than the 129 MB L2",
        "parallelism": "replicas",
    }


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if bus_id:
            cmd += ["--id=" + bus_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        rows = []
        for line in Path(self.f.name).read_text().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append(dict(t=ts, sm=float(parts[2]), smax=float(parts[3]),
                                 reasons={"hw_slowdown": parts[6], "hw_thermal_slowdown": parts[7],
                                          "sw_thermal_slowdown": parts[8], "sw_power_cap": parts[9]}))
            except (ValueError, IndexError):
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        inside = [r for r in rows if self.t0 is not None and self.t0 - 1.0 <= r["t"] <= self.t1 + 1.0] or rows
        reasons = sorted({k for r in inside for k, v in r["reasons"].items() if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r["sm"] for r in inside), "sm_max_mhz": max(r["smax"] for r in inside),
                "reasons": reasons, "samples": len(inside)}


# ---------------------------------------------------------------- helpers

def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return json.loads(p.read_text())
    return {}


def short_range_traffic(n_launch_atoms):
    """Per-launch DRAM traffic of the short-range kernel from the committed ncu summary,
    or None if the kernel source changed since the counters were taken."""
    f = ROOT / "profiles" / "short_range_water1M_traffic.json"
    if not f.exists():
        return None
    rec = json.loads(f.read_text())
    src = ROOT / "paper_1309_1889_gb300" / "csrc" / "k_short.cu"
    if hashlib.sha256(src.read_bytes()).hexdigest() != rec.get("source_sha256"):
        return None
    return rec["dram_bytes_per_atom"] * n_launch_atoms


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(t_ms, world, device):
    """The job's time: the largest of the ranks' times (one all_reduce; the value itself at N = 1)."""
    if world == 1:
        return t_ms
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(n_atoms, steps, world, t_ms):
    """Atom-steps per second of the whole job: every rank's replica over the slowest rank's time."""
    return n_atoms * steps * world / (t_ms / 1e3)


def dev_system(torch, s, dev):
    from paper_1309_1889_gb300 import inputs
    t = lambda x: torch.tensor(np.asarray(x), dtype=torch.float64, device=dev)
    return inputs.System(pos=t(s.pos), q=t(s.q), mass=t(s.mass), box=s.box, vel=t(s.vel), n_mol=s.n_mol,
                         lj=torch.tensor(s.lj, device=dev))


# ------------------------------------------------------------------- ours

def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_1309_1889_gb300 import api, inputs

    rank, world, local = env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg, config = workload_config(a.workload)
    s = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=1.0, seed=0, vel_seed=1)
    n = s.n
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- FP32 path: the timed run
    m32 = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp32", model="water", **WALL)
    d = dev_system(torch, s, dev)
    m32.md_run(d, DT, a.warmup, record=False)
    torch.cuda.synchronize()
    bus = None
    try:
        bus = torch.cuda.get_device_properties(dev).pci_bus_id if hasattr(torch.cuda.get_device_properties(dev), "pci_bus_id") else None
    except Exception:
        bus = None
    clocks = ClockSampler(bus) if rank == 0 else None
    time.sleep(0.5 if clocks else 0)
    l0 = api.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.mark_start()
    ev0.record(stream)
    uk = m32.md_run(d, DT, a.steps, record=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    if clocks:
        clocks.mark_end()
    launches = api.kernel_launches() - l0
    t_ms = ev0.elapsed_time(ev1)
    # per-stage CUDA-event times: the same trajectory continued for a few eager
    # (profiled, graph-free) steps right after the timed region
    m32.profile(True)
    m32.profile_read(reset=True)
    m32.md_run(d, DT, a.profile_steps, record=True)
    torch.cuda.synchronize()
    m32.profile(False)
    prof = m32.profile_read(reset=True)
    t_prof = sum(v[0] for v in prof.values())
    t_ms = max_over_ranks(t_ms, world, dev)
    clk = clocks.stop() if clocks else None
    uk = uk.cpu().numpy()
    etot = uk.sum(1)
    pairs = m32.count_pairs()

    value = whole_job_value(n, a.steps, world, t_ms)

    # ---- FP64 path on the same start state
    m64 = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp64", model="water", **WALL)
    d64 = dev_system(torch, s, dev)
    m64.md_run(d64, DT, 1, record=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    m64.md_run(d64, DT, a.fp64_steps, record=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1)
    value64 = n * a.fp64_steps / (t64 / 1e3)

    # ---- forces at t = 0: FP32 and FP64 GPU paths against the FP64 oracle
    d0 = dev_system(torch, s, dev)
    _, f32, _ = m32.system_forces(d0)
    _, f64, _ = m64.system_forces(d0)
    f32 = f32.cpu().numpy(); f64 = f64.cpu().numpy()
    err = {"fp32_vs_fp64_gpu": float(np.sqrt(((f32 - f64) ** 2).sum() / (f64 ** 2).sum()))}
    cpu_baseline = None
    if rank == 0 and not a.no_oracle:
        import oracle
        oracle.build()
        t = time.perf_counter()
        ref = oracle.model_forces(s, A, H, cfg["levels"], **WALL)
        t_cpu = time.perf_counter() - t
        fo = ref["forces"]
        den = np.sqrt((fo ** 2).sum())
        err["fp32_vs_oracle"] = float(np.sqrt(((f32 - fo) ** 2).sum()) / den)
        err["fp64_vs_oracle"] = float(np.sqrt(((f64 - fo) ** 2).sum()) / den)
        cpu_baseline = {"value": n / t_cpu, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                        "sample": f"one oracle force evaluation (MSM + water completion, FP64, plain C) of the "
                                  f"full {n:,}-atom box at t = 0 ({t_cpu:.1f} s); a step is this evaluation plus "
                                  f"O(N) integrator work"}

    # ---- end to end: public API with pinned host buffers, forces carried between calls
    hx = torch.tensor(s.pos).pin_memory().numpy()
    hv = torch.tensor(s.vel).pin_memory().numpy()
    hf = torch.zeros((n, 3), dtype=torch.float64).pin_memory().numpy()
    hq = torch.tensor(s.q).pin_memory().numpy()
    hm = torch.tensor(s.mass).pin_memory().numpy()
    hl = torch.tensor(s.lj).pin_memory().numpy()
    hs = inputs.System(pos=hx, q=hq, mass=hm, box=s.box, vel=hv, n_mol=s.n_mol, lj=hl)
    hs.force = hf
    m32.md_run(hs, DT, 1, record=True)            # warm: forces of the start state
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(a.e2e_steps):
        m32.md_run(hs, DT, 1, record=True)
    t_e2e_ms = max_over_ranks((time.perf_counter() - t) * 1e3, world, dev)
    e2e = {"value": whole_job_value(n, a.e2e_steps, world, t_e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": int(hx.nbytes + hv.nbytes + hf.nbytes + hq.nbytes + hm.nbytes + hl.nbytes),
           "d2h_bytes_per_step": int(hx.nbytes + hv.nbytes + hf.nbytes + 2 * 2 * 8)}

    batched = run_batch_leg(a, torch, api, inputs, dev) if a.batch_steps > 0 else None
    parareal = run_parareal_leg(a, torch, api, inputs, dev) if a.parareal else None
    paper_scale = run_paper_scale_leg(a, torch, api, inputs, dev) if a.paper_scale else None

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (short range): FP32 ALU bound
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = sm_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    sr_ms, sr_n = prof["short_range"]
    sr_avg_s = sr_ms / sr_n / 1e3
    achieved = pairs * FLOPS_PER_PAIR / sr_avg_s / 1e12
    traffic = short_range_traffic(n)
    # second stage: the lattice cutoff, FP32 ALU bound (2 flops per tap inside the sphere |n| h < 2a,
    # per point of levels 0..l-2; the kernel issues about half of them, rows +-dy sharing a weight row)
    rad = int(np.ceil(2 * A / H))
    rng_ = np.arange(-rad, rad + 1)
    dx_, dy_, dz_ = np.meshgrid(rng_, rng_, rng_, indexing="ij")
    taps = int((np.sqrt(dx_ ** 2 + dy_ ** 2 + dz_ ** 2) * H < 2 * A).sum())
    st_points = sum(int(np.prod(m32.grid_shape(k)[0])) for k in range(cfg["levels"] - 1))
    st_ms, st_n = prof["lattice_cutoff"]
    st_avg_s = st_ms / st_n / 1e3
    st_achieved = 2 * taps * st_points / st_avg_s / 1e12
    stage_ms = {k: round(v[0] / max(v[1], 1), 4) for k, v in prof.items() if v[1]}
    step_share = {k: round(v[0] / t_prof, 4) for k, v in prof.items() if v[1]}
    drift = float(etot[-1] - etot[0])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": t_ms / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic", "config": config,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved / peak_tflops, "traffic": traffic,
                     "kernel": "k_short (short-range g* sum)",
                     "peak_source": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz "
                                    "(max SM clock from MEASURED_PEAKS.json)",
                     "work": f"{pairs} ordered pairs within a per launch x {FLOPS_PER_PAIR} flops",
                     "duration": f"{sr_avg_s * 1e3:.4f} ms average of {sr_n} launches (CUDA events on the "
                                 f"launching stream, {a.profile_steps} eager steps continuing the timed run)"},
        "roofline_lattice_cutoff": {"bound": "alu", "achieved": st_achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                                    "frac": st_achieved / peak_tflops, "kernel": "k_stencil (levels 0..l-2)",
                                    "work": f"{taps} taps x 2 flops x {st_points} grid points per launch",
                                    "duration": f"{st_avg_s * 1e3:.4f} ms average of {st_n} launches"},
        "cpu_baseline": cpu_baseline,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "fp64_gpu": {"value": value64, "unit": UNIT, "steps": a.fp64_steps, "ms_per_step": t64 / a.fp64_steps,
                     "fp32_speedup": value / world / value64},
        "force_error": err,
        "nve": {"steps": a.steps, "energy_drift_kj_mol": drift,
                "max_abs_dev_kj_mol": float(np.abs(etot - etot[0]).max()), "kinetic_kj_mol": float(uk[-1, 1])},
        "stage_ms_per_launch": stage_ms,
        "stage_share_of_step": step_share,
        "timed_region": ("CUDA-graph replay of every step after the first (profiler off; the grid chain runs on a "
                         "second stream beside the pair kernels); stage times come from a serialised profiled pass"),
        "uneven_batch": batched,
        "parareal": parareal,
    }
    if paper_scale is not None:
        line["paper_scale"] = paper_scale
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------ extra legs

BATCH_SIZES = (20_000, 50_000, 100_000, 150_000, 200_000, 230_000, 250_000)


def run_batch_leg(a, torch, api, inputs, dev):
    """The uneven batch: 7 independent water boxes (20k ... 250k atoms, 1.02 M in
    total, density of the 1M box) stepped together, one launch per stage."""
    dens = 1_000_000 / 21.5 ** 3
    boxes = [inputs.water_box(n, (n / dens) ** (1 / 3), margin=1.0, seed=100 + k, vel_seed=200 + k)
             for k, n in enumerate(BATCH_SIZES)]
    m = api.MSM(a=A, h=H, levels=5, precision="fp32", model="water", **WALL)
    devs = [dev_system(torch, s, dev) for s in boxes]
    m.md_run_batched(devs, DT, 5, record=False)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = api.kernel_launches()
    e0.record(stream)
    uk = m.md_run_batched(devs, DT, a.batch_steps, record=True)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1)
    launches = api.kernel_launches() - l0
    n = sum(s.n for s in boxes)
    etot = uk.sum(-1).cpu().numpy()
    return {"value": n * a.batch_steps / (t / 1e3), "unit": UNIT, "atoms": n, "systems": list(BATCH_SIZES),
            "steps": a.batch_steps, "ms_per_step": t / a.batch_steps, "gpu_launches": launches,
            "launches_per_step": launches / a.batch_steps,
            "max_energy_drift_kj_mol": float(np.abs(etot[:, -1] - etot[:, 0]).max()),
            "layout": "one launch per stage for all 7 systems; steps after the first replay a CUDA graph"}


KB = 0.0083144626              # kJ/mol/K


def relaxed_state(api, inputs, s, steps=40, chunk=50, temp=300.0):
    """The jittered-lattice start relaxes violently (the potential energy falls by
    ~10^5 kJ/mol in the first picoseconds).  Parareal is run from a relaxed state:
    `steps` x `chunk` fine steps with the velocities rescaled to `temp` between
    chunks (a plain velocity-rescaling thermostat; not timed)."""
    dof = 6 * s.n_mol + 3 * (s.n - 3 * s.n_mol)
    m = api.MSM(a=A, h=H, levels=3, precision="fp32", model="water", **WALL)
    hs = inputs.System(pos=s.pos.copy(), q=s.q, mass=s.mass, box=s.box, vel=s.vel.copy(), n_mol=s.n_mol, lj=s.lj)
    for _ in range(steps):
        uk = m.md_run(hs, DT, chunk)
        hs.vel *= np.sqrt(0.5 * dof * KB * temp / uk[-1, 1])
    return hs


def run_parareal_leg(a, torch, api, inputs, dev):
    """Parareal on the 10,000-atom box from a relaxed 300 K state: 32 slices of
    50 fine steps (a = 1.2 nm, h = 0.25 nm, 3 levels, 2 fs) corrected by the
    coarse propagator (a = 0.8 nm, h = 0.5 nm, 2 levels, 4 fs), FP32 bulk with
    FP64 corrections, iterated until max |dx| <= 1e-6 nm (at the latest after 32
    iterations, when every slice is exact), against the serial fine trajectory;
    and the same with 4 fine steps per slice."""
    s0 = inputs.water_box(10_000, 4.65, margin=1.0, seed=0, vel_seed=1)
    s = relaxed_state(api, inputs, s0)
    n_slices, tol = 32, 1e-6
    out = {"atoms": s.n, "slices": n_slices, "tol_nm": tol,
           "start": "relaxed: 2 ps of fine dynamics with velocities rescaled to 300 K every 0.1 ps"}
    stream = torch.cuda.current_stream()
    for fsteps in (50, 4):
        F = dict(a=1.2, h=0.25, levels=3, dt=0.002, steps=fsteps, **WALL)
        G = dict(a=0.8, h=0.5, levels=2, dt=0.004, steps=fsteps // 2, **WALL)
        mf = api.MSM(a=F["a"], h=F["h"], levels=F["levels"], precision="fp32", model="water", **WALL)
        d = dev_system(torch, s, dev)
        mf.md_run(d, F["dt"], 2, record=False)                  # warm (graph capture, autotune)
        d = dev_system(torch, s, dev)
        serial = [d.pos.clone()]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n_slices):
            mf.md_run(d, F["dt"], F["steps"], record=False)
            serial.append(d.pos.clone())
        e1.record(stream)
        torch.cuda.synchronize()
        t_serial = e0.elapsed_time(e1) / 1e3
        serial = torch.stack(serial).cpu().numpy()
        hs = inputs.System(pos=s.pos.copy(), q=s.q, mass=s.mass, box=s.box, vel=s.vel.copy(), n_mol=s.n_mol,
                           lj=s.lj)
        t = time.perf_counter()
        xs, vs, it, dx, conv = api.parareal_run(G, F, hs, n_slices, n_slices, tol, precision="fp32")
        t_par = time.perf_counter() - t
        out[f"fine_steps_{fsteps}"] = {
            "iterations": it, "converged": bool(conv), "last_max_dx_nm": dx,
            "max_error_vs_serial_nm": float(np.abs(xs - serial).max()),
            "serial_fine_s": t_serial, "parareal_s": t_par, "speedup": t_serial / t_par}
    out["note"] = ("speedup = serial fine time / parareal time, both on this one GPU; F of all open slices runs "
                   "as one batch, G slice by slice")
    return out


def run_paper_scale_leg(a, torch, api, inputs, dev):
    """The paper-scale box: 12.7 M atoms of the water-like model in a 30 x 65 x 65 nm
    box, a = 1.2 nm, h = 0.25 nm, 6 levels, FP32 bulk with FP64 reductions.  One
    evaluation (timed, with the device memory in use), then an 8-slice parareal run
    of 20 fine steps per slice with the 10,000-atom leg's coarse propagator
    (a = 0.8 nm, h = 0.5 nm, 2 levels, 4 fs) against the serial fine trajectory, from
    a state relaxed by 5 x 20 fine steps with velocities rescaled to 300 K."""
    cfg = inputs.WORKLOADS["water12.7M"]
    s0 = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=1.0, seed=0, vel_seed=1)
    out = {"atoms": s0.n, "box_nm": [float(v) for v in s0.box[3:]], "levels": cfg["levels"]}
    stream = torch.cuda.current_stream()
    free0 = torch.cuda.mem_get_info()[0]
    m = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp32", model="water", **WALL)
    d = dev_system(torch, s0, dev)
    m.system_forces(d)                                          # sizes buffers, autotunes
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    e, _, _ = m.system_forces(d)
    e1.record(stream)
    torch.cuda.synchronize()
    out["evaluation_ms"] = e0.elapsed_time(e1)
    out["energy_kj_mol"] = float(e)
    out["device_gb_one_system"] = (free0 - torch.cuda.mem_get_info()[0]) / 1e9
    del m, d
    # relax the lattice start (not timed), as the 10,000-atom leg does
    dof = 6 * s0.n_mol + 3 * (s0.n - 3 * s0.n_mol)
    mf = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp32", model="water", **WALL)
    hs = inputs.System(pos=s0.pos.copy(), q=s0.q, mass=s0.mass, box=s0.box, vel=s0.vel.copy(), n_mol=s0.n_mol,
                       lj=s0.lj)
    for _ in range(5):
        uk = mf.md_run(hs, DT, 20)
        hs.vel *= np.sqrt(0.5 * dof * KB * 300.0 / uk[-1, 1])
    n_slices, fsteps, tol = 8, 20, 1e-6
    F = dict(a=A, h=H, levels=cfg["levels"], dt=DT, steps=fsteps, **WALL)
    G = dict(a=0.8, h=0.5, levels=2, dt=2 * DT, steps=fsteps // 2, **WALL)
    d = dev_system(torch, hs, dev)
    serial = [d.pos.clone()]
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n_slices):
        mf.md_run(d, F["dt"], F["steps"], record=False)
        serial.append(d.pos.clone())
    e1.record(stream)
    torch.cuda.synchronize()
    t_serial = e0.elapsed_time(e1) / 1e3
    del mf, d
    t = time.perf_counter()
    free1 = torch.cuda.mem_get_info()[0]
    try:
        xs, vs, it, dx, conv = api.parareal_run(G, F, hs, n_slices, n_slices, tol, precision="fp32")
    except api.MSMError as err:
        out["parareal"] = {"error": str(err)}
        return out
    t_par = time.perf_counter() - t
    err_nm = max(float((torch.from_numpy(xs[k]).to(dev) - serial[k]).abs().max()) for k in range(n_slices + 1))
    out["parareal"] = {"slices": n_slices, "fine_steps": fsteps, "iterations": it, "converged": bool(conv),
                       "last_max_dx_nm": dx, "max_error_vs_serial_nm": err_nm, "serial_fine_s": t_serial,
                       "parareal_s": t_par, "speedup": t_serial / t_par,
                       "device_gb_free_before": free1 / 1e9}
    return out


# -------------------------------------------------------------- reference

def run_reference(a):
    """The FP64 CPU oracle, as it stands, timed on this machine's host cores."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle
    from paper_1309_1889_gb300 import inputs

    oracle.build()
    cfg, config = workload_config(a.workload)
    # Each step is a bounded sample of the workload: one oracle force evaluation of a smaller
    # box of the same density and parameters (the cost per atom does not depend on the size).
    budget_s = 150.0
    n_s = 20_000
    L = cfg["region"] if np.isscalar(cfg["region"]) else float(np.prod(cfg["region"])) ** (1 / 3)
    dens = cfg["n_atoms"] / (L ** 3)

    def make(n):
        return inputs.water_box(n, (n / dens) ** (1 / 3), margin=1.0, seed=0, vel_seed=1)

    s = make(n_s)
    t = time.perf_counter()
    oracle.model_forces(s, A, H, cfg["levels"], **WALL)
    t1 = time.perf_counter() - t
    steps = a.steps + a.warmup
    if t1 * steps > budget_s:
        n_s = max(3000, int(n_s * budget_s / (t1 * steps)))
        s = make(n_s)
    for _ in range(a.warmup):
        oracle.model_forces(s, A, H, cfg["levels"], **WALL)
    t = time.perf_counter()
    for _ in range(a.steps):
        oracle.model_forces(s, A, H, cfg["levels"], **WALL)
    dt = time.perf_counter() - t
    value = s.n * a.steps / dt
    sample = (f"one oracle force evaluation per step (MSM + water completion, FP64, plain C) of a "
              f"{s.n:,}-atom box of the workload's density and parameters")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
