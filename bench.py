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
    p.add_argument("--relax-chunks", type=int, default=20,
                   help="relaxation of the lattice start before anything is timed: chunks of 50 fine steps with "
                        "velocities rescaled to 300 K after each (0: start from the lattice)")
    p.add_argument("--nve-steps", type=int, default=200, help="NVE leg: FP32 and FP64 energy drift side by side")
    p.add_argument("--list-skin", type=float, default=0.0, help="Verlet-list skin (nm) of the timed FP32 run")
    p.add_argument("--cluster-pairs", type=int, default=0, help="short-range Coulomb pass of the timed FP32 run on cluster pairs")
    p.add_argument("--bricks", type=int, default=0, help="pair passes of the timed FP32 run on bricks of cells instead of 32-atom groups")
    p.add_argument("--mts-steps", type=int, default=200,
                   help="timed steps of the multiple-time-stepping leg (grid part every 2 and 4 steps; 0: skip)")
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


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), and its core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"model": name or "unknown", "host_cores": os.cpu_count()}


def cpu_thread_scaling(oracle, inputs, cfg):
    """The oracle on 1 thread and on all cores, on a bounded sample: a box of 1/16
    of the workload's atoms at its density and parameters.  The oracle's cost per
    atom grows with N (its O-O Lennard-Jones is an all-pairs loop, its top level
    dense), so the sample's rate is not the full box's: the full box is timed on
    all cores separately."""
    n_s = cfg["n_atoms"] // 16
    L = cfg["region"] if np.isscalar(cfg["region"]) else float(np.prod(cfg["region"])) ** (1 / 3)
    dens = cfg["n_atoms"] / L ** 3
    ss = inputs.water_box(n_s, (n_s / dens) ** (1 / 3), margin=1.0, seed=0, vel_seed=1)
    k = oracle.num_threads()
    out = {}
    for label, th in (("single_thread", 1), ("all_cores", k)):
        oracle.set_num_threads(th)
        t = time.perf_counter()
        oracle.model_forces(ss, A, H, cfg["levels"], **WALL)
        dt = time.perf_counter() - t
        out[label] = {"value": ss.n / dt, "unit": UNIT, "cores": th,
                      "sample": f"one oracle force evaluation of a {ss.n:,}-atom box of the workload's density "
                                f"({dt:.1f} s)"}
    oracle.set_num_threads(k)
    return out


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
    s0 = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=1.0, seed=0, vel_seed=1)
    n = s0.n
    stream = torch.cuda.current_stream()
    # relaxed start (not timed): the lattice start would time a ~900 K box
    t_relax = time.perf_counter()
    s = relaxed_state(api, inputs, s0, steps=a.relax_chunks, levels=cfg["levels"], torch=torch, dev=dev) \
        if a.relax_chunks > 0 else s0
    t_relax = time.perf_counter() - t_relax
    dof = 6 * s.n_mol + 3 * (s.n - 3 * s.n_mol)
    config["start"] = (f"relaxed: {a.relax_chunks} x 50 fine steps from the jittered lattice, velocities rescaled to "
                       f"300 K after each chunk (not timed)" if a.relax_chunks > 0 else "jittered lattice (unrelaxed)")

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- FP32 path: the timed run
    m32 = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp32", model="water", list_skin=a.list_skin,
                  cluster_pairs=bool(a.cluster_pairs), bricks=bool(a.bricks), **WALL)
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

    # ---- NVE: FP32 and FP64 paths side by side from the same relaxed state
    nve = None
    if a.nve_steps > 0:
        nve = {"steps": a.nve_steps, "dt_ps": DT, "start": config["start"]}
        for prec, mm in (("fp32", m32), ("fp64", m64)):
            dn = dev_system(torch, s, dev)
            ukn = mm.md_run(dn, DT, a.nve_steps, record=True).cpu().numpy()
            et = ukn.sum(1)
            nve[prec] = {"energy_drift_kj_mol": float(et[-1] - et[0]),
                         "max_abs_dev_kj_mol": float(np.abs(et - et[0]).max()),
                         "rel_drift_of_kinetic": float((et[-1] - et[0]) / ukn[:, 1].mean()),
                         "temperature_k": float(2 * ukn[:, 1].mean() / (dof * KB))}
            del dn

    # ---- multiple time stepping (grid part every k steps): step time and energy at outer steps
    mts = None
    if a.mts_steps > 0:
        mts = {"note": "impulse method: short range, LJ and wall every 2 fs step, the grid part every k steps "
                       "(Sec. 3); energy drift over the NVE leg's steps from the same relaxed state, total energy "
                       "at the ends of outer steps"}
        for k in (2, 4):
            mk = api.MSM(a=A, h=H, levels=cfg["levels"], precision="fp32", model="water", mts=k, **WALL)
            dk = dev_system(torch, s, dev)
            mk.md_run(dk, DT, 2 * k, record=False)
            torch.cuda.synchronize()
            nst = (a.mts_steps // k) * k
            e0.record(stream)
            mk.md_run(dk, DT, nst, record=False)
            e1.record(stream)
            torch.cuda.synchronize()
            tk = e0.elapsed_time(e1) / nst
            entry = {"ms_per_step": tk, "value": n / (tk / 1e3), "unit": UNIT, "speedup_vs_every_step": t_ms / a.steps / tk}
            if a.nve_steps > 0:
                dn = dev_system(torch, s, dev)
                ukn = mk.md_run(dn, DT, (a.nve_steps // k) * k, record=True).cpu().numpy()
                et = ukn.sum(1)[::k]
                entry.update({"energy_drift_kj_mol": float(et[-1] - et[0]),
                              "max_abs_dev_kj_mol": float(np.abs(et - et[0]).max()),
                              "temperature_k": float(2 * ukn[:, 1].mean() / (dof * KB))})
                del dn
            mts[f"k{k}"] = entry
            mk.close()
            del dk

    # ---- forces and energy at the start: FP32 and FP64 GPU paths against the FP64 oracle
    d0 = dev_system(torch, s, dev)
    u32, f32, _ = m32.system_forces(d0)
    u64, f64, _ = m64.system_forces(d0)
    u32, u64 = float(u32), float(u64)
    f32 = f32.cpu().numpy(); f64 = f64.cpu().numpy()
    frms64 = np.sqrt((f64 ** 2).sum(1).mean())
    err = {"fp32_vs_fp64_gpu": float(np.sqrt(((f32 - f64) ** 2).sum() / (f64 ** 2).sum())),
           "fp32_vs_fp64_gpu_max_atom_over_rms": float(np.linalg.norm(f32 - f64, axis=1).max() / frms64),
           "energy_rel_fp32_vs_fp64_gpu": abs(u32 - u64) / abs(u64)}
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
        err["fp32_vs_oracle_max_atom_over_rms"] = float(np.linalg.norm(f32 - fo, axis=1).max()
                                                        / np.sqrt((fo ** 2).sum(1).mean()))
        err["energy_rel_fp32_vs_oracle"] = abs(u32 - ref["energy"]) / abs(ref["energy"])
        err["energy_rel_fp64_vs_oracle"] = abs(u64 - ref["energy"]) / abs(ref["energy"])
        cpu_baseline = {"value": n / t_cpu, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                        "cpu_model": cpu_model(),
                        "sample": f"one oracle force evaluation (MSM + water completion, FP64, plain C, all cores) "
                                  f"of the full {n:,}-atom box at the start ({t_cpu:.1f} s); a step is this "
                                  f"evaluation plus O(N) integrator work"}
        cpu_baseline.update(cpu_thread_scaling(oracle, inputs, cfg))

    # ---- end to end: public API, one md_run call per step with the state (x, v) in pinned host
    # buffers, copied in and out by every call; the model's constant arrays (q, m, LJ flags) and
    # the carried forces stay on the device, as a host-driven MD loop keeps them
    hx = torch.tensor(s.pos).pin_memory().numpy()
    hv = torch.tensor(s.vel).pin_memory().numpy()
    dq = torch.tensor(s.q, dtype=torch.float64, device=dev)
    dm = torch.tensor(s.mass, dtype=torch.float64, device=dev)
    dl = torch.tensor(s.lj, device=dev)
    hs = inputs.System(pos=hx, q=dq, mass=dm, box=s.box, vel=hv, n_mol=s.n_mol, lj=dl)
    hs.force = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    m32.md_run(hs, DT, 1, record=True)            # warm: forces of the start state
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(a.e2e_steps):
        uk_h = m32.md_run(hs, DT, 1, record=True)  # x, v back in host memory; (U, K) to the host
    t_e2e_ms = max_over_ranks((time.perf_counter() - t) * 1e3, world, dev)
    e2e = {"value": whole_job_value(n, a.e2e_steps, world, t_e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": int(hx.nbytes + hv.nbytes),
           "d2h_bytes_per_step": int(hx.nbytes + hv.nbytes + 2 * 2 * 8),
           "resident": "q, m, LJ flags and the carried forces (device arrays, uploaded once)"}

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
                     "pairs_per_s": pairs / sr_avg_s, "unique_pairs_per_s": 0.5 * pairs / sr_avg_s,
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
        "timed_run_energy": {"steps": a.steps, "energy_drift_kj_mol": drift,
                             "max_abs_dev_kj_mol": float(np.abs(etot - etot[0]).max()),
                             "kinetic_kj_mol": float(uk[-1, 1]),
                             "temperature_k": float(2 * uk[:, 1].mean() / (dof * KB))},
        "nve": nve,
        "mts": mts,
        "relax_s": t_relax,
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


def relaxed_state(api, inputs, s, steps=40, chunk=50, temp=300.0, levels=3, torch=None, dev=None):
    """The jittered-lattice start relaxes violently (the potential energy falls by
    ~10^5 kJ/mol in the first picoseconds, heating a 1M-atom box to ~900 K).
    Runs are timed from a relaxed state: `steps` x `chunk` fine steps with the
    velocities rescaled to `temp` between chunks (a plain velocity-rescaling
    thermostat; not timed).  Returns a host System."""
    dof = 6 * s.n_mol + 3 * (s.n - 3 * s.n_mol)
    m = api.MSM(a=A, h=H, levels=levels, precision="fp32", model="water", **WALL)
    if torch is not None:
        d = dev_system(torch, s, dev)
        for _ in range(steps):
            uk = m.md_run(d, DT, chunk)
            k = float(uk[-1, 1])
            d.vel.mul_(float(np.sqrt(0.5 * dof * KB * temp / k)))
        torch.cuda.synchronize()
        out = inputs.System(pos=d.pos.cpu().numpy(), q=s.q, mass=s.mass, box=s.box, vel=d.vel.cpu().numpy(),
                            n_mol=s.n_mol, lj=s.lj)
    else:
        out = inputs.System(pos=s.pos.copy(), q=s.q, mass=s.mass, box=s.box, vel=s.vel.copy(), n_mol=s.n_mol,
                            lj=s.lj)
        for _ in range(steps):
            uk = m.md_run(out, DT, chunk)
            out.vel *= np.sqrt(0.5 * dof * KB * temp / uk[-1, 1])
    m.close()
    return out


# coarse propagators of the parareal leg: the configured MSM G (shorter cutoff, coarser
# grid, longer step: Sec. 5's "shorter cutoff" and "coarse grid") and the two cutoff
# methods Sec. 5 keeps, the simple cutoff (its chosen G; also at the fine propagator's
# own cutoff, as in the paper's 12 A example) and Wolf summation
COARSE = {
    "msm_a0.8_h0.5": dict(a=0.8, h=0.5, levels=2, method="msm"),
    "cutoff_a0.8": dict(a=0.8, h=0.5, levels=1, method="cutoff"),
    "cutoff_a1.2": dict(a=1.2, h=0.5, levels=1, method="cutoff"),
    "wolf_a0.8": dict(a=0.8, h=0.5, levels=1, method="wolf", wolf_alpha=2.5),
}


def _step_ms(torch, api, s, dev, p, dt, steps=50):
    """CUDA-event time per md step of one propagator on one system (graph-replayed)."""
    m = api.MSM(a=p["a"], h=p["h"], levels=p["levels"], precision="fp32", model="water",
                method=p.get("method", "msm"), wolf_alpha=p.get("wolf_alpha", 0.0), **WALL)
    d = dev_system(torch, s, dev)
    m.md_run(d, dt, 3, record=False)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    m.md_run(d, dt, steps, record=False)
    e1.record(stream)
    torch.cuda.synchronize()
    m.close()
    return e0.elapsed_time(e1) / steps


def run_parareal_leg(a, torch, api, inputs, dev):
    """Parareal on the 10,000-atom box from a relaxed 300 K state: 32 slices of
    50 fine steps (a = 1.2 nm, h = 0.25 nm, 3 levels, 2 fs) corrected by a coarse
    propagator at 4 fs -- the configured MSM G (a = 0.8 nm, h = 0.5 nm, 2 levels),
    the paper's simple cutoff (a = 0.8 nm) and Wolf summation (a = 0.8 nm,
    alpha = 2.5/nm) -- FP32 bulk with FP64 corrections, iterated until max |dx| <=
    1e-6 nm (at the latest after 32 iterations, when every slice is exact),
    against the serial fine trajectory; the same with 4 fine steps per slice; and
    the simple cutoff G over a sliding window of 8 slices."""
    s0 = inputs.water_box(10_000, 4.65, margin=1.0, seed=0, vel_seed=1)
    s = relaxed_state(api, inputs, s0)
    n_slices, tol = 32, 1e-6
    out = {"atoms": s.n, "slices": n_slices, "tol_nm": tol,
           "start": "relaxed: 4 ps of fine dynamics with velocities rescaled to 300 K every 0.1 ps"}
    stream = torch.cuda.current_stream()
    Fp = dict(a=1.2, h=0.25, levels=3)
    # cost ratio Q_F/G of the paper's model (Sec. 6.1.3), measured as time per slice:
    # one fine step at 2 fs against the coarse steps covering the same time at 4 fs
    tf = _step_ms(torch, api, s, dev, Fp, 0.002)
    out["fine_step_ms"] = tf
    out["q_f_over_g"] = {}
    for gname, gp in COARSE.items():
        tg = _step_ms(torch, api, s, dev, gp, 0.004)
        out["q_f_over_g"][gname] = {"coarse_step_ms": tg, "measured": 2 * tf / tg,
                                    "paper": "453 (Sec. 6.1.3: simple cutoff 12 A vs MSM a = 12 A, h = 2 A, "
                                             "flop counts, no hardware)"}
    for fsteps in (50, 4):
        F = dict(Fp, dt=0.002, steps=fsteps, **WALL)
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
        runs = [(g, None) for g in COARSE] + ([("cutoff_a0.8", 8)] if fsteps == 50 else [])
        for gname, window in runs:
            G = dict(COARSE[gname], dt=0.004, steps=fsteps // 2, **WALL)
            hs = inputs.System(pos=s.pos.copy(), q=s.q, mass=s.mass, box=s.box, vel=s.vel.copy(),
                               n_mol=s.n_mol, lj=s.lj)
            t = time.perf_counter()
            try:
                xs, vs, it, dx, conv = api.parareal_run(G, F, hs, n_slices, n_slices, tol, precision="fp32",
                                                        window=window)
            except api.MSMError as err:
                out[f"fine_steps_{fsteps}/{gname}"] = {"error": str(err)}
                continue
            t_par = time.perf_counter() - t
            key = f"fine_steps_{fsteps}/{gname}" + (f"/window_{window}" if window else "")
            out[key] = {"iterations": it, "converged": bool(conv), "last_max_dx_nm": dx,
                        "max_error_vs_serial_nm": float(np.abs(xs - serial).max()),
                        "serial_fine_s": t_serial, "parareal_s": t_par, "speedup": t_serial / t_par}
    out["note"] = ("speedup = serial fine time / parareal time, both on this one GPU; F of all open slices runs "
                   "as one batch, G slice by slice with no host synchronisation inside a sweep; q_f_over_g = time "
                   "of one fine step x 2 / one coarse step (the coarse step is twice as long)")
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
    """The FP64 CPU oracle, as it stands, timed on this machine's host cores on the
    workload itself: a step is one oracle force evaluation of the full box (the
    oracle's cost per atom grows with N -- its O-O Lennard-Jones is an all-pairs
    loop and its top level dense -- so a smaller box would not stand for it).  One
    untimed evaluation is the warm-up and sizes the run: at most --steps
    evaluations are timed, as many as fit in about 150 s (at least one)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle
    from paper_1309_1889_gb300 import inputs

    oracle.build()
    cfg, config = workload_config(a.workload)
    s = inputs.water_box(cfg["n_atoms"], cfg["region"], margin=1.0, seed=0, vel_seed=1)
    config["start"] = "jittered lattice (the oracle's cost does not depend on the state)"
    budget_s = 150.0
    t = time.perf_counter()
    oracle.model_forces(s, A, H, cfg["levels"], **WALL)           # warm-up, and the step's duration
    t1 = time.perf_counter() - t
    steps = max(1, min(a.steps, int(budget_s // max(t1, 1e-9))))
    t = time.perf_counter()
    for _ in range(steps):
        oracle.model_forces(s, A, H, cfg["levels"], **WALL)
    dt = time.perf_counter() - t
    value = s.n * steps / dt
    sample = (f"{steps} oracle force evaluation(s) (MSM + water completion, FP64, plain C, all cores) of the full "
              f"{s.n:,}-atom box, {dt / steps:.1f} s each; a step of the workload is this evaluation plus O(N) "
              f"integrator work; 1 untimed warm-up evaluation")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": 1,
            "steps_requested": a.steps, "warmup_requested": a.warmup,
            "ms_per_step": dt / steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": config, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": sample},
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
