"""Benchmark: MLUPS and fraction of the HBM roofline of the stream-collide step.

Workload (default): the turbulent channel of the paper's Sec. 5.1 benchmark class, as a
synthetic stand-in: 512 x 256 x 256 cells, D3Q19 TRT + Smagorinsky (C_s = 0.1), float32
populations, walls at the y faces, periodic x/z, body force for Re_tau ~ 180, initial
state = equilibrium of the seeded perturbed parabola.  One step = one lattice update of
every cell (one kernel launch; two-grid pull streaming by default, the in-place AA pattern
is reported as a form).  MLUPS counts all cells, like the paper (Sec. 5.2).

Roofline (Sec. 5.2, Eq. roofline: P_max = b_s / n_b): n_b = 2 q s + 1 bytes per update
(q populations of s bytes read and written, one flag byte), b_s = the measured copy
bandwidth of this GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torchrun): every rank runs an independent replica (the method needs no
exchange on one lattice per GPU; "replicas only"), barrier + max over ranks.
--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the
same workload (128 x 64 x 64 sub-lattice).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS & % of HBM roofline per form (FP32/FP16/MLP closure) at stated error"
FALLBACK_HBM_GBS = 6800.0
WORKLOAD = "turbulent channel 512x256x256 D3Q19 TRT+Smagorinsky FP32 (two-grid pull)"
FACES_CHANNEL = ("periodic", "periodic", "wall", "wall", "periodic", "periodic")


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _profile_value(kernel_tag, key):
    """A value ("- key: `v`" line) of the committed ncu summary of this kernel, if it was taken
    on step kernels identical to the ones running now (same kernel-source hash); else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    try:
        stamp = open(os.path.join(ROOT, "paper_2305_09910_gb300", "liblbm.so.kernel.sha256")).read().strip()
    except OSError:
        return None
    if vals.get("kernel_sha256") != stamp:
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def _profile_traffic(kernel_tag):
    """Per-launch DRAM bytes (read + write) from the committed ncu summary, or None."""
    return _profile_value(kernel_tag, "dram_bytes_per_launch")


SMS, SCHEDULERS = 152, 4  # GB300: 4 warp schedulers per SM, each issuing one warp instruction per clock


def _issue_roofline(mlups, inst_per_cell, sm_mhz, hbm):
    """Instruction-issue roofline of a kernel bound by its arithmetic: achieved thread
    instructions per second (instructions per cell from the ncu summary of the same kernel x
    cell updates per second) against SMs x 4 schedulers x 32 lanes x the SM clock."""
    peak = SMS * SCHEDULERS * 32 * sm_mhz * 1e6 / 1e9
    if inst_per_cell is None:
        return {"bound": "issue", "achieved": None, "peak": round(peak, 1), "unit": "Ginst/s", "frac": None,
                "traffic": None, "inst_per_cell": None, "sm_mhz": sm_mhz,
                "note": "no ncu instruction count taken on this kernel build", "hbm": hbm}
    achieved = inst_per_cell * mlups * 1e6 / 1e9
    return {"bound": "issue", "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "Ginst/s",
            "frac": round(achieved / peak, 4), "traffic": None, "inst_per_cell": inst_per_cell, "sm_mhz": sm_mhz,
            "hbm": hbm}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.rows = []
        self.proc = None
        self.active = False
        self.lock = threading.Lock()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            with self.lock:
                if self.active:
                    self.rows.append([s.strip() for s in line.split(",")])

    def start(self):
        with self.lock:
            self.active = True

    def stop(self):
        with self.lock:
            self.active = False
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(num(r[2]) or 0 for r in rows),
                "power_w_max": max(num(r[3]) or 0 for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1, 0
    import torch
    import torch.distributed as dist

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl")
    return dist, dist.get_rank(), ws, local


def _barrier_max(dist, value):
    """Maximum of a per-rank value over the ranks (device tensor under NCCL, host under gloo)."""
    if dist is None:
        return value
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _channel_lattice(nx, ny, nz, precision, closure="smag", streaming="pull", collision="trt"):
    import torch

    from paper_2305_09910_gb300 import inputs, lbm

    par = inputs.channel_parameters(ny)
    lat = lbm.Lattice(nx, ny, nz, stencil=19, tau=par["tau"], precision=precision, closure=closure,
                      cs_smag=0.1, faces=FACES_CHANNEL, streaming=streaming, collision=collision)
    lat.set_force(par["force"])
    rho = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    u = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    step = max(1, nz // 8)
    for z0 in range(0, nz, step):  # generate slab by slab to bound host memory
        z1 = min(nz, z0 + step)
        r, v = inputs.channel_init(nx, ny, nz, z_range=(z0, z1))
        rho[z0:z1].copy_(torch.from_numpy(r))
        u[:, z0:z1].copy_(torch.from_numpy(v))
    lat.init_equilibrium(rho, u)
    del rho, u
    return lat, par


def _bluff_lattice(nx, ny, nz, precision, streaming="pull"):
    """The landing-gear tunnel of the bluff-body form (D3Q27 TRT + Smagorinsky, inflow 0.05 at
    x = 0, outflow at x = nx-1, free-slip y/z), geometry scaled by nx / 768, started from the
    uniform inflow state."""
    import torch

    from paper_2305_09910_gb300 import inputs, lbm

    scale = nx / 768
    tau = 0.5 + 3 * 0.05 * (80 * scale) / 1e4
    lat = lbm.Lattice(nx, ny, nz, stencil=27, tau=tau, precision=precision, closure="smag", cs_smag=0.1,
                      faces=("inflow", "outflow", "freeslip", "freeslip", "freeslip", "freeslip"),
                      u_inflow=(0.05, 0.0, 0.0), streaming=streaming)
    flags = inputs.landing_gear_flags(nx, ny, nz, scale=scale)
    lat.set_flags(torch.from_numpy(flags).cuda())
    u = torch.zeros((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    u[0] = 0.05
    lat.init_equilibrium(None, u)
    del u
    return lat, {"tau": tau, "force": 0.0, "fluid_cells": int((flags == 0).sum())}


def _closure_params():
    """Network weights of the learned-closure form (fixed seed; the cost of the fused inference
    does not depend on them)."""
    import numpy as np

    from paper_2305_09910_gb300 import closure

    params = closure.init_params(7)
    params[closure.OUT_LAYER] = np.random.default_rng(7).normal(0, 0.1, 33).astype(np.float32)
    return params


def _time_steps(lat, steps, warmup, dist, stats_every=0):
    """Device time of `steps` single-launch steps (CUDA events on the handle's stream); with
    stats_every > 0 the profile statistics of the state every stats_every-th step starts from
    are sampled inside the timed region (the turbulent-channel job accumulates mean and RMS
    profiles), by that step's own kernel (lbm_step_stats)."""
    import torch

    from paper_2305_09910_gb300 import lbm

    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        lbm.lbm_step(lat.h, 1)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if stats_every:
        lbm.lbm_stats_reset(lat.h)
    t0.record(stream)
    for k in range(steps):
        starts[k].record(stream)
        if stats_every and k % stats_every == 0:
            lbm.lbm_step_stats(lat.h, 1, 1)
        else:
            lbm.lbm_step(lat.h, 1)
        ends[k].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    lat.sync()
    return total_ms, per


def _roofline(ncell, bytes_per_update, per_launch_ms, peak, peak_kind, traffic):
    avg_s = statistics.mean(per_launch_ms) * 1e-3
    achieved = ncell * bytes_per_update / avg_s / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6.8 TB/s",
            "bytes_per_update": bytes_per_update, "avg_launch_ms": round(avg_s * 1e3, 4)}


def _form_line(lat, nsteps, warmup, peak, peak_kind, fluid=None):
    """MLUPS over all cells (as the paper counts), MFLUPS over the fluid cells when some are
    solid, and the HBM roofline of the mean launch."""
    ms, per = _time_steps(lat, nsteps, warmup, None)
    line = {"MLUPS": round(lat.ncell * nsteps / (ms * 1e-3) / 1e6, 1), "cells": lat.ncell}
    if fluid is not None:
        line["MFLUPS"] = round(fluid * nsteps / (ms * 1e-3) / 1e6, 1)
        line["fluid_cells"] = int(fluid)
    line["roofline"] = _roofline(lat.ncell, lat.bytes_per_update, per, peak, peak_kind, None)
    return line


def _extra_forms(nsteps, warmup, peak, peak_kind, sm_mhz):
    """The other benchmark shapes, timed the same way (state values do not change the cost
    of a step; these start from rest or from uniform flow):
      * precision form: channel 1024x512x512 (268M cells), FP32 and FP16-shifted storage;
      * bluff body: 768x384x384 D3Q27 TRT+Smagorinsky tunnel (inflow 0.05, outflow, free-slip)
        with the landing-gear flags, FP32 and FP16-shifted storage;
      * learned closure: channel 256x128x128 and 512x256x256, fused MLP closure (tensor-core
        hidden layer) vs Smagorinsky (network weights from a fixed seed: the cost of the fused
        inference does not depend on them).
    All forms use two-grid pull streaming except those named _aa (in-place AA pattern)."""
    import numpy as np
    import torch

    from paper_2305_09910_gb300 import closure, inputs, lbm

    out = {}
    par = inputs.channel_parameters(512)
    for prec in ("f32", "f16"):
        lat = lbm.Lattice(1024, 512, 512, stencil=19, tau=par["tau"], precision=prec, closure="smag",
                          cs_smag=0.1, faces=FACES_CHANNEL, streaming="pull")
        lat.set_force(par["force"])
        lat.init_equilibrium()
        out[f"channel1024_{prec}"] = _form_line(lat, max(20, nsteps // 4), warmup, peak, peak_kind)
        lat.close()
        torch.cuda.empty_cache()
    flags = torch.from_numpy(inputs.landing_gear_flags(768, 384, 384)).cuda()
    tau = 0.5 + 3 * 0.05 * 80 / 1e4
    for prec in ("f32", "f16"):
        lat = lbm.Lattice(768, 384, 384, stencil=27, tau=tau, precision=prec, closure="smag", cs_smag=0.1,
                          faces=("inflow", "outflow", "freeslip", "freeslip", "freeslip", "freeslip"),
                          u_inflow=(0.05, 0.0, 0.0), streaming="pull")
        lat.set_flags(flags)
        u = torch.zeros((3, 384, 384, 768), dtype=torch.float32, device="cuda")
        u[0] = 0.05
        lat.init_equilibrium(None, u)
        del u
        out[f"bluffbody768_q27_{prec}"] = _form_line(lat, max(20, nsteps // 4), warmup, peak, peak_kind,
                                                     fluid=int((flags == 0).sum().item()))
        lat.close()
        torch.cuda.empty_cache()
    params = _closure_params()
    for size, name in ((256, "smag"), (256, "mlp"), (512, "mlp")):
        lat = closure.channel(size, size // 2, size // 2, closure=name, streaming="pull")
        if name == "mlp":
            lbm.lbm_set_closure_f32(lat.h, params, 600.0, 3000.0)
            lbm.lbm_set_closure_floor(lat.h, 0.1)
        line = _form_line(lat, nsteps, warmup, peak, peak_kind)
        if name == "mlp":  # issue-bound: the network's arithmetic, with the HBM fraction beside it
            inst = _profile_value(f"k_step_q19_f32_mlp_pull_channel{size}", "inst_per_cell")
            if inst is None:
                inst = _profile_value("k_step_q19_f32_mlp_pull_channel256", "inst_per_cell")
            line["roofline"] = _issue_roofline(line["MLUPS"], inst, sm_mhz, line["roofline"])
        out[f"channel{size}_{name}"] = line
        lat.close()
        torch.cuda.empty_cache()
    return out


def _slab_form(nslab, nsteps, warmup, peak, peak_kind):
    """The channel split into nslab z slabs on this GPU, a halo exchange after every step
    (lbm_halo_pack/unpack of the 5 crossing directions per face): cost of the domain split."""
    import torch

    from paper_2305_09910_gb300 import inputs, slabs

    par = inputs.channel_parameters(256)
    sl = slabs.ZSlabs(512, 256, 256, nslab, stencil=19, tau=par["tau"], closure="smag", cs_smag=0.1,
                      faces=FACES_CHANNEL)
    sl.set_force(par["force"])
    sl.init_equilibrium()
    sl.step(warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    sl.step(nsteps)
    t1.record(stream)
    torch.cuda.synchronize()
    sl.sync()
    ms = t0.elapsed_time(t1) / nsteps
    ncell = sl.ncell
    halo = sum(b.numel() for b in sl.bufs)
    sl.close()
    achieved = ncell * 153 / (ms * 1e-3) / 1e9
    return {"MLUPS": round(ncell / (ms * 1e-3) / 1e6, 1), "cells": ncell, "halo_bytes_per_step": halo,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None,
                         "bytes_per_update": 153.0, "ms_per_step": round(ms, 4)}}


def _small_form(streaming, nsteps=2000):
    """The 64x32x32 Poiseuille lattice (walls as solid rows, body force), launch-bound: time
    per step of lbm_step(n), which runs several steps per launch (multi-step cooperative
    launches or graph replays)."""
    import torch

    from paper_2305_09910_gb300 import inputs, lbm

    nx, ny, nz = 64, 32, 32
    lat = lbm.Lattice(nx, ny, nz, stencil=19, tau=0.8, streaming=streaming)
    lat.set_flags(inputs.poiseuille_flags(nx, ny, nz))
    lat.set_force(1e-6)
    lat.init_equilibrium()
    lat.step(20)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    lat.step(nsteps)
    t1.record(stream)
    torch.cuda.synchronize()
    lat.sync()
    us = t0.elapsed_time(t1) * 1e3 / nsteps
    lat.close()
    fluid = nx * (ny - 2) * nz  # rows y = 0 and ny - 1 are solid
    return {"MLUPS": round(nx * ny * nz / us, 1), "MFLUPS": round(fluid / us, 1), "fluid_cells": fluid,
            "us_per_step": round(us, 2), "steps": nsteps}


def _refined_form(nsteps, warmup, peak, peak_kind, precision="f32"):
    """A 256x128x128 coarse box (periodic, body force along x, TRT + Smagorinsky) whose planes
    z = 32..95 are refined 2:1 into a 512x256x128 fine lattice: per coarse step every coarse
    cell is updated once and every fine cell twice, plus the explosion and coalescence of the
    two interfaces.  Throughput counts cell updates of both levels."""
    import torch

    from paper_2305_09910_gb300 import inputs, refine

    par = inputs.channel_parameters(128)
    rs = refine.RefinedSlab(256, 128, 128, 32, 96, stencil=19, tau=par["tau"], force=(par["force"], 0.0, 0.0),
                            closure="smag", cs_smag=0.1, precision=precision)
    rs.init_equilibrium()
    rs.step(warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    rs.step(nsteps)
    t1.record(stream)
    torch.cuda.synchronize()
    rs.sync()
    ms = t0.elapsed_time(t1) / nsteps
    upd = rs.updates_per_step
    bpu = float(rs.fine.bytes_per_update)
    launches = 3 * len(rs.interfaces) + 2 * len(rs.fines) + len(rs.coarse)  # transfers; steps
    rs.close()
    achieved = upd * bpu / (ms * 1e-3) / 1e9
    return {"MLUPS": round(upd / (ms * 1e-3) / 1e6, 1), "updates_per_coarse_step": upd,
            "launches_per_coarse_step": launches,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None,
                         "bytes_per_update": bpu, "ms_per_coarse_step": round(ms, 4)}}


def _time_oracle(threads, target_s):
    """(MLUPS, steps, seconds) of the FP64 oracle on a 128x64x64 sub-lattice of the channel."""
    import numpy as np

    import oracle
    from paper_2305_09910_gb300 import inputs

    nx, ny, nz = 128, 64, 64
    par = inputs.channel_parameters(ny)
    ora = oracle.Oracle(nx, ny, nz, q=19, tau=par["tau"], closure="smag", cs=0.1,
                        faces=FACES_CHANNEL, force=(par["force"], 0, 0))
    rho, u = inputs.channel_init(nx, ny, nz)
    ora.init_equilibrium(rho.astype(np.float64), u.astype(np.float64))
    t = time.perf_counter()
    ora.step(1, threads=threads)
    one = max(time.perf_counter() - t, 1e-3)
    steps = max(2, int(target_s / one))
    t = time.perf_counter()
    ora.step(steps, threads=threads)
    dt = time.perf_counter() - t
    return nx * ny * nz * steps / dt / 1e6, steps, dt


def _cpu_baseline(target_s=12.0, target_one_s=6.0):
    """The FP64 oracle on this host's cores (all of them, and one), on a 128x64x64 sub-lattice
    of the channel."""
    threads = os.cpu_count() or 1
    mlups, steps, dt = _time_oracle(threads, target_s)
    m1, s1, d1 = _time_oracle(1, target_one_s)
    return {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"FP64 oracle, channel 128x64x64 D3Q19 TRT+Smagorinsky, {steps} steps "
                      f"({dt:.1f} s, OpenMP over z on {threads} threads)",
            "one_thread": {"value": round(m1, 3), "unit": "MLUPS", "cores": 1,
                           "sample": f"the same sub-lattice, {s1} steps ({d1:.1f} s) on 1 thread"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2305_09910_gb300 import inputs

    nx, ny, nz = 128, 64, 64
    par = inputs.channel_parameters(ny)
    threads = os.cpu_count() or 1
    ora = oracle.Oracle(nx, ny, nz, q=19, tau=par["tau"], closure="smag", cs=0.1,
                        faces=FACES_CHANNEL, force=(par["force"], 0, 0))
    rho, u = inputs.channel_init(nx, ny, nz)
    ora.init_equilibrium(rho.astype(np.float64), u.astype(np.float64))
    ora.step(args.warmup, threads=threads)
    t = time.perf_counter()
    ora.step(args.steps, threads=threads)
    dt = time.perf_counter() - t
    mlups = nx * ny * nz * args.steps / dt / 1e6
    sample = (f"FP64 oracle on the host cores, channel sub-lattice {nx}x{ny}x{nz} (1/64 of the "
              f"512x256x256 workload) D3Q19 TRT+Smagorinsky, {args.steps} timed steps")
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " -- oracle sample 128x64x64", "parallelism": "host threads"},
            "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-forms", action="store_true", help="skip the FP16/BF16 forms")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    ap.add_argument("--size", default="512x256x256", help="lattice NXxNYxNZ (profiling runs)")
    ap.add_argument("--form", default="f32", choices=["f32", "f16", "bf16"],
                    help="storage precision of the main line (profiling runs)")
    ap.add_argument("--streaming", default="pull", choices=["pull", "aa"],
                    help="streaming pattern of the main line (profiling runs)")
    ap.add_argument("--closure", default="smag", choices=["smag", "mlp"],
                    help="closure of the main line (profiling runs of the learned-closure kernel)")
    ap.add_argument("--workload", default="channel", choices=["channel", "bluffbody"],
                    help="main-line workload (profiling runs of the D3Q27 bluff-body kernel)")
    ap.add_argument("--collision", default="trt", choices=["trt", "mrt", "reg"],
                    help="collision of the channel main line (profiling runs of the MRT / regularised steps)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_2305_09910_gb300 import build as lib_build
    from paper_2305_09910_gb300 import lbm

    dist, rank, world, local = _dist()
    if rank == 0:
        lib_build.build()
    if dist is not None:
        dist.barrier()
    torch.cuda.set_device(local)
    peak, peak_kind = _peak_hbm()
    gpu_uuid = str(torch.cuda.get_device_properties(local).uuid)
    gpu_id = gpu_uuid if gpu_uuid.startswith("GPU-") else f"GPU-{gpu_uuid}"

    nx, ny, nz = (int(v) for v in args.size.lower().split("x"))
    ncell = nx * ny * nz
    channel = args.workload == "channel"
    if channel:
        lat, par = _channel_lattice(nx, ny, nz, args.form, closure=args.closure, streaming=args.streaming,
                                    collision=args.collision)
        if args.closure == "mlp":
            lbm.lbm_set_closure_f32(lat.h, _closure_params(), 600.0, 3000.0)
            lbm.lbm_set_closure_floor(lat.h, 0.1)
    else:
        lat, par = _bluff_lattice(nx, ny, nz, args.form, streaming=args.streaming)
    clocks = ClockSampler(gpu_id)
    time.sleep(1.0)  # let nvidia-smi start
    for _ in range(args.warmup):
        lbm.lbm_step(lat.h, 1)
    torch.cuda.synchronize()
    clocks.start()
    total_ms, per = _time_steps(lat, args.steps, 3, dist, stats_every=10 if channel else 0)
    clocks.stop()
    clock_summary = clocks.summary()
    total_ms = _barrier_max(dist, total_ms)
    value = world * ncell * args.steps / (total_ms * 1e-3) / 1e6
    fluid = ncell if channel else par["fluid_cells"]  # the channel's walls are faces: every cell is fluid
    mflups = world * fluid * args.steps / (total_ms * 1e-3) / 1e6
    q = 19 if channel else 27
    coll = "" if args.collision == "trt" else f"_{args.collision}"
    tag = f"k_step_q{q}_{args.form}_{args.closure}{coll}_{args.streaming}_{args.workload}{nx}"
    traffic = _profile_traffic(tag)
    roof = _roofline(ncell, lat.bytes_per_update, per, peak, peak_kind, traffic)
    mass = lat.reduce()[0]
    lat_bytes = ncell * q * lat.bytes_per_pop
    nsample = (args.steps + 9) // 10 if channel else 0
    # our kernel launches in the timed region: one per step, plus per statistics sample the
    # plane-sum pass (fused sampling) or the two reduction kernels (learned closure).  (With
    # --form f16/bf16 a pull step whose boundary list exceeds 2^18 cells launches the list on
    # its own; the default FP32 line never does.)
    launches = args.steps + (2 * nsample if args.closure == "mlp" else nsample)

    # end to end through the C ABI with host buffers: upload (rho, u) from pinned memory,
    # K steps, read the moments back to pinned memory
    from paper_2305_09910_gb300 import inputs

    rho_h = torch.empty((nz, ny, nx), dtype=torch.float32).pin_memory()
    u_h = torch.empty((3, nz, ny, nx), dtype=torch.float32).pin_memory()
    step = max(1, nz // 8)
    for z0 in range(0, nz, step):
        z1 = min(nz, z0 + step)
        r, v = inputs.channel_init(nx, ny, nz, z_range=(z0, z1))
        rho_h[z0:z1].copy_(torch.from_numpy(r))
        u_h[:, z0:z1].copy_(torch.from_numpy(v))
    rho_o = torch.empty_like(rho_h).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t = time.perf_counter()
    lbm.lbm_init_equilibrium(lat.h, rho_h, u_h)
    lbm.lbm_step(lat.h, args.steps)
    lbm.lbm_moments(lat.h, rho_o, u_o)
    lat.sync()
    e2e_s = _barrier_max(dist, time.perf_counter() - t)
    e2e = {"value": round(world * ncell * args.steps / e2e_s / 1e6, 1), "unit": "MLUPS",
           "h2d_bytes_per_step": int(16 * ncell / args.steps),
           "d2h_bytes_per_step": int(16 * ncell / args.steps),
           "what": "lbm_init_equilibrium from pinned host (rho,u) + K lbm_step + lbm_moments to pinned host"}
    lat.close()

    forms = {}
    if not args.no_forms:
        nsteps = max(50, args.steps // 4)
        for prec, streaming in (("f32", "aa"), ("f16", "pull"), ("bf16", "pull"), ("f16", "aa")):
            fl, _ = _channel_lattice(nx, ny, nz, prec, streaming=streaming)
            tag = "" if streaming == "pull" else "_aa"
            name = f"channel{nx}_{prec}{tag}" if prec == "f32" else f"channel{nx}_{prec}_shifted{tag}"
            forms[name] = _form_line(fl, nsteps, args.warmup, peak, peak_kind)
            fl.close()
            torch.cuda.empty_cache()
        sm_mhz = clock_summary.get("sm_mhz") or 2070.0
        forms.update(_extra_forms(nsteps, args.warmup, peak, peak_kind, sm_mhz))
        forms["channel512_f32_2slabs_halo"] = _slab_form(2, nsteps, args.warmup, peak, peak_kind)
        for streaming in ("pull", "aa"):
            forms[f"poiseuille64_f32_{streaming}"] = _small_form(streaming)
        for prec in ("f32", "f16"):
            forms[f"box256_refined2to1_{prec}"] = _refined_form(nsteps // 2, args.warmup, peak, peak_kind, prec)
            torch.cuda.empty_cache()
        for coll in ("mrt", "reg"):
            fl, _ = _channel_lattice(nx, ny, nz, "f32", collision=coll)
            forms[f"channel{nx}_f32_{coll}"] = _form_line(fl, nsteps, args.warmup, peak, peak_kind)
            fl.close()
            torch.cuda.empty_cache()

    if (nx, ny, nz, args.form, args.streaming, args.closure, args.collision, channel) == \
            (512, 256, 256, "f32", "pull", "smag", "trt", True):
        workload = WORKLOAD
    elif channel:
        workload = (f"turbulent channel {nx}x{ny}x{nz} D3Q19 {args.collision.upper()}+" +
                    ("learned closure" if args.closure == "mlp" else "Smagorinsky") + f" {args.form} ({args.streaming})")
    else:
        workload = f"bluff body {nx}x{ny}x{nz} D3Q27 TRT+Smagorinsky {args.form} ({args.streaming})"
    out = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload, "storage": args.form, "nx": nx, "ny": ny, "nz": nz, "stencil": q,
                      "tau": round(par["tau"], 6), "force": par["force"], "cs_smag": 0.1,
                      "global_batch": world * ncell, "parallelism": f"replicas x{world}",
                      "stats": ("mean/RMS profile sample (FP64 plane sums) every 10 steps, taken by the step kernel, "
                                "inside the timed region") if channel else "none",
                      "l2": f"inputs larger than L2 ({lat_bytes / 1e9:.2f} GB population array vs 129 MB L2)"},
           "mflups": round(mflups, 1), "roofline": roof, "e2e": e2e, "gpu_launches": launches,
           "clocks": clock_summary, "mass_after": mass, "forms": forms}
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = _cpu_baseline()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
