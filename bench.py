#!/usr/bin/env python3
"""Throughput benchmark of the fused linear-LB step on GB300.

Workload: the 4096^2 two-layer medium (contrast 1:2 at mid-depth), D2Q5 BGK
tau = 1/2, FP32 populations, 40-cell sponge, Ricker point source, 512
receivers (the paper's recommended scheme, Sec. 5.1).  One bench step is one
LB time step of the whole grid (stream + collide + source + sponge + receiver
gather, one fused launch).  Metric: GLUPS (1e9 lattice-site updates / s).

--impl reference times the FP64 CPU oracle on this machine's host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
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

from paper_1704_03172_gb300 import workloads as W  # noqa: E402

METRIC = "GLUPS & % of HBM roofline (D2Q5 step, FP32 vs BF16); served shots/s, p50/p99"
UNIT = "GLUPS"
N_GRID = 4096
FALLBACK_HBM_GBS = 6800.0
ELEM_BYTES = {"f32": 4, "bf16": 2, "f16": 2}


# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant kernel on the
# 4096^2 two-layer workload, from one ncu capture (the summaries under profiles/ give the
# commands), keyed by (kernel, medium index) and stamped with the hash of the kernel's
# source files at the capture.  A kernel without an entry, or whose sources hash
# differently now, reports null.
KERNEL_SOURCES = {
    "lbk::step_kernel": ("lb_kernels.cuh",),
    "stream_step_kernel": ("lb_kernels.cuh", "aa_sites.cuh", "stream_step.cu"),
    "lbtb5::tb5_kernel": ("lb_kernels.cuh", "tblock5.cuh"),
}
NCU_TRAFFIC = {
    ("lbk::step_kernel<5,false,false,float>", True):
        (638.5e6, "df1c40b8bd02", "profiles/step_kernel_d2q5_f32_4096.md"),
    ("stream_step_kernel<5,false,false,__nv_bfloat16>", True):
        (300.3e6, "3a52a69fc363", "profiles/stream_step_kernel_d2q5_bf16_4096.md"),
    ("lbtb5::tb5_kernel<false,4,false,float>", True):
        (656.4e6, "be28d81b9dd6", "profiles/tb5_kernel_d2q5_4096.md"),
    ("lbtb5::tb5_kernel<false,4,false,__nv_bfloat16>", True):
        (314.8e6, "be28d81b9dd6", "profiles/tb5_kernel_d2q5_4096.md"),
    ("lbtb5::tb5_kernel<false,8,false,float>", True):
        (671.9e6, "be28d81b9dd6", "profiles/tb5_kernel_d2q5_4096.md"),
}


def source_hash(kname):
    """sha1 (12 hex digits) of the source files a kernel is built from"""
    import hashlib
    files = KERNEL_SOURCES.get(kname.split("<")[0])
    if files is None:
        return None
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_1704_03172_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def ncu_traffic(kname, indexed):
    """(bytes per launch or None, why) from NCU_TRAFFIC for the kernel as built now"""
    ent = NCU_TRAFFIC.get((kname, bool(indexed)))
    if ent is None:
        return None, "no capture of this kernel"
    nbytes, stamp, prof = ent
    if stamp != source_hash(kname):
        return None, "kernel source changed since its capture"
    return nbytes, f"ncu capture, {prof}"


def bytes_per_site(Q, storage, indexed):
    """Algorithmic HBM bytes of one site update: read and write every population once,
    plus the medium read (a 1-byte medium index, or 4-byte eta^2 per site)."""
    return 2 * Q * ELEM_BYTES[storage] + (1 if indexed else 4)


def _indexed(sim):
    return sim.info()[4] > 0      # distinct speeds behind the 1-byte medium index (0: none)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            if d.get("hbm_gbs"):
                return float(d["hbm_gbs"]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_rate(sec, units, ws, device="cuda"):
    """Whole-job throughput of ws independent replicas: the units all ranks processed over
    the slowest rank's timed seconds (sum and max over ranks).  Returns (units / s, s)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(sec)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        u = torch.tensor([float(units)], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        sec, units = float(t.item()), float(u.item())
    return units / sec, sec


def _workload(lattice=5, storage="f32", collision="bgk"):
    wl = W.two_layer_workload(N_GRID, lattice=lattice, collision=collision)
    wl["storage"] = storage
    return wl


def _make_sim(LBSim, wl, nt_cap):
    sim = LBSim(wl["c_map"], lattice=wl["lattice"], collision=wl["collision"], tau=wl["tau"],
                s=wl.get("s"), storage=wl["storage"], c_ref=wl["c_ref"],
                sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"],
                w_ref=wl["w_ref"], time_block=wl.get("time_block", 1),
                step_kernel=wl.get("step_kernel", "auto"), streaming=wl.get("streaming", "ab"))
    sx, sy, wav = wl["source"]
    sim.set_source(sx, sy, wav)
    sim.set_receivers(wl["receivers"], nt_cap)
    sim.init_pressure(None)
    return sim


def _time_steps(torch, sim, steps, warmup):
    sim.step(warmup)
    torch.cuda.synchronize()
    stream = sim.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def _variant(torch, LBSim, lattice, storage, collision, steps, warmup, time_block=1,
             streaming="ab"):
    wl = _workload(lattice, storage, collision)
    wl["time_block"] = time_block
    wl["streaming"] = streaming
    sim = _make_sim(LBSim, wl, steps + warmup)
    try:
        # the D2Q9 tile-blocked kernel reads eta^2 per site; the others the medium index
        indexed = _indexed(sim) and (time_block <= 1 or lattice == 5)
        sec = _time_steps(torch, sim, steps, warmup)
    finally:
        sim.close()
    sites = N_GRID * N_GRID
    glups = sites * steps / sec / 1e9
    bps = bytes_per_site(lattice, storage, indexed)
    out = {"glups": round(glups, 2), "bytes_per_site": bps,
           "achieved_gbs": round(glups * bps, 1), "ms_per_step": round(sec / steps * 1e3, 4)}
    if streaming == "aa":
        out["frac_of_measured_hbm"] = round(glups * bps / _peaks()[0], 4)
        out["population_gb"] = round(lattice * sites * ELEM_BYTES[storage] / 1e9, 3)
        out["streaming"] = "in place: one population buffer (two-buffer form: twice this)"
    return out


_LAYERED = {}


def _layered(n):
    """The layered workload (20 layers, faults, 1500-5500 m/s) at n^2, generated once."""
    if n not in _LAYERED:
        _LAYERED[n] = W.layered_workload(n)
    return _LAYERED[n]


def _layered_variant(torch, LBSim, storage, steps, warmup, n=8192):
    """The 8192^2 layered workload: D2Q5 BGK tau = 1/2, 40-cell sponge, Ricker source at
    (4096, 80), 512 receivers on the source row; GLUPS and the algorithmic HBM rate."""
    wl = dict(_layered(n))
    wl["storage"] = storage
    sim = LBSim(wl["c_map"], lattice=5, tau=0.5, storage=storage, c_ref=wl["c_ref"],
                sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"])
    try:
        sim.set_source(*wl["source"])
        sim.set_receivers(wl["receivers"], steps + warmup)
        sim.init_pressure(None)
        indexed = _indexed(sim)
        sec = _time_steps(torch, sim, steps, warmup)
    finally:
        sim.close()
    glups = n * n * steps / sec / 1e9
    bps = bytes_per_site(5, storage, indexed)
    return {"glups": round(glups, 2), "bytes_per_site": bps, "achieved_gbs": round(glups * bps, 1),
            "frac_of_measured_hbm": round(glups * bps / _peaks()[0], 4),
            "ms_per_step": round(sec / steps * 1e3, 4), "grid": f"{n}^2", "steps": steps,
            "state_gb": round(2 * 5 * n * n * ELEM_BYTES[storage] / 1e9, 2)}


def _refined_variant(torch, LBSim, steps, warmup):
    """Slow-block workload: 2048^2 coarse grid + 1025^2-node fine patch (2x in space and
    time).  One fine site-step counts as one update: 2048^2 + 2 * 1025^2 per coarse step."""
    wl = W.refined_block_workload(2048)
    sim = LBSim(wl["c_map"], lattice=5, collision="mrt", s=wl["s"], c_ref=wl["c_ref"],
                sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"],
                patch=wl["patch"])
    sim.set_source(*wl["source"])
    sim.set_receivers(wl["receivers"], steps + warmup)
    sim.init_pressure(None)
    try:
        sec = _time_steps(torch, sim, steps, warmup)
    finally:
        sim.close()
    nf = 2 * wl["patch"][2] + 1
    updates = 2048 * 2048 + 2 * nf * nf
    return {"glups": round(updates * steps / sec / 1e9, 2), "updates_per_coarse_step": updates,
            "ms_per_coarse_step": round(sec / steps * 1e3, 4),
            "launches_per_coarse_step": 3,
            "launches": "coarse step + snapshot transfer; fine step + midpoint transfer; fine "
                        "step + fine -> coarse correction (each coupling task in extra blocks of a step launch)"}


def _upsample2(c):
    """The medium on a grid refined by 2 everywhere: node (a, b) at coarse position
    (a / 2, b / 2), the average of the coarse nodes around it (as for a refined patch)."""
    c = np.asarray(c, np.float64)
    ny, nx = c.shape
    cx = np.concatenate([c[:, 1:], c[:, -1:]], axis=1)      # x + 1, clamped
    cy = np.concatenate([c[1:], c[-1:]], axis=0)            # y + 1, clamped
    cxy = np.concatenate([cy[:, 1:], cy[:, -1:]], axis=1)
    f = np.empty((2 * ny, 2 * nx))
    f[0::2, 0::2] = c
    f[0::2, 1::2] = (c + cx) / 2
    f[1::2, 0::2] = (c + cy) / 2
    f[1::2, 1::2] = (c + cx + cy + cxy) / 4
    return f.astype(np.float32)


def _refined_vs_fine_variant(torch, LBSim):
    """The slow-block workload's stated comparison (Sec. 5.2, Fig. 11 experiment): the
    2048^2 coarse grid with its 2x patch for all 4000 coarse steps, the same problem on a
    uniformly fine 4096^2 grid for 8000 steps, and the coarse grid alone.  Reported: the
    trace error of the refined and of the coarse-only run against the uniformly fine one,
    per receiver region (upstream of the patch, inside it, downstream), and the upstream
    difference between the refined and the coarse-only run (what the interface reflects,
    with the block's own reflection in both)."""
    wl = W.refined_block_workload(2048)
    steps = wl["steps"]
    sx, sy, wav = wl["source"]
    rec = wl["receivers"]
    x0, y0, nxp, _ = wl["patch"]
    kw = dict(lattice=5, collision="mrt", s=wl["s"], c_ref=wl["c_ref"])
    out = {}

    def run(c, patch, src, receivers, nt, sponge, smax):
        sim = LBSim(c, sponge_width=sponge, sponge_sigma_max=smax, patch=patch, **kw)
        try:
            sim.set_source(*src)
            sim.set_receivers(receivers, nt)
            sim.init_pressure(None)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.step(nt)
            tr = sim.traces(nt).cpu().numpy().astype(np.float64)
            sec = time.perf_counter() - t0
        finally:
            sim.close()
        return tr, sec

    tr_ref, s_ref = run(wl["c_map"], wl["patch"], wl["source"], rec, steps, wl["sponge_width"],
                        wl["sponge_sigma_max"])
    tr_crs, s_crs = run(wl["c_map"], None, wl["source"], rec, steps, wl["sponge_width"],
                        wl["sponge_sigma_max"])
    # the same physical problem refined by 2 everywhere: twice the nodes, the source at the
    # coincident node with S_f(t) = 2 S(t / 2) (the same source density per unit time), the
    # sponge twice as wide and half as strong per (half-length) step
    fc0 = (0.5 ** 0.5) / 32.0
    wav_f = 2.0 * W.ricker(2 * steps, fc0 / 2)
    tr_f, s_f = run(_upsample2(wl["c_map"]), None, (2 * sx, 2 * sy, wav_f), 2 * rec, 2 * steps,
                    2 * wl["sponge_width"], wl["sponge_sigma_max"] / 2)
    tr_f = tr_f[::2]
    regions = {"upstream": rec[:, 0] < x0, "inside": (rec[:, 0] >= x0) & (rec[:, 0] <= x0 + nxp),
               "downstream": rec[:, 0] > x0 + nxp}
    for name, m in regions.items():
        den = np.linalg.norm(tr_f[:, m])
        out[name] = {"receivers": int(m.sum()),
                     "refined_vs_fine": round(float(np.linalg.norm(tr_ref[:, m] - tr_f[:, m]) / den), 5),
                     "coarse_vs_fine": round(float(np.linalg.norm(tr_crs[:, m] - tr_f[:, m]) / den), 5)}
    up = regions["upstream"]
    out["upstream_refined_minus_coarse_over_peak"] = round(
        float(np.abs(tr_ref[:, up] - tr_crs[:, up]).max() / np.abs(tr_crs[:, up]).max()), 5)
    out["seconds"] = {"refined": round(s_ref, 3), "coarse": round(s_crs, 3),
                      "uniform_fine": round(s_f, 3)}
    out["workload"] = ("2048^2 coarse (slow block c/3), 1025^2-node 2x patch, MRT s = (1, 1, 1, 2, "
                       "2), Ricker source, 256 receivers on y = 1024, 4000 coarse steps; uniform "
                       "fine 4096^2 for 8000 steps; traces at coincident times")
    return out


def _l2_variant(torch, LBSim, n, storage, steps, warmup=50, time_block=1):
    """The two-layer workload scaled to n^2 (64 receivers), small enough that both state
    buffers stay in the 129 MB L2: reported apart from the HBM-bound lines, against no
    roofline.  time_block 8 takes 8 steps per launch, which matters where a step lasts
    only a few microseconds."""
    wl = W.two_layer_workload(n, nrec=64)
    wl["storage"] = storage
    wl["time_block"] = time_block
    sim = _make_sim(LBSim, wl, steps + warmup)
    try:
        sec = _time_steps(torch, sim, steps, warmup)
        pitch = sim.info()[1]
    finally:
        sim.close()
    state = 2 * 5 * n * pitch * ELEM_BYTES[storage]
    return {"glups": round(n * n * steps / sec / 1e9, 2), "ms_per_step": round(sec / steps * 1e3, 5),
            "state_mb": round(state / 1e6, 1), "l2_resident": state < 129e6,
            "grid": f"{n}^2", "steps": steps, "time_block": time_block}


def _nested_variant(torch, LBSim, steps, warmup):
    """The slow-block workload with a nested patch: 2048^2 coarse grid, a 1025^2-node patch
    (2x) and inside it a 1025^2-node nested patch (4x to the coarse grid).  One site-step of
    any level counts as one update: 2048^2 + 2 * 1025^2 + 4 * 1025^2 per coarse step."""
    wl = W.refined_nested_workload(2048)
    sim = LBSim(wl["c_map"], lattice=5, collision="mrt", s=wl["s"], c_ref=wl["c_ref"],
                sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"],
                patch=wl["patches"])
    sim.set_source(*wl["source"])
    sim.set_receivers(wl["receivers"], steps + warmup)
    sim.init_pressure(None)
    try:
        sec = _time_steps(torch, sim, steps, warmup)
    finally:
        sim.close()
    n1 = 2 * wl["patches"][0][2] + 1
    n2 = 2 * wl["patches"][1][2] + 1
    updates = 2048 * 2048 + 2 * n1 * n1 + 4 * n2 * n2
    return {"glups": round(updates * steps / sec / 1e9, 2), "updates_per_coarse_step": updates,
            "ms_per_coarse_step": round(sec / steps * 1e3, 4),
            "launches_per_coarse_step": 7,
            "launches": "coarse step + level-1 snapshot; per level-1 step: that step with its "
                        "transfer or correction and the level-2 snapshot, then two level-2 steps "
                        "with theirs"}


_OBSERVED = {}


def _observed(torch, LBSim, n, nt):
    """Data d of the misfit: the 512 traces of a Gaussian-smoothed (sigma = 20 cells) copy of
    the layered model at n^2 (FP32, same source and receivers), computed once per size."""
    if (n, nt) not in _OBSERVED:
        from scipy.ndimage import gaussian_filter
        wl = _layered(n)
        cs = gaussian_filter(np.asarray(wl["c_map"], np.float32), 20.0, mode="nearest")
        sim = LBSim(cs, lattice=5, tau=0.5, c_ref=wl["c_ref"], sponge_width=40)
        try:
            sim.set_source(wl["source"][0], wl["source"][1], W.ricker(nt, W.SERVED_FC))
            sim.set_receivers(wl["receivers"], nt)
            sim.init_pressure(None)
            sim.step(nt)
            _OBSERVED[(n, nt)] = sim.traces(nt).clone()
        finally:
            sim.close()
    return _OBSERVED[(n, nt)]


def _adjoint_variant(torch, LBSim, n=4096, nt=1000, every=200, storage="f32", mode="ckpt"):
    """Gradient of J = 1/2 sum (p - d)^2 over 512 receiver traces w.r.t. the sound-speed map
    and the source, for the 20-layer faulted model (the layered workload at n^2), with d the
    traces of a smoothed copy of the model: forward run with checkpoints, then lb_adjoint
    (replay + reverse sweep); mode "tape": the forward run records rho (n^2 nt 4 bytes) and
    lb_adjoint is the reverse sweep alone.  Rates count n^2 * nt site-steps of the gradient
    call; peak device memory of the whole shot."""
    d = _observed(torch, LBSim, n, nt)
    wl = _layered(n)
    sim = LBSim(wl["c_map"], lattice=5, tau=0.5, c_ref=wl["c_ref"], sponge_width=40,
                storage=storage)
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    mem0 = torch.cuda.memory_allocated()
    try:
        sim.set_source(wl["source"][0], wl["source"][1], W.ricker(nt, W.SERVED_FC))
        sim.set_receivers(wl["receivers"], nt)
        sim.init_pressure(None)
        if mode == "tape":
            sim.record_rho(nt)
        else:
            sim.checkpoint_every(every)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(nt)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
        R = sim.traces(nt) - d  # dJ/dp
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gc, gs, _ = sim.adjoint(R, nt)
        torch.cuda.synchronize()
        t_adj = time.perf_counter() - t0
        finite = bool(torch.isfinite(gc).all().item())
        indexed = _indexed(sim)
        peak_gb = (torch.cuda.max_memory_allocated() - mem0) / 1e9
    finally:
        sim.close()
    T = min(every, (16 << 30) // (n * n * 4))
    levels = 1 if T >= every else 2
    if storage == "f32":  # replays run 8 steps per launch (the D2Q5 wavefront kernel)
        bps_fwd = bytes_per_site(5, storage, indexed) / 8
    else:
        bps_fwd = bytes_per_site(5, storage, indexed)
    # per adjoint site-step: the wavefront reverse sweep, 4 levels per launch: lambda read and
    # written, eta^2 read and the FP64 gradient read-modify-write once per 4 levels, and the
    # rho tape read at every level
    bps_adj = (2 * 5 * 4 + 4 + 16) / 4 + 4
    bps = round(bps_adj if mode == "tape" else levels * bps_fwd + 4 + bps_adj, 2)
    upd = n * n * nt
    out = {"gradient_glups": round(upd / t_adj / 1e9, 2),
           "forward_with_checkpoints_glups" if mode != "tape" else "forward_with_rho_tape_glups":
               round(upd / t_fwd / 1e9, 2),
           "bytes_per_site_step": bps, "achieved_gbs": round(upd * bps / t_adj / 1e9, 1),
           "seconds": round(t_adj, 4), "finite": finite,
           "peak_device_gb": round(peak_gb, 2),
           "workload": f"{n}x{n} 20-layer faulted model, D2Q5 BGK {storage.upper()}, {nt} steps, "
                       + (f"forward rho tape ({n * n * nt * 4 / 1e9:.0f} GB), no replay"
                          if mode == "tape" else f"checkpoint every {every}")
                       + ", 512 receivers, J = 1/2 sum (p - d)^2 with d from the model "
                         "smoothed by a Gaussian of 20 cells, wall time of lb_adjoint"}
    if mode != "tape":
        out["replay_levels"] = levels
        out["checkpoint_every"] = every
    return out


def _d3q7_variant(torch, LBSim, storage, n=256, steps=300, warmup=10):
    """The 3-D (D3Q7) step on a two-layer n^3 medium (contrast 1:2 at mid-depth along z),
    BGK tau = 1/2, 16-cell sponge, Ricker source, 64 receivers on a line."""
    c = np.ones((n, n, n), np.float32)
    c[n // 2:] = 2.0
    sim = LBSim(c, lattice=7, tau=0.5, storage=storage, c_ref=2.0, sponge_width=16)
    try:
        fc = 0.5 / math.sqrt(3.0) / (n / 30.0)
        sim.set_source(n // 2, n // 2, n // 4, W.ricker(steps + warmup, fc))
        rec = np.stack([np.arange(16, n - 16, (n - 32) // 64)[:64], np.full(64, n // 2),
                        np.full(64, n // 4)], 1)
        sim.set_receivers(rec, steps + warmup)
        sim.init_pressure(None)
        indexed = _indexed(sim)
        sec = _time_steps(torch, sim, steps, warmup)
    finally:
        sim.close()
    glups = n ** 3 * steps / sec / 1e9
    bps = 2 * 7 * ELEM_BYTES[storage] + (1 if indexed else 4)
    return {"glups": round(glups, 2), "bytes_per_site": bps, "achieved_gbs": round(glups * bps, 1),
            "ms_per_step": round(sec / steps * 1e3, 4), "grid": f"{n}^3"}


def _dispersion_variant(n=128, steps=256):
    """Fig. 3 / Fig. 4 style: phase speed / c_s of the acoustic branch, measured on the GPU
    (single-mode runs batched in one periodic grid, FP64 projections, matrix pencil fit),
    at theta = 0 and 45 degrees, for D2Q5 and two D2Q9 weight sets, BGK tau = 1/2."""
    from paper_1704_03172_gb300 import dispersion as D
    modes = [(32, 0), (16, 0), (8, 0), (4, 0), (16, 16), (8, 8), (4, 4)]
    out = {}
    for name, kw in (("d2q5", dict(lattice=5)),
                     ("d2q9_conventional_weights", dict(lattice=9, w_ref=(4 / 9, 1 / 9, 1 / 36))),
                     ("d2q9_w0_0.01_0.24", dict(lattice=9, w_ref=(0.0, 0.01, 0.24)))):
        rows = D.phase_speed(modes, n, steps, **kw)
        out[name] = [{"ppw": round(r["ppw"], 2), "theta_deg": round(r["theta_deg"], 1),
                      "phase_speed_ratio": round(r["phase_speed_ratio"], 6),
                      "damping": round(r["damping"], 8)} for r in rows]
    return out


def _e2e(torch, LBSim, steps_shot):
    """One full shot through the public API with host buffers (create .. traces .. destroy)."""
    from paper_1704_03172_gb300.sim import LBSim as _S  # noqa: F401
    wl = _workload()
    # the caller's buffers: pinned host memory, allocated before the timed region
    c_host = torch.from_numpy(np.ascontiguousarray(wl["c_map"], dtype=np.float32)).pin_memory().numpy()
    sx, sy, wav = wl["source"]
    rec = wl["receivers"]
    out = torch.empty((steps_shot, len(rec)), dtype=torch.float32, pin_memory=True).numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = LBSim(c_host, lattice=5, collision="bgk", tau=0.5, c_ref=wl["c_ref"],
                sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"])
    sim.set_source(sx, sy, wav)
    sim.set_receivers(rec, steps_shot)
    sim.init_pressure(None)
    sim.step(steps_shot)
    from paper_1704_03172_gb300 import lbac
    import ctypes
    n = lbac.lb_record_receivers(sim.ctx, ctypes.c_void_p(out.ctypes.data), steps_shot, 0)
    sim.close()
    sec = time.perf_counter() - t0
    assert n == steps_shot
    h2d = c_host.nbytes + len(wav) * 8 + rec.nbytes
    return {"value": round(N_GRID * N_GRID * steps_shot / sec / 1e9, 2), "unit": UNIT,
            "h2d_bytes_per_step": round(h2d / steps_shot, 1),
            "d2h_bytes_per_step": round(out.nbytes / steps_shot, 1),
            "h2d_bytes_per_shot": int(h2d), "d2h_bytes_per_shot": int(out.nbytes),
            "step": f"one {steps_shot}-step shot: lb_create(host c_map) .. lb_step .. "
                    "lb_record_receivers(host) .. lb_destroy", "host_buffers": "pinned",
            "seconds": round(sec, 4)}


def _served(n_req, n_cal, seed=W.DEFAULT_SEED + 5, load=0.7, max_active=64):
    """Served shot stream through lb_server_*: ``n_req`` shots with Poisson arrivals at
    ``load`` x the closed-loop capacity measured on ``n_cal`` calibration shots.

    Each shot: grid side from {256, 512, 1024, 2048}, 2000-8000 steps, its own seeded
    layered-fault model (4-12 layers), FP32 or BF16 storage with p = 1/2, and with
    p = 1/4 an adjoint gradient of J = 1/2 sum p^2 (zero observed data, checkpoint every
    200 steps).  Latency = result ready - submit (the arrival).  GLUPS counts forward
    site updates only."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_1704_03172_gb300.sim import LBServer

    descs = W.served_requests(n_req, seed)
    cal = W.served_requests(n_cal, seed + 1, id0=1_000_000)
    t_gen = time.perf_counter()
    with ThreadPoolExecutor(8) as ex:
        shots = list(ex.map(W.served_shot, descs))
        cal_shots = list(ex.map(W.served_shot, cal))
    t_gen = time.perf_counter() - t_gen

    def submit(srv, s):
        kw = dict(s)
        c = kw.pop("c_map")
        if kw["want_gradient"]:
            kw["observed"] = np.zeros((kw["nt"], len(kw["receivers"])), np.float32)
            kw["checkpoint_every"] = 0  # the forward rho tape when it is small, else 200
        return srv.submit(c, **kw)

    def collect(srv, ids, out):
        for i in ids:
            srv.wait(i)
            out.append(srv.result(i))

    def one_by_one(shots_):
        """The same shots through the plain per-shot API (LBSim), one after another."""
        import torch
        from paper_1704_03172_gb300.sim import LBSim
        tape_limit = 0.4 * torch.cuda.mem_get_info()[0]  # the server's rule: budget / 2
        t0 = time.monotonic()
        for s in shots_:
            sim = LBSim(s["c_map"], lattice=5, tau=s["tau"], storage=s["storage"],
                        sponge_width=s["sponge_width"], sponge_sigma_max=s["sponge_sigma_max"],
                        c_ref=s["c_ref"])
            sim.set_source(*s["source"])
            sim.set_receivers(s["receivers"], s["nt"])
            sim.init_pressure(None)
            if s["want_gradient"]:
                n = s["c_map"].shape[0]
                if s["nt"] * n * (-(-n // 32) * 32) * 4 <= tape_limit:
                    sim.record_rho(s["nt"])
                else:
                    sim.checkpoint_every(200)
            sim.step(s["nt"])
            tr = sim.traces(s["nt"])
            tr.cpu()
            if s["want_gradient"]:
                gc, gs, _ = sim.adjoint(tr, s["nt"])
                gc.cpu()
            sim.close()
        torch.cuda.synchronize()
        return time.monotonic() - t0

    srv = LBServer(max_active=max_active, rounds_per_pass=16, adjoint_workers=4)
    try:
        t0 = time.monotonic()
        ids = [submit(srv, s) for s in cal_shots]
        done = []
        collect(srv, ids, done)
        cal_s = time.monotonic() - t0
        capacity = n_cal / cal_s
        lam = load * capacity
        arrivals = np.cumsum(np.random.default_rng(seed + 2).exponential(1.0 / lam, n_req))
        launches0 = srv.stats()["launches"]
        ids, res = [], []
        import queue
        q = queue.Queue()
        th = threading.Thread(target=lambda: collect(srv, iter(q.get, None), res), daemon=True)
        th.start()
        t0 = time.monotonic()
        for k, s in enumerate(shots):
            dt = t0 + arrivals[k] - time.monotonic()
            if dt > 0:
                time.sleep(dt)
            rid = submit(srv, s)
            ids.append(rid)
            q.put(rid)
        q.put(None)
        th.join()
        launches = srv.stats()["launches"] - launches0
    finally:
        srv.close()
    plain_s = one_by_one(cal_shots)
    lat = np.array([r["done"] - r["submit"] for r in res])
    span = max(r["done"] for r in res) - min(r["submit"] for r in res)
    fwd = sum(d["n"] ** 2 * d["nt"] for d in descs)
    finite = all(np.isfinite(r["traces"]).all() for r in res)
    return {"requests": n_req, "shots_per_s": round(n_req / span, 3),
            "p50_latency_s": round(float(np.percentile(lat, 50)), 4),
            "p99_latency_s": round(float(np.percentile(lat, 99)), 4),
            "mean_latency_s": round(float(lat.mean()), 4),
            "forward_glups": round(fwd / span / 1e9, 2), "span_s": round(span, 2),
            "offered_rate_per_s": round(lam, 3), "load": load,
            "calibrated_capacity_per_s": round(capacity, 3),
            "calibration": f"{n_cal} shots of the same distribution submitted at once, "
                           f"{cal_s:.2f} s", "launches": int(launches),
            "one_by_one_capacity_per_s": round(n_cal / plain_s, 3),
            "batching_gain": round(plain_s / cal_s, 3),
            "one_by_one": f"the {n_cal} calibration shots run one after another through the "
                          f"per-shot API (LBSim: create, step, traces, adjoint), {plain_s:.2f} s",
            "gradients": sum(d["grad"] for d in descs),
            "bf16": sum(d["storage"] == "bf16" for d in descs),
            "forward_updates": fwd, "finite": bool(finite), "max_active": max_active,
            "input_generation_s": round(t_gen, 2),
            "shot": "D2Q5 BGK tau=1/2, layered-fault model (4-12 layers, c 1500-5500 m/s), "
                    "Ricker 10 ppw at 1500 m/s, 40-cell sponge, 128 receivers; side from "
                    "{256,512,1024,2048}, 2000-8000 steps"}


def _served_classes(n_per_class=32, nt=2000, sizes=W.SERVED_SIZES, seed=W.DEFAULT_SEED + 7):
    """Batching gain per grid size: n_per_class FP32 forward shots of one size (layered
    models, Ricker source, 128 receivers, nt steps) submitted at once to the server,
    against the same shots one after another through LBSim (create, step, traces)."""
    import torch
    from paper_1704_03172_gb300.sim import LBServer, LBSim
    out = {}
    for n in sizes:
        descs = [dict(id=seed + 100 * n + k, n=n, nt=nt, storage="f32", grad=False, layers=8)
                 for k in range(4)]
        shots = [W.served_shot(d) for d in descs]
        shots = [shots[k % len(shots)] for k in range(n_per_class)]

        def kw(s):
            d = dict(s)
            d.pop("c_map")
            return d

        srv = LBServer(max_active=n_per_class, rounds_per_pass=16, adjoint_workers=1)
        try:
            t0 = time.monotonic()
            ids = [srv.submit(s["c_map"], **kw(s)) for s in shots]
            res = []
            for i in ids:
                srv.wait(i)
                res.append(srv.result(i))
            served_s = time.monotonic() - t0
        finally:
            srv.close()
        torch.cuda.synchronize()
        t0 = time.monotonic()
        for s in shots:
            sim = LBSim(s["c_map"], lattice=5, tau=0.5, sponge_width=s["sponge_width"],
                        sponge_sigma_max=s["sponge_sigma_max"], c_ref=s["c_ref"])
            sim.set_source(*s["source"])
            sim.set_receivers(s["receivers"], nt)
            sim.init_pressure(None)
            sim.step(nt)
            sim.traces(nt).cpu()
            sim.close()
        torch.cuda.synchronize()
        plain_s = time.monotonic() - t0
        upd = n * n * nt * n_per_class
        out[f"{n}^2"] = {"shots": n_per_class, "steps": nt,
                         "served_shots_per_s": round(n_per_class / served_s, 2),
                         "one_by_one_shots_per_s": round(n_per_class / plain_s, 2),
                         "batching_gain": round(plain_s / served_s, 3),
                         "served_glups": round(upd / served_s / 1e9, 2),
                         "one_by_one_glups": round(upd / plain_s / 1e9, 2),
                         "finite": bool(all(np.isfinite(r["traces"]).all() for r in res))}
    return out


def _cpu_sample(target_s=12.0, lattice=5):
    """Time the FP64 oracle on a bounded sample of the workload (rows of the 4096^2 grid)."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    wl = _workload(lattice)
    rows = 256
    c = wl["c_map"][: rows]
    P = oracle.Problem(lattice, N_GRID, rows, c, c_ref=wl["c_ref"], tau=wl["tau"],
                       sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"],
                       w_ref=wl["w_ref"])
    g = P.zeros()
    oracle.run(P, g, 1)                     # warm the thread pool
    t0 = time.perf_counter()
    oracle.run(P, g, 1)
    chunk = max(1, int(1.0 / max(time.perf_counter() - t0, 1e-6)))   # ~1 s per call
    steps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < target_s:
        oracle.run(P, g, chunk)
        steps += chunk
    sec = time.perf_counter() - t0
    glups = N_GRID * rows * steps / sec / 1e9
    # one thread, on a shorter sample of the same band (the oracle's thread count is a
    # process setting: restored to all cores afterwards)
    def band(nthreads):
        return oracle.Problem(lattice, N_GRID, rows, c, c_ref=wl["c_ref"], tau=wl["tau"],
                              sponge_width=wl["sponge_width"],
                              sponge_sigma_max=wl["sponge_sigma_max"], w_ref=wl["w_ref"],
                              nthreads=nthreads)
    P1 = band(1)
    steps1, t1 = 0, time.perf_counter()
    while time.perf_counter() - t1 < target_s / 4:
        oracle.run(P1, g, 1)
        steps1 += 1
    sec1 = time.perf_counter() - t1
    oracle.run(band(cores), g, 1)
    return {"value": round(glups, 4), "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "single_thread_value": round(N_GRID * rows * steps1 / sec1 / 1e9, 5),
            "sample": f"{steps} steps of a {N_GRID}x{rows} band of the two-layer workload "
                      f"(FP64 C, OpenMP over rows), {sec:.1f} s; single thread: {steps1} steps, "
                      f"{sec1:.1f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    wl = _workload()
    rows = max(4, min(N_GRID, int(os.environ.get("LB_REF_ROWS", "64"))))
    c = wl["c_map"][: rows]
    P = oracle.Problem(5, N_GRID, rows, c, c_ref=wl["c_ref"], tau=wl["tau"],
                       sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"])
    g = P.zeros()
    for _ in range(args.warmup):
        g, _ = oracle.run(P, g, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g, _ = oracle.run(P, g, 1)
    sec = time.perf_counter() - t0
    glups = N_GRID * rows * args.steps / sec / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(glups, 5), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"two-layer {N_GRID}x{N_GRID} D2Q5 BGK tau=1/2, sponge 40, "
                                   f"sampled as a {N_GRID}x{rows} band per step",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": round(glups, 5), "unit": UNIT, "cores": oracle.max_threads(),
                             "kind": "oracle",
                             "sample": f"one LB step of a {N_GRID}x{rows} band per bench step"},
            "e2e": {"value": round(glups, 5), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_slabs(args, torch, LBSim, ws, rank, local):
    """One shot of the 8192^2 layered workload split into ws row slabs, one per rank, the
    cut rows exchanged after every step (torch.distributed point-to-point, NCCL): strong
    scaling.  value = the grid's site updates over the slowest rank's timed seconds."""
    from paper_1704_03172_gb300 import slabs
    import torch.distributed as dist
    wl = _layered(8192)
    n = wl["nx"]
    slab = slabs.DistSlab(wl["c_map"], rank, ws, lattice=5, tau=0.5, c_ref=wl["c_ref"],
                          sponge_width=wl["sponge_width"], sponge_sigma_max=wl["sponge_sigma_max"])
    slab.set_source(*wl["source"])
    slab.set_receivers(wl["receivers"], args.steps + args.warmup)
    slab.init_pressure(None)
    slab.step(args.warmup)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        e0.record(slab.sim.stream)
        slab.step(args.steps)
        e1.record(slab.sim.stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    rows = slab.y1 - slab.y0
    rate, sec = job_rate(e0.elapsed_time(e1) / 1e3, rows * n * args.steps, ws)
    tr = slab.traces(args.steps + args.warmup)
    slab.close()
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": round(rate / 1e9, 3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(sec / args.steps * 1e3, 4), "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "layered 8192x8192 (20 layers, faults, 1500-5500 m/s), D2Q5 "
                                   "BGK tau=1/2, FP32, 40-cell sponge, Ricker source, 512 "
                                   "receivers; one shot split into row slabs",
                       "parallelism": f"{ws} row slabs, cut rows exchanged every step",
                       "l2": "inputs larger than L2 (population buffers >= 168 MB per slab "
                             "up to 8 slabs)"},
            "gpu_launches": args.steps, "clocks": clk.summary(),
            "finite": bool(np.isfinite(tr).all())}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1704_03172_gb300 import build
    build.build()
    from paper_1704_03172_gb300.sim import LBSim

    if args.decompose == "slabs":
        return run_slabs(args, torch, LBSim, ws, rank, local)
    if args.variant:  # one variant alone (profiling runs)
        name = args.variant
        if name.startswith("adjoint_"):  # adjoint_f32, adjoint_bf16, adjoint_tape_f32, ...
            out = _adjoint_variant(torch, LBSim, n=args.adj_n, nt=args.adj_nt,
                                   every=args.adj_every, storage=name.rsplit("_", 1)[1],
                                   mode="tape" if "_tape_" in name else "ckpt")
        elif name == "refined_vs_fine":
            out = _refined_vs_fine_variant(torch, LBSim)
        elif name.startswith("refined_nested"):
            out = _nested_variant(torch, LBSim, args.steps, args.warmup)
        elif name.startswith("refined"):
            out = _refined_variant(torch, LBSim, args.steps, args.warmup)
        elif name == "dispersion":
            out = _dispersion_variant()
        elif name.startswith("l2_resident"):  # l2_resident_<n>_<storage>[_tb8]
            parts = name.split("_")
            st = next(p for p in parts if p in ELEM_BYTES)
            out = _l2_variant(torch, LBSim, int(parts[2]), st, args.steps, args.warmup,
                              time_block=8 if "tb8" in parts else 1)
        elif name.startswith("aa_"):  # aa_d2q<Q>_<collision>_<storage>: in-place streaming
            _, q, coll, st = name.split("_")
            out = _variant(torch, LBSim, int(q[3:]), st, coll, args.steps, args.warmup,
                           streaming="aa")
        elif name.startswith("d3q7"):
            out = _d3q7_variant(torch, LBSim, name.rsplit("_", 1)[1])
        elif name.startswith("layered_8192"):  # layered_8192_<storage>
            out = _layered_variant(torch, LBSim, name.rsplit("_", 1)[1], args.steps, args.warmup)
        elif name == "served":
            out = _served(args.served_requests, args.served_calibration)
        elif name == "served_classes":
            out = _served_classes()
        else:
            raise SystemExit(f"unknown variant {name}")
        if rank == 0:
            print(json.dumps({"variant": name, **out}), flush=True)
        return 0

    wl = _workload(args.lattice, args.storage, args.collision)
    wl["time_block"] = args.time_block
    wl["step_kernel"] = args.step_kernel
    sim = _make_sim(LBSim, wl, args.steps + args.warmup)
    sim.step(args.warmup)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.3)            # let the sampler start before the timed region
        t0 = time.perf_counter()
        e0.record(sim.stream)
        sim.step(args.steps)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if ws > 1:
        dist.barrier()
    sites = N_GRID * N_GRID
    rate, sec = job_rate(e0.elapsed_time(e1) / 1e3, sites * args.steps, ws)
    tr = sim.traces(args.steps + args.warmup)
    finite = bool(torch.isfinite(tr).all().item())
    indexed = _indexed(sim)
    sim.close()
    value = rate / 1e9
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return 0
    peak, peak_kind = _peaks()
    K = max(1, args.time_block)
    # the one-step and the D2Q5 wavefront kernels read the 1-byte medium index; the D2Q9
    # tile-blocked kernel reads eta^2 per site
    medium_idx = indexed and (K == 1 or args.lattice == 5)
    bps = bytes_per_site(args.lattice, args.storage, medium_idx)
    launches = (args.steps + K - 1) // K
    per_launch_s = sec / launches
    achieved = bps * sites * K / per_launch_s / 1e9   # algorithmic one-step bytes per update
    staged = K == 1 and (args.step_kernel == "staged" or
                         (args.step_kernel == "auto" and args.storage != "f32"))
    st_name = dict(f32='float', bf16='__nv_bfloat16', f16='__half')[args.storage]
    mrt = "true" if args.collision == "mrt" else "false"
    tb5 = K > 1 and args.lattice == 5
    kname = (f"lbtb5::tb5_kernel<{mrt},{K},false,{st_name}>" if tb5 else
             f"tb_kernel<{args.lattice},{mrt},false,{K}>" if K > 1 else
             f"stream_step_kernel<{args.lattice},{mrt},false,{st_name}>" if staged else
             f"lbk::step_kernel<{args.lattice},{mrt},false,{st_name}>")
    traffic, traffic_src = ncu_traffic(kname, indexed)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(sec / args.steps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": {"workload": f"two-layer {N_GRID}x{N_GRID} (c 1:2 at mid-depth), "
                               f"D2Q{args.lattice} " + ("BGK tau=1/2" if args.collision == "bgk"
                                                         else "MRT (seeded rates)") +
                               f", {args.storage.upper()} populations, "
                               "40-cell sponge, Ricker source, 512 receivers; one bench step = "
                               "one LB time step" + (f" ({K} steps fused per launch)" if K > 1 else ""),
                   "parallelism": f"replicas x{ws} (independent shots)",
                   "l2": "inputs larger than L2 (each population buffer >= 168 MB; 129 MB L2)",
                   "medium": "1-byte medium index + eta^2 table" if medium_idx
                             else "eta^2 per site (FP32)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "traffic_source": traffic_src, "kernel": kname,
                     "algorithmic_bytes_per_launch": bps * sites * K,
                     "note": "achieved counts the one-step algorithmic bytes of every fused "
                             "step (one-step equivalent bandwidth)"
                     if K > 1 else "one launch per step"},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "wall_s": round(wall, 4),
        "finite": finite,
    }
    if not args.no_variants:
        v = {}
        for lat, st, coll in ((5, "bf16", "bgk"), (5, "f16", "bgk"), (5, "f32", "mrt"),
                              (9, "f32", "bgk"), (9, "f32", "mrt"), (9, "bf16", "bgk")):
            try:
                v[f"d2q{lat}_{coll}_{st}"] = _variant(torch, LBSim, lat, st, coll,
                                                       max(200, args.steps // 5), 10)
            except Exception as ex:  # report, do not hide
                v[f"d2q{lat}_{coll}_{st}"] = {"error": str(ex)[:200]}
        for st, K in (("f32", 2), ("f32", 4), ("f32", 6), ("f32", 8), ("bf16", 4), ("bf16", 8)):
            name = f"d2q5_bgk_{st}_tb{K}"
            try:
                v[name] = _variant(torch, LBSim, 5, st, "bgk", max(400, args.steps // 5) // 24 * 24,
                                   24, time_block=K)
                v[name]["one_step_roofline_glups"] = round(
                    _peaks()[0] / bytes_per_site(5, st, True), 1)
            except Exception as ex:
                v[name] = {"error": str(ex)[:200]}
        for lat, st, coll in ((5, "f32", "bgk"), (5, "bf16", "bgk"), (9, "f32", "mrt")):
            name = f"aa_d2q{lat}_{coll}_{st}"
            try:
                v[name] = _variant(torch, LBSim, lat, st, coll, max(200, args.steps // 5), 10,
                                   streaming="aa")
            except Exception as ex:
                v[name] = {"error": str(ex)[:200]}
        for n, nsteps in ((256, 20000), (1024, 5000)):
            for st, tb in (("f32", 1), ("bf16", 1), ("f32", 8)):
                name = f"l2_resident_{n}_d2q5_bgk_{st}" + ("_tb8" if tb > 1 else "")
                try:
                    v[name] = _l2_variant(torch, LBSim, n, st, nsteps, time_block=tb)
                except Exception as ex:
                    v[name] = {"error": str(ex)[:200]}
        try:
            v["refined_block_2048_d2q5_mrt_f32"] = _refined_variant(torch, LBSim, 400, 10)
        except Exception as ex:
            v["refined_block_2048_d2q5_mrt_f32"] = {"error": str(ex)[:200]}
        try:
            v["refined_nested_2048_d2q5_mrt_f32"] = _nested_variant(torch, LBSim, 400, 10)
        except Exception as ex:
            v["refined_nested_2048_d2q5_mrt_f32"] = {"error": str(ex)[:200]}
        try:
            v["refined_block_2048_vs_uniform_fine"] = _refined_vs_fine_variant(torch, LBSim)
        except Exception as ex:
            v["refined_block_2048_vs_uniform_fine"] = {"error": str(ex)[:200]}
        for st in ("f32", "bf16"):
            try:
                v[f"adjoint_tape_4096_d2q5_{st}"] = _adjoint_variant(torch, LBSim, storage=st,
                                                                     mode="tape")
            except Exception as ex:
                v[f"adjoint_tape_4096_d2q5_{st}"] = {"error": str(ex)[:200]}
        for st in ("f32", "bf16"):
            try:
                v[f"adjoint_4096_d2q5_{st}"] = _adjoint_variant(torch, LBSim, storage=st)
            except Exception as ex:
                v[f"adjoint_4096_d2q5_{st}"] = {"error": str(ex)[:200]}
        for st in ("f32", "bf16", "f16"):
            name = f"layered_8192_d2q5_bgk_{st}"
            try:
                v[name] = _layered_variant(torch, LBSim, st, max(200, args.steps // 5), 10)
            except Exception as ex:
                v[name] = {"error": str(ex)[:200]}
        try:
            v["adjoint_8192_d2q5_f32"] = _adjoint_variant(torch, LBSim, n=8192, nt=1000,
                                                           every=200, storage="f32")
        except Exception as ex:
            v["adjoint_8192_d2q5_f32"] = {"error": str(ex)[:200]}
        for st in ("f32", "bf16"):
            try:
                v[f"d3q7_bgk_{st}_256"] = _d3q7_variant(torch, LBSim, st)
            except Exception as ex:
                v[f"d3q7_bgk_{st}_256"] = {"error": str(ex)[:200]}
        try:
            v["dispersion_bgk_tau0.5"] = _dispersion_variant()
        except Exception as ex:
            v["dispersion_bgk_tau0.5"] = {"error": str(ex)[:200]}
        line["variants"] = v
    if not args.no_e2e:
        line["e2e"] = _e2e(torch, LBSim, args.e2e_steps)
    if args.served_requests > 0:
        try:
            line["served"] = _served(args.served_requests, args.served_calibration)
        except Exception as ex:  # report, do not hide
            line["served"] = {"error": str(ex)[:300]}
        try:
            line["served_by_size"] = _served_classes()
        except Exception as ex:
            line["served_by_size"] = {"error": str(ex)[:300]}
    if not args.no_cpu:
        line["cpu_baseline"] = _cpu_sample(args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=5000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--variant", default="",
                    help="run one variant alone: adjoint_f32, adjoint_bf16, adjoint_tape_f32, "
                         "adjoint_tape_bf16, refined, refined_nested, refined_vs_fine, served, "
                         "served_classes, aa_d2q<Q>_<collision>_<storage>, "
                         "layered_8192_<storage>, l2_resident_<n>_<storage>[_tb8], d3q7_<storage>, "
                         "dispersion")
    ap.add_argument("--adj-n", type=int, default=4096, help="adjoint variant grid side")
    ap.add_argument("--adj-nt", type=int, default=1000, help="adjoint variant steps")
    ap.add_argument("--adj-every", type=int, default=200, help="adjoint checkpoint interval")
    ap.add_argument("--served-requests", type=int, default=512,
                    help="shots in the served stream (0 skips it)")
    ap.add_argument("--served-calibration", type=int, default=64,
                    help="closed-loop shots that set the Poisson arrival rate")
    ap.add_argument("--collision", choices=["bgk", "mrt"], default="bgk",
                    help="main line only (profiling runs): BGK or MRT with the seeded rates")
    ap.add_argument("--lattice", type=int, choices=[5, 9], default=5,
                    help="main line's lattice (D2Q5 is the paper's recommended scheme)")
    ap.add_argument("--storage", choices=["f32", "bf16", "f16"], default="f32")
    ap.add_argument("--step-kernel", choices=["auto", "direct", "staged"], default="auto",
                    help="auto (TMA-staged for wide 16-bit rows), direct (register-streaming) "
                         "or staged (TMA-staged persistent)")
    ap.add_argument("--decompose", choices=["replicas", "slabs"], default="replicas",
                    help="N > 1: independent shots, one per rank (weak scaling), or one 8192^2 "
                         "shot split into row slabs with a cut-row exchange (strong scaling)")
    ap.add_argument("--time-block", type=int, default=1,
                    help="steps fused per launch for the main line (temporal blocking)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
