#!/usr/bin/env python3
"""Benchmark of the fused D3Q19 + D3Q7 time step (thermal pseudopotential MRT-LBM, arXiv 2206.00946).

Workload (one "step" = one lattice-Boltzmann time step over the whole domain),
by default the heated-surface droplet: a 256 x 256 x 128 lattice, hemispherical
droplet of radius 30 on a bounce-back bottom wall at 0.96 T_c (contact angle
90 degrees), constant-pressure top face (rho_b = rho_v, T_s), periodic in x
and y, FP32 populations (1.75 GB double-buffered, far above L2).  Metric:
million lattice updates per second (MLUPS), whole job, and the fraction of the
measured HBM copy bandwidth that the 208 bytes of algorithmic traffic per
lattice update reach.  --workload droplet selects the d^2-law droplet
(128^3, radius 15, open faces on all six sides) instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload sessile|droplet] [--storage f32|f16|bf16|f16local]
                    [--schedule slabs|phases|fused]

The JSON line also carries the roofline of the dominant kernel (each kernel timed
alone with CUDA events in the phase schedule, charged its own algorithmic bytes),
the end-to-end rate through host buffers, the FP64 CPU oracle on a bounded sample
on all host cores and on one (cpu_baseline), the 128^3 d^2-law droplet
(droplet_128), the paper's own geometries of Secs. 4.2 and 4.3 (paper_cases), the adjoint/forward cost on a 64^3 droplet over 2000 steps with
checkpoints every 100 (adjoint), 48 uneven droplet domains stepped as one batch
(batched), and the 512^3 heated-plate pool with 64 droplets in FP16-shifted
storage (large), the step time with the correction term of Eq. 16
(vartheta = 1) against without (vartheta), and the rate in each population
storage form (storage_forms: FP32, FP16 and BF16 with one global shift, FP16
with per-cell references); --no-adjoint / --no-batched / --no-large /
--no-vartheta / --no-storage / --no-droplet / --no-paper-cases / --no-cpu-baseline skip those.

N > 1 (torchrun, one rank per GPU) runs N independent replicas of the domain
(weak scaling, no collective on the data path).  --impl reference times the
FP64 CPU oracle on host cores on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2206_00946_gb300 import workloads as W  # noqa: E402

METRIC = "fused D3Q19+D3Q7 MLUPS"
UNIT = "MLUPS"
BYTES_PER_LU = 208  # f and g (19 + 7 FP32 populations) read once and written once per lattice update
STORAGE = {"f32": (0, 4), "f16": (1, 2), "bf16": (2, 2), "f16local": (3, 2)}  # lbm_storage code, bytes per population


def kernel_alg_bytes(kernel: str, esize: int):
    """Algorithmic bytes per cell of one launch of `kernel` (populations it must read and write once)."""
    return {"phaseC": 2 * 19 * esize,   # D3Q19 collide + push: f read and written
            "phaseC7": 2 * 7 * esize,   # D3Q7 collide + relaxed push: g read and written
            "phaseA": 26 * esize,       # macroscopic fields: f and g read
            "fused": 2 * 26 * esize}.get(kernel)
WORKLOADS = {
    "sessile": "droplet on a heated surface 256x256x128, R=30, W=5, bottom wall 0.96 T_c (theta 90), "
               "open top rho_b=rho_v at T_s, periodic x/y",
    "droplet": "d2-law droplet 128^3, R=15, W=5, open (Zou-He) faces rho_b=rho_v, T_faces=T_c, seed 2206",
}


def workload(name, Tc, rv, rl, n=None):
    """(params, rho0, T0) of a named workload (n: side of the droplet lattice)."""
    if name == "sessile":
        return W.sessile(Tc, rv, rl)
    return W.droplet(Tc, rv, rl, n=n or 128, R=15.0)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def src_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2206_00946_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


# the per-cell and phase code of the step kernels, and the block of lbm_api.cu that defines
# the phase kernels (their launch bounds and loops)
KERNEL_HEADERS = ("lbm_cell.cuh", "lbm_lattice.cuh", "lbm_phases.cuh", "lbm_stage.cuh")
KERNEL_BLOCK = ("// Phase kernels over the cell range", "// FP64 block reduction")


def code_only(text: str) -> str:
    """C++ source without its // and /* */ comments, runs of whitespace collapsed."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_digest():
    """Digest of the step kernels' own code (comments and layout left out), so that host-side
    edits of the library and edits of comments do not void an ncu traffic figure taken on
    unchanged kernels."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2206_00946_gb300", "csrc")
    for f in KERNEL_HEADERS:
        h.update(code_only(open(os.path.join(csrc, f)).read()).encode())
    api = open(os.path.join(csrc, "lbm_api.cu")).read()
    h.update(code_only(api[api.index(KERNEL_BLOCK[0]):api.index(KERNEL_BLOCK[1])]).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, kernel_digest: str, n_cells: int):
    """DRAM bytes per launch from the committed ncu summary of `kernel`, if it was taken on this kernel source."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel}.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("kernel_src_sha") != kernel_digest:
        return None
    return d["dram_bytes_per_cell"] * n_cells


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_throughput(dist, local_s: float, units_per_rank: int, device="cpu"):
    """Whole-job throughput of weakly scaled replicas: every rank processed
    units_per_rank units in local_s seconds; the job took the slowest rank's
    time.  Returns (max seconds over ranks, total units / that time)."""
    world = dist.get_world_size() if dist else 1
    if dist:
        import torch
        t = torch.tensor([local_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_s = float(t.item())
    return local_s, world * units_per_rank / local_s


def adjoint_cost(lbm, Tc, rv, rl, schedule, stream, n=2000, K=100, side=64):
    """Adjoint / forward cost on a side^3 droplet of radius 10 side/64 with open
    faces (64^3, R = 10 by default): the time of lbm_adjoint_step over n recorded
    steps (segment recompute included) over the time of n forward steps, both CUDA
    events on the context stream."""
    import torch
    p, rho0, T0 = W.droplet(Tc, rv, rl, n=side, R=10.0 * side / 64)
    p["schedule"] = schedule
    rho_d = torch.tensor(rho0.reshape(-1), dtype=torch.float32, device="cuda")
    T_d = torch.tensor(T0.reshape(-1), dtype=torch.float32, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)
    lat = lbm.Lattice(p, rho_d, T_d, stream=stream.cuda_stream)
    lat.lbm_step(20)
    e = [ev() for _ in range(6)]
    torch.cuda.synchronize()
    e[0].record(stream)
    lat.lbm_step(n)
    e[1].record(stream)
    lat.close()
    lat = lbm.Lattice(p, rho_d, T_d, stream=stream.cuda_stream)
    e[2].record(stream)
    lat.lbm_record(n, K)
    e[3].record(stream)
    rho = torch.empty_like(rho_d)
    lat.lbm_macros(rho=rho)
    mid, w = 0.5 * (rl + rv), 0.1 * (rl - rv)
    th = torch.tanh((rho - mid) / w)
    seed = (0.5 * (1 + th) + rho * 0.5 * (1 - th * th) / w).contiguous()  # d(liquid mass)/d rho
    dT0 = torch.empty(lat.N, dtype=torch.float64, device="cuda")
    dTf = torch.empty(6 * side * side, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    e[4].record(stream)
    lat.lbm_adjoint_step(n, seed, None, dTf, dT0)
    e[5].record(stream)
    torch.cuda.synchronize()
    lat.close()
    fwd, rec, adj = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3]), e[4].elapsed_time(e[5])
    return {"workload": f"d2-law droplet {side}^3, R={10.0 * side / 64:g}, open faces, loss = smooth liquid mass "
                        f"after {n} steps, "
                        f"checkpoint every {K} steps; gradients w.r.t. T0 and the six face-temperature fields",
            "forward_ms_per_step": fwd / n, "record_ms_per_step": rec / n, "adjoint_ms_per_step": adj / n,
            "ratio": adj / fwd, "ratio_with_record": (adj + rec) / fwd}


def batched_throughput(lbm, Tc, rv, rl, stream, ndom=48, steps=100, seed=2206):
    """48 droplet domains with sides drawn from {32, 48, 64, 96} and radius side/4
    (open faces, rho_b = rho_v, T = T_c): one persistent launch per step over all
    of them (shape from the autotuner) against stepping the domains one after
    another with the single-lattice schedule."""
    import torch
    sides = [32, 48, 64, 96]
    draws = W.uniform(seed, ndom, stream=7)
    lats = []
    for k in range(ndom):
        n = sides[min(3, int(draws[k] * 4))]
        p, rho0, T0 = W.droplet(Tc, rv, rl, n=n, R=n / 4.0, seed=seed + k)
        p["schedule"] = lbm.SCHED_SLABS
        lats.append(lbm.Lattice(p, torch.tensor(rho0.reshape(-1), dtype=torch.float32, device="cuda"),
                                torch.tensor(T0.reshape(-1), dtype=torch.float32, device="cuda"),
                                stream=stream.cuda_stream))
    cells = sum(l.N for l in lats)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    # one domain after another
    for l in lats:
        l.lbm_step(8)
    e0, e1 = ev(), ev()
    torch.cuda.synchronize()
    e0.record(stream)
    for l in lats:
        l.lbm_step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    b = lbm.Batch(lats)
    shape = b.lbm_batch_tune()
    b.lbm_batch_step(8)
    e2, e3 = ev(), ev()
    torch.cuda.synchronize()
    e2.record(stream)
    b.lbm_batch_step(steps)
    e3.record(stream)
    torch.cuda.synchronize()
    st = b.lbm_batch_sync()
    bat_ms = e2.elapsed_time(e3)
    b.close()
    for l in lats:
        l.close()
    if st != lbm.OK:
        raise SystemExit(f"batched run failed: {lbm.lbm_status_string(st)}")
    mlups = cells * steps / (bat_ms * 1e-3) / 1e6
    return {"workload": f"{ndom} droplet domains, sides drawn from {{32,48,64,96}} (seed {seed}), R = side/4, "
                        f"open faces, {cells} cells, {steps} steps",
            "value": mlups, "unit": "MLUPS", "ms_per_step": bat_ms / steps,
            "shape": {"threads": shape[0], "ctas_per_sm": shape[1], "tile_cells": shape[2],
                      "mode": "one launch per phase" if shape[1] == 0 else "persistent cooperative launch"},
            "one_after_another_MLUPS": cells * steps / (seq_ms * 1e-3) / 1e6,
            "step_effective_GBs": BYTES_PER_LU * mlups * 1e6 / 1e9}


def large_pool(lbm, Tc, rv, rl, stream, steps=100, warmup=10):
    """512^3 heated-plate pool with 64 droplets (R in [10, 25), seeded), periodic in
    x and y, bottom wall at 0.96 T_c, open top, FP16-shifted storage, slab
    schedule: throughput over `steps` steps after `warmup`, and the step's
    effective bandwidth for its 104 algorithmic bytes per lattice update (26
    16-bit populations read and written) against the measured HBM peak."""
    import torch
    p, rho0, T0 = W.pool(Tc, rv, rl)
    p["schedule"] = lbm.SCHED_SLABS
    rho_d = torch.from_numpy(rho0.reshape(-1)).to("cuda")
    T_d = torch.from_numpy(T0.reshape(-1)).to("cuda")
    del rho0, T0
    lat = lbm.Lattice(p, rho_d, T_d, stream=stream.cuda_stream)
    lat.lbm_step(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.lbm_step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    st = lat.lbm_sync()
    N = lat.N
    lat.close()
    if st != lbm.OK:
        raise SystemExit(f"pool run failed: {lbm.lbm_status_string(st)}")
    ms = e0.elapsed_time(e1) / steps
    mlups = N / (ms * 1e-3) / 1e6
    step_bytes = 26 * 2 * STORAGE["f16"][1]
    peak = peaks().get("hbm_gbs", 6800.0)
    return {"workload": "heated-plate pool 512^3, 64 droplets R in [10,25) (seed 2206), periodic x/y, "
                        "bottom wall 0.96 T_c, open top, FP16-shifted storage, slab schedule",
            "cells": N, "steps": steps, "warmup": warmup, "value": mlups, "unit": "MLUPS", "ms_per_step": ms,
            "step_bytes_per_lu": step_bytes, "step_effective_GBs": step_bytes * mlups * 1e6 / 1e9,
            "step_frac": step_bytes * mlups * 1e6 / 1e9 / peak}


def vartheta_cost(lbm, p, rho0, T0, stream, steps=2000, warmup=50):
    """Step time of the workload with the correction term of Eq. 16 (vartheta = 1) against
    without, both in the slab schedule; the paper compares the two in CPU time (Table 1)."""
    import torch
    rho_d = torch.tensor(rho0.reshape(-1), dtype=torch.float32, device="cuda")
    T_d = torch.tensor(T0.reshape(-1), dtype=torch.float32, device="cuda")
    ms = {}
    for vt in (0, 1):
        lat = lbm.Lattice(dict(p, vartheta=vt, schedule=lbm.SCHED_SLABS), rho_d, T_d, stream=stream.cuda_stream)
        lat.lbm_step(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.lbm_step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        st = lat.lbm_sync()
        lat.close()
        if st != lbm.OK:
            raise SystemExit(f"vartheta={vt} run failed: {lbm.lbm_status_string(st)}")
        ms[vt] = e0.elapsed_time(e1) / steps
    return {"ms_per_step_vartheta0": ms[0], "ms_per_step_vartheta1": ms[1], "ratio": ms[1] / ms[0],
            "paper_cpu_ratio": 55983.6 / 54461.5, "steps": steps}


def storage_cost(lbm, p, rho0, T0, stream, steps=2000, warmup=50):
    """MLUPS of the workload in each population storage form (slab schedule): FP32, FP16 and
    BF16 with one global shift, and FP16 with per-cell references.  A form whose run reports an error
    status is recorded with that status instead of a rate."""
    import torch
    rho_d = torch.tensor(rho0.reshape(-1), dtype=torch.float32, device="cuda")
    T_d = torch.tensor(T0.reshape(-1), dtype=torch.float32, device="cuda")
    N = p["nx"] * p["ny"] * p["nz"]
    out = {"steps": steps}
    for name in ("f32", "f16", "bf16", "f16local"):
        lat = None
        try:
            lat = lbm.Lattice(dict(p, storage=STORAGE[name][0], schedule=lbm.SCHED_SLABS), rho_d, T_d,
                              stream=stream.cuda_stream)
            lat.lbm_step(warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            lat.lbm_step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            st = lat.lbm_sync()
            ms = e0.elapsed_time(e1) / steps
            out[name] = {"mlups": N / (ms * 1e-3) / 1e6, "ms_per_step": ms} if st == lbm.OK else \
                {"status": lbm.lbm_status_string(st)}
        except Exception as exc:  # a form that fails is reported in its entry, not fatal to the line
            out[name] = {"status": f"{type(exc).__name__}: {exc}"}
        finally:
            if lat is not None:
                lat.close()
    for name in ("f16", "bf16", "f16local"):
        if "mlups" in out["f32"] and "mlups" in out[name]:
            out[f"{name}_over_f32"] = out[name]["mlups"] / out["f32"]["mlups"]
    return out


def paper_cases(lbm, Tc, rv, rl, stream, steps=400, warmup=20):
    """Rates of the paper's own geometries, FP32, slab schedule: the d^2-law droplet of Sec. 4.2
    as the paper runs it (100^3, R = 25, periodic velocity field, every boundary node layer held
    at T_c) and the droplet on a heated surface of Sec. 4.3 (160 x 160 x 100, diameter 70,
    contact angle 120 degrees, wall at 0.8931 T_c, the paper's a = 3/49)."""
    import torch
    out = {}
    pa = W.base_params(4, 4, 4, a=3.0 / 49.0)
    Tc3 = lbm.lbm_Tc(pa)
    cases = {"sec42_droplet_100": W.droplet(Tc, rv, rl, n=100, R=25.0, faces=W.PERIODIC),
             "sec43_heated_surface_160x160x100": W.heated_surface(Tc3, rv, rl)}
    for name, (p, rho0, T0) in cases.items():
        p = dict(p, schedule=lbm.SCHED_SLABS)
        N = p["nx"] * p["ny"] * p["nz"]
        lat = lbm.Lattice(p, torch.tensor(rho0.reshape(-1), dtype=torch.float32, device="cuda"),
                          torch.tensor(T0.reshape(-1), dtype=torch.float32, device="cuda"), stream=stream.cuda_stream)
        lat.lbm_step(warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.lbm_step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        st = lat.lbm_sync()
        lat.close()
        ms = e0.elapsed_time(e1) / steps
        out[name] = ({"cells": N, "steps": steps, "value": N / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms}
                     if st == lbm.OK else {"status": lbm.lbm_status_string(st)})
    return out


def thermo_product():
    """T_c and the coexistence densities from the library's host helpers (not the oracle)."""
    from paper_2206_00946_gb300 import lbm
    p = W.base_params(4, 4, 4)
    Tc = lbm.lbm_Tc(p)
    rv, rl, _ = lbm.lbm_maxwell(p, 0.86 * Tc)
    return Tc, rv, rl


def cpu_oracle_sample(p, rho0, T0, steps: int, omp: bool = False):
    """Oracle (FP64, as it stands; omp=True: the same source built with OpenMP over z, all
    host cores) on the workload for `steps` steps; returns (MLUPS, seconds, threads)."""
    from oracle import Oracle
    o = Oracle(p, omp=omp)
    threads = o.threads()
    f, g = o.init_state(rho0, T0)
    t0 = time.perf_counter()
    st, f, g = o.run(f, g, steps)
    dt = time.perf_counter() - t0
    return p["nx"] * p["ny"] * p["nz"] * steps / dt / 1e6, dt, threads


def sub_box(p, rho0, T0, s, sz):
    """A centred s x s x sz sub-box of a workload (z from the bottom: the wall and the
    droplet stay in it), the same face kinds."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    s, sz = min(s, nx, ny), min(sz, nz)
    x0, y0 = (nx - s) // 2, (ny - s) // 2
    z0 = 0 if p["face_kind"][4] == W.WALL else (nz - sz) // 2
    sl = (slice(z0, z0 + sz), slice(y0, y0 + s), slice(x0, x0 + s))
    r, t = (np.ascontiguousarray(a.reshape(nz, ny, nx)[sl]) for a in (rho0, T0))
    return dict(p, nx=s, ny=s, nz=sz), r, t


def run_reference(args, rank, world):
    """The oracle on all host cores (its OpenMP build): each timed step one lattice update of
    the workload, or of a centred sub-box of it when the whole run would exceed ~2 minutes."""
    if rank != 0:
        return 0
    from oracle import Oracle
    o0 = Oracle(W.base_params(4, 4, 4))
    Tc = o0.Tc()
    rv, rl, _ = o0.maxwell(0.86 * Tc)
    p, rho0, T0 = workload(args.workload, Tc, rv, rl)
    # calibrate the rate on a small box, then size the sample to the budget
    q, r, t = sub_box(p, rho0, T0, 32, 32)
    rate, _, threads = cpu_oracle_sample(q, r, t, 2, omp=True)
    budget_s = 120.0
    cells = int(budget_s * rate * 1e6 / max(1, args.steps + args.warmup))
    N = p["nx"] * p["ny"] * p["nz"]
    if cells >= N:
        q, r, t = p, rho0, T0
        sample = f"the whole {args.workload} workload, one lattice update per timed step"
    else:
        frac = (cells / N) ** (1.0 / 3.0)
        sxy = max(8, int(frac * min(p["nx"], p["ny"])))
        sz = max(8, int(frac * p["nz"]))
        q, r, t = sub_box(p, rho0, T0, sxy, sz)
        sample = (f"{q['nx']}x{q['ny']}x{q['nz']} centred sub-box of the {args.workload} workload, "
                  f"one lattice update per timed step")
    o = Oracle(q, omp=True)
    f, g = o.init_state(r, t)
    _, f, g = o.run(f, g, args.warmup)
    t0 = time.perf_counter()
    _, f, g = o.run(f, g, args.steps)
    dt = time.perf_counter() - t0
    mlups = q["nx"] * q["ny"] * q["nz"] * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "sample": sample},
            "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def droplet_rate(lbm, Tc, rv, rl, stream, steps=2000, warmup=50):
    """Steady rate of the 128^3 d^2-law droplet (open faces on all six sides), slab schedule, FP32."""
    import torch
    p, rho0, T0 = workload("droplet", Tc, rv, rl)
    p["schedule"] = lbm.SCHED_SLABS
    N = p["nx"] * p["ny"] * p["nz"]
    lat = lbm.Lattice(p, torch.tensor(rho0.reshape(-1), dtype=torch.float32, device="cuda"),
                      torch.tensor(T0.reshape(-1), dtype=torch.float32, device="cuda"), stream=stream.cuda_stream)
    lat.lbm_step(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.lbm_step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    st = lat.lbm_sync()
    lat.close()
    if st != lbm.OK:
        raise SystemExit(f"droplet run failed: {lbm.lbm_status_string(st)}")
    ms = e0.elapsed_time(e1) / steps
    mlups = N / (ms * 1e-3) / 1e6
    peak = peaks().get("hbm_gbs", 6800.0)
    return {"workload": WORKLOADS["droplet"], "steps": steps, "value": mlups, "unit": UNIT, "ms_per_step": ms,
            "step_frac": BYTES_PER_LU * mlups * 1e6 / 1e9 / peak}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sessile", choices=list(WORKLOADS))
    ap.add_argument("--n", type=int, default=128, help="lattice side of the droplet workload (128)")
    ap.add_argument("--schedule", default="slabs", choices=["fused", "phases", "slabs"])
    ap.add_argument("--storage", default="f32", choices=list(STORAGE))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward cost measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-domains measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the 512^3 FP16 pool measurement")
    ap.add_argument("--adjoint-side", type=int, default=64, help="cube side of the adjoint workload (64)")
    ap.add_argument("--no-vartheta", action="store_true", help="skip the vartheta = 1 cost measurement")
    ap.add_argument("--no-storage", action="store_true", help="skip the storage-form comparison")
    ap.add_argument("--no-droplet", action="store_true", help="skip the 128^3 droplet rate")
    ap.add_argument("--no-paper-cases", action="store_true", help="skip the Sec. 4.2 and 4.3 geometries")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank, world, local = dist_env()

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    from paper_2206_00946_gb300 import lbm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    Tc, rv, rl = thermo_product()
    p, rho0, T0 = workload(args.workload, Tc, rv, rl, args.n)
    p["schedule"] = {"fused": lbm.SCHED_FUSED, "phases": lbm.SCHED_PHASES, "slabs": lbm.SCHED_SLABS}[args.schedule]
    p["storage"], esize = STORAGE[args.storage]
    step_bytes = 26 * 2 * esize  # algorithmic bytes per lattice update in this storage
    N = p["nx"] * p["ny"] * p["nz"]
    stream = torch.cuda.current_stream()
    rho_d = torch.tensor(rho0.reshape(-1), dtype=torch.float32, device="cuda")
    T_d = torch.tensor(T0.reshape(-1), dtype=torch.float32, device="cuda")
    lat = lbm.Lattice(p, rho_d, T_d, stream=stream.cuda_stream)
    launches = lat.lbm_step_launches(args.steps)

    # warm-up
    lat.lbm_step(args.warmup)
    torch.cuda.synchronize()
    st = lat.lbm_sync()
    if st != lbm.OK:
        raise SystemExit(f"warm-up failed: {lbm.lbm_status_string(st)}")

    # timed region: K steps, bracketed by barrier + synchronize, CUDA events on the launch stream
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        time.sleep(0.5)  # let the sampler start before the timed region
        e0.record(stream)
        lat.lbm_step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    st = lat.lbm_sync()
    if st != lbm.OK:
        raise SystemExit(f"timed run failed: {lbm.lbm_status_string(st)}")
    dev = "cuda" if (dist and dist.get_backend() == "nccl") else "cpu"
    s_max, lups = job_throughput(dist, ms * 1e-3, N * args.steps, dev)
    ms_step = s_max * 1e3 / args.steps
    value = lups / 1e6

    lat.close()

    # Per-kernel device time from the library's launch timing (CUDA events on each
    # kernel's launch stream).  The slab schedule runs every phase as many
    # concurrent sub-range launches, so its kernels are timed here in the phase
    # schedule: the same kernels, one launch per phase over the whole lattice.
    nl = min(args.steps, 200)
    q = dict(p, schedule=p["schedule"] if args.schedule == "fused" else lbm.SCHED_PHASES)
    latp = lbm.Lattice(q, rho_d, T_d, stream=stream.cuda_stream)
    latp.lbm_step(args.warmup)
    latp.lbm_profile(True)
    latp.lbm_step(nl)
    prof = latp.lbm_profile_read()
    latp.lbm_profile(False)
    latp.close()
    dom = max(prof, key=lambda k: prof[k][1])
    per_launch_ms = prof[dom][1] / prof[dom][0]

    # end to end through the C ABI with host buffers: init from host fields, K steps, macros to host
    # host buffers in pinned (page-locked) memory, the form a caller streaming fields would use
    def pinned(n):
        return torch.empty(n, dtype=torch.float32, pin_memory=True).numpy()
    rho_h, T_h = pinned(N), pinned(N)
    rho_h[:] = rho0.reshape(-1)
    T_h[:] = T0.reshape(-1)
    outs = {k: pinned(N) for k in ("rho", "ux", "uy", "uz", "T")}
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    lat2 = lbm.Lattice(p, rho_h, T_h, stream=stream.cuda_stream)
    lat2.lbm_step(args.steps)
    st2 = lat2.lbm_macros(**outs)
    e2e_s = time.perf_counter() - t0
    lat2.close()
    if st2 != lbm.OK:
        raise SystemExit(f"e2e run failed: {lbm.lbm_status_string(st2)}")
    e2e_value = job_throughput(dist, e2e_s, N * args.steps, dev)[1] / 1e6

    adj = None
    if args.storage == "f32" and not args.no_adjoint:
        adj = adjoint_cost(lbm, Tc, rv, rl, p["schedule"], stream, side=args.adjoint_side)
    batched = None
    if args.storage == "f32" and not args.no_batched:
        batched = batched_throughput(lbm, Tc, rv, rl, stream)
    large = None
    if args.storage == "f32" and not args.no_large:
        large = large_pool(lbm, Tc, rv, rl, stream)
    vartheta = None
    if args.storage == "f32" and not args.no_vartheta:
        vartheta = vartheta_cost(lbm, p, rho0, T0, stream)
    storage_forms = None
    if args.storage == "f32" and not args.no_storage:
        storage_forms = storage_cost(lbm, p, rho0, T0, stream)
    droplet = None
    if args.workload != "droplet" and not args.no_droplet:
        droplet = droplet_rate(lbm, Tc, rv, rl, stream)
    papers = None
    if args.storage == "f32" and not args.no_paper_cases:
        papers = paper_cases(lbm, Tc, rv, rl, stream)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    pk = peaks()
    peak = pk.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in pk else "fallback"
    alg = kernel_alg_bytes(dom, esize)
    achieved = alg * N / (per_launch_ms * 1e-3) / 1e9 if alg else None
    digest = kernel_digest()
    traffic = ncu_traffic(dom + ("" if args.storage == "f32" else "_" + args.storage), digest, N)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        # the oracle as it stands on all host cores (OpenMP over z) and on one core, on whole
        # steps of the same workload
        mlups_omp, dt_omp, threads = cpu_oracle_sample(p, rho0, T0, 2, omp=True)
        mlups_1, dt_1, _ = cpu_oracle_sample(p, rho0, T0, 1)
        cpu = {"value": mlups_omp, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"2 full steps of the {args.workload} workload ({dt_omp:.1f} s, OpenMP over z, "
                         f"{threads} threads)",
               "single_thread": {"value": mlups_1, "unit": UNIT, "cores": 1,
                                 "sample": f"1 full step of the {args.workload} workload ({dt_1:.1f} s)"}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": (WORKLOADS[args.workload] if args.workload == "sessile" or args.n == 128
                                else WORKLOADS["droplet"].replace("128^3", f"{args.n}^3")),
                   "cells": N, "schedule": args.schedule, "parallelism": f"replicas x{world}",
                   "storage": {"f32": "f32", "f16": "f16 shifted by w_i rho_ref / w_i T_ref",
                               "bf16": "bf16 shifted by w_i rho_ref / w_i T_ref",
                               "f16local": "f16 shifted by w_i rho / w_i T of the cell before the step"}[args.storage],
                   "l2": f"inputs larger than L2: {2 * 26 * esize * N / 1e6:.0f} MB of double-buffered populations"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": traffic,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)",
                     "kernel": dom, "alg_bytes_per_cell": alg, "per_launch_ms": per_launch_ms,
                     "kernel_timing": "CUDA events on the kernel's stream, phase schedule, whole-lattice launches",
                     "kernel_src_sha": digest,
                     "step_bytes_per_lu": step_bytes,
                     "step_effective_GBs": step_bytes * N / (ms_step * 1e-3) / 1e9,
                     "step_frac": step_bytes * N / (ms_step * 1e-3) / 1e9 / peak,
                     "kernels": {k: {"launches": v[0], "ms_per_launch": v[1] / v[0],
                                     "share": v[1] / sum(w[1] for w in prof.values())} for k, v in prof.items()}},
        "cpu_baseline": cpu,
        "droplet_128": droplet,
        "paper_cases": papers,
        "adjoint": adj,
        "batched": batched,
        "large": large,
        "vartheta": vartheta,
        "storage_forms": storage_forms,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * N / args.steps,
                "d2h_bytes_per_step": 5 * 4 * N / args.steps},
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
