#!/usr/bin/env python
"""Benchmark of the coupled pore-scale CDI path on GB300.

One step = the whole hot path on one synthetic electrode image: Stokes flow
by lattice Boltzmann to steady state, the potential solve, the explicit time
step bound, the Nernst-Planck transport steps, and the outputs (adsorbed
amount, outlet concentration, mass balance).  The metric is coupled
lattice-site updates per second,
    (flow steps x flow sites + transport steps x cells) / time,
in MLUPS, with the dominant kernel's bandwidth against the measured HBM peak.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   (the FP64 CPU oracle, as it stands)
    python bench.py --accuracy [--workload NAME]   (per-field error of the
        benchmark's storage against FP64 storage at full size and horizon)

The default workload is the 3D 256^3 sphere pack: its working set (2.3 GB of
populations) is far above the 129 MB L2, so the roofline fraction measures
HBM bandwidth.  The 2D 1024x512 pack stays reachable with --workload.

Under torchrun each rank runs its own instance (independent problems, no
data-path collective; weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2110_13055_gb300 import cdi, inputs  # noqa: E402

METRIC = "coupled MLUPS & % HBM peak; sweep solves/s + p99 latency vs plain, equal error"

WORKLOADS = {
    "2d-1024x512": dict(
        desc=("2D 1024x512 polydisperse discs r~U[4,16] lu (overlap), porosity 0.5, seed 1; "
              "D2Q9 BGK tau=1, body force 1e-6 lu, Stokes to K-lag residual 1e-8 (FP64 "
              "residual, K=100), mirror along x, periodic laterally; screened potential at "
              "0.8 V (c_bulk 10 mol/m^3, dx 100 nm); Na+/Cl- z=+1/-1, D=1.33e-9/2.03e-9 m^2/s, "
              "c0=10 mol/m^3, Ka=1e-6 m/s, pore-mean velocity 1e-4 m/s; 50000 explicit "
              "Nernst-Planck steps; FP32 arithmetic: populations stored as FP32 pairs "
              "(plain FP32 stalls at residual 7e-7 with a 4e-5 velocity error here), "
              "transport in FP32 with FP32-pair concentrations"),
        mask=lambda: inputs.disc_pack_1024x512()[0], prec=cdi.FP32_SPLIT, V=0.8, U=1e-4, c0=10.0,
        np_steps=50000, flow_tol=1e-8, max_flow=1_000_000),
    "2d-2048x1024": dict(
        desc=("2D 2048x1024 polydisperse discs r~U[4,16] lu (overlap), porosity 0.5, seed 1; "
              "as 2d-1024x512 but the populations exceed L2; flow to 1e-8; "
              "50000 Nernst-Planck steps; FP32 pair populations and concentrations"),
        mask=lambda: inputs.grain_pack((1024, 2048), 0.5, 4.0, 16.0, seed=1)[0],
        prec=cdi.FP32_SPLIT, V=0.8, U=1e-4, c0=10.0, np_steps=50000, flow_tol=1e-8,
        max_flow=1_000_000),
    "3d-256": dict(
        desc=("3D 256^3 sphere pack r~U[6,12] lu (overlap), porosity 0.45, seed 2; D3Q19 BGK "
              "tau=1, body force 1e-6 lu, mirror along x; Stokes to K-lag residual 1e-7 (FP64 "
              "residual, K=100; 11200 steps on this pack), capped at 20000; 1.2 V, "
              "c0=20 mol/m^3, pore-mean "
              "velocity 1e-6 m/s; 20000 Nernst-Planck steps; FP32 populations, transport "
              "in FP32 with FP32-pair concentrations (plain FP32 concentrations drift to a "
              "1e-5 adsorbed-amount error over the 20000 steps)"),
        mask=lambda: inputs.sphere_pack_256()[0], prec=cdi.FP32_CPAIR, V=1.2, U=1e-6, c0=20.0,
        np_steps=20000, flow_tol=1e-7, max_flow=20000),
    "3d-160": dict(
        desc=("3D 160^3 sphere pack r~U[6,12] lu (overlap), porosity 0.45, seed 2 (a profiling "
              "case of the 256^3 recipe whose populations still exceed L2); D3Q19 tau=1; flow "
              "capped at 20000 steps; 1.2 V, c0=20 mol/m^3; 20000 Nernst-Planck steps; FP32"),
        mask=lambda: inputs.grain_pack((160, 160, 160), 0.45, 6.0, 12.0, seed=2)[0],
        prec=cdi.FP32_CPAIR, V=1.2, U=1e-6, c0=20.0, np_steps=20000, flow_tol=1e-7,
        max_flow=20000),
    "2d-128x64": dict(
        desc=("2D 128x64 non-overlapping discs r=6 lu, porosity 0.6, seed 0; D2Q9 tau=1, "
              "Stokes to residual 1e-8; 1.0 V; Na+/Cl-, c0=10 mol/m^3; 2000 Nernst-Planck "
              "steps; FP64"),
        mask=lambda: inputs.disc_pack_128x64()[0], prec=cdi.FP64, V=1.0, U=1e-4, c0=10.0,
        np_steps=2000, flow_tol=1e-8, max_flow=1_000_000),
}

Z, D = (1, -1), (1.33e-9, 2.03e-9)
REASONS = {  # nvidia-smi clocks_event_reasons bit names
    0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
    0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
    0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
    0x100: "display_clock_setting"}


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Clocks:
    """nvidia-smi samples (SM clock, max clock, throttle reasons) every 200 ms."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 3:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                bits = int(parts[2], 16)
            except ValueError:
                continue
            for b, name in REASONS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


KERNEL_SOURCES = {"k_lbm_step": "flow.cu", "k_np_step": "transport.cu"}


def kernel_hash(kernel):
    """Hash of the source file that defines the kernel and the shared header."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2110_13055_gb300", "csrc")
    for f in (KERNEL_SOURCES[kernel], "cdi_internal.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """Per-launch DRAM bytes of the kernel on this workload from a committed
    ncu summary, if it was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p)).get(kernel, {}).get(workload)
    except (OSError, ValueError, AttributeError):
        return None
    if not rec or rec.get("source_sha") != kernel_hash(kernel):
        return None
    return rec.get("dram_bytes_per_launch")


def roofline_bound(traffic, abytes, layout):
    """"l2" when the recorded DRAM traffic per launch is well below the bytes
    the kernel touches (its working set stayed in L2 between launches), else
    "hbm" (also when no traffic was recorded on the current source)."""
    if traffic is not None and traffic < 0.8 * (abytes + layout):
        return "l2"
    return "hbm"


def aggregate(elapsed, units):
    """Whole-job figures under torchrun: the max over ranks of the timed
    region and the sum of the units every rank processed (a host-side gloo
    reduction of two numbers; the ranks' solves never exchange data)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return elapsed, float(units)
    t = torch.tensor([float(elapsed)], dtype=torch.float64)
    u = torch.tensor([float(units)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return t.item(), u.item()


def algorithmic_bytes(prec, dim, n_flow_pore, n_pore, ns=2):
    """Per-launch algorithmic bytes of the two step kernels, counted from the
    method alone (populations and fields, per site and per cell):
    LBM: Q populations read and written per pore site (4 B FP32, 8 B FP64 or
    an FP32 pair, 2 B BF16); transport: ns concentrations read and written,
    dim velocity components, the potential (4 B in FP32 storage, 8 B in FP64)
    and a 1-byte solid mask per pore cell.  Returned beside them, the bytes
    the compact layout adds per launch: the odd LBM step's neighbour data
    (averaged over the even/odd pair) and the transport step's potential low
    words, rank metadata and lateral neighbour ranks."""
    Tp = {cdi.FP64: 8, cdi.FP32: 4, cdi.FP32_SPLIT: 8, cdi.BF16_POP: 2,
          cdi.FP32_CPAIR: 4}[prec]
    Tt = 8 if prec == cdi.FP64 else 4
    Tc = 8 if prec in (cdi.FP64, cdi.FP32_SPLIT, cdi.FP32_CPAIR) else 4  # a pair is 8 B
    Q = 9 if dim == 2 else 19
    lbm = n_flow_pore * Q * 2 * Tp
    # odd step: a 4-byte flag word, one byte per lateral row offset (2 in 2D,
    # 8 in 3D; in 4-byte words) and a 32-site tile's 4-byte bases once per
    # tile; the even step reads none
    n_off = 2 if dim == 2 else 8
    lbm_layout = (n_flow_pore * (4 + (4 if dim == 2 else 8))
                  + n_off * 4 * ((n_flow_pore + 31) // 32)) // 2
    npb = n_pore * (ns * 2 * Tc + dim * Tt + Tt + 1)
    # potential low words (FP32), 2-byte face flags instead of the mask byte,
    # 2 (d - 1) lateral neighbour ranks
    np_layout = n_pore * ((8 - Tt) + 1 + 2 * (dim - 1) * 4)
    return lbm, lbm_layout, npb, np_layout


def run_pipeline(dom, w):
    """The hot path on a resident domain; returns the step's counters."""
    steps, res, st = dom.solve_flow(tol=w["flow_tol"], max_steps=w["max_flow"],
                                    U_target=w["U"], allow_not_converged=True)
    dom.set_potential(w["V"], c_bulk=w["c0"], tol=1e-12)
    dom.init_transport(Z, D, c0=w["c0"], Ka=1e-6)
    dom.step(w["np_steps"])
    G = dom.adsorbed()
    Cout = dom.outlet()
    M, _, I, O = dom.mass_balance()
    return dict(flow_steps=steps, flow_residual=res, flow_status=st, Gamma=G, C_out=Cout)


def ours(args, w, mask):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    res = cdi.TorchResources(local)
    dim = mask.ndim
    nx = mask.shape[-1]
    N = mask.size
    n_pore = int((mask == 0).sum())
    Nf = 2 * N
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    dom = cdi.Domain(mask, precision=w["prec"], torch_resources=res)
    if args.launch_shapes:
        dom.set_launch_shapes(*args.launch_shapes)
    for _ in range(args.warmup):
        run_pipeline(dom, w)
    torch.cuda.synchronize()
    dom.timing(reset=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    units = 0
    info = None
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(res.stream)
        for _ in range(args.steps):
            with torch.cuda.stream(res.stream):
                flush.zero_()          # evict the previous step's data from L2
            info = run_pipeline(dom, w)
            units += info["flow_steps"] * Nf + w["np_steps"] * N
        ev1.record(res.stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    dev_ms = ev0.elapsed_time(ev1)
    tim = dom.timing(reset=True)
    elapsed = dev_ms / 1e3
    elapsed_all, units_all = aggregate(elapsed, units)

    # dominant kernel and its roofline: algorithmic bytes per launch (the
    # method's populations and fields) over the kernel's mean launch time
    # (CUDA events the library records on the launching stream); the bytes
    # the compact layout adds are reported beside them, not counted
    n_flow_pore = 2 * n_pore
    lbm_bytes, lbm_layout, np_bytes, np_layout = algorithmic_bytes(
        w["prec"], dim, n_flow_pore, n_pore)
    lbm_avg = tim["flow_ms"] / max(tim["flow_launches"], 1) / 1e3
    np_avg = tim["np_ms"] / max(tim["np_launches"], 1) / 1e3
    if tim["flow_ms"] >= tim["np_ms"]:
        kname, abytes, layout, avg = "k_lbm_step", lbm_bytes, lbm_layout, lbm_avg
    else:
        kname, abytes, layout, avg = "k_np_step", np_bytes, np_layout, np_avg
    peak, peak_kind = measured_peak_gbs()
    achieved = abytes / avg / 1e9 if avg > 0 else 0.0
    traffic = recorded_traffic(kname, args.workload)
    bound = roofline_bound(traffic, abytes, layout)

    # end to end through the C ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        t0 = time.perf_counter()
        d2h = 0
        for _ in range(args.e2e_steps):
            d2 = cdi.Domain(mask, precision=w["prec"], torch_resources=res)   # H2D of the mask
            if args.launch_shapes:
                d2.set_launch_shapes(*args.launch_shapes)
            run_pipeline(d2, w)
            C = d2.C()                                                          # D2H of the fields
            d2.close()
            d2h = C.nbytes + 8 * 2 * 6
        torch.cuda.synchronize()
        e2e_t = time.perf_counter() - t0
        e2e = {"value": units / args.steps * args.e2e_steps / e2e_t / 1e6 * world,
               "unit": "MLUPS", "h2d_bytes_per_step": int(mask.nbytes),
               "d2h_bytes_per_step": int(d2h), "steps": args.e2e_steps}
    dom.close()

    if rank != 0:
        return None
    line = {
        "metric": METRIC,
        "value": units_all / elapsed_all / 1e6,
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if w["prec"] == cdi.FP64 else "f32",  # arithmetic type
        "storage": {cdi.FP64: "fp64", cdi.FP32: "fp32",
                    cdi.FP32_SPLIT: "fp32-pair populations and concentrations",
                    cdi.FP32_CPAIR: "fp32 populations, fp32-pair concentrations",
                    cdi.BF16_POP: "bf16 populations, fp32 transport"}[w["prec"]],
        "data": "synthetic",
        "config": {"workload": w["desc"], "name": args.workload,
                   "flow_sites": Nf, "cells": N, "pore_cells": n_pore,
                   "flow_steps": info["flow_steps"], "flow_residual": info["flow_residual"],
                   "flow_converged": info["flow_status"] == 0,
                   "np_steps": w["np_steps"], "Gamma_mol_per_m": list(info["Gamma"]),
                   "launch_shapes": (list(args.launch_shapes) if args.launch_shapes
                                     else "autotuned"),
                   "C_out_molm3": list(info["C_out"]),
                   "l2": ("flushed between steps (256 MB write); the populations "
                          f"({lbm_bytes / 2e6:.0f} MB) "
                          + ("exceed the 129 MB L2" if n_flow_pore * (9 if dim == 2 else 19) * 4 > 129e6
                             else "fit in the 129 MB L2 within a step")),
                   "phase_ms_per_step": {
                       "flow": tim["flow_ms"] / args.steps,
                       "flow_check": tim["flow_check_ms"] / args.steps,
                       "psi": tim["psi_ms"] / args.steps,
                       "np": tim["np_ms"] / args.steps},
                   "wall_s": wall},
        "roofline": {"bound": bound, "kernel": kname, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": abytes,
                     "layout_bytes_per_launch": layout,
                     "avg_launch_us": avg * 1e6,
                     "other": {
                         "k_lbm_step": {"GBps": lbm_bytes / lbm_avg / 1e9 if lbm_avg else None,
                                        "frac": lbm_bytes / lbm_avg / 1e9 / peak
                                        if lbm_avg else None,
                                        "avg_launch_us": lbm_avg * 1e6,
                                        "algorithmic_bytes_per_launch": lbm_bytes,
                                        "layout_bytes_per_launch": lbm_layout,
                                        "block": tim["lbm_block"],
                                        "shape": tim["lbm_shape"]},
                         "k_np_step": {"GBps": np_bytes / np_avg / 1e9 if np_avg else None,
                                       "frac": np_bytes / np_avg / 1e9 / peak
                                       if np_avg else None,
                                       "avg_launch_us": np_avg * 1e6,
                                       "algorithmic_bytes_per_launch": np_bytes,
                                       "layout_bytes_per_launch": np_layout,
                                       "block": tim["np_block"],
                                       "shape": tim["np_shape"]}}},
        "e2e": e2e,
        "gpu_launches": int(tim["kernel_launches"]),
        "clocks": clk.summary(),
    }
    return line


def accuracy(args, w, mask):
    """Per-field error of the workload's storage precision against FP64
    storage, both on the GPU, same mask, same parameters, full size and full
    horizon (flow to its tolerance, all transport steps).  The FP64 path
    itself matches the FP64 oracle to 1e-11 on the parity cases of the test
    suite (the oracle cannot run these sizes to convergence)."""
    import torch
    torch.cuda.set_device(0)

    def run(prec):
        with cdi.Domain(mask, precision=prec) as d:
            t0 = time.perf_counter()
            info = run_pipeline(d, dict(w, prec=prec))
            out = dict(info, u=d.u(), C=d.C(), seconds=time.perf_counter() - t0)
            out["M"], _, out["In"], out["Out"] = d.mass_balance()
        return out

    ref = run(cdi.FP64)
    got = run(w["prec"])

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    return {"metric": "per-field relative error vs FP64 storage", "data": "synthetic",
            "config": {"workload": w["desc"], "name": args.workload},
            "storage": {cdi.FP32: "fp32", cdi.FP32_SPLIT: "fp32-pair populations and "
                        "concentrations", cdi.FP32_CPAIR: "fp32 populations, fp32-pair "
                        "concentrations", cdi.BF16_POP: "bf16 populations",
                        cdi.FP64: "fp64"}[w["prec"]],
            "flow_steps": {"fp64": ref["flow_steps"], "tested": got["flow_steps"]},
            "flow_residual": {"fp64": ref["flow_residual"], "tested": got["flow_residual"]},
            "rel_l2_u": rel(got["u"], ref["u"]),
            "rel_l2_C": [rel(got["C"][k], ref["C"][k]) for k in range(len(ref["C"]))],
            "rel_Gamma": [float(abs(g - r) / abs(r)) for g, r in zip(got["Gamma"], ref["Gamma"])],
            "rel_C_out": [float(abs(g - r) / abs(r)) for g, r in zip(got["C_out"], ref["C_out"])],
            "bars": {"u": 1e-5, "C": 1e-4, "Gamma": 1e-6},
            "seconds": {"fp64": ref["seconds"], "tested": got["seconds"]}}


SWEEP_V = (0.2, 0.6, 1.0, 1.2)
SWEEP_U = (1e-5, 1e-4, 1e-3)


def sweep_bench(args):
    """Batched sweep against two one-solve-at-a-time GPU loops, at equal
    results.  Geometries: seeds 10, 11, ... of the sweep recipe (2D disc packs
    of uneven sizes 256x256 to 1024x512, porosity ~U[0.4, 0.7]); every
    (geometry, V, U) is one solve of flow + potential + transport.
      batched: all geometries' flows in one batched solve (one launch per step
        over every geometry still running, each stopping at its own check),
        then every member of every geometry in one fused transport launch per
        step (cdi_sweep_batch);
      plain: each solve from scratch through the C ABI (create, flow,
        potential, transport, queries, destroy);
      per-geometry loop: each geometry's flow solved once (Eq. 2 is linear,
        so one flow serves every velocity), then its combinations one at a
        time (rescale, potential, transport, queries).
    The BF16 population variant runs the batched transport on flows advanced
    by the same step counts and reports its difference from the FP32-pair
    results."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    torch.cuda.set_device(0)
    geoms = [inputs.sweep_instance(10 + k)[0] for k in range(args.sweep_geometries)]
    combos = [(U, V) for V in SWEEP_V for U in SWEEP_U]
    n_np = args.np_steps or 5000
    prec = cdi.FP32_SPLIT
    kw = dict(tol=1e-8, max_steps=2_000_000)

    def batched(masks):
        doms = [cdi.Domain(m, precision=prec) for m in masks]
        try:
            steps, res, st = cdi.flow_batch(doms, U_target=1e-4, allow_not_converged=True, **kw)
            g, c, _ = cdi.batch(doms, combos, n_steps=n_np)
        finally:
            for d in doms:
                d.close()
        return g, c, [int(x) for x in steps], [float(x) for x in res], [int(x) for x in st]

    def bf16(masks, flow_steps):
        doms = [cdi.Domain(m, precision=cdi.BF16_POP) for m in masks]
        try:
            def flow(i):
                return doms[i].solve_flow(U_target=1e-4, tol=1e-8, max_steps=flow_steps[i],
                                          allow_not_converged=True)[0]
            with ThreadPoolExecutor(len(doms)) as ex:
                list(ex.map(flow, range(len(doms))))
            g, c, _ = cdi.batch(doms, combos, n_steps=n_np)
        finally:
            for d in doms:
                d.close()
        return g, c

    def transport(d, U, V):
        d.set_velocity(U)
        d.set_potential(V, c_bulk=10.0, tol=1e-12)
        d.init_transport(Z, D, c0=10.0, Ka=1e-6)
        d.step(n_np)
        return d.adsorbed(), d.outlet()

    def plain(m, U, V):
        with cdi.Domain(m, precision=prec) as d:
            d.solve_flow(U_target=U if U else 1e-4, allow_not_converged=True, **kw)
            return transport(d, U, V)

    batched([inputs.sweep_instance(9)[0]])          # warm-up (kernel loading, graphs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g_b, c_b, steps, residuals, status = batched(geoms)
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    g_h, c_h = bf16(geoms, steps)
    t_h = time.perf_counter() - t0
    # per-geometry loop: one flow per geometry, combinations one at a time
    lat_g, g_g, c_g = [], [], []
    t0 = time.perf_counter()
    for m in geoms:
        t = time.perf_counter()
        with cdi.Domain(m, precision=prec) as d:
            d.solve_flow(U_target=1e-4, allow_not_converged=True, **kw)
            t_flow = time.perf_counter() - t
            for U, V in combos:
                t = time.perf_counter()
                g, c = transport(d, U, V)
                lat_g.append(time.perf_counter() - t + t_flow / len(combos))
                g_g.append(g)
                c_g.append(c)
    t_g = time.perf_counter() - t0
    g_g = np.array(g_g).reshape(g_b.shape)
    c_g = np.array(c_g).reshape(c_b.shape)
    n_solves = len(geoms) * len(combos)
    lat_b = [t_b] * n_solves                       # every member finishes with the batch
    out = {
        "metric": "sweep solves/s (batched vs one-at-a-time GPU loops, equal results)",
        "value": n_solves / t_b, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "storage": "fp32-pair populations and concentrations",
        "data": "synthetic",
        "config": {"workload": (f"{len(geoms)} 2D disc packs of the sweep recipe (seeds 10.."
                                f"{9 + len(geoms)}; sizes "
                                + ", ".join(f"{m.shape[1]}x{m.shape[0]}" for m in geoms)
                                + f") x V {SWEEP_V} x U {SWEEP_U}; flow to 1e-8 per geometry; "
                                f"{n_np} Nernst-Planck steps per solve; wall-clock through the "
                                "C ABI with host buffers"),
                   "solves": n_solves, "flow_steps": steps, "flow_residuals": residuals,
                   "flows_converged": sum(1 for x in status if x == 0),
                   "flow_cap_steps": kw["max_steps"]},
        "batched": {"value": n_solves / t_b, "p50_s": float(np.percentile(lat_b, 50)),
                    "p99_s": float(np.percentile(lat_b, 99)), "seconds": t_b},
        "per_geometry_loop": {"value": n_solves / t_g, "p50_s": float(np.percentile(lat_g, 50)),
                              "p99_s": float(np.percentile(lat_g, 99)), "seconds": t_g,
                              "results_bitwise_equal": bool(np.array_equal(g_b, g_g)
                                                            and np.array_equal(c_b, c_g))},
        "speedup_vs_per_geometry_loop": t_g / t_b,
        "bf16_populations": {
            "value": n_solves / t_h, "seconds": t_h,
            "max_rel_gamma_diff_vs_fp32_pair": float(np.max(np.abs(g_h - g_b) / np.abs(g_b))),
            "max_rel_cout_diff_vs_fp32_pair": float(np.max(np.abs(c_h - c_b) / np.abs(c_b)))},
    }
    if args.sweep_plain:
        lat_p, g_p, c_p = [], [], []
        t0 = time.perf_counter()
        for m in geoms:
            for U, V in combos:
                t = time.perf_counter()
                g, c = plain(m, U, V)
                lat_p.append(time.perf_counter() - t)
                g_p.append(g)
                c_p.append(c)
        t_p = time.perf_counter() - t0
        g_p = np.array(g_p).reshape(g_b.shape)
        c_p = np.array(c_p).reshape(c_b.shape)
        out["plain"] = {"value": n_solves / t_p, "p50_s": float(np.percentile(lat_p, 50)),
                        "p99_s": float(np.percentile(lat_p, 99)), "seconds": t_p,
                        "results_bitwise_equal": bool(np.array_equal(g_b, g_p)
                                                      and np.array_equal(c_b, c_p))}
        out["speedup_vs_plain"] = t_p / t_b
    return out


_SERVE_MASKS = {}


def serve_requests(n, seed=100):
    """Mixed request stream of the serving recipe (seeds seed, seed + 1, ...):
    half 2D 512x512 disc packs (FP32-pair flow to 1e-8, U = 1e-4 m/s), half 3D
    sphere packs n^3, n in {64, 96, 128, 160, 192} (FP32 flow to 1e-7, U =
    1e-6 m/s, c0 = 20 mM); porosity ~U[0.4, 0.6], potential ~U[0.2, 1.2] V,
    2000 transport steps per request."""
    from paper_2110_13055_gb300 import serve
    reqs = []
    for i in range(n):
        if seed + i not in _SERVE_MASKS:
            _SERVE_MASKS[seed + i] = inputs.serve_instance(seed + i)
        m, V = _SERVE_MASKS[seed + i]
        if m.ndim == 2:
            reqs.append(serve.Request(m, V, 1e-4, 2000, precision=cdi.FP32_SPLIT,
                                      flow_tol=1e-8, tag=i))
        else:
            reqs.append(serve.Request(m, V, 1e-6, 2000, precision=cdi.FP32_CPAIR, flow_tol=1e-7,
                                      max_flow_steps=200_000, c0=20.0, tag=i))
    return reqs


def serve_bench(args):
    """Poisson arrivals at rates around the sequential capacity, the
    continuous-batching server against the plain sequential loop."""
    from paper_2110_13055_gb300 import serve
    n = args.serve_requests
    # the request geometries, built on all host cores before the first GPU
    # call (a spawned pool: no CUDA state is forked)
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    seeds = [7] + [100 + i for i in range(n)]
    with ProcessPoolExecutor(max_workers=os.cpu_count(),
                             mp_context=mp.get_context("spawn")) as ex:
        for sd, mv in zip(seeds, ex.map(inputs.serve_instance, seeds, chunksize=4)):
            _SERVE_MASKS[sd] = mv
    import torch
    torch.cuda.set_device(0)
    serve.solve(serve_requests(1, seed=7)[0])           # warm-up
    # capacity of the plain loop (back-to-back, no waiting)
    probe = serve_requests(n, seed=100)
    t0 = time.perf_counter()
    serve.run_sequential(probe, [0.0] * n)
    cap = n / (time.perf_counter() - t0)
    out = {"metric": "served solves/s and p99 latency vs plain sequential loop",
           "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
           "config": {"requests_per_rate": n, "mix": serve_requests.__doc__.strip(),
                      "sequential_capacity_solves_per_s": cap, "slots": args.serve_slots,
                      "memory_budget_GiB": args.serve_budget_gib},
           "rates": []}
    rs = np.random.default_rng(5)
    for frac in args.serve_rates:
        rate = frac * cap
        arrivals = list(np.cumsum(rs.exponential(1.0 / rate, size=n)))
        seq = serve.run_sequential(serve_requests(n, seed=100), arrivals)
        srv = serve.run_served(serve_requests(n, seed=100), arrivals, slots=args.serve_slots,
                               memory_budget=int(args.serve_budget_gib * (1 << 30)))
        same = all(np.array_equal(a.result["Gamma"], b.result["Gamma"])
                   for a, b in zip(sorted(seq, key=lambda r: r.tag),
                                   sorted(srv, key=lambda r: r.tag)))
        out["rates"].append({"offered_fraction_of_capacity": frac, "rate_per_s": rate,
                             "sequential": serve.latency_stats(seq),
                             "served": serve.latency_stats(srv),
                             "results_bitwise_equal": same})
    best = max(r["served"]["solves_per_s"] for r in out["rates"])
    out["value"] = best
    return out


def oracle_sample(mask, w, flow_steps, np_steps, threads=1):
    """Time the FP64 oracle as it stands on a bounded sample of the workload:
    flow_steps LBM steps on the full flow grid, the potential solve, np_steps
    transport steps on the full grid, on `threads` host threads.  Returns
    (MLUPS, seconds, sample text)."""
    import oracle as O
    O.build()
    O.set_threads(threads)
    N = mask.size
    t0 = time.perf_counter()
    uf, *_ = O.lbm(mask, tol=0.0, check_every=flow_steps, max_steps=flow_steps)
    u, _ = O.velocity_export(mask, uf, w["U"])
    ps, *_ = O.psi(mask, -w["V"], c_bulk=w["c0"], tol=1e-12)
    dt = O.np_dt(mask, u, ps, Z, D)
    O.np_run(mask, u, ps, Z, D, c0=w["c0"], dt=dt, n_steps=np_steps)
    t = time.perf_counter() - t0
    units = flow_steps * 2 * N + np_steps * N
    return units / t / 1e6, t, (f"{flow_steps} LBM steps on the full {2 * N}-site flow grid + "
                                f"potential solve + {np_steps} transport steps on {N} cells, "
                                f"{threads} host thread{'s' if threads > 1 else ''}")


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def cpu_baselines(mask, w, flow_steps, np_steps):
    """The oracle on one host core and on all host cores (OpenMP), each on a
    bounded sample of the workload (the all-core sample is scaled up by the
    core count so that both take comparable time)."""
    cores = host_cores()
    v1, t1, s1 = oracle_sample(mask, w, flow_steps, np_steps, 1)
    fs = max(2, (flow_steps * cores) // 2 * 2)
    v, t, s = oracle_sample(mask, w, fs, max(1, np_steps * cores), cores)
    return {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle", "sample": s,
            "seconds": t,
            "single_core": {"value": v1, "unit": "MLUPS", "cores": 1, "sample": s1,
                            "seconds": t1}}


def reference(args, w, mask):
    rank, world, local = dist_info()
    if rank != 0:
        return None
    cores = host_cores()
    fs = max(2, (args.ref_flow_steps * cores) // 2 * 2)
    ns = max(1, args.ref_np_steps * cores)
    for _ in range(args.warmup):
        oracle_sample(mask, w, max(2, fs // 10) // 2 * 2, max(1, ns // 10), cores)
    vals, ts = [], []
    for _ in range(args.steps):
        v, t, sample = oracle_sample(mask, w, fs, ns, cores)
        vals.append(v)
        ts.append(t)
    value = float(np.mean(vals))
    return {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(ts)) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": w["desc"], "name": args.workload},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="3d-256", choices=list(WORKLOADS))
    ap.add_argument("--accuracy", action="store_true",
                    help="per-field error of the workload's storage against FP64 storage "
                         "on the GPU, at full size and horizon")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--ref-flow-steps", type=int, default=0,
                    help="oracle sample: LBM steps (0: about 1e8 site updates)")
    ap.add_argument("--ref-np-steps", type=int, default=0,
                    help="oracle sample: transport steps (0: about 2e7 cell updates)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--launch-shapes", type=int, nargs=2, default=None,
                    metavar=("LBM", "NP"),
                    help="fix the LBM (0-5) and transport (0-9) launch shapes instead of "
                         "autotuning (a profiler's serialised launches mislead the tuner)")
    ap.add_argument("--flow-steps", type=int, default=0,
                    help="run exactly this many flow steps (multiple of 100) instead of "
                         "converging; for short profiling runs")
    ap.add_argument("--np-steps", type=int, default=0,
                    help="override the number of transport steps")
    ap.add_argument("--precision", choices=["fp64", "fp32", "fp32-pair", "fp32-cpair", "bf16"],
                    default=None,
                    help="override the workload's storage precision")
    ap.add_argument("--sweep", action="store_true",
                    help="batched parameter sweep against the plain loop (solves/s)")
    ap.add_argument("--sweep-geometries", type=int, default=64)
    ap.add_argument("--sweep-plain", action="store_true",
                    help="also run the plain loop that re-solves the flow for every solve")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[0.25, 0.5, 1.0, 1.5, 2.0],
                    help="offered load as fractions of the sequential capacity")
    ap.add_argument("--serve", action="store_true",
                    help="continuous-batching server against the sequential loop")
    ap.add_argument("--serve-requests", type=int, default=500)
    ap.add_argument("--serve-slots", type=int, default=6)
    ap.add_argument("--serve-budget-gib", type=float, default=64.0)
    args = ap.parse_args()
    rank, world, local = dist_info()
    if args.sweep or args.serve:
        if rank == 0:
            print(json.dumps(sweep_bench(args) if args.sweep else serve_bench(args)), flush=True)
        return
    w = dict(WORKLOADS[args.workload])
    if args.precision:
        w["prec"] = {"fp64": cdi.FP64, "fp32": cdi.FP32, "fp32-pair": cdi.FP32_SPLIT,
                     "fp32-cpair": cdi.FP32_CPAIR, "bf16": cdi.BF16_POP}[args.precision]
        w["desc"] += f" [override: {args.precision} storage]"
    if args.flow_steps:
        w.update(flow_tol=0.0, max_flow=args.flow_steps)
        w["desc"] += f" [override: exactly {args.flow_steps} flow steps]"
    if args.np_steps:
        w["np_steps"] = args.np_steps
        w["desc"] += f" [override: {args.np_steps} transport steps]"
    mask = w["mask"]()
    if args.accuracy:
        if rank == 0:
            print(json.dumps(accuracy(args, w, mask)), flush=True)
        return
    # bounded oracle sample (10-30 s of single-thread CPU work on any workload)
    if not args.ref_flow_steps:
        args.ref_flow_steps = max(2, int(round(1e8 / (2 * mask.size) / 2)) * 2)
    if not args.ref_np_steps:
        args.ref_np_steps = max(1, int(round(2e7 / mask.size)))
    if args.impl == "reference":
        # the oracle runs on rank 0 alone; the other ranks exit without work
        line = reference(args, w, mask)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if True:
        line = ours(args, w, mask)
        if line is not None and not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baselines(mask, w, args.ref_flow_steps, args.ref_np_steps)
        elif line is not None:
            line["cpu_baseline"] = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
