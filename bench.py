#!/usr/bin/env python3
"""Benchmark of the ternary free-energy LB time step (arXiv:1511.02155) on GB300.

A "step" is one full time step of the method over the whole lattice (moments,
derivatives, chemical potentials, pressure-tensor equilibria, BGK collision,
streaming, FP64 mass totals).  Metric: million lattice-node updates per second
(MLUPS) and the step kernel's fraction of the measured HBM roofline.

Default workload: D3Q19 256^3 periodic ternary spinodal decomposition (FP32),
populations 3.8 GB per copy (larger than L2, so every step streams from HBM).
The default run also times the FP16 and BF16 storage formats on the same
lattice and reports them under "companions" (MLUPS, kernel time, roofline
fractions, largest |dC_m| against the FP32 run after the same steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload spinodal256|lens512|probe8192|wells4096|sweep96]
                  [--precision fp32|fp64|fp16|bf16] [--coupling pressure_tensor|forcing]

--coupling forcing times the Guo body-force coupling (three kernels per step:
moments, pressure tensor and chemical potentials, collide+stream) on the
periodic workloads; its roofline keeps the algorithmic 1 read + 1 write of the
populations per node, so the fraction is against the ideal one-pass step.

Under torchrun (N > 1) every rank runs an independent replica of the workload on
its own GPU (weak scaling, no collective in the data path); timing takes the
maximum over ranks and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1511_02155_gb300 import workloads as W  # noqa: E402

METRIC = "MLUPS and % HBM roofline per ternary step (FP32 vs FP16-store) at fixed error"


def bytes_per_node(Q: int, precision: str) -> int:
    """Algorithmic bytes of one node update: every stored population read once and
    written once.  FP64/FP32 store 3Q values; the 16-bit formats store the 3(Q-1)
    moving populations in 2 bytes and the three rest populations in 4."""
    if precision in ("fp16", "bf16"):
        return 2 * (3 * (Q - 1) * 2 + 3 * 4)
    return 2 * 3 * Q * {"fp64": 8, "fp32": 4}[precision]


SWEEP_LABEL = ("96 D2Q9 square-well contact-angle runs of uneven size (128x64 .. 768x384), "
               "target angles in [30, 150] deg, batched (one launch per step) under a CUDA graph")


def workload(name: str, size: int = 0):
    """(config dict, label).  size overrides the edge of the spinodal / probe
    lattices (used for small profiling cases of the same kernel)."""
    if name == "spinodal256":
        n = size or 256
        return W.spinodal_3d(n, seed=3), f"D3Q19 {n}^3 periodic ternary spinodal decomposition"
    if name == "lens512":
        return W.lens_512x256(), "D2Q9 512x256 periodic liquid lens, radius 60 (L2-resident)"
    if name == "probe8192":
        n = size or 8192
        return W.probe_2d(n), f"D2Q9 {n}^2 periodic ternary spinodal mixture"
    if name == "wells4096":
        nx = size or 4096
        return (W.wells_2d(nx, nx // 2),
                f"D2Q9 {nx}x{nx // 2} walls with 32 square wells, wetting on all fluids")
    raise SystemExit(f"unknown workload {name}")


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_from_profiles(kernel_tag: str, source_digest: str, nodes: int):
    """DRAM bytes (read + write) of one launch of this configuration, from the
    committed ncu summary profiles/traffic.json, scaled by node count from the
    captured case; None if there is no capture of this configuration or it was
    taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel_tag)
    if not e or e.get("source_sha256") != source_digest:
        return None
    return round(float(e["dram_bytes_per_node"]) * nodes)


def kernel_source_digest():
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1511_02155_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cuh", ".cu", ".h")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows
                                    if r[3].replace(".", "").isdigit()), default=None)}


def cpu_baseline(cfg_name: str, cfg: dict, budget_s: float = 12.0):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload:
    the same recipe on a smaller lattice, OpenMP over all host cores."""
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle
    Q = cfg["Q"]
    solid = None
    if Q == 19:
        n = 48
        C = W.spinodal((n, n, n), seed=3)
        shape = (n, n, n)
        sample = f"D3Q19 {n}^3 sub-lattice of the same spinodal recipe"
    else:
        ny, nx = (128, 256) if cfg_name == "lens512" else (256, 256)
        solid = None
        if cfg_name == "lens512":
            C = W.lens(nx, ny, 30.0, 1.0, 0.0, 64.0, (128.0, 64.0))
        elif cfg_name == "wells4096":
            wc = W.wells_2d(nx, ny, 2)
            C, solid = wc["C"], wc["solid"]
        elif cfg_name == "sweep96":
            C, solid = W.square_well(nx, ny // 2, 70, 35, floor=8)
            ny = ny // 2
        else:
            C = W.spinodal((ny, nx), seed=5)
        shape = (nx, ny, 1)
        sample = (f"D2Q9 {nx}x{ny} square well of the same recipe (one member-sized lattice)"
                  if cfg_name == "sweep96" else f"D2Q9 {nx}x{ny} sub-lattice of the same recipe")
    p = oracle.make_params(Q, *shape, cfg["kappa"], cfg["alpha"], cfg["tau_f"], cfg["M_phi"], cfg["M_psi"],
                           cfg.get("h", (0.0, 0.0, 0.0)))
    rho, phi, psi = W.to_aux(*C)
    if solid is not None:
        for a in (rho, phi, psi):
            a[solid != 0] = 0.0
    f, g, k = oracle.init_equilibrium(p, rho, phi, psi, solid=solid)
    N = int(np.prod(shape))
    t0 = time.perf_counter()
    oracle.step(p, f, g, k, 1, solid)
    one = time.perf_counter() - t0
    nsteps = max(1, int(budget_s / max(one, 1e-6)))
    t0 = time.perf_counter()
    oracle.step(p, f, g, k, nsteps, solid)
    dt = time.perf_counter() - t0
    return {"value": round(N * nsteps / dt / 1e6, 4), "unit": "MLUPS",
            "cores": int(os.environ.get("OMP_NUM_THREADS", cores)), "kind": "oracle",
            "sample": f"{sample}, {nsteps} steps ({dt:.1f} s, FP64)"}


def run_reference(args, cfg_name, cfg, label):
    """Reference arm: the FP64 CPU oracle on a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle
    Q = cfg["Q"]
    if Q == 19:
        n = 32
        C = W.spinodal((n, n, n), seed=3)
        shape = (n, n, n)
        sample = f"D3Q19 {n}^3 sub-lattice per step"
    else:
        C = W.spinodal((128, 128), seed=5) if cfg_name != "lens512" else W.lens(256, 128, 30.0, 1.0, 0.0, 64.0, (128.0, 64.0))
        shape = (C[0].shape[1], C[0].shape[0], 1)
        sample = f"D2Q9 {shape[0]}x{shape[1]} sub-lattice per step"
    p = oracle.make_params(Q, *shape, cfg["kappa"], cfg["alpha"], cfg["tau_f"], cfg["M_phi"], cfg["M_psi"])
    f, g, k = oracle.init_equilibrium(p, *W.to_aux(*C))
    N = int(np.prod(shape))
    oracle.step(p, f, g, k, args.warmup)
    t0 = time.perf_counter()
    oracle.step(p, f, g, k, args.steps)
    dt = time.perf_counter() - t0
    v = N * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": round(v, 4), "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": label, "sample": sample, "lattice_nodes": N},
            "cpu_baseline": {"value": round(v, 4), "unit": "MLUPS",
                             "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sweep_members(precision: str, count: int = 96):
    """Engines of the contact-angle sweep, h from each member's first admissible
    target pair (the library's wetting inversion)."""
    import paper_1511_02155_gb300 as tl
    members = W.sweep_wells(count)
    engines, hosts = [], []
    for m in members:
        for a in m["angles"]:
            try:
                m["h"] = tl.wetting_from_angles(m["kappa"], m["alpha"], *a)
                m["target"] = a
                break
            except tl.TLBMError:
                continue
        rho, phi, psi = W.to_aux(*m["C"])
        m["C"] = None
        for a in (rho, phi, psi):
            a[m["solid"] != 0] = 0.0
        eng = tl.TernaryLB(9, m["nx"], m["ny"], 1, m["kappa"], m["alpha"], m["tau_f"], m["M_phi"],
                           m["M_psi"], m["h"], m["solid"], precision)
        eng.init_fields(rho, phi, psi)
        engines.append(eng)
        hosts.append((rho, phi, psi))
    return members, engines, hosts


def run_sweep(args):
    """Batched contact-angle sweep: every member advanced by one launch per step."""
    import torch
    import paper_1511_02155_gb300 as tl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    members, engines, hosts = sweep_members(args.precision)
    N = sum(m["nx"] * m["ny"] for m in members)
    n_fluid = sum(int(m["nx"] * m["ny"] - np.count_nonzero(m["solid"])) for m in members)
    batch = tl.TernaryBatch(engines)
    tile = batch.autotune(trial_steps=5)  # real steps: part of the warm-up
    batch.set_graph(True)
    batch.step(args.warmup)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        e0.record(stream)
        batch.step(args.steps)
        e1.record(stream)
        barrier()
    ms = reduce_max(e0.elapsed_time(e1), dist)
    clocks = clk.summary()
    for e in engines:
        e.step_mass()  # raises on a non-finite total
    value = job_mlups(world, N, args.steps, ms / 1e3)

    # the same members stepped one by one (two launches each per step), for comparison
    ks = max(3, min(args.steps, 20))
    barrier()
    e0.record(stream)
    for _ in range(ks):
        for e in engines:
            e.step(1)
    e1.record(stream)
    barrier()
    lone_mlups = job_mlups(world, N, ks, reduce_max(e0.elapsed_time(e1), dist) / 1e3)

    # main-kernel duration (CUDA events on the members' stream around each batched launch)
    batch.set_timing(True)
    batch.step(min(args.steps, 50))
    kms, ksteps = batch.kernel_time()
    batch.set_timing(False)
    kernel_ms = kms / max(ksteps, 1)
    bpn = bytes_per_node(9, args.precision)
    alg_bytes = bpn * n_fluid + N
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (kernel_ms / 1e3) / 1e9
    tag = f"batch:sweep96:{args.precision}"  # captured at the tile the autotuner chose in that run
    traffic = traffic_from_profiles(tag, kernel_source_digest(), N)

    # end to end: upload every member's fields from pinned host memory, K batched
    # steps, download C_1..3 of every member and their mass totals
    pin = [[torch.from_numpy(np.ascontiguousarray(a.reshape(-1))).pin_memory() for a in h] for h in hosts]
    outs = [[torch.empty(m["nx"] * m["ny"], dtype=torch.float64).pin_memory() for _ in range(3)]
            for m in members]
    barrier()
    t0 = time.perf_counter()
    for e, p in zip(engines, pin):
        e.init_from_host_ptrs(*(t.data_ptr() for t in p))
    batch.step(args.steps)
    for e, o in zip(engines, outs):
        e.fields_into(*(t.data_ptr() for t in o))
        _ = e.mass()
    barrier()
    e2e_s = reduce_max(time.perf_counter() - t0, dist)
    e2e = {"value": round(job_mlups(world, N, args.steps, e2e_s), 2), "unit": "MLUPS",
           "h2d_bytes_per_step": round(3 * 8 * N / args.steps, 1),
           "d2h_bytes_per_step": round((3 * 8 * N + 24 * len(members)) / args.steps, 1),
           "job": f"upload rho/phi/psi of 96 members (fp64, pinned) + equilibrium init, {args.steps} "
                  "batched steps, download C1..C3 (fp64) + mass totals of every member"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f16-store/f32",
                                           "bf16": "bf16-store/f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": SWEEP_LABEL, "members": len(members), "nodes_per_gpu": N,
                       "fluid_nodes_per_gpu": n_fluid, "lattice": "D2Q9", "precision": args.precision,
                       "kernel": "batched fused (solid-aware)", "tile": list(tile),
                       "blocks_per_launch": batch.blocks,
                       "lone_engines_mlups": round(lone_mlups, 2),
                       "l2": "populations exceed L2 (no flush needed)", "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                         "kernel_ms": round(kernel_ms, 4),
                         "algorithmic_bytes_per_launch": alg_bytes, "bytes_per_node": bpn},
            "e2e": e2e,
            "gpu_launches": args.steps * 2,
            "clocks": clocks,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline("sweep96", {"Q": 9, "kappa": (0.01, 0.01, 0.01), "alpha": 1.0,
                                                             "tau_f": 1.0, "M_phi": 0.5, "M_psi": 1.0 / 6.0})
        print(json.dumps(line), flush=True)
    batch.close()
    for e in engines:
        e.close()
    if dist is not None:
        dist.destroy_process_group()


def reduce_max(value: float, dist, device="cuda") -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world: int, nodes_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank advances its own lattice `steps` times."""
    return world * nodes_per_rank * steps / seconds / 1e6


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="spinodal256",
                    choices=["spinodal256", "lens512", "probe8192", "wells4096", "sweep96"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16", "bf16"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "fused", "split"])
    ap.add_argument("--coupling", default="pressure_tensor", choices=["pressure_tensor", "forcing"],
                    help="forcing: the Guo body-force coupling (periodic workloads, split kernels)")
    ap.add_argument("--tile", default="0,0")
    ap.add_argument("--size", type=int, default=0, help="lattice edge override (profiling cases)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-companions", action="store_true",
                    help="skip the FP16/BF16 storage companions of the default FP32 run")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.workload == "sweep96":
        run_sweep(args)
        return
    cfg, label = workload(args.workload, args.size)

    if args.impl == "reference":
        run_reference(args, args.workload, cfg, label)
        return

    import torch
    import paper_1511_02155_gb300 as tl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)

    Q = cfg["Q"]
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    N = nx * ny * nz
    if world > 1 and rank > 0 and cfg.get("C") is not None and Q == 19:
        cfg["C"] = W.spinodal((nz, ny, nx), seed=3 + rank)  # an independent replica per rank
    rho, phi, psi = W.to_aux(*cfg["C"])
    cfg["C"] = None
    solid = cfg.get("solid")
    if solid is not None:
        for a in (rho, phi, psi):
            a[solid != 0] = 0.0
    n_fluid = N if solid is None else int(N - np.count_nonzero(solid))
    fields = (rho, phi, psi)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if args.coupling == "forcing" and solid is not None:
        raise SystemExit("--coupling forcing runs on periodic workloads only")
    with_companions = (args.precision == "fp32" and args.workload == "spinodal256" and not args.no_companions
                       and args.coupling == "pressure_tensor")
    main_run = measure(args, cfg, fields, solid, args.precision, args.tile, args.kernel, world, local, dist,
                       barrier, keep_fields=with_companions)
    value, ms, clocks, m_after = main_run["value"], main_run["ms"], main_run["clocks"], main_run["mass"]
    kernel_ms, kind, e2e, launches = (main_run["kernel_ms"], main_run["kind"], main_run["e2e"],
                                      main_run["launches"])
    bpn = bytes_per_node(Q, args.precision)
    # every population of a fluid node read once and written once, plus one mask
    # byte per node where solid nodes exist
    alg_bytes = bpn * n_fluid + (0 if solid is None else N)
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (kernel_ms / 1e3) / 1e9
    tag = f"{kind}:{args.workload}:{args.precision}:{args.tile}"
    if args.coupling != "pressure_tensor":
        tag += f":{args.coupling}"
    traffic = traffic_from_profiles(tag, kernel_source_digest(), N)

    # the 16-bit storage companions of the FP32 headline (the metric compares
    # FP32 and FP16 storage): same lattice and timing; roofline fractions against
    # 228 B/node (every population in 16 bits) and against the 240 B/node the
    # packed format stores (rest populations in FP32); the largest |dC_m|
    # against the FP32 run after the same steps from the same fields
    companions = None
    if with_companions:
        companions = {}
        for prec in ("fp16", "bf16"):
            c = measure(args, cfg, fields, solid, prec, "0,0", "auto", world, local, dist, barrier,
                        keep_fields=True)
            dC = max(float(np.abs(a - b).max()) for a, b in zip(c["C"], main_run["C"]))
            b228, b240 = 2 * 3 * Q * 2, bytes_per_node(Q, prec)
            companions[prec] = {
                "value": round(c["value"], 2), "unit": "MLUPS",
                "ms_per_step": round(c["ms"] / args.steps, 4), "kernel_ms": round(c["kernel_ms"], 4),
                "frac_228": round(b228 * n_fluid / (c["kernel_ms"] / 1e3) / 1e9 / peak, 4),
                "frac_240": round(b240 * n_fluid / (c["kernel_ms"] / 1e3) / 1e9 / peak, 4),
                "e2e_mlups": c["e2e"]["value"], "clocks": c["clocks"],
                "max_dC_vs_fp32": dC, "steps_compared": args.steps,
            }
        main_run.pop("C", None)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp16": "f16-store/f32",
                                           "bf16": "bf16-store/f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": label, "nodes_per_gpu": N, "fluid_nodes_per_gpu": n_fluid,
                       "lattice": f"D{3 if Q == 19 else 2}Q{Q}",
                       "precision": args.precision, "kernel": kind, "coupling": args.coupling,
                       "l2": "populations exceed L2 (no flush needed)" if alg_bytes / 2 > 129e6
                       else "L2-resident lattice", "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                         "kernel_ms": round(kernel_ms, 4),
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "bytes_per_node": bpn},
            "e2e": e2e,
            "gpu_launches": args.steps * launches,
            "clocks": clocks,
            "mass_totals": [float(v) for v in m_after],
        }
        if companions:
            line["companions"] = companions
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload, cfg)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def measure(args, cfg, fields, solid, precision, tile, kernel, world, local, dist, barrier, keep_fields=False):
    """Time one engine of the workload in one storage format: W warm-up steps,
    K timed steps (CUDA events on the engine's stream, clocks sampled), the main
    kernel's own duration in timing mode, and the end-to-end job through the
    public API with host buffers.  keep_fields: also return the end-to-end job's
    C_1..3 (host arrays)."""
    import torch
    import paper_1511_02155_gb300 as tl
    Q = cfg["Q"]
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    N = nx * ny * nz
    rho, phi, psi = fields
    eng = tl.TernaryLB(Q, nx, ny, nz, cfg["kappa"], cfg["alpha"], cfg["tau_f"], cfg["M_phi"],
                       cfg["M_psi"], cfg["h"], solid, precision)
    if kernel != "auto":
        eng.set_kernel(kernel)
    if getattr(args, "coupling", "pressure_tensor") != "pressure_tensor":
        eng.set_coupling(args.coupling)
    tv, tc = (int(v) for v in tile.split(","))
    eng.set_tile(tv, tc)
    eng.init_fields(rho, phi, psi)
    stream = torch.cuda.current_stream()

    # warm-up
    eng.step(args.warmup)
    barrier()

    # timed region: K steps, inputs (3.8 GB populations) far larger than L2
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        e0.record(stream)
        eng.step(args.steps)
        e1.record(stream)
        barrier()
    ms = reduce_max(e0.elapsed_time(e1), dist)
    clocks = clk.summary()
    m_after = eng.step_mass()  # raises on a non-finite total
    value = job_mlups(world, N, args.steps, ms / 1e3)

    # main-kernel duration, CUDA events on the engine's stream around each launch
    eng.set_timing(True)
    eng.step(min(args.steps, 50))
    kms, ksteps = eng.kernel_time()
    eng.set_timing(False)
    kernel_ms = kms / max(ksteps, 1)

    # end to end through the public API with host buffers: upload the fields from
    # pinned memory, K steps, download C_1..3 and the mass totals
    pin = [torch.from_numpy(np.ascontiguousarray(a.reshape(-1))).pin_memory() for a in (rho, phi, psi)]
    outs = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(3)]
    barrier()
    t0 = time.perf_counter()
    eng.init_from_host_ptrs(*(t.data_ptr() for t in pin))
    eng.step(args.steps)
    eng.fields_into(*(t.data_ptr() for t in outs))
    _ = eng.mass()
    barrier()
    e2e_s = reduce_max(time.perf_counter() - t0, dist)
    e2e = {"value": round(job_mlups(world, N, args.steps, e2e_s), 2), "unit": "MLUPS",
           "h2d_bytes_per_step": round(3 * 8 * N / args.steps, 1),
           "d2h_bytes_per_step": round((3 * 8 * N + 24) / args.steps, 1),
           "job": f"upload rho/phi/psi (fp64, pinned) + equilibrium init, {args.steps} steps, "
                  "download C1..C3 (fp64) + mass totals"}
    out = {"value": value, "ms": ms, "clocks": clocks, "mass": m_after, "kernel_ms": kernel_ms,
           "kind": eng.kernel, "e2e": e2e, "launches": eng.launches_per_step}
    eng.close()
    if keep_fields:
        out["C"] = [t.numpy() for t in outs]
    return out


if __name__ == "__main__":
    main()
