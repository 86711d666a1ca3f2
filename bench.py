"""Throughput benchmark of the per-step lattice update (near-contact interaction + regularized
LB hydrodynamics + conservative Allen-Cahn phase field) on one GB300 per rank.

Workload: the 3D head-on collision at 256x128x128 (D3Q19, R = 24, density ratio 100), seeded
synthetic fields. One step = one near-contact pass, one hydrodynamic pass and one phase-field
pass over all cells. The populations (2 x 319 MB in FP32) exceed the 129 MB L2, so no flush is
needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--store f32|f16|bf16]

Prints one JSON line (rank 0). Multi-GPU (torchrun): every rank runs its own independent copy of
the workload (weak scaling, no data-path collective); the slowest rank's time is used.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & HBM-roofline fraction, FP32 vs FP16-store at stated φ error vs FP64"
WORKLOAD = "3D head-on droplet collision 256x128x128 D3Q{Q}, R=24, W=4, density ratio 100"
HBM_FALLBACK_GBS = 6800.0
# Algorithmic bytes per cell update (stored state only): populations read + written, phi read +
# written, velocity written + read.
def nci_kernels(cfg):
    """Kernels of one near-contact pass: normals and scan and, on 3D grids whose sides are multiples
    of 4, the brick prefilter between them."""
    if not cfg["nci_on"]:
        return 0
    prefilter = cfg["dim"] == 3 and all(cfg[k] % 4 == 0 for k in ("nx", "ny", "nz"))
    return 3 if prefilter else 2


# scan blocks of the split step compared against the one-stream step (one resident block per SM
# is 152 on a GB300), in alternating chunks of SPLIT_CHUNK steps
SPLIT_SCAN_BLOCKS = (38, 76, 152)
SPLIT_CHUNK = 25
# the timed region records events around one hydrodynamic launch in HYDRO_SAMPLE
HYDRO_SAMPLE = 10


def split_applies(cfg):
    """The split step of lbm_step (hydro as two launches, one concurrent with the near-contact pass):
    3D with the near-contact pass on, nx even and Q N <= 2^32."""
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    return bool(cfg["nci_on"]) and cfg["dim"] == 3 and cfg["nx"] % 2 == 0 and cfg["Q"] * n <= 2 ** 32


def kernels_per_step(cfg, overlap=False):
    """Kernels one lbm_step launches: the near-contact pass, hydro (two launches in the split step)
    and phase."""
    return nci_kernels(cfg) + (2 if overlap and split_applies(cfg) else 1) + 1


def step_bytes_per_cell(Q, pop_bytes):
    return 2 * Q * pop_bytes + 8 + 24


def hydro_bytes_per_cell(Q, pop_bytes):
    # hydrodynamic kernel: populations read + written, phi read, velocity written
    return 2 * Q * pop_bytes + 4 + 12


RECORD_BYTES = 64  # the moment-record store: one 16-float record per cell instead of Q populations


def store_bytes_per_cell(Q, store):
    """(hydro kernel, whole step) algorithmic bytes per cell update for a store: populations (or
    records) read + written, phi read (+ written by phase), velocity written + read."""
    if store == "mom":
        return 2 * RECORD_BYTES + 4 + 12, 2 * RECORD_BYTES + 8 + 24
    pb = 4 if store == "f32" else 2
    return hydro_bytes_per_cell(Q, pb), step_bytes_per_cell(Q, pb)


# DRAM traffic of one hydrodynamic launch on the full workload, from the ncu capture summarised in
# profiles/ (dram__bytes_read.sum + dram__bytes_write.sum), keyed by the hydro kernel source hash:
# a changed kernel reports null until it is profiled again.
HYDRO_TRAFFIC = {
    # 337.76 MB read + 323.17 MB written (ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,
    # one step launch of k_hydro2 on the 256x128x128 case; profiles/launches_collision_256x128x128.md)
    ("f32", 19, "86bb24acb2461a5c"): 660.93e6,
}


def _src_hash(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2603_17481_gb300", "csrc", n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, cells_per_rank, steps, ms_local, device=None):
    """Weak scaling: every rank advances its own copy of the workload; the job's throughput is all
    ranks' cell updates over the slowest rank's time. Returns (MLUPS, max ms)."""
    ms_max = max_over_ranks(world, ms_local, device=device)
    return world * cells_per_rank * steps / (ms_max * 1e-3) / 1e6, ms_max


# Fixed horizons of the store-variant comparison, independent of --steps/--warmup (each on fresh
# contexts): phi is compared point by point at EARLY, before the droplets meet; after contact the
# flow is chaotic (a 2^-30 change of phi in one cell grows to max|dphi| ~ 0.2 by step 2000 in
# FP32), so the LATE checkpoint compares the droplet centroids.
EARLY = 200
LATE = 1000


def centroids(cfg, phi):
    """phi-weighted mean x of the left and right halves of the box (one droplet each)."""
    import numpy as np
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    p = np.asarray(phi).reshape(nz, ny, nx)
    X = np.arange(nx, dtype=np.float64)
    out = []
    for sl in (slice(0, nx // 2), slice(nx // 2, nx)):
        q = p[:, :, sl].sum(axis=(0, 1))
        out.append(float((q * X[sl]).sum() / q.sum()))
    return out


def make_workload(Q=19):
    from paper_2603_17481_gb300 import workloads as W
    cfg, phi, u = W.droplets_head_on_3d(Q=Q)
    phi = W.to_q30_grid(phi)
    return cfg, phi, u


def cpu_oracle_run(cfg, phi, u, budget_s, max_steps=20, min_steps=1):
    """Times the FP64 oracle (as it stands) on the full grid for a bounded number of steps; also
    returns its phi and velocity after those steps."""
    import oracle
    P = oracle.make_params(cfg)
    f = oracle.init(P, phi, u)
    N = cfg["nx"] * cfg["ny"] * cfg["nz"]
    steps, t_total = 0, 0.0
    ph = phi
    while steps < max_steps and (steps < min_steps or t_total < budget_s):
        t0 = time.perf_counter()
        f, ph, _ = oracle.step(P, f, ph, 1)
        t_total += time.perf_counter() - t0
        steps += 1
    _, u_o = oracle.moments(P, f, ph)
    return N * steps / t_total / 1e6, steps, t_total, ph, u_o


def run_plan(args, world, rank):
    """What one default run does, as plain numbers: every step count is non-negative whatever
    --steps and --warmup are (the store variants use their own fixed horizons)."""
    variants = bool(args.variants and args.store == "f32" and world == 1)
    return {
        "warmup": max(args.warmup, 0), "timed": max(args.steps, 0),
        "split_steps": max(min(args.steps, 500), 1),
        "split_compare_steps": max(min(args.steps, 500), 1) if args.split_compare else 0,
        "e2e_steps": max(args.steps, 1) if not args.no_e2e else 0,
        "variant_stores": ("f16", "bf16", "mom") if variants else (),
        "variant_timed": max(args.steps, 1), "early": EARLY, "late": LATE,
        "cpu_baseline": rank == 0 and world == 1 and not args.no_cpu_baseline,
    }


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2603_17481_gb300 import binding as B
    from paper_2603_17481_gb300 import build as lbm_build

    plan = run_plan(args, world, rank)
    torch.cuda.set_device(local)
    lbm_build.build()
    cfg, phi, u = make_workload(args.lattice)
    N = cfg["nx"] * cfg["ny"] * cfg["nz"]
    Q = cfg["Q"]
    stream = torch.cuda.Stream()
    sim = B.Lbm(cfg, store=args.store, stream=stream.cuda_stream)
    sim.init_fields(phi, u)
    m0, _ = sim.mass()

    # warm-up
    sim.step(plan["warmup"])
    sim.synchronize()

    # timed region: K steps, with events on the library stream around the hydrodynamic kernel of one
    # step in HYDRO_SAMPLE (events around every pass would add time between kernels); the
    # per-kernel split is taken after it, untimed
    sampler = ClockSampler(local)
    sim.profile_kinds(["hydro"])
    sim.profile_sample(HYDRO_SAMPLE)
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(plan["timed"]):
        sim.step(1)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    prof = sim.profile_read()
    sim.profile(False)
    ms_total = ev0.elapsed_time(ev1)
    mlups, ms_max = whole_job_mlups(world, N, args.steps, ms_total, device=f"cuda:{local}")
    m1, _ = sim.mass()
    split_steps = plan["split_steps"]
    sim.profile_sample(1)  # every pass of the untimed split
    sim.profile(True)
    sim.step(split_steps)
    split = sim.profile_read()
    sim.profile(False)

    # the split step (lbm_set_overlap) against the one-stream step over the same steps: chunks of
    # the two alternate, so both see the same phase of the collision
    split_step = None
    if split_applies(cfg) and args.store != "mom" and plan["split_compare_steps"]:  # populations only
        ko = plan["split_compare_steps"]
        chunk = min(ko, SPLIT_CHUNK)
        split_step = {"unit": "MLUPS", "steps_each": ko, "chunk": chunk}

        def timed_chunk(blocks):
            sim.set_overlap(blocks)
            sim.step(2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(chunk)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)

        for blocks in SPLIT_SCAN_BLOCKS:
            t_one = t_split = 0.0
            done = 0
            while done < ko:
                t_one += timed_chunk(0)
                t_split += timed_chunk(blocks)
                done += chunk
            split_step[f"scan_blocks_{blocks}"] = {
                "value": round(N * done / (t_split * 1e-3) / 1e6, 1),
                "one_stream_value": round(N * done / (t_one * 1e-3) / 1e6, 1),
                "vs_one_stream": round(t_one / t_split, 4)}
        sim.set_overlap(0)

    hydro_b, step_b = store_bytes_per_cell(Q, args.store)
    peak, peak_kind = measured_peaks()
    # one hydrodynamic launch per sampled step (one stream)
    hydro_ms, hydro_n = prof["hydro"]
    hydro_avg = hydro_ms / max(hydro_n, 1)
    per_launch_bytes = hydro_b * N
    achieved = per_launch_bytes / (hydro_avg * 1e-3) / 1e9
    key = (args.store, Q, _src_hash("hydro_impl.cuh", "lbm_device.cuh"))
    traffic = HYDRO_TRAFFIC.get(key)
    gpu_launches = kernels_per_step(cfg) * args.steps

    step_frac = mlups / world * 1e6 * step_b / (peak * 1e9)

    # end-to-end through the C ABI with pinned host buffers: H2D of the initial fields, one
    # lbm_step call per step, D2H of the final fields
    e2e = None
    if plan["e2e_steps"]:
        phi_h = torch.from_numpy(np.ascontiguousarray(phi)).pin_memory()
        u_h = torch.from_numpy(np.ascontiguousarray(u)).reshape(-1).pin_memory()
        out_phi = torch.empty(N, dtype=torch.float64).pin_memory()
        out_u = torch.empty(3 * N, dtype=torch.float64).pin_memory()
        out_ps = torch.empty(N, dtype=torch.float64).pin_memory()
        ke = plan["e2e_steps"]
        # pinned arrays are read and written in place by the library's conversion kernels (no staging
        # buffer); one read before the clock starts, as a long-running caller would have made
        sim.read_fields(phi=out_phi, u=out_u, pstar=out_ps)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.init_fields(phi_h, u_h)
        for _ in range(ke):
            sim.step(1)
        sim.read_fields(phi=out_phi, u=out_u, pstar=out_ps)
        t1 = time.perf_counter()
        dt = max_over_ranks(world, t1 - t0, device=f"cuda:{local}")
        h2d = (phi_h.numel() + u_h.numel()) * 8
        d2h = (out_phi.numel() + out_u.numel() + out_ps.numel()) * 8
        e2e = {"value": round(world * N * ke / dt / 1e6, 1), "unit": "MLUPS",
               "h2d_bytes_per_step": round(h2d / ke, 1), "d2h_bytes_per_step": round(d2h / ke, 1),
               "steps": ke, "what": "lbm_init_fields(pinned host) + steps x lbm_step(1) + lbm_read_fields(pinned host); "
                       "the pinned arrays cross the host link inside the conversion kernels"}
    sim.close()

    def fresh(store, steps):
        """phi after `steps` steps of the workload from its initial state, in a new context."""
        s = B.Lbm(cfg, store=store, stream=stream.cuda_stream)
        s.init_fields(phi, u)
        s.step(steps)
        ph_s = s.read_fields(want=("phi",))[0]
        s.close()
        return ph_s

    variants = {}
    if plan["variant_stores"]:
        # FP32 references at the fixed horizons
        ph32_early, ph32_late = fresh("f32", plan["early"]), fresh("f32", plan["late"])
        c32 = centroids(cfg, ph32_late)
        for st in plan["variant_stores"]:
            s2 = B.Lbm(cfg, store=st, stream=stream.cuda_stream)
            s2.init_fields(phi, u)
            mv0, _ = s2.mass()
            s2.step(plan["warmup"])
            s2.synchronize()
            kv = plan["variant_timed"]
            s2.profile_kinds(["hydro"])  # as in the FP32 timed region
            s2.profile_sample(HYDRO_SAMPLE)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(kv):
                s2.step(1)
            e1.record(stream)
            e1.synchronize()
            pr = s2.profile_read()
            s2.profile(False)
            mv1, _ = s2.mass()
            s2.close()
            msv = e0.elapsed_time(e1)
            hm, hn = pr["hydro"]
            hm = hm / max(hn, 1) * kv  # the sampled mean, as a total over kv steps
            v_mlups = N * kv / (msv * 1e-3) / 1e6
            d_early = np.abs(fresh(st, plan["early"]) - ph32_early)
            ph_late = fresh(st, plan["late"])
            variants[st] = {
                "value": round(v_mlups, 1), "steps": kv, "vs_f32": round(v_mlups / mlups, 4),
                "hydro_gbs": round(store_bytes_per_cell(Q, st)[0] * N / (hm / kv * 1e-3) / 1e9, 1),
                "hydro_ms": round(hm / kv, 5),
                "step_roofline_frac": round(v_mlups * 1e6 * store_bytes_per_cell(Q, st)[1] / (peak * 1e9), 4),
                "phi_diff_vs_f32": {
                    f"after_{plan['early']}_steps": {"max": float(d_early.max()),
                                                     "q999": float(np.quantile(d_early, 0.999))},
                    f"after_{plan['late']}_steps": {
                        "max": float(np.max(np.abs(ph_late - ph32_late))),
                        "centroid_max_cells": max(abs(a - b) for a, b in zip(centroids(cfg, ph_late), c32))}},
                "phi_mass_drift": abs(mv1 - mv0) / abs(mv0),
            }

    cpu, vs_oracle = None, None
    if plan["cpu_baseline"]:
        v, steps, tt, ph_o, u_o = cpu_oracle_run(cfg, phi, u, budget_s=args.cpu_budget)
        cpu = {"value": round(v, 4), "unit": "MLUPS", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{steps} FP64 oracle step(s) of the full {cfg['nx']}x{cfg['ny']}x{cfg['nz']} grid, "
                         f"{tt:.1f} s, OpenMP over all host cores"}
        # every store against the FP64 oracle after the same steps, on the full grid
        vs_oracle = {"steps": steps}
        # (the record store starts from the equilibrium records, which stream f_eq of the
        # neighbours: another initial state, compared with the oracle in the parity tests)
        for st in ("f32",) + tuple(v for v in plan["variant_stores"] if v != "mom"):
            s = B.Lbm(cfg, store=st, stream=stream.cuda_stream)
            s.init_fields(phi, u)
            s.step(steps)
            ph_g, u_g, _ = s.read_fields(want=("phi", "u"))
            s.close()
            vs_oracle[st] = {"max_dphi": float(np.max(np.abs(ph_g - ph_o))),
                             "max_du": float(np.max(np.abs(u_g - u_o)))}

    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.store == "f32" else f"f32 ({args.store} store)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD.format(Q=Q), "cells": N,
                   "lattice": f"D3Q{Q} hydro, D3Q27 phase-field stencils",
                   "store": args.store, "near_contact": "on (w=3, q_th=0.125, eta=0.1, cos=-0.8)",
                   "l2": "inputs larger than L2 (2 x %.0f MB %s), no flush" % (
                       (hydro_b - 16) / 2 * N / 1e6, "records" if args.store == "mom" else "populations"),
                   "parallelism": f"{world} independent replica(s), one per GPU"},
        "roofline": {"bound": "hbm", "kernel": "hydro", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "bytes_per_cell": hydro_b, "avg_ms": round(hydro_avg, 5),
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback"},
        "step_roofline": {"bytes_per_cell": step_b, "frac_of_measured": round(step_frac, 4),
                          "frac_of_8TBs": round(step_frac * peak / 8000.0, 4)},
        "kernels_ms_per_step": {k: round(ms / split_steps, 5) for k, (ms, n) in split.items() if n},
        "kernels_split_steps": split_steps,
        "split_step": split_step,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "phi_mass_drift": abs(m1 - m0) / abs(m0),
    }
    if vs_oracle:
        line["vs_fp64_oracle"] = vs_oracle
    if variants:
        line["variants"] = variants
    return line


SWEEP_WORKLOAD = ("batched sweep: {n} independent 3D D3Q19 collisions on grids drawn from {{48,64,80,96}}^3, "
                  "R=L/6, W=4, density ratio 10, sigma=1e-3, Weber log-uniform in [1,100] via speed, "
                  "b ~ U[0,1]*2R")


def run_sweep(args, world, rank, local):
    """The batched sweep: every case advanced through one CUDA graph per two steps (lbm_batch_step):
    fused (one launch per pass over all cases, autotuned) and as a graph of per-case steps, against
    the same cases advanced by per-case lbm_step calls, one case after another."""
    import numpy as np
    import torch

    from paper_2603_17481_gb300 import binding as B
    from paper_2603_17481_gb300 import build as lbm_build
    from paper_2603_17481_gb300 import workloads as W

    torch.cuda.set_device(local)
    lbm_build.build()
    cfgs = W.collision_sweep(args.cases, seed=17481 + rank)
    stream = torch.cuda.Stream()
    sims, m0 = [], []
    for cfg in cfgs:
        phi, u = W.sweep_case_fields(cfg)
        s = B.Lbm(cfg, stream=stream.cuda_stream)
        s.init_fields(phi, u)
        m0.append(s.mass()[0])
        sims.append(s)
    cells = sum(s.N for s in sims)
    launches_fused = sum(nci_kernels(c) for c in cfgs) + 2  # near-contact per case, 2 batched
    launches_case = sum(kernels_per_step(c) for c in cfgs)
    steps = args.steps + (args.steps & 1)  # whole graph launches

    def timed(run, k):
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run(k)
        e1.record(stream)
        e1.synchronize()
        barrier(world)
        return e0.elapsed_time(e1)

    def per_case(k):
        for s in sims:
            s.step(k)

    per_case(args.warmup)
    ms_single = timed(per_case, steps)
    mlups_single, ms_single_max = whole_job_mlups(world, cells, steps, ms_single, device=f"cuda:{local}")

    # the per-case graph (every context's own steps on concurrent branches), the fused batch as is
    # (one launch per pass over all cases, tile shape 64x4x2 and 4 march rows), and the autotuned
    # batch (tile shape and march rows tuned, then the faster of fused and per-case), at each
    # branch count
    results, graph_results, fused_results, configs = {}, {}, {}, {}
    sampler = ClockSampler(local)
    for ns in args.streams:
        for mode in ("graph", "fused", "tuned"):
            flags = {"graph": B.LBM_BATCH_PER_CASE, "fused": B.LBM_BATCH_NO_TUNE, "tuned": 0}[mode]
            batch = B.LbmBatch(sims, nstreams=ns, stream=stream.cuda_stream, flags=flags)
            batch.step(args.warmup + (args.warmup & 1), sync=True)
            if mode == "tuned" and ns == args.streams[-1]:
                sampler.start()
                time.sleep(0.3)
            ms = timed(lambda k: batch.step(k, sync=False), steps)
            {"graph": graph_results, "fused": fused_results, "tuned": results}[mode][ns] = whole_job_mlups(
                world, cells, steps, ms, device=f"cuda:{local}")
            if mode == "tuned":
                configs[ns] = batch.config()
            batch.close()
    clocks = sampler.stop()
    best = max(results, key=lambda ns: results[ns][0])
    mlups, ms_max = results[best]
    drift, nonfinite = 0.0, 0
    for s, m in zip(sims, m0):
        m1, _ = s.mass()
        if not np.isfinite(m1):
            nonfinite += 1
        else:
            drift = max(drift, abs(m1 - m) / abs(m))
    for s in sims:
        s.close()
    if rank != 0:
        return None
    peak, peak_kind = measured_peaks()
    frac = mlups / world * 1e6 * step_bytes_per_cell(19, 4) / (peak * 1e9)
    return {
        "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": SWEEP_WORKLOAD.format(n=len(cfgs)), "cases": len(cfgs), "cells": cells,
                   "graph_branches": best, "l2": "inputs larger than L2 (%.1f GB of populations), no flush"
                   % (2 * 19 * 4 * cells / 1e9),
                   "parallelism": f"{world} independent replica(s), one per GPU"},
        "per_case_launches": {"value": round(mlups_single, 1), "unit": "MLUPS",
                              "ms_per_step": round(ms_single_max / steps, 5),
                              "what": "lbm_step(K) per case, cases one after another on one stream"},
        "batched_vs_per_case": round(mlups / mlups_single, 3),
        "per_case_graph": {"by_branches": {str(ns): round(v[0], 1) for ns, v in graph_results.items()},
                           "what": "CUDA graph of every case's own lbm_step kernels on concurrent branches"},
        "fused_untuned": {"by_branches": {str(ns): round(v[0], 1) for ns, v in fused_results.items()},
                          "what": "one hydrodynamic and one phase-field launch over all cases per step, "
                                  "64x4x2 tiles, 4 march rows"},
        "tuned_by_branches": {str(ns): round(v[0], 1) for ns, v in results.items()},
        "tuned_config": configs[best],
        "tuned_vs_per_case_graph": round(mlups / max(v[0] for v in graph_results.values()), 3),
        "step_roofline": {"bytes_per_cell": step_bytes_per_cell(19, 4), "frac_of_measured": round(frac, 4),
                          "peak": peak, "peak_source": peak_kind},
        "gpu_launches": (launches_fused if configs[best]["fused"] else launches_case) * steps,
        "clocks": clocks,
        "phi_mass_drift_max": drift, "nonfinite_cases": nonfinite,
    }


SWARM_WORKLOAD = ("3D buoyant bubble swarm, {L}^3 periodic D3Q19, {nb} bubbles R ~ U[8,12] at seeded "
                  "positions with surface gaps >= {gap} eps (gas fraction {gf:.3f}), W=4, density ratio 100, g=1e-6")


def count_bubbles(gas, volumes=False):
    """Connected components (6-neighbour) of a boolean (nz, ny, nx) mask on a periodic grid; with
    ``volumes`` also the cell count of each component."""
    import numpy as np
    from scipy import ndimage
    lab, n = ndimage.label(gas)
    parent = list(range(n + 1))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for ax in range(3):
        a = lab.take(0, axis=ax).ravel()
        b = lab.take(-1, axis=ax).ravel()
        m = (a > 0) & (b > 0)
        for i, j in set(zip(a[m].tolist(), b[m].tolist())):
            ri, rj = find(i), find(j)
            if ri != rj:
                parent[max(ri, rj)] = min(ri, rj)
    roots = [find(i) for i in range(1, n + 1)]
    if not volumes:
        return len(set(roots))
    sizes = np.bincount(lab.ravel(), minlength=n + 1)[1:]
    vol = {}
    for r, v in zip(roots, sizes.tolist()):
        vol[r] = vol.get(r, 0) + v
    return len(vol), sorted(vol.values())


def run_swarm(args, world, rank, local):
    """The bubble swarm with the near-contact repulsion on and off: throughput of each, and the
    number of distinct bubbles (gas components) left after --swarm-steps steps."""
    import numpy as np
    import torch

    from paper_2603_17481_gb300 import binding as B
    from paper_2603_17481_gb300 import build as lbm_build
    from paper_2603_17481_gb300 import workloads as W

    torch.cuda.set_device(local)
    lbm_build.build()
    cfg, cs, rs = W.bubble_swarm(L=args.swarm_L, nb=args.swarm_bubbles, seed=17481 + rank, gap_eps=args.swarm_gap)
    phi, u = W.bubble_swarm_fields(cfg, cs, rs)
    N = W.ncells(cfg)
    L = cfg["nx"]
    nb0 = count_bubbles((phi < 0.5).reshape(L, L, L))
    stream = torch.cuda.Stream()
    runs = {}
    for name, nci, store in (("nci_on", 1, "f32"), ("nci_off", 0, "f32"), ("nci_on_f16", 1, "f16")):
        c = dict(cfg, nci_on=nci)
        sim = B.Lbm(c, store=store, stream=stream.cuda_stream)
        sim.init_fields(phi, u)
        m0, _ = sim.mass()
        sim.step(args.warmup)
        sim.synchronize()
        sim.profile(True)
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            sim.step(1)
        e1.record(stream)
        e1.synchronize()
        barrier(world)
        prof = sim.profile_read()
        sim.profile(False)
        mlups, ms_max = whole_job_mlups(world, N, args.steps, e0.elapsed_time(e1), device=f"cuda:{local}")
        done = args.warmup + args.steps
        counts = {}
        for mark in sorted(set(args.swarm_count_at) | {args.swarm_steps}):
            if mark <= done:
                continue
            sim.step(mark - done)
            done = mark
            if mark != args.swarm_steps:
                pm, _, _ = sim.read_fields(want=("phi",))
                counts[str(mark)] = count_bubbles((pm < 0.5).reshape(L, L, L)) if np.all(np.isfinite(pm)) else None
        ph, _, _ = sim.read_fields(want=("phi",))
        m1, _ = sim.mass()
        kap = sim.curvature(0.0, 0.5, 50)  # kappa = div n, Eq. 78: 2 / R for R in [8, 12] is 0.17-0.25
        Ek = sim.energy_spectrum(min(L // 2, 1024))
        kb = L / 20.0  # bubble wavenumber L / d_b
        ks = np.arange(Ek.size)
        band = (ks >= kb) & (ks <= 4 * kb) & (Ek > 0)
        slope = float(np.polyfit(np.log(ks[band]), np.log(Ek[band]), 1)[0]) if band.sum() > 3 else None
        pick = np.unique(np.geomspace(1, Ek.size - 1, 24).astype(int))
        deq = None
        if np.all(np.isfinite(ph)):
            _, vols = count_bubbles((ph < 0.5).reshape(L, L, L), volumes=True)
            d = (6.0 * np.asarray(vols, dtype=np.float64) / np.pi) ** (1.0 / 3.0)
            deq = {"mean": round(float(d.mean()), 3), "std": round(float(d.std()), 3),
                   "hist_1lu_0_40": np.histogram(d, bins=40, range=(0, 40))[0].tolist()}
        runs[name] = {"value": round(mlups, 1), "ms_per_step": round(ms_max / args.steps, 5),
                      "kernels_ms_per_step": {k: round(ms / args.steps, 5) for k, (ms, n) in prof.items() if n},
                      "bubbles_after": count_bubbles((ph < 0.5).reshape(L, L, L)) if np.all(np.isfinite(ph)) else None,
                      "after_steps": max(args.swarm_steps, args.warmup + args.steps),
                      "bubbles_at": counts,
                      "kappa": {"mean": round(kap["mean"], 5), "band_cells": kap["band_cells"],
                                "hist_0_0.5_50": kap["hist"].tolist()},
                      "D_eq": deq,
                      "E_k": {"shells": pick.tolist(), "E": [float(f"{v:.4g}") for v in Ek[pick]],
                              "slope_kb_to_4kb": slope, "total": float(Ek.sum())},
                      "phi_mass_drift": abs(m1 - m0) / abs(m0)}
        sim.close()
    if rank != 0:
        return None
    peak, peak_kind = measured_peaks()
    on = runs["nci_on"]["value"]
    return {
        "metric": METRIC, "value": on, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": runs["nci_on"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": SWARM_WORKLOAD.format(L=L, nb=len(cs), gap=args.swarm_gap, gf=float((phi < 0.5).mean())),
                   "cells": N,
                   "l2": "inputs larger than L2, no flush",
                   "parallelism": f"{world} independent replica(s), one per GPU"},
        "step_roofline": {"bytes_per_cell": step_bytes_per_cell(19, 4),
                          "frac_of_measured": round(on / world * 1e6 * step_bytes_per_cell(19, 4) / (peak * 1e9), 4),
                          "peak": peak, "peak_source": peak_kind},
        "nci_overhead": round(runs["nci_off"]["value"] / on - 1.0, 4),
        "bubbles_initial": nb0, "runs": runs,
        "gpu_launches": int(kernels_per_step(dict(cfg, nci_on=1)) * args.steps),
    }


IMPACT_WORKLOAD = ("the paper's {case} droplet impact, {L}^3 periodic D3Q19, D_lu = {D:g}, density ratio 1000, "
                   "sigma = 0.02, We = {we}, B = {B}, nu_l = {nul}, nu_g = {nug}")


def run_impact(args, world, rank, local):
    """The paper's droplet impacts of Sec. 3.1 (E1 head-on We 4.6, E2 off-axis We 4.8, B 0.32) at
    density ratio 1000 as synthetic stress workloads: throughput of the FP32 and FP16-store paths,
    exact phi mass and finite fields after the timed steps."""
    import numpy as np
    import torch

    from paper_2603_17481_gb300 import binding as B
    from paper_2603_17481_gb300 import build as lbm_build
    from paper_2603_17481_gb300 import workloads as W

    torch.cuda.set_device(local)
    lbm_build.build()
    cfg, phi, u = W.droplets_paper_impact(args.case, L=args.impact_L, D=args.impact_D)
    phi = W.to_q30_grid(phi)
    N = W.ncells(cfg)
    stream = torch.cuda.Stream()
    runs = {}
    for store in ("f32", "f16"):
        sim = B.Lbm(cfg, store=store, stream=stream.cuda_stream)
        sim.init_fields(phi, u)
        m0, _ = sim.mass()
        sim.step(args.warmup)
        sim.synchronize()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            sim.step(1)
        e1.record(stream)
        e1.synchronize()
        barrier(world)
        mlups, ms_max = whole_job_mlups(world, N, args.steps, e0.elapsed_time(e1), device=f"cuda:{local}")
        m1, mom = sim.mass()
        ph, uu, _ = sim.read_fields(want=("phi", "u"))
        runs[store] = {"value": round(mlups, 1), "ms_per_step": round(ms_max / args.steps, 5),
                       "phi_mass_drift": abs(m1 - m0) / abs(m0), "finite": bool(np.all(np.isfinite(uu))),
                       "max_u": float(np.max(np.abs(uu))), "after_steps": args.warmup + args.steps}
        sim.close()
    if rank != 0:
        return None
    peak, peak_kind = measured_peaks()
    v = runs["f32"]["value"]
    return {
        "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": runs["f32"]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": IMPACT_WORKLOAD.format(case=args.case, L=args.impact_L, D=args.impact_D, we=cfg["We"],
                                                      B=cfg["B"], nul=cfg["nu_l"], nug=cfg["nu_g"]),
                   "cells": N, "l2": "inputs larger than L2, no flush",
                   "parallelism": f"{world} independent replica(s), one per GPU"},
        "step_roofline": {"bytes_per_cell": step_bytes_per_cell(19, 4),
                          "frac_of_measured": round(v / world * 1e6 * step_bytes_per_cell(19, 4) / (peak * 1e9), 4),
                          "peak": peak, "peak_source": peak_kind},
        "runs": runs,
        "gpu_launches": int(kernels_per_step(cfg) * args.steps),
    }


def run_selftune(args, world, rank, local):
    """Film statistics over D x sigma x A_rep / sigma (Sec. 3.3): every case advanced in one batch,
    lbm_nci_diagnostics every --diag-every steps, each case's record taken at its maximum film
    volume (the instant of maximum activation)."""
    import torch

    from paper_2603_17481_gb300 import binding as B
    from paper_2603_17481_gb300 import build as lbm_build
    from paper_2603_17481_gb300 import workloads as W

    torch.cuda.set_device(local)
    lbm_build.build()
    cfgs = W.selftune_cases()
    stream = torch.cuda.Stream()
    sims = []
    for cfg in cfgs:
        phi, u = W.sweep_case_fields(cfg)
        s = B.Lbm(cfg, stream=stream.cuda_stream)
        s.init_fields(phi, u)
        sims.append(s)
    cells = sum(s.N for s in sims)
    batch = B.LbmBatch(sims, nstreams=16, stream=stream.cuda_stream)
    best = [None] * len(sims)
    every = args.diag_every + (args.diag_every & 1)
    steps, ms = 0, 0.0
    while steps < args.steps:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.step(every, sync=False)
        e1.record(stream)
        batch.synchronize()
        ms += e0.elapsed_time(e1)
        steps += every
        for k, s in enumerate(sims):
            d = s.nci_diagnostics()
            if best[k] is None or d["V_film"] > best[k]["V_film"]:
                best[k] = dict(d, step=steps)
    batch.close()
    for s in sims:
        s.close()
    if rank != 0:
        return None
    rows = []
    for cfg, b in zip(cfgs, best):
        rows.append({"D": cfg["diameter"], "sigma": cfg["sigma"], "A_rep_over_sigma": cfg["A_over_sigma"],
                     "step": b["step"], "R_n": round(b["R_n"], 5), "max_Frep": b["max_rep"],
                     "mean_Frep": b["mean_rep"], "V_film_over_D2": round(b["V_film"] / cfg["diameter"] ** 2, 5)})
    mlups = cells * steps / (ms * 1e-3) / 1e6
    return {
        "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world, "steps": steps,
        "warmup": 0, "ms_per_step": round(ms / steps, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "film statistics sweep: head-on collisions, D in {24,32,48}, sigma in "
                               "{0.005,0.01,0.02}, A_rep/sigma in {0.5,1,2}, We=4.6, density ratio 10",
                   "cases": len(cfgs), "cells": cells, "diag_every": every},
        "gpu_launches": None,
        "film_at_max_activation": rows,
    }


def run_reference(args, world, rank):
    """The FP64 CPU oracle as the reference arm, each step a bounded crop of the same workload."""
    if rank != 0:
        return None
    import numpy as np

    import oracle
    from paper_2603_17481_gb300 import workloads as W
    oracle.build()
    cfg, phi, u = make_workload(args.lattice)
    # calibrate: oracle throughput on a 64x32x32 crop of the workload
    budget = args.ref_budget / max(args.steps + args.warmup, 1)

    def crop(nx, ny, nz):
        g = phi.reshape(cfg["nz"], cfg["ny"], cfg["nx"])
        x0, y0, z0 = (cfg["nx"] - nx) // 2 - 28, (cfg["ny"] - ny) // 2, (cfg["nz"] - nz) // 2
        x0 = max(x0, 0)
        p = g[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx].ravel().copy()
        uu = u.reshape(3, cfg["nz"], cfg["ny"], cfg["nx"])[:, z0:z0 + nz, y0:y0 + ny, x0:x0 + nx].reshape(3, -1).copy()
        c = dict(cfg, nx=nx, ny=ny, nz=nz)
        return c, p, uu

    c, p, uu = crop(64, 32, 32)
    P = oracle.make_params(c)
    f = oracle.init(P, p, uu)
    t0 = time.perf_counter()
    oracle.step(P, f, p, 1)
    rate = 64 * 32 * 32 / (time.perf_counter() - t0)
    side = max(8, int(round((rate * budget / 2) ** (1 / 3))))
    nx, ny, nz = min(2 * side, cfg["nx"]), min(side, cfg["ny"]), min(side, cfg["nz"])
    c, p, uu = crop(nx, ny, nz)
    P = oracle.make_params(c)
    f = oracle.init(P, p, uu)
    ph = p
    for _ in range(args.warmup):
        f, ph, _ = oracle.step(P, f, ph, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, ph, _ = oracle.step(P, f, ph, 1)
    dt = time.perf_counter() - t0
    N = nx * ny * nz
    v = N * args.steps / dt / 1e6
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(Q=args.lattice), "sample": f"{nx}x{ny}x{nz} central crop per step"},
        "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": round(v, 4), "unit": "MLUPS",
                         "sample": f"each step: one FP64 oracle step on a {nx}x{ny}x{nz} crop of the workload"},
        "e2e": {"value": round(v, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--store", choices=["f32", "f16", "bf16", "mom"], default="f32")
    ap.add_argument("--lattice", type=int, choices=[19, 27], default=19,
                    help="collision: hydrodynamic lattice D3Q19 (the benchmark's) or D3Q27 (the paper's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--no-split-compare", dest="split_compare", action="store_false",
                    help="skip the split-step comparison (profiling runs)")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle time for cpu_baseline")
    ap.add_argument("--ref-budget", type=float, default=120.0, help="seconds for the whole reference arm")
    ap.add_argument("--workload", choices=["collision", "sweep", "swarm", "selftune", "impact"], default="collision",
                    help="collision: the 256x128x128 head-on case; sweep: the batched sweep of independent "
                         "cases; swarm: the 512^3 bubble swarm with the near-contact repulsion on and off; "
                         "selftune: film statistics over D x sigma x A_rep; impact: the paper's E1/E2 "
                         "droplet impacts at density ratio 1000")
    ap.add_argument("--cases", type=int, default=512, help="sweep: number of cases")
    ap.add_argument("--streams", type=int, nargs="+", default=[16], help="sweep: graph branch counts to time")
    ap.add_argument("--swarm-L", type=int, default=512)
    ap.add_argument("--swarm-bubbles", type=int, default=1500)
    ap.add_argument("--swarm-steps", type=int, default=0, help="swarm: total steps before counting bubbles")
    ap.add_argument("--swarm-count-at", type=int, nargs="*", default=[], help="swarm: also count bubbles at these steps")
    ap.add_argument("--swarm-gap", type=float, default=2.0, help="swarm: minimum initial surface gap in units of eps")
    ap.add_argument("--diag-every", type=int, default=20, help="selftune: steps between film statistics")
    ap.add_argument("--case", choices=["E1", "E2"], default="E1", help="impact: which of the paper's impacts")
    ap.add_argument("--impact-L", type=int, default=512, help="impact: periodic box edge")
    ap.add_argument("--impact-D", type=float, default=80.0, help="impact: droplet diameter in lattice units")
    args = ap.parse_args(argv)
    if args.steps < 1 or args.warmup < 0:
        ap.error("--steps must be >= 1 and --warmup >= 0")
    return args


def main():
    args = parse_args()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    elif args.workload == "sweep":
        line = run_sweep(args, world, rank, local)
    elif args.workload == "swarm":
        line = run_swarm(args, world, rank, local)
    elif args.workload == "selftune":
        line = run_selftune(args, world, rank, local)
    elif args.workload == "impact":
        line = run_impact(args, world, rank, local)
    else:
        line = run_ours(args, world, rank, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
