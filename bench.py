#!/usr/bin/env python
"""Throughput of the GB300 mDPD hot path: particle-steps/s (and pair-evals/s).

One bench step = one velocity-Verlet time step of the whole hot path (binning,
density pass, force pass fused with the half-kicks, drift and reflection, FP64
reductions) over the synthetic workload.  Prints one JSON line.

  python bench.py [--gpus N --steps K --warmup W] [--workload slab|bulk|slit|rock|batch]
                  [--precision fp32|fp64] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload on the host cores.
Multi-GPU (torchrun): each rank advances an independent replica (the path is
replicated, not sharded); value = all ranks' particle-steps / slowest rank.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 2 ** 20
ISSUE_LANES_PER_SM_CLK = 128          # 4 schedulers x 32 lanes, one instruction each per clock
NUM_SMS = 152
# Hand count of the FP32/INT32 lane operations one pair evaluation needs by its
# formula (Sec. 2.1, Eq. 1): separation 3, r^2 3, cutoff test 1, rsqrt 1, r 1,
# w_C 1, A term 1, rho_i+rho_j 1, w_d 1, B term 2, v_ij 3, e.v 4, F^D 3,
# Philox-4x32-10 ten rounds of 2 mul-hi + 2 mul-lo + 2 xor = 60, counter 2,
# xi 4, F^R 3, sum 2, scale 1, accumulate 3.
OPS_PER_PAIR = 100
# Hand count for one candidate test of the density pass (Sec. 2.1): separation
# 3, r^2 3, cutoff compare 1, select 1.
OPS_PER_CANDIDATE = 8

DESC = {
    "slab": "liquid-vapour slab, periodic 60x20x20, 20x20x20 liquid block at density 6, "
            "N=48000, A=-40 B=25 gamma=4.5 kT=1 rc=1 rd=0.75 dt=0.01",
    "bulk": "bulk liquid, periodic 10x10x10, N=6000 uniform random, A=-40 B=25 "
            "gamma=4.5 kT=1 rc=1 rd=0.75 dt=0.01",
    "slit": "slit pore 100x40 periodic x,y, height 20, walls from a voxel mask "
            "(voxel 0.5, 1 rc shell at density 6, A_fs=-30), g_x=0.02, fluid density 6",
    "rock": "synthetic porous rock, 256^3 voxel Gaussian random field (corr 4 voxels) at "
            "porosity 0.15, voxel 0.5 rc, 1 rc wall shell at density 6, fluid density 6, g_x=0.01",
    "batch": "256 independent liquid slabs in one batch (one launch per kernel for all), "
             "N_r ~ U[2000,20000] (2.94M in all), A_r ~ U[-50,-30], B_r ~ U[15,35], "
             "box 3L x L x L with L = (N_r/6)^(1/3), liquid middle third at density 6",
}


def make_workload(name: str, precision: int, seed: int, nvox: int = 256, nrep: int = 256):
    from paper_1903_10134_gb300 import inputs as I
    if name == "bulk":
        return I.bulk(seed=seed, precision=precision)
    if name == "slab":
        return I.slab(seed=seed, precision=precision)
    if name == "slit":
        return I.slit(seed=seed, precision=precision)
    if name == "rock":
        return I.rock(nvox=nvox, seed=seed, precision=precision)
    if name == "batch":
        return I.batch_slabs(nrep=nrep, seed=seed, precision=precision)
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def oracle_throughput(w, budget_s: float, max_steps: int = 1000):
    """Time the FP64 oracle on the workload: particle-steps/s over a bounded
    number of steps (at least one) chosen to fill about budget_s seconds."""
    from oracle import oracle as O
    walls = _oracle_walls(w)
    t0 = time.perf_counter()
    o = O.Oracle(w.params.copy(), w.pos, w.vel, w.type, w.seed, use_cells=True, **walls)
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.run(1)
    one = time.perf_counter() - t0
    steps = int(max(0, min(max_steps - 1, (budget_s - one) / max(one, 1e-6))))
    t1 = time.perf_counter()
    if steps:
        o.run(steps)
    el = time.perf_counter() - t1 + one
    total = steps + 1
    return {"value": o.n * total / el, "steps": total, "seconds": el, "setup_s": setup,
            "cores": O.num_threads(), "n": o.n}


def oracle_throughput_batch(ws, budget_s: float):
    """The FP64 oracle on a batch: one step of replica after replica (each a
    system of its own, as the oracle has no batching) until about budget_s
    seconds are spent; particle-steps/s over the replicas done."""
    from oracle import oracle as O
    done_n, el, k = 0, 0.0, 0
    while k < len(ws) and (k == 0 or el < budget_s):
        w = ws[k]
        o = O.Oracle(w.params.copy(), w.pos, w.vel, w.type, w.seed, use_cells=True)
        t0 = time.perf_counter()
        o.run(1)
        el += time.perf_counter() - t0
        done_n += o.n
        k += 1
    return {"value": done_n / el, "steps": 1, "replicas": k, "seconds": el,
            "cores": O.num_threads(), "n": done_n}


def _oracle_walls(w) -> dict:
    """Wall particles and mask for the oracle (its own packing of the image)."""
    if w.mask is None:
        return {}
    import numpy as np
    from oracle import oracle as O
    wpos, _ = O.place_walls(w.mask, w.params.periodic, w.voxel, w.origin, w.wall_density,
                            w.shell, w.wall_seed)
    w.pos = np.concatenate([w.pos, wpos])
    w.vel = np.concatenate([w.vel, np.zeros_like(wpos)])
    w.type = np.concatenate([w.type, np.full(len(wpos), w.wall_type, np.int32)])
    w.mask_applied = True
    return {"mask": w.mask, "voxel": w.voxel, "origin": w.origin}


def kernel_traffic(workload: str, precision: str) -> dict:
    """DRAM bytes per launch of each profiled kernel from the committed ncu
    summary profiles/traffic_<workload>.txt ({} when there is none, the
    precision is not FP32, or a source file of that kernel changed since the
    counters were taken: each kernel line carries the SHA-1 of its sources)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    if precision != "fp32" or not os.path.exists(path):
        return {}
    out = {}
    try:
        for line in open(path):
            # kernel <name> bytes <n> sha1 <hex> sources <a,b,...>
            f = line.split()
            if len(f) < 8 or f[0] != "kernel":
                continue
            h = hashlib.sha1()
            for src in f[7].split(","):
                with open(os.path.join(ROOT, src), "rb") as fh:
                    h.update(fh.read())
            if h.hexdigest() == f[5]:
                out[f[1]] = int(f[3])
    except (OSError, ValueError):
        return {}
    return out


def _cell_counts(x, params, nc):
    import numpy as np
    lo = np.array(params.box_lo, dtype=float)
    L = np.array(params.box, dtype=float)
    q = np.floor((x - lo) / (L / nc)).astype(np.int64)
    q = np.clip(q, 0, nc - 1)
    counts = np.zeros(tuple(nc[::-1]), dtype=np.int64)       # [z, y, x]
    np.add.at(counts, (q[:, 2], q[:, 1], q[:, 0]), 1)
    return counts


def _neighbourhood_sum(counts, periodic):
    """For every cell, the sum of counts over its 27 neighbour cells."""
    import numpy as np
    neigh = np.zeros_like(counts)
    for oz in (-1, 0, 1):
        for oy in (-1, 0, 1):
            for ox in (-1, 0, 1):
                sh = counts
                for axis, o, k in ((0, oz, 2), (1, oy, 1), (2, ox, 0)):
                    if o == 0:
                        continue
                    if periodic[k]:
                        sh = np.roll(sh, -o, axis=axis)
                    else:
                        pad = np.zeros_like(sh)
                        idx = [slice(None)] * 3
                        src = [slice(None)] * 3
                        if o > 0:
                            idx[axis] = slice(0, sh.shape[axis] - 1)
                            src[axis] = slice(1, None)
                        else:
                            idx[axis] = slice(1, None)
                            src[axis] = slice(0, sh.shape[axis] - 1)
                        pad[tuple(idx)] = sh[tuple(src)]
                        sh = pad
                neigh += sh
    return neigh


def candidate_tests(x, params, ncell, frozen=None) -> int:
    """Candidate tests of one density pass: every particle is tested against
    every particle of its 27 neighbour cells (itself included), so the count
    is sum over cells c of n_c times the particles in c's neighbourhood.  With
    `frozen` (a per-particle flag; the split density pass), only mobile
    particles scan: a frozen particle's density is its constant frozen-frozen
    part plus the terms its mobile neighbours scatter to it."""
    import numpy as np
    nc = np.array(ncell, dtype=np.int64)
    counts = _cell_counts(x, params, nc)
    neigh = _neighbourhood_sum(counts, params.periodic)
    if frozen is None or not np.any(frozen):
        return int((counts * neigh).sum())
    cm = counts - _cell_counts(x[frozen], params, nc)
    return int((cm * neigh).sum())


OBS_NAMES = ("px", "py", "pz", "ke", "kT", "Wxx", "Wyy", "Wzz", "Wxy", "Wxz", "Wyz",
             "sum_vx2", "sum_vy2", "sum_vz2")


def fp64_leg(mdpd, args, stream, workload=None):
    """The same workload with FP64 pair arithmetic: autotuned, warmed up, then
    min(K, 100) steps timed with CUDA events (same L2 rule as the FP32 run)."""
    import torch
    workload = workload or args.workload
    w = make_workload(workload, 0, seed=1, nvox=args.nvox, nrep=args.nrep)
    if workload == "batch":
        s = mdpd.Batch.from_workloads(w, stream=stream)
    else:
        s = mdpd.System.from_workload(w, stream=stream)
    try:
        s.autotune()
        for _ in range(3):
            s.step(1)
        s.sync()
        n = s.n
        K = max(3, min(args.steps, 100))
        working_set = n * (32 + 32 + 8 + 4 + 2 * 3 * 24 + 8)
        flush = working_set < 4 * L2_BYTES
        flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32,
                                device=torch.cuda.current_device()) if flush else None
        torch.cuda.synchronize()
        if flush:
            ms = 0.0
            for _ in range(K):
                with torch.cuda.stream(stream):
                    flush_buf.fill_(1.0)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s.step(1)
                b.record(stream)
                torch.cuda.synchronize()
                ms += a.elapsed_time(b)
        else:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(K)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
        s.sync()
        pairs = s.pair_count()
        value = n * K / (ms * 1e-3)
        return {"value": value, "unit": "particle-steps/s", "ms_per_step": ms / K, "steps": K,
                "pair_evals_per_s": value * pairs / 2 / n, "dtype": "f64",
                "l2": "flushed between timed steps" if flush else "working set > L2"}
    finally:
        s.close()


def precision_error(mdpd, s, w, workload):
    """Error of the FP32 pair arithmetic against the FP64 path (itself pinned
    to the FP64 oracle at 1e-12 by the tests) on the bench's final state: an
    FP64 handle is built from the same particles (wall particles included as
    their frozen type), step index and seed; both evaluate forces, densities
    and observables once.  For a batch, replica 0."""
    import numpy as np
    x, v, t, _ = s.state()
    step = mdpd.mdpd_step_count(s.h)
    f32, rho32 = s.forces()
    if workload == "batch":
        w0 = w[0]
        a, b = 0, w0.n
        x, v, t, f32, rho32 = x[a:b], v[a:b], t[a:b], f32[a:b], rho32[a:b]
        obs32 = s.observables()[0]
        p, seed = w0.params, w0.seed
    else:
        obs32 = s.observables()
        p, seed = w.params, w.seed
    with mdpd.System(p.copy(precision=0), x, v, t, seed) as d:
        mdpd.mdpd_set_step(d.h, step)
        f64, rho64 = d.forces()
        obs64 = d.observables()
    fn = np.linalg.norm(f64, axis=1)
    rms = float(np.sqrt(np.mean(fn ** 2)))
    ferr = np.linalg.norm(f32 - f64, axis=1) / np.maximum(fn, rms)
    rerr = np.abs(rho32 - rho64) / np.maximum(np.abs(rho64), max(float(np.mean(rho64)), 1e-30))
    # momentum is a cancelling sum: its error is stated relative to sum |m v|
    scale = {k: abs(obs64[k]) for k in range(14)}
    for k in range(3):
        scale[k] = float(np.abs(v[:, k]).sum())
    obs_err = {OBS_NAMES[k]: float(abs(obs32[k] - obs64[k]) / max(scale[k], 1e-30))
               for k in range(14)}
    return {"vs": "FP64 pair arithmetic on the GPU (pinned to the FP64 oracle at 1e-12)",
            "n": int(len(x)), "force_rel_max": float(ferr.max()),
            "force_rel_rms": float(np.sqrt(np.mean(ferr ** 2))),
            "density_rel_max": float(rerr.max()), "observables_rel": obs_err,
            "note": "per particle |f32 - f64| / max(|f64|, rms f64) and |rho32 - rho64| / "
                    "max(rho64, mean rho64); momentum relative to sum |v|; one force evaluation "
                    "at the final state"}


def oracle_error(mdpd, s, w, workload):
    """Error of the FP32 path against the FP64 oracle on
    the bench's final state: the GPU evaluates densities, forces and
    observables once at its current state and step index (mdpd_forces), and
    the oracle evaluates the same state (positions, velocities, types, wall
    particles included, same seed and step) in FP64 on the host cores.  Every
    particle is compared; for a batch, replica 0."""
    import numpy as np
    from oracle import oracle as O
    x, v, t, _ = s.state()
    step = mdpd.mdpd_step_count(s.h)
    f32, rho32 = s.forces()
    if workload == "batch":
        w0 = w[0]
        a, b = 0, w0.n
        x, v, t, f32, rho32 = x[a:b], v[a:b], t[a:b], f32[a:b], rho32[a:b]
        obs32 = s.observables()[0]
        p, seed = w0.params, w0.seed
    else:
        obs32 = s.observables()
        p, seed = w.params, w.seed
    t0 = time.perf_counter()
    o = O.Oracle(p.copy(precision=0), x, v, t, seed, use_cells=True, step=step)
    el = time.perf_counter() - t0
    f64, rho64 = o.a, o.rho
    obs64 = o.observables()
    mob = ~np.isin(t, np.array(p.frozen_types, dtype=np.int32))
    fn = np.linalg.norm(f64[mob], axis=1)
    rms = float(np.sqrt(np.mean(fn ** 2))) if fn.size else 1.0
    ferr = np.linalg.norm(f32[mob] - f64[mob], axis=1) / np.maximum(fn, rms)
    rerr = np.abs(rho32 - rho64) / np.maximum(np.abs(rho64), max(float(np.mean(rho64)), 1e-30))
    scale = {k: abs(obs64[k]) for k in range(14)}
    for k in range(3):
        scale[k] = float(np.abs(v[mob, k]).sum())
    obs_err = {OBS_NAMES[k]: float(abs(obs32[k] - obs64[k]) / max(scale[k], 1e-30))
               for k in range(14)}
    return {"vs": "FP64 CPU oracle (oracle/), same state, step index and seed",
            "n": int(len(x)), "mobile": int(mob.sum()), "oracle_seconds": el,
            "force_rel_max": float(ferr.max()) if ferr.size else 0.0,
            "force_rel_rms": float(np.sqrt(np.mean(ferr ** 2))) if ferr.size else 0.0,
            "density_rel_max": float(rerr.max()), "observables_rel": obs_err,
            "tolerance": {"force": 1e-5, "density": 2e-6},
            "note": "per mobile particle |f32 - f64| / max(|f64|, rms f64); every particle's "
                    "|rho32 - rho64| / max(rho64, mean rho64); momentum relative to sum |v|; "
                    "the virial from the oracle's full force evaluation"}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The FP64 oracle on the host cores, same workload: W warm-up steps and up
    to K timed steps, stopped early once about args.ref_seconds have been spent
    (the bounded sample is stated in the output)."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from oracle import oracle as O
    w = make_workload(args.workload, 0, seed=1, nvox=args.nvox, nrep=args.nrep)
    if args.workload == "batch":
        info = oracle_throughput_batch(w, args.ref_seconds)
        value = info["value"]
        sample = (f"one FP64 oracle step of each of the first {info['replicas']} of "
                  f"{len(w)} replicas ({info['n']} particles), {info['seconds']:.1f} s")
        print(json.dumps({
            "impl": "reference", "metric": "particle-steps/s", "value": value,
            "unit": "particle-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(x.n for x in w) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": DESC[args.workload],
                       "n": sum(x.n for x in w), "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s",
                             "cores": info["cores"], "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}), flush=True)
        return
    walls = _oracle_walls(w)
    o = O.Oracle(w.params.copy(), w.pos, w.vel, w.type, w.seed, use_cells=True, **walls)
    t0 = time.perf_counter()
    for _ in range(args.warmup):
        o.run(1)
        if time.perf_counter() - t0 > args.ref_seconds / 4:
            break
    done, el = 0, 0.0
    while done < args.steps and (done == 0 or el < args.ref_seconds):
        t1 = time.perf_counter()
        o.run(1)
        el += time.perf_counter() - t1
        done += 1
    value = o.n * done / el
    sample = (f"{done} of {args.steps} timed FP64 oracle steps of the full {args.workload} "
              f"workload (N={o.n}), {el:.1f} s")
    line = {
        "impl": "reference", "metric": "particle-steps/s", "value": value,
        "unit": "particle-steps/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": DESC[args.workload], "n": o.n,
                   "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": O.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def aggregate_ranks(ms: float, n: int, steps: int, world: int, device=None):
    """Whole-job throughput of independent replicas, one per rank: the slowest
    rank's timed milliseconds (MAX all-reduce) and all ranks' particle-steps
    divided by it.  Works with any torch.distributed backend (nccl on GPUs,
    gloo on CPU)."""
    import torch
    t = torch.tensor([ms, float(n)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        m = t[:1].clone()
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
        tot = t[1:].clone()
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
        ms_max, n_all = float(m.item()), float(tot.item())
    else:
        ms_max, n_all = float(ms), float(n)
    return ms_max, n_all * steps / (ms_max * 1e-3)


def replica_seed(rank: int) -> int:
    """Seed of the replica advanced by a rank (independent replicas)."""
    return 1 + rank


def slab_leg(mdpd, args, stream):
    """The liquid-vapour slab (N = 48,000) beside the headline: FP32
    throughput (L2 flushed between timed steps), the same with FP64 pair
    arithmetic, and the FP32 error against both the FP64 GPU path and the FP64
    oracle on the final state."""
    import torch
    w = make_workload("slab", 1, seed=1)
    s = mdpd.System.from_workload(w, stream=stream)
    try:
        res = s.autotune()
        for _ in range(5):
            s.step(1)
        s.sync()
        K = max(3, min(args.steps, 200))
        flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32,
                                device=torch.cuda.current_device())
        ms = 0.0
        for _ in range(K):
            with torch.cuda.stream(stream):
                flush_buf.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(1)
            b.record(stream)
            torch.cuda.synchronize()
            ms += a.elapsed_time(b)
        s.sync()
        pairs = s.pair_count()
        value = s.n * K / (ms * 1e-3)
        out = {"workload": "slab", "desc": DESC["slab"], "n": s.n, "steps": K,
               "value": value, "unit": "particle-steps/s", "ms_per_step": ms / K,
               "pair_evals_per_s": value * pairs / 2 / s.n, "dtype": "f32",
               "autotune": {"density": {mdpd.KERNELS_NLIST: "nlist",
                                        mdpd.KERNELS_NLIST_THREAD: "nlist-thread"}[res[0]],
                            "force_lanes": res.lanes},
               "l2": "flushed between timed steps"}
        if not args.no_error:
            out["fp32_error"] = precision_error(mdpd, s, w, "slab")
        if not args.no_oracle_error:
            out["oracle_error"] = oracle_error(mdpd, s, w, "slab")
    finally:
        s.close()
    if not args.no_fp64:
        out["fp64"] = fp64_leg(mdpd, args, stream, workload="slab")
        out["fp32_speedup_vs_fp64"] = out["value"] / out["fp64"]["value"]
    return out


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1903_10134_gb300 import mdpd

    dev = torch.cuda.current_device()
    prec = 0 if args.precision == "fp64" else 1
    w = make_workload(args.workload, prec, seed=replica_seed(rank), nvox=args.nvox,
                      nrep=args.nrep)
    stream = torch.cuda.Stream()
    if args.workload == "batch":
        s = mdpd.Batch.from_workloads(w, stream=stream)
    else:
        s = mdpd.System.from_workload(w, stream=stream)
    tuned = None
    if args.kernels == "auto":
        res = s.autotune()
        chosen, tms = res
        tuned = {"chosen": {mdpd.KERNELS_NLIST: "nlist", mdpd.KERNELS_NLIST_THREAD: "nlist-thread"}[chosen],
                 "density_ms": {"nlist": tms[0], "nlist-thread": tms[1]},
                 "density_shape": res.shape,
                 "force_lanes": res.lanes,
                 "force_ms": {str(l): t for l, t in zip((1, 2, 4), res.force_ms) if t >= 0}}
    elif args.kernels != "nlist":
        s.set_option(mdpd.OPT_KERNELS, {"scan": mdpd.KERNELS_SCAN,
                                        "nlist-thread": mdpd.KERNELS_NLIST_THREAD}[args.kernels])
    if args.kernels != "auto" and args.density_shape is not None:
        s.set_option(mdpd.OPT_DENSITY_SHAPE, args.density_shape)
    if args.kernels != "auto" and args.force_lanes is not None:
        s.set_option(mdpd.OPT_FORCE_LANES, args.force_lanes)
    n = s.n
    working_set = n * (16 + 16 + 4 + 4 + 2 * 3 * 24 + 8)
    flush = working_set < 4 * L2_BYTES
    flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev) if flush else None

    def l2_flush():
        with torch.cuda.stream(stream):
            flush_buf.fill_(1.0)

    # warm-up (also captures the step graphs)
    for _ in range(max(args.warmup, 3)):
        s.step(1)
    s.step(2)
    s.sync()
    pairs = s.pair_count()

    K = args.steps
    s.set_option(mdpd.OPT_PROFILE, 0 if args.no_profile else K)
    s.set_option(mdpd.OPT_PROFILE_EVERY, args.profile_every)
    clocks = ClockSampler(dev) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if flush:
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for k in range(K):
            l2_flush()
            starts[k].record(stream)
            s.step(1)
            ends[k].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    else:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    s.sync()
    prof, prof_steps, launches = s.profile()

    ms_max, value = aggregate_ranks(ms, n, K, world, device=dev)

    # candidate tests of the density pass, counted from the state after the
    # timed steps (rank 0; the other ranks hold replicas of the same workload)
    cand = None
    if rank == 0:
        import numpy as np
        xs, _, ts, _ = s.state()
        ws = w if args.workload == "batch" else [w]
        split_density = (tuned and tuned["chosen"] == "nlist-thread") or \
            args.kernels == "nlist-thread"
        off = 0
        cand = 0
        for wr in ws:
            nr = wr.n if args.workload == "batch" else n
            p = wr.params
            ncell = [max(1, int(math.floor(p.box[k] / p.rc))) for k in range(3)]
            # the thread-per-particle pass of a single system with frozen
            # particles runs the frozen split
            fz = None
            if args.workload != "batch" and p.frozen_types and split_density:
                fz = np.isin(ts[off:off + nr], np.array(p.frozen_types))
            cand += candidate_tests(xs[off:off + nr], p, ncell, fz)
            off += nr

    # end-to-end through the host-pointer C ABI: every step uploads the state
    # a caller resumes from (x, v and the accelerations of the next
    # half-kick) from pinned host memory with mdpd_set_state_accel (which
    # evaluates no forces), advances one step, and reads the same three arrays
    # back into pinned host memory
    e2e = None
    if not args.no_e2e:
        x, v, _, _ = s.state()
        acc = mdpd.mdpd_get_accel(s.h)
        hx = torch.from_numpy(x).pin_memory().numpy()
        hv = torch.from_numpy(v).pin_memory().numpy()
        ha = torch.from_numpy(acc).pin_memory().numpy()
        ke = max(3, min(K, 50 if n > 10 ** 6 else 200))

        def e2e_step():
            mdpd.mdpd_set_state_accel(s.h, hx, hv, ha)
            s.step(1)
            mdpd.mdpd_get_state(s.h, hx, hv, want_type=False, want_rho=False)
            mdpd.mdpd_get_accel(s.h, ha)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        el = time.perf_counter() - t0
        et = torch.tensor([el], dtype=torch.float64, device=dev)
        if world > 1:
            torch.distributed.all_reduce(et, op=torch.distributed.ReduceOp.MAX)
        e2e = {"value": world * n * ke / float(et.item()), "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(hx.nbytes + hv.nbytes + ha.nbytes),
               "d2h_bytes_per_step": int(hx.nbytes + hv.nbytes + ha.nbytes),
               "steps": ke,
               "api": "mdpd_set_state_accel + mdpd_step(1) + mdpd_get_state + mdpd_get_accel "
                      "(host buffers; no force evaluation besides the step's own)"}

    if rank == 0:
        peaks = measured_peaks()
        clk_mhz = peaks.get("sm_max_mhz", 2070.0)
        alu_nominal = NUM_SMS * ISSUE_LANES_PER_SM_CLK * clk_mhz * 1e6 / 1e12     # Tlane-op/s
        try:
            alu_peak = mdpd.mdpd_measure_fma_peak()[0] / 1e12
            alu_peak_of = "measured: FP32 FMA issue-rate microbenchmark (mdpd_measure_fma_peak)"
        except mdpd.MDPDError:
            alu_peak = alu_nominal
            alu_peak_of = "nominal: 152 SMs x 128 lanes x sm_max_mhz"
        per = max(prof_steps, 1)
        dens_ms = prof.get("density", 0.0) / per
        force_ms = prof.get("force", 0.0) / per
        traffic = kernel_traffic(args.workload, args.precision)
        hbm_peak = peaks.get("hbm_gbs", 6790.0)
        # lists: 4 B per directed partner; FP32 tiles 16 B (FP64 32 B)
        tile = 16 if prec == 1 else 32
        npart = pairs / max(n, 1)
        dens_name = "k_density_cell" if (tuned and tuned["chosen"] == "nlist") or \
            args.kernels == "nlist" else "k_density_nl"

        def entry(name, work, ms_k, bytes_pp, what):
            if ms_k <= 0:
                return None
            ach = work / (ms_k * 1e-3) / 1e12
            gbs = n * bytes_pp / (ms_k * 1e-3) / 1e9
            return {"kernel": name, "what": what, "ms": ms_k, "achieved": ach,
                    "frac": ach / alu_peak, "traffic": traffic.get(name),
                    "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm_peak, "frac": gbs / hbm_peak,
                            "bytes_per_particle": bytes_pp, "peak_of": "measured"}}
        kern = {
            "density": entry(dens_name, cand * OPS_PER_CANDIDATE, dens_ms,
                             tile + 8 + tile // 4 + 4 * npart + 4,
                             f"{cand} candidate tests x {OPS_PER_CANDIDATE} ops"),
            "force": entry("k_force_nl", pairs * OPS_PER_PAIR, force_ms,
                           (tile * 2 + tile // 4) + 4 * npart + 4 + 96,
                           f"{pairs} directed pairs x {OPS_PER_PAIR} ops"),
        }
        dom = max((k for k in kern if kern[k]), key=lambda k: kern[k]["ms"], default=None)
        fp64 = None
        if prec == 1 and not args.no_fp64:
            fp64 = fp64_leg(mdpd, args, stream)
        err = orc_err = None
        if prec == 1 and not args.no_error:
            err = precision_error(mdpd, s, w, args.workload)
        if not args.no_oracle_error:
            orc_err = oracle_error(mdpd, s, w, args.workload)
        slab = None
        if args.workload != "slab" and not args.no_slab and world == 1:
            slab = slab_leg(mdpd, args, stream)
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            wc = make_workload(args.workload, 0, seed=1, nvox=args.nvox, nrep=args.nrep)
            if args.workload == "batch":
                info = oracle_throughput_batch(wc, args.cpu_seconds)
                sample = (f"one FP64 oracle step of each of the first {info['replicas']} of "
                          f"{len(wc)} replicas ({info['n']} particles), {info['seconds']:.1f} s")
            else:
                info = oracle_throughput(wc, args.cpu_seconds, max_steps=200)
                sample = (f"{info['steps']} FP64 oracle steps of the full {args.workload} "
                          f"workload (N={info['n']}), {info['seconds']:.1f} s")
            cpu = {"value": info["value"], "unit": "particle-steps/s", "cores": info["cores"],
                   "kind": "oracle", "sample": sample}
            # the same oracle on one thread (its sums do not depend on the thread
            # count), when one step of it fits the budget: estimated from the
            # all-thread step time
            from oracle import oracle as O
            nthr = O.num_threads()
            per_step = info["seconds"] / max(info["steps"], 1)
            if args.workload == "batch" or per_step * nthr <= args.cpu_seconds / 3:
                O.set_num_threads(1)
                try:
                    wc1 = make_workload(args.workload, 0, seed=1, nvox=args.nvox, nrep=args.nrep)
                    if args.workload == "batch":
                        i1 = oracle_throughput_batch(wc1, args.cpu_seconds / 3)
                        s1 = f"one step of each of the first {i1['replicas']} replicas"
                    else:
                        i1 = oracle_throughput(wc1, args.cpu_seconds / 3, max_steps=200)
                        s1 = f"{i1['steps']} steps of the full workload"
                finally:
                    O.set_num_threads(nthr)
                cpu["one_thread"] = {"value": i1["value"], "cores": 1,
                                     "sample": f"{s1}, {i1['seconds']:.1f} s"}
            else:
                cpu["one_thread"] = {"value": None, "cores": 1,
                                     "sample": f"skipped: one step takes about "
                                               f"{per_step * nthr:.0f} s on one thread"}
        line = {
            "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
            "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == 1 else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": DESC[args.workload], "n": n,
                       "nvox": args.nvox if args.workload == "rock" else None,
                       "replicas": len(w) if args.workload == "batch" else None,
                       "precision": args.precision, "kernels": args.kernels, "autotune": tuned,
                       "l2": "flushed between timed steps" if flush else "working set > L2",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "pair_evals_per_s": value * pairs / 2 / n,
            "roofline": ({"bound": "alu", "kernel": kern[dom]["kernel"], "pass": dom,
                          "achieved": kern[dom]["achieved"], "peak": alu_peak,
                          "unit": "Tlane-op/s", "frac": kern[dom]["frac"],
                          "traffic": kern[dom]["traffic"], "work": kern[dom]["what"],
                          "peak_of": alu_peak_of, "peak_nominal": alu_nominal,
                          "hbm": kern[dom]["hbm"], "all": kern} if dom else None),
            "kernel_ms_per_step": {k: v / max(prof_steps, 1) for k, v in prof.items()},
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "fp32_error": err,
            "oracle_error": orc_err,
            "fp64": fp64,
            "slab": slab,
            "e2e": e2e,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(DESC), default="rock")
    ap.add_argument("--precision", choices=("fp32", "fp64"), default="fp32")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile", action="store_true",
                    help="no per-kernel events in the timed region (no roofline)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the FP64 throughput leg after the FP32 run")
    ap.add_argument("--no-error", action="store_true",
                    help="skip the FP32-vs-FP64 error evaluation after the timed steps")
    ap.add_argument("--no-oracle-error", action="store_true",
                    help="skip the FP32-vs-oracle error evaluation after the timed steps")
    ap.add_argument("--no-slab", action="store_true",
                    help="skip the slab leg (FP32 vs FP64) beside a non-slab headline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--nvox", type=int, default=256, help="rock image edge in voxels")
    ap.add_argument("--nrep", type=int, default=256, help="replicas of the batch workload")
    ap.add_argument("--kernels", choices=("auto", "nlist", "nlist-thread", "scan"), default="auto")
    ap.add_argument("--density-shape", type=int, choices=(0, 1), default=None,
                    help="code shape of the thread-per-particle density kernel when "
                         "--kernels is not auto")
    ap.add_argument("--force-lanes", type=int, choices=(1, 2, 4), default=None,
                    help="lanes per particle of the force pass when --kernels is not auto")
    ap.add_argument("--profile-every", type=int, default=10,
                    help="record per-kernel events on every k-th timed step")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
