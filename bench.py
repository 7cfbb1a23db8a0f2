#!/usr/bin/env python
"""Benchmark of the IC(k) hot path: numeric factorization (value scatter + the
persistent Chol/Trsm/Herk/Gemm task-DAG kernel) followed by a PCG solve with the
factor as preconditioner.

Workload (default): 27-point constant-coefficient Laplacian on a 96^3 grid
(884,736 rows, 23,393,656 nonzeros), geometric nested dissection (separator planes cut
into strips of at most 4096 rows, each numbered in 2x2 colour classes), 2D blocks of at
most 4096 rows, IC(2), FP64, b ~ N(0,1), PCG to relative residual 1e-10.

A step is one numeric factorization plus one PCG solve, which runs as one CUDA graph
(the library's loop on the device).  value = algorithmic factor flops / factor time
(GFLOP/s, the time of the factorization's kernels, CUDA events recorded on the
launching stream before and after them).  The per-kernel times of the roofline
objects come from a pass of three more steps with the library's own CUDA events
around every kernel (PCG then loops on the host).  e2e repeats the step through the C
ABI from pinned host buffers, with the host-to-device copies of A's values and b and
the device-to-host copy of x inside the timed region.

With one GPU the line also carries, outside the timed region, the other workloads of
the method (each with a few fixed repetitions): c4_shift (Q1 elasticity, FP32 +
learned shift vs plain FP64, time to 1e-8), c3_batch (512 diffusion cubes in one
launch) and c5 (160^3 7-point diffusion IC(3), FP32 vs FP64 time to 1e-8).  --shift,
--c3 and --c5 print each of them as a line of its own instead.

--impl reference times the CPU oracle (the single-threaded FP64 reference the
parity tests use): one numeric factorization of the same workload per step.
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

METRIC = "IC(k) factor GFLOP/s & HBM GB/s; PCG time-to-1e-8 vs plain FP64 on GB300"
FP64_NOMINAL_GFLOPS = 1250.0  # GB300's nominal FP64 rate, used only if the probe cannot run
# DRAM bytes (read + write) per launch of a solve kernel of the 27-point IC(2) problem,
# per factor entry: ncu captures (dram__bytes_read.sum + dram__bytes_write.sum, one
# launch each) of the 48^3 and 64^3 problems gave 14.89 / 14.76 (forward) and 14.98 /
# 14.97 (backward) bytes per entry; the 64^3 figures are scaled to the factor at hand
SOLVE_TRAFFIC_PER_ENTRY = {(2, "forward_dag"): 14.76, (2, "backward_dag"): 14.97}
# The captures above and below ordered the separators lexicographically (sep_colours
# 0); under another separator order the traffic fields are left null, not reused
CAPTURED_SEP_COLOURS = 0
# DRAM bytes (read + write) per factor entry of one launch of the numeric task kernel
# of the 27-point IC(k) problem, by k: ncu captures of the 48^3, 64^3 and 80^3
# problems gave 50.4, 57.8 and 55.1 bytes per entry; the 80^3 figure is scaled to the
# factor at hand
NUMERIC_TRAFFIC_PER_ENTRY = {2: 55.1}


def timed_solve(ick, torch, h, av, b, x, tol, stream=None):
    """One factorization and PCG solve with the library's per-kernel timing off, so that
    pcg_solve runs as one graph (its loop on the device).  Returns the CUDA events
    recorded on the stream before and after the factorization and after the solve,
    the iterations and the residual; the factorization's status is checked."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(stream)
    ick.ic_numeric_async(h, av, stream)
    ev[1].record(stream)
    it, rel = ick.pcg_solve(h, av, b, x, tol, 5000, stream)
    ev[2].record(stream)
    ick.ic_numeric_status(h)
    return ev, it, rel


def factor_kernel_ms(ick, h, av, stream=None, reps=3):
    """Mean time of the factorization's own kernels (value scatter + task-DAG kernel),
    from the library's CUDA events around them: reps factorizations with the
    library's per-kernel timing on (switched off again afterwards)."""
    ick.ic_set_timing(h, True)
    t = []
    for _ in range(reps):
        ick.ic_numeric(h, av, stream)
        tm = ick.ic_get_timing(h)
        t.append(tm["prepare_ms"] + tm["numeric_ms"])
    ick.ic_set_timing(h, False)
    return sum(t) / len(t)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=96)
    ap.add_argument("--k", type=int, default=2)
    ap.add_argument("--block-rows", type=int, default=4096)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--pcg-host-loop", action="store_true",
                    help="keep the library's per-kernel timing on in the timed steps, so that PCG loops on "
                         "the host (the same kernels, no graph): for profilers")
    ap.add_argument("--numeric-only", action="store_true",
                    help="time only the numeric factorization (for profiling runs)")
    ap.add_argument("--no-f32", action="store_true", help="skip the mixed-precision arm")
    ap.add_argument("--solve-mode", type=int, default=0, choices=[0, 1],
                    help="triangular solves: 0 block-DAG, 1 row-level")
    ap.add_argument("--solve-lanes", type=int, default=0, help="lanes per row of the solves (0: default)")
    ap.add_argument("--solve-ctas", type=int, default=0, help="CTAs per SM of the solves (0: default)")
    ap.add_argument("--shift", action="store_true",
                    help="learned-shift workload instead: Q1 elasticity, FP32 + learned shift vs plain FP64")
    ap.add_argument("--ne", type=int, default=48, help="elements per side of the --shift workload")
    ap.add_argument("--c3", action="store_true",
                    help="batch workload instead: 512 7-point diffusion cubes, IC(1), FP32, one launch")
    ap.add_argument("--c5", action="store_true",
                    help="7-point diffusion workload instead: 160^3 (--side), sigma 2, z faces x100, IC(3)")
    ap.add_argument("--leaf-rows", type=int, default=0,
                    help="nested-dissection leaf size (the pruning of the ND tree); 0: --block-rows")
    ap.add_argument("--sep-colours", type=int, default=2,
                    help="ND separator planes cut into block-sized strips numbered in C x C colour "
                         "classes (0: lexicographic)")
    ap.add_argument("--leaf-colours", type=int, default=0,
                    help="number each ND leaf box in C x C x C colour classes (0: lexicographic)")
    ap.add_argument("--no-sub", action="store_true",
                    help="leave the C4 / C3 / C5 workloads out of the default line")
    a = ap.parse_args()
    if a.leaf_rows <= 0:
        a.leaf_rows = a.block_rows
    return a


def workload_name(a):
    leaf = "" if a.leaf_rows == a.block_rows else f" (ND leaves <= {a.leaf_rows} rows)"
    if a.sep_colours >= 2:
        leaf += f", separator strips in {a.sep_colours}x{a.sep_colours} colour classes"
    if a.leaf_colours >= 2:
        c = a.leaf_colours
        leaf += f", leaves in {c}x{c}x{c} colour classes"
    solves = {0: "block-DAG", 1: "row-level"}[a.solve_mode]
    return (f"27-point Laplacian {a.side}^3 (n={a.side ** 3}), geometric ND{leaf}, 2D blocks <= "
            f"{a.block_rows} rows, IC({a.k}) FP64 factor + FP64 PCG to {a.tol:g}, {solves} triangular solves")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                rows.append(parts)
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")

        util = [num(r[4]) for r in rows]
        loaded = [r for r, u in zip(rows, util) if u >= 50] or rows
        sm = [num(r[1]) for r in loaded]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in loaded:
            for nm, v in zip(names, r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": num(loaded[0][2]),
                "samples": len(loaded), "reasons": sorted(reasons)}


def oracle_problem(side, k, leaf_rows, sep_colours, leaf_colours):
    """The oracle's symbolic phase of the side^3 27-point problem, as the GPU arm orders
    it (geometric ND with the same leaf size, separator and leaf orders)."""
    import oracle
    import synth
    prob = synth.laplace3d_27pt(side)
    perm, _ = oracle.nd_grid(side, side, side, 1, leaf_rows, sep_colours=sep_colours, leaf_colours=leaf_colours)
    return prob, oracle.OracleIC.from_problem(prob, perm, k)


def time_oracle_numeric(prob, h):
    t0 = time.perf_counter()
    st = h.numeric(prob.vals)
    t = time.perf_counter() - t0
    assert st == 0
    return t


def max_over_ranks(values, world, device="cuda"):
    """Element-wise maximum of `values` (floats) over the ranks of the default process
    group (a no-op for one rank): the job's time is its slowest replica's."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(values), device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rate(units_per_replica, world, seconds):
    """Whole-job throughput of `world` replicas each processing units_per_replica in
    at most `seconds`."""
    return world * units_per_replica / seconds


def reference_arm(a, rank, world):
    if rank != 0:
        return
    # each step: one oracle numeric factorization of the full workload (single thread)
    prob, h = oracle_problem(a.side, a.k, a.leaf_rows, a.sep_colours, a.leaf_colours)
    for _ in range(a.warmup):
        time_oracle_numeric(prob, h)
    ts = [time_oracle_numeric(prob, h) for _ in range(a.steps)]
    t = sum(ts) / len(ts)
    fl = h.flops
    v = fl / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GFLOP/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "sample": f"the full {a.side}^3 workload, IC({a.k})"},
            "cpu_baseline": {"value": v, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": f"one oracle numeric IC({a.k}) of the full {a.side}^3 27-point "
                                       f"problem per step ({fl:.4g} flops)"},
            "e2e": {"value": v, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SHIFT_NU_TRAIN = (0.40, 0.44, 0.46, 0.47, 0.475, 0.48, 0.485, 0.49, 0.493, 0.496, 0.499)
SHIFT_NU_TEST = (0.4725, 0.4875, 0.4965)
SHIFT_ALPHAS = [0.0] + [1e-3 * 2 ** j for j in range(13)]
SHIFT_NE_TRAIN = (6, 8, 12, 16, 24)


def shift_workload(a, steps):
    """Q1 hex elasticity (ne^3 elements, clamped face, IC(0), geometric ND): time to a
    relative residual of 1e-8, all factorization attempts included, for the plain FP64
    form (FP64 factor, shift 0 then 1e-3 doubling) and the FP32 + learned-shift form
    (FP32 factor with FP64 pivots, first shift from the network trained on shift
    sweeps of 6^3 to 24^3 meshes, doubling as the fallback).  Poisson ratios of the
    timed instances are held out of training."""
    import torch
    import synth
    import paper_1601_05871_gb300 as ick
    from paper_1601_05871_gb300 import shift_train as T
    from paper_1601_05871_gb300.build import build

    build()
    ick.load()
    t0 = time.perf_counter()
    X, y = [], []
    for ne in SHIFT_NE_TRAIN:
        for nu in SHIFT_NU_TRAIN:
            p = synth.elasticity3d_q1(ne, nu=nu)
            perm, ranges = ick.ic_nd_grid(*p.grid, 3, 256, p.keep)
            h = ick.ic_symbolic(p.rowptr, p.colind, 0, perm, ranges, block_rows=256, dtype=ick.IC_F32,
                               warps_per_cta=a.warps)
            av = torch.from_numpy(p.vals).cuda()
            b = torch.from_numpy(synth.rhs(p.n, 11)).cuda()
            x = torch.empty_like(b)
            X.append(ick.ic_shift_features(h, av, nu))
            y.append(T.label(T.sweep(h, av, b, x, SHIFT_ALPHAS)))
    mlp, loss = T.train(np.array(X), np.array(y), steps=1500, lr=1e-2, seed=1)
    train_s = time.perf_counter() - t0
    rows = []
    for nu in SHIFT_NU_TEST:
        p = synth.elasticity3d_q1(a.ne, nu=nu)
        perm, ranges = ick.ic_nd_grid(*p.grid, 3, 4096, p.keep)
        av = torch.from_numpy(p.vals).cuda()
        b = torch.from_numpy(synth.rhs(p.n, 13)).cuda()
        x = torch.empty_like(b)
        res = {}
        for name, dtype, model in (("fp64_plain", ick.IC_F64, None), ("fp32_learned", ick.IC_F32, mlp)):
            h = ick.ic_symbolic(p.rowptr, p.colind, 0, perm, ranges, block_rows=4096, dtype=dtype,
                               warps_per_cta=a.warps)
            T.solve(h, av, b, x, mlp=model, nu=nu)  # warm-up
            runs = [T.solve(h, av, b, x, mlp=model, nu=nu) for _ in range(max(1, steps))]
            r = min(runs, key=lambda q: q["seconds"])
            xh = x.cpu().numpy()
            r["true_relres"] = float(np.linalg.norm(p.scipy() @ xh - synth.rhs(p.n, 13)) /
                                     np.linalg.norm(synth.rhs(p.n, 13)))
            r["ms"] = r.pop("seconds") * 1e3
            res[name] = r
            del h
        rows.append({"nu": nu, "n": p.n, "nnz": int(p.rowptr[-1]), **res,
                     "speedup": res["fp64_plain"]["ms"] / res["fp32_learned"]["ms"]})
    tot64 = sum(r["fp64_plain"]["ms"] for r in rows)
    tot32 = sum(r["fp32_learned"]["ms"] for r in rows)
    line = {"metric": "elasticity IC(0) time to PCG relres 1e-8, FP32 + learned shift vs plain FP64",
            "value": tot64 / tot32, "unit": "x (plain FP64 time / FP32 learned-shift time)", "n_gpus": 1,
            "steps": steps, "warmup": 1, "higher_is_better": True, "dtype": "f32 factor, f64 PCG",
            "data": "synthetic",
            "config": {"workload": f"Q1 hex elasticity {a.ne}^3 elements (clamped face, 3 dof/node), E = 1, "
                                   f"held-out nu {list(SHIFT_NU_TEST)}, geometric ND, IC(0), b ~ N(0,1)",
                       "training": f"shift sweeps of {list(SHIFT_NE_TRAIN)}^3-element meshes, "
                                   f"nu {list(SHIFT_NU_TRAIN)}",
                       "train_seconds": train_s, "train_loss": loss},
            "instances": rows, "total_ms_fp64_plain": tot64, "total_ms_fp32_learned": tot32}
    return line


def c3_workload(a, warmup, steps):
    """512 independent 7-point diffusion cubes of side U{8..32} (kappa ~ LogNormal(0, 1)),
    IC(1), FP32 factors with FP64 pivots, all factored by one persistent launch, then
    batched FP64 PCG to 1e-8 (one captured CUDA graph iteration replayed).  Each step:
    the numeric phase of all systems + the batched solve."""
    import torch
    import synth
    import paper_1601_05871_gb300 as ick
    from paper_1601_05871_gb300.build import build

    build()
    ick.load()
    probs = synth.config_problem(3)
    nd = [ick.ic_nd_grid(*p.grid, 1, 4096) for p in probs]
    pats = [(p.rowptr, p.colind) for p in probs]
    h = ick.ic_symbolic_batch(pats, 1, [x[0] for x in nd], [x[1] for x in nd], dtype=ick.IC_F32, block_rows=4096,
                              warps_per_cta=a.warps)
    st = ick.ic_stats(h)
    vals = torch.from_numpy(np.concatenate([p.vals for p in probs])).cuda()
    b_host = np.concatenate([synth.rhs(p.n, 3000 + s) for s, p in enumerate(probs)])
    b = torch.from_numpy(b_host).cuda()
    x = torch.empty_like(b)
    ick.ic_set_timing(h, True)
    for _ in range(warmup):
        ick.ic_numeric(h, vals)
        ick.pcg_solve_batch(h, vals, b, x, 1e-8, 1000)
    torch.cuda.synchronize()
    fact, tts = [], []
    its = rels = None
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ick.ic_numeric(h, vals)
        t = ick.ic_get_timing(h)
        its, rels = ick.pcg_solve_batch(h, vals, b, x, 1e-8, 1000)
        e1.record()
        torch.cuda.synchronize()
        fact.append(t["prepare_ms"] + t["numeric_ms"])
        tts.append(e0.elapsed_time(e1))
    mf = statistics.median(fact)
    line = {"metric": "batched IC(1) factor GFLOP/s and time to 1e-8 of 512 systems (one launch)",
            "value": st["flops"] / (mf * 1e-3) / 1e9, "unit": "GFLOP/s", "n_gpus": 1, "steps": steps,
            "warmup": warmup, "higher_is_better": True, "dtype": "f32 factor, f64 PCG", "data": "synthetic",
            "config": {"workload": "512 7-point diffusion cubes, side U{8..32}, kappa ~ LogNormal(0, 1), "
                                   "geometric ND, IC(1), one persistent launch",
                       "systems": len(probs), "n": st["n"], "nnz_l": st["nnz_l"], "tasks": st["ntasks"],
                       "flops": st["flops"]},
            "factor_ms": mf, "time_to_solution_ms": statistics.median(tts),
            "pcg_iters_min": int(its.min()), "pcg_iters_max": int(its.max()), "max_relres": float(rels.max())}
    return line


def c5_workload(a, side, warmup, steps, densities=True):
    """7-point variable-coefficient diffusion (kappa ~ LogNormal(0, 2), z faces x100),
    geometric ND, 2D blocks <= 4096 rows, IC(3): FP32 factor + FP64 PCG to 1e-8, with
    the FP64 form beside it.  Reports the largest block density of the factor (the
    dense-block tensor-core path applies only to dense blocks)."""
    import torch
    import synth
    import paper_1601_05871_gb300 as ick
    from paper_1601_05871_gb300.build import build

    build()
    ick.load()
    p = synth.config_problem(5, scale=side)
    perm, ranges = ick.ic_nd_grid(side, side, side, 1, a.block_rows)
    av = torch.from_numpy(p.vals).cuda()
    b_host = synth.rhs(p.n, 5000)
    b = torch.from_numpy(b_host).cuda()
    x = torch.empty_like(b)
    out = {}
    st = None
    for name, dtype in (("fp32", ick.IC_F32), ("fp64", ick.IC_F64)):
        h = ick.ic_symbolic(p.rowptr, p.colind, 3, perm, ranges, block_rows=a.block_rows, dtype=dtype,
                            warps_per_cta=a.warps)
        st = ick.ic_stats(h)
        for _ in range(warmup):
            timed_solve(ick, torch, h, av, b, x, 1e-8)
        torch.cuda.synchronize()
        tts, its = [], 0
        for _ in range(steps):
            ev, its, rel = timed_solve(ick, torch, h, av, b, x, 1e-8)
            torch.cuda.synchronize()
            tts.append(ev[0].elapsed_time(ev[2]))
        true_rel = float(np.linalg.norm(p.scipy() @ x.cpu().numpy() - b_host) / np.linalg.norm(b_host))
        mf = factor_kernel_ms(ick, h, av)
        out[name] = {"factor_ms": mf, "factor_gflops": st["flops"] / (mf * 1e-3) / 1e9,
                     "time_to_solution_ms": statistics.median(tts), "pcg_iters": int(its), "relres": float(rel),
                     "true_relres": true_rel}
        del h
    line = {"metric": "IC(3) FP32 factor + FP64 PCG time to 1e-8 (7-point diffusion)",
            "value": out["fp32"]["time_to_solution_ms"], "unit": "ms", "n_gpus": 1, "steps": steps,
            "warmup": warmup, "higher_is_better": False, "dtype": "f32 factor, f64 PCG", "data": "synthetic",
            "config": {"workload": f"7-point diffusion {side}^3, kappa ~ LogNormal(0, 2), z faces x100, "
                                   f"geometric ND, 2D blocks <= {a.block_rows} rows, IC(3)",
                       "n": st["n"], "nnz_a": st["nnz_a"], "nnz_l": st["nnz_l"], "blocks": st["nblocks"],
                       "tasks": st["ntasks"], "flops": st["flops"]},
            **out,
            "speedup_fp32_vs_fp64": out["fp64"]["time_to_solution_ms"] / out["fp32"]["time_to_solution_ms"]}
    if not densities:
        return line
    # largest block density: entries of each (row range, column range) block over its area
    hh = ick.ic_symbolic(p.rowptr, p.colind, 3, perm, ranges, block_rows=a.block_rows, host_only=1)
    urp, ucol, _, _, _ = ick.ic_get_upper(hh)
    rg, _, _ = ick.ic_get_blocks(hh)
    blk = np.searchsorted(rg, np.arange(p.n), side="right") - 1
    rows = np.repeat(np.arange(p.n), np.diff(urp))
    nb = len(rg) - 1
    cnt = np.bincount(blk[rows].astype(np.int64) * nb + blk[ucol], minlength=nb * nb).reshape(nb, nb)
    sz = np.diff(rg).astype(np.float64)
    area = np.outer(sz, sz)
    area[np.diag_indices(nb)] = sz * (sz + 1) / 2
    dens = np.where(cnt > 0, cnt / area, 0.0)
    line["max_block_density"] = float(dens.max())
    line["blocks_denser_than_5pct"] = int((dens >= 0.05).sum())
    return line


def main():
    a = parse()
    if a.shift:
        print(json.dumps(shift_workload(a, a.steps)), flush=True)
        return
    if a.c5:
        print(json.dumps(c5_workload(a, a.side if a.side != 96 else 160, a.warmup, a.steps)), flush=True)
        return
    if a.c3:
        print(json.dumps(c3_workload(a, a.warmup, a.steps)), flush=True)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if a.impl == "reference":
        reference_arm(a, rank, world)
        return

    import torch
    import torch.distributed as dist
    import synth
    import paper_1601_05871_gb300 as ick
    from paper_1601_05871_gb300.build import build

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    ick.load()

    prob = synth.laplace3d_27pt(a.side)
    perm, ranges = ick.ic_nd_grid(a.side, a.side, a.side, 1, a.leaf_rows, sep_colours=a.sep_colours,
                                  leaf_colours=a.leaf_colours)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, a.k, perm, ranges, block_rows=a.block_rows,
                        warps_per_cta=a.warps, solve_mode=a.solve_mode, solve_lanes=a.solve_lanes,
                        solve_ctas_per_sm=a.solve_ctas)
    st = ick.ic_stats(h)
    # the library's per-kernel timing stays off in the timed steps, so that pcg_solve runs
    # as one graph; the kernels are timed afterwards, in a pass of their own
    ick.ic_set_timing(h, a.pcg_host_loop)
    stream = torch.cuda.current_stream()
    av = torch.from_numpy(prob.vals).cuda()
    b_host = synth.rhs(prob.n, 2000 + rank)
    b = torch.from_numpy(b_host).cuda()
    x = torch.empty(prob.n, dtype=torch.float64, device="cuda")

    def step():
        if a.numeric_only:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            ick.ic_numeric_async(h, av, stream)
            ev[1].record(stream)
            stream.synchronize()
            ick.ic_numeric_status(h)
            return ev, 0, 0.0
        return timed_solve(ick, torch, h, av, b, x, a.tol, stream)

    if a.numeric_only:
        a.no_e2e = True
        a.no_cpu_baseline = True

    # arithmetic roofs of the numeric phase, measured on this GPU by the library's FMA
    # throughput kernel (before the timed region)
    try:
        fp64_peak, fp64_src = ick.ic_fma_peak(ick.IC_F64), "measured (ic_fma_peak, FP64 FMA chains)"
        fp32_peak = ick.ic_fma_peak(ick.IC_F32)
    except ick.IckError:
        fp64_peak, fp64_src, fp32_peak = FP64_NOMINAL_GFLOPS, "nominal GB300 FP64 rate", None

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    ick.ic_reset_timing(h)
    fevs, iters, rels = [], [], []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(a.steps):
            ev, it, rel = step()
            fevs.append(ev)
            iters.append(it)
            rels.append(rel)
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    total_ms = ev0.elapsed_time(ev1)
    launches = ick.ic_get_timing(h)["launches"]  # kernels of the timed steps
    clocks = clk.summary()
    # the factorization phase of a step as the timed steps saw it (scatter, task kernel
    # and the solves' operand copies of the factor)
    phase_ms = [e[0].elapsed_time(e[1]) for e in fevs]
    mean_phase = sum(phase_ms) / len(phase_ms)
    # per-kernel times: a few more steps with the library's CUDA events around every
    # kernel (PCG then loops on the host, one synchronisation per iteration); the
    # factor time of value is the scatter plus the task kernel
    ks = 3
    ick.ic_set_timing(h, True)
    ick.ic_reset_timing(h)
    fact_ms, kern = [], []
    for _ in range(ks):
        ick.ic_numeric(h, av, stream)
        tm = ick.ic_get_timing(h)
        fact_ms.append(tm["prepare_ms"] + tm["numeric_ms"])
        kern.append(tm["numeric_ms"])
        if not a.numeric_only:
            ick.pcg_solve(h, av, b, x, a.tol, 5000, stream)
    torch.cuda.synchronize()
    tim = ick.ic_get_timing(h)
    ick.ic_set_timing(h, False)
    mean_fact = sum(fact_ms) / len(fact_ms)
    total_ms, mean_fact, mean_phase = max_over_ranks([total_ms, mean_fact, mean_phase], world)
    ms_per_step = total_ms / a.steps
    value = job_rate(st["flops"], world, mean_fact * 1e-3) / 1e9
    hbm = job_rate(st["bytes"], world, mean_fact * 1e-3) / 1e9
    apply_ms_step = tim["apply_ms"] / ks
    mean_kern = sum(kern) / len(kern)

    # true residual of the last solve, in FP64 on the host
    xh = x.cpu().numpy()
    true_rel = (float(np.linalg.norm(prob.scipy() @ xh - b_host) / np.linalg.norm(b_host))
                if not a.numeric_only else None)

    # dominant kernel by measured share of the step: numeric task kernel vs triangular solves
    peak_hbm = 6783.5
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        peak_hbm = float(peaks.get("hbm_gbs", peak_hbm))
        peak_src = "measured"
    except Exception:
        peak_src = "fallback"
    n, nnz_l = st["n"], st["nnz_l"]
    # one solve launch reads every factor entry once (8-byte value + 4-byte index) and
    # four row vectors (row pointer, right-hand side, reciprocal diagonal, result)
    solve_bytes = nnz_l * 12 + n * 8 * 4
    # the FP64 factor's arithmetic floor (flops / FP64 peak) lies above its HBM floor
    # (compulsory bytes / bandwidth), so the FP64 FMA rate is its roof; the FP32 factor
    # takes the same time, so what limits the kernel is instruction issue while every
    # CTA is busy and the dependence chain of the top separators at the end
    captured = a.leaf_rows == a.block_rows and a.sep_colours == CAPTURED_SEP_COLOURS and a.leaf_colours < 2
    traffic_entry = NUMERIC_TRAFFIC_PER_ENTRY.get(a.k) if captured else None
    roof_numeric = {"kernel": "numeric_persistent (+ numeric_prepare scatter)",
                    "bound": "alu", "achieved": st["flops"] / (mean_fact * 1e-3) / 1e9,
                    "peak": fp64_peak, "unit": "GFLOP/s", "peak_source": fp64_src,
                    "fp32_fma_peak_gflops": fp32_peak,
                    "limiter": "instruction issue while all CTAs are busy, then the top separators' "
                               "dependence chain (the FP32 factor takes as long)",
                    "hbm_achieved_gbs": st["bytes"] / (mean_fact * 1e-3) / 1e9,
                    "hbm_peak_gbs": peak_hbm, "algorithmic_bytes": st["bytes"],
                    "traffic": traffic_entry * nnz_l if traffic_entry else None}
    roof_numeric["frac"] = roof_numeric["achieved"] / roof_numeric["peak"]
    calls = max(1, tim["apply_calls"])
    roofs = {"numeric": (mean_fact, roof_numeric)}
    names = {0: ("forward_dag", "backward_dag"), 1: ("forward_solve_v", "backward_solve_v")}[a.solve_mode]
    for name, key in zip(names, ("fwd_ms", "bwd_ms")):
        per = tim[key] / calls
        r = {"kernel": name, "bound": "hbm",
             "achieved": solve_bytes / (per * 1e-3) / 1e9 if per > 0 else 0.0,
             "peak": peak_hbm, "unit": "GB/s", "peak_source": peak_src,
             "launch_ms": per, "algorithmic_bytes": solve_bytes,
             "traffic": (SOLVE_TRAFFIC_PER_ENTRY[(a.k, name)] * nnz_l
                         if captured and (a.k, name) in SOLVE_TRAFFIC_PER_ENTRY else None)}
        r["frac"] = r["achieved"] / r["peak"]
        roofs[name] = (tim[key] / ks, r)
    dominant = max(roofs.values(), key=lambda v: v[0])[1]
    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "n": n, "nnz_a": st["nnz_a"], "nnz_l": nnz_l,
                       "k": a.k, "block_rows": a.block_rows, "ranges": st["nranges"],
                       "blocks": st["nblocks"], "tasks": st["ntasks"], "items": st["nitems"],
                       "critical_path_tasks": st["critical_path"], "warps_per_cta": st["warps_per_cta"],
                       "grid_ctas": st["grid_ctas"], "flops": st["flops"], "bytes": st["bytes"],
                       "l2": "inputs larger than L2 (factor values alone 8*nnz(L) bytes)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "hbm_gbs": hbm, "factor_ms": mean_fact, "numeric_kernel_ms": mean_kern,
            "factor_phase_ms": mean_phase,
            "pcg": {"iters": iters[-1], "relres": rels[-1], "true_relres": true_rel,
                    "tol": a.tol, "apply_ms_per_step": apply_ms_step,
                    "time_to_solution_ms": ms_per_step},
            "roofline": dominant, "roofline_numeric": roof_numeric,
            "roofline_solves": [roofs[names[0]][1], roofs[names[1]][1]],
            "ms_per_step_by_kernel": {k: v[0] for k, v in roofs.items()},
            "gpu_launches": int(launches), "clocks": clocks}

    if not a.no_e2e:
        ab = torch.from_numpy(prob.vals).pin_memory()
        bb = torch.from_numpy(b_host).pin_memory()
        xb = torch.empty(prob.n, dtype=torch.float64).pin_memory()
        av2 = torch.empty_like(av)
        b2 = torch.empty_like(b)

        def e2e_step():
            av2.copy_(ab, non_blocking=True)
            b2.copy_(bb, non_blocking=True)
            ick.ic_numeric(h, av2, stream)
            ick.pcg_solve(h, av2, b2, x, a.tol, 5000, stream)
            xb.copy_(x, non_blocking=True)
            stream.synchronize()

        for _ in range(a.warmup):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            e2e_step()
        t_e2e = (time.perf_counter() - t0) / a.steps
        t_e2e = max_over_ranks([t_e2e], world)[0]
        line["e2e"] = {"value": job_rate(st["flops"], world, t_e2e) / 1e9, "unit": "GFLOP/s",
                       "h2d_bytes_per_step": int(prob.vals.nbytes + b_host.nbytes),
                       "d2h_bytes_per_step": int(xh.nbytes), "ms_per_step": t_e2e * 1e3,
                       "note": "factor flops / end-to-end step time (copies + factor + PCG)"}

    # mixed precision arm: FP32 factor values and solves, FP64 pivots and PCG, same
    # workload, timed the same way; the plain FP64 arm above is its comparison
    h32 = None
    if not a.numeric_only and not a.no_f32:
        h32 = ick.ic_symbolic(prob.rowptr, prob.colind, a.k, perm, ranges, block_rows=a.block_rows,
                              warps_per_cta=a.warps, dtype=ick.IC_F32, solve_mode=a.solve_mode,
                              solve_lanes=a.solve_lanes, solve_ctas_per_sm=a.solve_ctas)
        x32 = torch.empty_like(x)
        for _ in range(a.warmup):
            timed_solve(ick, torch, h32, av, b, x32, a.tol, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f32_evs, f32_it, f32_rel = [], 0, 0.0
        e0.record(stream)
        for _ in range(a.steps):
            ev, f32_it, f32_rel = timed_solve(ick, torch, h32, av, b, x32, a.tol, stream)
            f32_evs.append(ev)
        e1.record(stream)
        torch.cuda.synchronize()
        t32 = e0.elapsed_time(e1) / a.steps
        f32_fact = [factor_kernel_ms(ick, h32, av, stream)]
        f32_true = float(np.linalg.norm(prob.scipy() @ x32.cpu().numpy() - b_host) / np.linalg.norm(b_host))
        mf32 = sum(f32_fact) / len(f32_fact)
        line["mixed_f32"] = {"factor_ms": mf32, "factor_gflops": st["flops"] / (mf32 * 1e-3) / 1e9,
                             "pcg_iters": f32_it, "relres": f32_rel, "true_relres": f32_true,
                             "time_to_solution_ms": t32,
                             "speedup_vs_f64_time_to_solution": ms_per_step / t32}

    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        import oracle
        operm, _ = oracle.nd_grid(a.side, a.side, a.side, 1, a.leaf_rows, sep_colours=a.sep_colours,
                                  leaf_colours=a.leaf_colours)
        if not np.array_equal(operm, perm):
            raise RuntimeError("the library's nested-dissection order differs from the oracle's")
        o = oracle.OracleIC.from_problem(prob, operm, a.k)
        t0 = time.perf_counter()
        assert o.numeric(prob.vals) == 0
        t = time.perf_counter() - t0
        fl = o.flops
        line["cpu_baseline"] = {"value": fl / t / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                                "sample": f"one oracle numeric IC({a.k}) of the full {a.side}^3 "
                                          f"workload ({t:.1f} s)"}
        # error of each GPU factor against the FP64 oracle on the full workload
        ref = o.values()
        amax = float(np.abs(prob.vals).max())
        orp, oci, _ = o.pattern()
        parity = {}
        for name, hh in (("f64", h), ("f32", h32)):
            if hh is None:
                continue
            rp, ci, lv, _ = ick.ic_get_factor(hh)
            parity[name] = {"pattern_equal": bool(np.array_equal(rp, orp) and np.array_equal(ci, oci)),
                            "max_abs_err_over_max_A": float(np.abs(lv - ref).max() / amax)}
        line["parity_vs_oracle"] = parity

    # the method's other workloads, outside the timed region, a few fixed repetitions
    # each (one GPU only: the replicas of a multi-GPU run measure the default workload)
    if world == 1 and not a.no_sub and not a.numeric_only:
        del h, h32
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        for key, run in (("c4_shift", lambda: shift_workload(a, steps=1)),
                         ("c3_batch", lambda: c3_workload(a, warmup=2, steps=3)),
                         ("c5", lambda: c5_workload(a, 160, warmup=1, steps=2, densities=False))):
            try:
                line[key] = run()
            except Exception as e:  # the default workload's line is still printed
                line[key] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()
        line["sub_workloads_wall_s"] = time.perf_counter() - t0
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
