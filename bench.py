"""Benchmark: cell-stage updates per second of the SSP-RK3 FVCW solver on the
2-D corner-blast workload at 4096^2 (FP32 line arithmetic with FP64 state
accumulation, with the plain FP64 form measured beside it).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

One JSON line on stdout (rank 0).  N > 1 (torchrun, one process per GPU) runs
N independent replicas of the workload (the grid is not split across GPUs):
value = the cell-stages of all ranks / the slowest rank's time.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-stage updates/s at 2D 4096^2, FP32 form vs FP64 plain, at stated L1 error"
UNIT = "cell-stage/s"
N_GRID = 4096


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            self.tmp.flush()
            rows = [r.split(",") for r in open(self.tmp.name).read().strip().splitlines()]
            os.unlink(self.tmp.name)
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def _json_default(o):
    """numpy scalars (counts and sums of per-problem arrays) as plain numbers"""
    if hasattr(o, "item"):
        return o.item()
    raise TypeError(f"not JSON serialisable: {type(o).__name__}")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _init_dist(ws: int, local: int):
    """One process per GPU under torchrun: NCCL when CUDA is present, else
    gloo (the host-side logic of the replica path runs on CPU that way)."""
    if ws == 1:
        return
    import torch
    import torch.distributed as dist
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist.init_process_group("gloo")


def _close_dist(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _barrier_max(x: float, ws: int) -> float:
    """Max of a per-rank scalar over the ranks (the slowest replica's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_value(ws: int, ncell: int, steps: int, ms_max: float) -> float:
    """Whole-job throughput of N independent replicas: the cell-stages of all
    ranks over the slowest rank's time (three stages per SSP-RK3 step)."""
    return ws * ncell * 3 * steps / (ms_max * 1e-3)


# Per-kernel algorithmic bytes per cell of a 2-D stage (4 conserved
# variables; a state value is 8 B: FP64, or an FP32 hi + lo pair).
# Plain form (2 sweeps per stage):
#   x sweep  reads U_k, writes D_x (8 B / variable)                   64 B
#   y sweep  reads U_k and D_x, U^n in stages 2-3 (2/3 on average),
#            writes U_{k+1}                                          117.3 B
# Mixed form (3 kernels per stage):
#   x sweep  reads the FP32 hi parts of U_k, writes D_x (FP32)        32 B
#   y sweep  reads the transposed hi parts, writes D_y transposed     32 B
#   combine  reads U_k, U^n (2/3), D_x, D_y; writes U_{k+1} and its
#            transposed hi and lo parts                              149.3 B
KERNEL_BYTES = {
    0: [("x_sweep", 64.0), ("y_sweep", 32 + 32 + 32 * 2.0 / 3.0 + 32)],
    1: [("x_sweep", 32.0), ("y_sweep_transposed", 32.0),
        ("stage_combine", 32 + 32 * 2.0 / 3.0 + 16 + 16 + 32 + 32)],
}

# Algorithmic arithmetic per cell of one line sweep (2-D, 4 variables),
# counted on the scheme's formulas as the FP64 oracle writes them (+, -, *,
# /, sqrt, |.|, min, max one operation each):
#   per variable  smoothness indicators 33, WENO-Z weights of both sides 44,
#                 rows of both compact systems 42, Thomas elimination and
#                 back substitution of both systems 16                  135
#   per cell      limiter (the unlimited path) 121, HLLC at one face 118,
#                 flux difference 8                                     247
#   x sweep, transposed y sweep: 4 x 135 + 247 = 787; the FP64 y sweep adds
#   the SSP-RK3 stage combination (20) and the admissibility check (15): 822.
# The stage combination of the mixed form is a stream (bound by HBM).
KERNEL_FLOPS = {
    0: {"x_sweep": 787.0, "y_sweep": 822.0},
    1: {"x_sweep": 787.0, "y_sweep_transposed": 787.0},
}
# ALU peaks from unit counts and clocks: FP32 152 SMs x 128 lanes x 2 flop x
# 2.07 GHz; FP64 the GB300 nominal 1.25 TFLOP/s.
ALU_PEAK_TFLOPS = {1: 152 * 128 * 2 * 2.07e9 / 1e12, 0: 1.25}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per cell of the
# dominant kernel, from one ncu capture, valid only for the kernel sources it
# was taken on (their SHA-256 below); any change to them voids it.
# Captured on the 3072^2 blast (`bench.py --profile-only mixed|fp64 --n 3072`,
# the first x sweep of the first step, `-s 6 -c 1` past the autotuner's
# trials): reads are the algorithmic bytes of a plain-form line (the blast's
# lines are flat to FP32 precision at that step); writes fall short of them by
# what is still dirty in L2 when the kernel ends.  The FP64 form's dominant
# kernel is its y sweep, for which no capture of these sources exists.
TRAFFIC_PER_CELL = {            # {(precision, kernel): bytes per cell}
    (1, "x_sweep"): 28.33,
    (0, "x_sweep"): 59.64,
}
TRAFFIC_SRC_SHA256 = "125b6e168b43838d09caa6c191c5d38175b8c94383bd35a6e8e9d3d6b2b84e5a"
KERNEL_SOURCES = ("line_sweep.cuh", "physics.cuh", "dfloat.cuh", "batch_lines.cuh")


def _kernel_src_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1402_5618_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def run_native(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_1402_5618_gb300 import binding as B
    from paper_1402_5618_gb300 import workloads as W

    torch.cuda.set_device(local)
    B.lib()
    p = W.blast_2d(N_GRID)
    U0 = np.ascontiguousarray(p.U0).ravel()
    ncell = p.nx * p.ny
    stream = torch.cuda.Stream()
    results = {}
    for prec, steps in ((1, args.steps), (0, args.fp64_steps)):
        s = B.Solver(B.config_from_problem(p, prec, cfl_positivity_cap=True), stream=stream)
        s.set_state(U0)
        s.enqueue_steps(args.warmup)
        torch.cuda.synchronize()
        # per-kernel durations with CUDA events on the solver's stream
        prof = [s.profile_step() for _ in range(args.profile_steps)]
        torch.cuda.synchronize()
        launches = s.launches_per_step()
        m_rows = s.rows_per_chunk()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st0 = s.stats()
        _barrier(ws)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            ev0.record(stream)
            s.enqueue_steps(steps)
            ev1.record(stream)
            torch.cuda.synchronize()
        _barrier(ws)
        ms = ev0.elapsed_time(ev1)
        st = s.stats()
        if prec == 0:   # the FP64 state and time, for the blast's stated accuracy
            U64, t64, _ = s.get_state()
        # throughput counts accepted steps only: a step redone by the face
        # check of eq. (CFL-CD) is work that does not advance the solution
        accepted = int(st.steps - st0.steps)
        results[prec] = dict(ms=ms, steps=accepted, attempts=steps, prof=prof, launches=launches,
                             clk=clk.summary(), rows_per_chunk=m_rows,
                             rejected=int(st.rejected - st0.rejected),
                             violations=st.violations, t=st.t, theta2=st.theta2_active)
        s.close()

    # the characteristic-wise form (Sec. 2.3) on the same workload at CFL
    # omega_1/2 (its positivity bound on the near-vacuum cases), in both
    # arithmetics: ms per step and the split between the reconstruction
    # kernel and the line kernel from CUDA events on the solver's stream
    charf = {}
    if args.characteristic:
        for prec, pname, steps in ((1, "mixed", args.char_steps), (0, "fp64", args.char_fp64_steps)):
            cfg = B.config_from_problem(p, prec, recon=B.RECON_CHARACTERISTIC)
            cfg.cfl = 1.0 / 24.0
            s = B.Solver(cfg, stream=stream)
            s.set_state(U0)
            s.enqueue_steps(2)
            torch.cuda.synchronize()
            prof = s.profile_step()
            torch.cuda.synchronize()
            ev0.record(stream)
            s.enqueue_steps(steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            st = s.stats()
            launches = s.launches_per_step()
            s.close()
            names = (["char_rows_x", "char_solve_x", "x_sweep", "char_rows_y", "char_solve_y",
                      "y_sweep_transposed", "stage_combine"] if prec == 1 else
                     ["char_rows_x", "char_solve_x", "x_sweep", "char_rows_y", "char_solve_y", "y_sweep"])
            per = prof[1:]           # prof[0]: the per-step dt kernel
            kms = {nm: sum(per[i::len(names)]) / max(1, len(per[i::len(names)]))
                   for i, nm in enumerate(names)}
            charf[pname] = {"value": ncell * 3 * steps / (ms * 1e-3), "unit": UNIT,
                            "steps": steps, "ms_per_step": ms / steps,
                            "kernel_ms": {k: round(v, 4) for k, v in kms.items()},
                            "gpu_launches_per_step": int(launches),
                            "violations": int(st.violations)}

    # end-to-end through the public API with host buffers: H2D initial state,
    # K steps, D2H final state, inside one wall-clock region
    s = B.Solver(B.config_from_problem(p, 1, cfl_positivity_cap=True), stream=stream)
    Uh = np.empty_like(U0)
    s.set_state(U0)
    s.enqueue_steps(args.warmup)
    torch.cuda.synchronize()
    _barrier(ws)
    t0 = time.perf_counter()
    s.set_state(U0)
    s.enqueue_steps(args.steps)
    s.get_state(Uh)
    e2e_s = time.perf_counter() - t0
    e2e_steps = int(s.stats().steps)   # accepted steps of the K enqueued
    s.close()

    # stated accuracy, measured live: (i) the blast itself, the mixed form
    # run from the same initial state to the FP64 run's final time, relative
    # L1 per variable against the FP64 state; (ii) smooth data, the
    # isentropic vortex on 1024^2 to t = 1 in both forms against its closed
    # form (one period on 2048^2, the 2048^2 configuration, is in the
    # --accuracy study: minutes of FP64)
    acc = {}
    sm = B.Solver(B.config_from_problem(p, 1, cfl_positivity_cap=True), stream=stream)
    sm.set_state(U0)
    sm.advance(t64, 10 ** 6, check=False)
    Um, tm, _ = sm.get_state()
    sm.close()
    Um, Ud = Um.reshape(p.U0.shape), U64.reshape(p.U0.shape)
    acc["blast_rel_l1"] = [float(np.abs(Um[v] - Ud[v]).sum() / np.abs(Ud[v]).sum()) for v in range(4)]
    acc["blast_t"] = float(t64)
    nv = args.accuracy_n
    pv = W.vortex_2d(nv, t_final=1.0)
    ex = W.vortex_2d(nv, t=1.0).U0[0]
    for prec in (0, 1):
        sv = B.Solver(B.config_from_problem(pv, prec), stream=stream)
        sv.set_state(np.ascontiguousarray(pv.U0).ravel())
        sv.advance(pv.t_final)
        Uv = sv.get_state()[0].reshape(pv.U0.shape)
        sv.close()
        acc[prec] = float(np.mean(np.abs(Uv[0] - ex)))

    batches = {}
    if args.batches:
        # the whole seeded 1-D set (the 168 problems whose exact solution
        # opens a vacuum included) and the 2-D four-quadrant set, at the
        # positivity CFL with eq. (CFL-CD) checked on the face values
        # (the 1-D set also in the characteristic-wise form: its data are
        # all discontinuous)
        rb = W.riemann_batch()
        for name, probs, steps, recon in (("riemann_1d", rb, (20, 20), 0),
                                          ("quadrant_2d", W.quadrant_batch(), (6, 6), 0),
                                          ("riemann_1d_characteristic", rb, (10, 3), 1)):
            U0b = np.concatenate([np.ascontiguousarray(q.U0).ravel() for q in probs])
            cells = np.array([q.nx * q.ny for q in probs], dtype=np.float64)
            row = {"problems": len(probs), "cells": int(cells.sum())}
            for prec, pname, steps in ((1, "mixed", steps[0]), (0, "fp64", steps[1])):
                sb = B.Solver(None, batch=[B.config_from_problem(q, prec, cfl_positivity_cap=True,
                                                                 recon=recon)
                                           for q in probs], stream=stream)
                sb.set_state(U0b)
                sb.enqueue_steps(3)
                torch.cuda.synchronize()
                k0 = np.array([sb.problem_stats(k).steps for k in range(len(probs))])
                ev0.record(stream)
                sb.enqueue_steps(steps)
                ev1.record(stream)
                torch.cuda.synchronize()
                ms = ev0.elapsed_time(ev1)
                per = [sb.problem_stats(k) for k in range(len(probs))]
                stb = sb.stats()
                sb.close()
                taken = np.array([ps.steps for ps in per]) - k0
                row[pname] = {"value": float((cells * 3 * taken).sum() / (ms * 1e-3)), "unit": UNIT,
                              "steps": steps, "ms_per_step": ms / steps,
                              "accepted_step_fraction": float(taken.sum() / (steps * len(probs))),
                              "redone_steps": int(stb.rejected),
                              "violations": int(stb.violations),
                              "problems_outside_G": int(sum(1 for ps in per if ps.violations))}
            batches[name] = row

    return dict(results=results, ncell=ncell, e2e_s=e2e_s, e2e_steps=e2e_steps, acc=acc,
                state_bytes=U0.nbytes, batches=batches, characteristic=charf)


def _roofline(r, prec, ncell, hbm_peak, peak_kind):
    """Roofline of the kernel with the largest share of the step time: its
    algorithmic work per launch over its mean CUDA-event duration (the line
    sweeps against the ALU peak of their precision, the stage combination
    against HBM), with the HBM view of every kernel beside it."""
    import numpy as np
    prof = np.array(r["prof"])          # [steps, launches]: dt kernel, then per stage
    kinds = KERNEL_BYTES[prec]
    # then (checked steps) the commit copy, the transposed-plane restore of
    # the mixed form and the step-end bookkeeping
    per = prof[:, 1:1 + 3 * len(kinds)].reshape(prof.shape[0], 3, len(kinds))
    tot = per.sum(axis=(0, 1))
    table = {}
    for i, (name, per_cell) in enumerate(kinds):
        t_ms = float(per[:, :, i].mean())
        gbs = per_cell * ncell / (t_ms * 1e-3) / 1e9
        row = {"avg_launch_ms": round(t_ms, 4), "share": round(float(tot[i] / prof.sum()), 3),
               "alg_bytes_per_cell": round(per_cell, 1), "hbm_gbs": round(gbs, 1),
               "hbm_frac": round(gbs / hbm_peak, 4)}
        fl = KERNEL_FLOPS[prec].get(name)
        if fl is not None:
            tf = fl * ncell / (t_ms * 1e-3) / 1e12
            row.update(bound="alu", alg_flops_per_cell=fl, tflops=round(tf, 3),
                       alu_frac=round(tf / ALU_PEAK_TFLOPS[prec], 4))
        else:
            row.update(bound="hbm")
        table[name] = row
    tail = prof[:, 1 + 3 * len(kinds):]
    if tail.shape[1]:
        table["step_end"] = {"avg_ms_per_step": round(float(tail.sum(axis=1).mean()), 4),
                             "share": round(float(tail.sum() / prof.sum()), 3),
                             "launches_per_step": int(tail.shape[1])}
    k = int(np.argmax(tot))
    name = kinds[k][0]
    row = table[name]
    traffic = None
    tpc = TRAFFIC_PER_CELL.get((prec, name))
    if tpc is not None and TRAFFIC_SRC_SHA256 == _kernel_src_sha256():
        traffic = round(tpc * ncell)
    if row["bound"] == "alu":
        out = {"kernel": name, "bound": "alu", "achieved": row["tflops"],
               "peak": round(ALU_PEAK_TFLOPS[prec], 2), "unit": "TFLOP/s",
               "frac": row["alu_frac"], "traffic": traffic,
               "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz" if prec == 1
                               else "nominal GB300 FP64 1.25 TFLOP/s"),
               "alg_flops_per_cell": row["alg_flops_per_cell"]}
    else:
        out = {"kernel": name, "bound": "hbm", "achieved": row["hbm_gbs"], "peak": hbm_peak,
               "unit": "GB/s", "frac": row["hbm_frac"], "traffic": traffic,
               "peak_source": peak_kind}
    out.update(avg_launch_ms=row["avg_launch_ms"],
               hbm={"achieved": row["hbm_gbs"], "peak": hbm_peak, "unit": "GB/s",
                    "frac": row["hbm_frac"], "alg_bytes_per_cell": row["alg_bytes_per_cell"],
                    "peak_source": peak_kind},
               kernels=table,
               kernel_ms={n: table[n]["avg_launch_ms"] for n in table if "avg_launch_ms" in table[n]},
               shares={n: table[n]["share"] for n in table})
    return out


def _cpu_baseline(seconds_target: float = 20.0):
    """The oracle as it stands on the host cores: full 4096^2 RK3 steps."""
    import numpy as np

    import oracle
    from paper_1402_5618_gb300 import workloads as W
    p = W.blast_2d(N_GRID)
    g = oracle.make_grid(p.ndim, p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc)
    U = np.ascontiguousarray(p.U0)
    dt = min(p.cfl, 1.0 / 12.0) / oracle.max_rate(g, U)
    t0 = time.perf_counter()
    n = 0
    while True:
        U = oracle.rk3_step(g, U, dt)
        n += 1
        el = time.perf_counter() - t0
        if el > seconds_target or n >= 4:
            break
    out = {"value": p.nx * p.ny * 3 * n / el, "unit": UNIT, "cores": oracle.num_threads(),
           "kind": "oracle", "sample": f"{n} SSP-RK3 step(s) of the 4096^2 blast in FP64 "
                                        f"({el:.1f} s, OpenMP over grid lines)"}
    # one core: a step of the blast on 1024^2, and a step of each of the
    # first 256 problems of the 1-D Riemann batch (a 1-D line is one
    # thread's work in the oracle)
    cores = oracle.num_threads()
    oracle.set_threads(1)
    try:
        q = W.blast_2d(1024)
        gq = oracle.make_grid(q.ndim, q.nx, q.ny, q.dx, q.dy, q.gamma, q.bc)
        Uq = np.ascontiguousarray(q.U0)
        t0 = time.perf_counter()
        oracle.rk3_step(gq, Uq, min(q.cfl, 1.0 / 12.0) / oracle.max_rate(gq, Uq))
        el1 = time.perf_counter() - t0
        rb = W.riemann_batch()[:256]
        cells = 0
        t0 = time.perf_counter()
        for r in rb:
            gr = oracle.make_grid(1, r.nx, 1, r.dx, 1.0, r.gamma, r.bc)
            Ur = np.ascontiguousarray(r.U0)
            oracle.rk3_step(gr, Ur, (1.0 / 24.0) / oracle.max_rate(gr, Ur))
            cells += r.nx
        el2 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    out["single_core"] = {"blast_1024": q.nx * q.ny * 3 / el1, "riemann_batch_256": cells * 3 / el2,
                          "unit": UNIT, "sample": f"one SSP-RK3 step of the 1024^2 blast ({el1:.1f} s); "
                                                  f"one step of each of the first 256 problems of the "
                                                  f"1-D Riemann batch, {cells} cells ({el2:.1f} s)"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--fp64-steps", type=int, default=12)
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--accuracy-n", type=int, default=1024,
                    help="grid of the vortex in the line's stated accuracy")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batches", type=int, default=1, help="also time the batch workloads (0: skip)")
    ap.add_argument("--characteristic", type=int, default=1,
                    help="also time the characteristic-wise form on the blast (0: skip)")
    ap.add_argument("--char-steps", type=int, default=20)
    ap.add_argument("--char-fp64-steps", type=int, default=3)
    ap.add_argument("--profile-only", choices=["mixed", "fp64"], default=None,
                    help="only run --steps steps of the blast on an --n^2 grid (for ncu)")
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--recon", type=int, default=0,
                    help="--profile-only: 0 component-wise, 1 characteristic-wise reconstruction")
    ap.add_argument("--accuracy", action="store_true",
                    help="accuracy study instead of the throughput line: the blast to t = 1 in "
                         "both forms at --blast-n, the vortex at --vortex-n against its closed form")
    ap.add_argument("--blast-n", type=int, default=512)
    ap.add_argument("--blast-steps", type=int, default=3000)
    ap.add_argument("--vortex-n", type=int, default=1024)
    ap.add_argument("--vortex-from", type=int, default=128, help="smallest vortex grid of the sweep")
    ap.add_argument("--vortex-t", type=float, default=1.0,
                    help="end time of the vortex runs (10: one period, the 2048^2 configuration)")
    ap.add_argument("--blast-rel-n", type=int, default=0,
                    help="> 0: also the mixed-vs-FP64 relative L1 of the blast on this grid after "
                         "--blast-rel-steps steps of each form from the same state")
    ap.add_argument("--blast-rel-steps", type=int, default=100)
    ap.add_argument("--skip-blast", action="store_true", help="accuracy study without the blast probe")
    args = ap.parse_args()
    if args.profile_only:
        profile_only(args)
        return
    if args.accuracy:
        accuracy_study(args)
        return
    ws, rank, local = _dist()
    if args.impl == "reference":
        # rank 0 alone times the oracle on the host cores; other ranks exit
        if rank == 0:
            run_reference(args, ws)
        return
    _init_dist(ws, local)

    out = run_native(args, ws, rank, local)
    ncell = out["ncell"]
    rm = out["results"][1]
    rd = out["results"][0]
    ms_m = _barrier_max(rm["ms"], ws)
    ms_d = _barrier_max(rd["ms"], ws)
    e2e = _barrier_max(out["e2e_s"], ws)
    if rank == 0:
        hbm, kind = _peaks()
        value = replica_value(ws, ncell, rm["steps"], ms_m)          # accepted steps
        value_fp64 = replica_value(ws, ncell, rd["steps"], ms_d)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_m / rm["steps"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "2-D corner blast (Sedov-type) 4096^2 on [0,1.1]^2, reflective "
                                   "x-lo/y-lo, transmissive x-hi/y-hi, SSP-RK3, FVCW "
                                   "component-wise with Zhang-Shu limiter and HLLC",
                       "cfl": "min(0.5, omega_1/2) = 1/24 with eq. (CFL-CD) checked on the "
                              "limited face values of every stage (a failing step is redone; "
                              "value counts accepted steps only): the stated CFL 0.5 exceeds "
                              "the positivity bound and breaks positivity on this workload; "
                              "throughput per cell-stage does not depend on the CFL number",
                       "precision": "mixed: FP32 line arithmetic, FP32 hi+lo compensated state, FP64 limiter factors",
                       "grid": [N_GRID, N_GRID], "cells": ncell,
                       "rows_per_chunk": rm["rows_per_chunk"],
                       "l2": "no flush: the state (537 MB FP64) and stage buffers exceed L2",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": _roofline(rm, 1, ncell, hbm, kind),
            "clocks": rm["clk"],
            "e2e": {"value": replica_value(ws, ncell, out["e2e_steps"], e2e * 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": out["state_bytes"] / args.steps,
                    "d2h_bytes_per_step": out["state_bytes"] / args.steps,
                    "note": "set_state from host, K steps, get_state to host, wall clock"},
            "gpu_launches": int(rm["launches"] * rm["steps"]),
            "fp64_plain": {"value": value_fp64, "unit": UNIT, "steps": rd["steps"],
                           "rows_per_chunk": rd["rows_per_chunk"],
                           "ms_per_step": ms_d / rd["steps"], "dtype": "f64",
                           "roofline": _roofline(rd, 0, ncell, hbm, kind), "clocks": rd["clk"]},
            "accuracy": {"blast": {"case": "this workload, mixed form vs FP64 form from the same "
                                           "state at the FP64 run's final time",
                                   "t": out["acc"]["blast_t"],
                                   "rel_l1_per_variable": out["acc"]["blast_rel_l1"]},
                         "smooth": {"case": f"isentropic vortex {args.accuracy_n}^2, t = 1, "
                                            "L1 of density vs the closed form",
                                    "l1_fp64": out["acc"][0], "l1_mixed": out["acc"][1],
                                    "ratio_mixed_over_fp64": out["acc"][1] / out["acc"][0]}},
            "positivity_violations": int(rm["violations"] + rd["violations"]),
            "redone_steps": {"mixed": rm["rejected"], "fp64": rd["rejected"]},
        }
        if out["batches"]:
            line["batches"] = {"note": "seeded batches of uneven problems at the positivity CFL "
                                       "(omega_1/2 = 1/24, eq. (CFL-CD) checked on the face values, "
                                       "value over accepted steps): all 4096 1-D Riemann problems "
                                       "of 256-8192 cells (168 open an exact vacuum), 256 2-D "
                                       "four-quadrant problems of 128^2-1024^2; the 1-D set also "
                                       "with the characteristic-wise reconstruction of Sec. 2.3",
                               **out["batches"]}
        if out["characteristic"]:
            line["characteristic"] = {"note": "the same 4096^2 blast with the characteristic-wise "
                                              "reconstruction of Sec. 2.3 (block tridiagonal "
                                              "systems, Roe-averaged eigenvectors), CFL 1/24",
                                      **out["characteristic"]}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = _cpu_baseline()
        print(json.dumps(line, default=_json_default), flush=True)
    _close_dist(ws)


def profile_only(args):
    """The blast on an n^2 grid, `steps` steps, nothing else (a small case for
    ncu captures of the line kernels)."""
    import numpy as np
    import torch

    from paper_1402_5618_gb300 import binding as B
    from paper_1402_5618_gb300 import workloads as W
    prec = B.PREC_MIXED if args.profile_only == "mixed" else B.PREC_FP64
    p = W.blast_2d(args.n)
    cfg = B.config_from_problem(p, prec, cfl_positivity_cap=True, recon=args.recon)
    s = B.Solver(cfg)
    s.set_state(np.ascontiguousarray(p.U0).ravel())
    s.enqueue_steps(args.steps)
    torch.cuda.synchronize()
    st = s.stats()
    print(json.dumps({"profile_only": args.profile_only, "recon": args.recon, "n": args.n,
                      "steps": st.steps,
                      "violations": st.violations, "rows_per_chunk": s.rows_per_chunk()}))
    s.close()


def accuracy_study(args):
    """The stated accuracy of the two forms, measured on the GPU path.

    Blast (the metric's workload, on an n^2 grid, at the positivity CFL, to
    the time a bounded probe run reaches): positivity over the whole run, the mixed form's density against the
    FP64 form's (relative L1), the shock radius along a wall and along the
    diagonal (the density maximum; a cylindrical blast has one radius), and
    the mirror symmetry U(i, j) = swap(U(j, i)).  Vortex (periodic, CFL 0.5,
    to t = 1, grids 128^2 doubling up to --vortex-n): L1 and Linf of density
    against the translated closed form."""
    import numpy as np
    import torch

    from paper_1402_5618_gb300 import binding as B
    from paper_1402_5618_gb300 import workloads as W
    out = {"accuracy_study": True}

    def run(p, prec, **kw):
        s = B.Solver(B.config_from_problem(p, prec, **kw))
        s.set_state(np.ascontiguousarray(p.U0).ravel())
        t0 = time.perf_counter()
        n, rc = s.advance(p.t_final, 10 ** 7, check=False)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        U, t, steps = s.get_state()
        st = s.stats()
        s.close()
        return U.reshape(p.U0.shape), dict(steps=int(steps), t=float(t), rc=int(rc), seconds=round(el, 2),
                                           violations=int(st.violations),
                                           limiter_theta1=int(st.theta1_active),
                                           limiter_theta2=int(st.theta2_active))

    if not args.skip_blast:
        out["blast"] = _blast_study(args, run)
    if args.blast_rel_n > 0:
        out["blast_rel"] = _blast_rel(args)
    _vortex_study(args, run, out)
    print(json.dumps(out), flush=True)


def _blast_rel(args):
    """The metric's stated accuracy (i): the mixed form's blast against the
    FP64 form's after the same number of steps from the same state (each
    with its own dt), relative L1 per variable, at the positivity CFL with
    the face check."""
    import numpy as np
    import torch

    from paper_1402_5618_gb300 import binding as B
    from paper_1402_5618_gb300 import workloads as W
    p = W.blast_2d(args.blast_rel_n)
    res = {}
    for prec, name in ((0, "fp64"), (1, "mixed")):
        s = B.Solver(B.config_from_problem(p, prec, cfl_positivity_cap=True))
        s.set_state(np.ascontiguousarray(p.U0).ravel())
        s.enqueue_steps(args.blast_rel_steps)
        U, t, steps = s.get_state()
        st = s.stats()
        s.close()
        torch.cuda.synchronize()
        res[name] = (U.reshape(p.U0.shape), float(t), int(steps), int(st.violations), int(st.rejected))
    U64, U32 = res["fp64"][0], res["mixed"][0]
    rel = [float(np.abs(U32[v] - U64[v]).sum() / np.abs(U64[v]).sum()) for v in range(4)]
    out = {"grid": [args.blast_rel_n] * 2, "attempted_steps": args.blast_rel_steps,
           "fp64": {"t": res["fp64"][1], "steps": res["fp64"][2], "violations": res["fp64"][3],
                    "redone": res["fp64"][4]},
           "mixed": {"t": res["mixed"][1], "steps": res["mixed"][2], "violations": res["mixed"][3],
                     "redone": res["mixed"][4]},
           "rel_l1_mixed_vs_fp64": rel}
    print(f"blast_rel: {out}", file=sys.stderr, flush=True)
    return out


def _blast_study(args, run):
    import numpy as np

    from paper_1402_5618_gb300 import binding as B
    from paper_1402_5618_gb300 import workloads as W
    n = args.blast_n
    p = W.blast_2d(n)
    h = p.dx
    # the blast's centre empties and heats, so dt keeps shrinking: probe how
    # far a bounded number of steps gets, then run both forms from the same
    # initial state to a common end time inside that reach
    s = B.Solver(B.config_from_problem(p, 1, cfl_positivity_cap=True))
    s.set_state(np.ascontiguousarray(p.U0).ravel())
    s.enqueue_steps(args.blast_steps)
    t_reach = s.get_state()[1]
    s.close()
    p.t_final = float(f"{0.8 * t_reach:.3g}")
    print(f"blast {n}^2: {args.blast_steps} steps reach t = {t_reach:.4g}; "
          f"both forms run to t = {p.t_final}", file=sys.stderr, flush=True)
    res = {}
    for prec, name in ((0, "fp64"), (1, "mixed")):
        U, info = run(p, prec, cfl_positivity_cap=True)
        print(f"  {name}: {info}", file=sys.stderr, flush=True)
        rho = U[0]
        i_ax = int(np.argmax(rho[0, :]))
        i_dg = int(np.argmax(np.diagonal(rho)))
        sym = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
        info.update(front_axis=round((i_ax + 0.5) * h, 5),
                    front_diagonal=round(np.sqrt(2.0) * (i_dg + 0.5) * h, 5),
                    front_gap_cells=round(abs(np.sqrt(2.0) * (i_dg + 0.5) - (i_ax + 0.5)), 2),
                    mirror_max_rel=float(np.max(np.abs(U - sym)) / np.max(np.abs(U))),
                    rho_min=float(rho.min()))
        res[name] = (U, info)
    r64, r32 = res["fp64"][0][0], res["mixed"][0][0]
    return {"grid": [n, n], "t_final": p.t_final,
            "cfl": "1/24 (positivity cap, face check)",
            "t_reach_probe": t_reach, "probe_steps": args.blast_steps,
            "fp64": res["fp64"][1], "mixed": res["mixed"][1],
            "rel_l1_rho_mixed_vs_fp64": float(np.abs(r32 - r64).sum() / np.abs(r64).sum())}


def _vortex_study(args, run, out):
    import numpy as np

    from paper_1402_5618_gb300 import workloads as W
    # vortex: refinement sweep up to --vortex-n; the FP64 error falls with
    # the scheme's order while the FP32 form levels off at its rounding floor
    sweep = []
    nv = args.vortex_from
    tv = args.vortex_t
    while nv <= args.vortex_n:
        pv = W.vortex_2d(nv, t_final=tv)
        ex = W.vortex_2d(nv, t=tv).U0[0]
        vres = {"grid": [nv, nv]}
        for prec, name in ((0, "fp64"), (1, "mixed")):
            U, info = run(pv, prec)
            d = U[0] - ex
            vres[name] = {"l1_rho": float(np.mean(np.abs(d))), "linf_rho": float(np.max(np.abs(d))),
                          "steps": info["steps"], "seconds": info["seconds"],
                          "violations": info["violations"]}
        vres["l1_ratio_mixed_over_fp64"] = vres["mixed"]["l1_rho"] / vres["fp64"]["l1_rho"]
        print(f"vortex {nv}^2: {vres}", file=sys.stderr, flush=True)
        sweep.append(vres)
        nv *= 2
    out["vortex"] = {"t_final": tv, "cfl": 0.5, "error": "density vs the translated closed form",
                     "sweep": sweep}


def run_reference(args, ws):
    """The oracle (FP64 CPU reference) as it stands, on the host cores; each
    step is one SSP-RK3 step of the blast on a 1024^2 grid (a bounded sample
    of the 4096^2 workload: same problem, same per-cell work)."""
    import numpy as np

    import oracle
    from paper_1402_5618_gb300 import workloads as W
    n = 1024
    p = W.blast_2d(n)
    g = oracle.make_grid(p.ndim, p.nx, p.ny, p.dx, p.dy, p.gamma, p.bc)
    U = np.ascontiguousarray(p.U0)
    cfl = min(p.cfl, 1.0 / 12.0)   # the positivity cap applied by the native arm
    for _ in range(args.warmup):
        U = oracle.rk3_step(g, U, cfl / oracle.max_rate(g, U))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = oracle.rk3_step(g, U, cfl / oracle.max_rate(g, U))
    el = time.perf_counter() - t0
    value = n * n * 3 * args.steps / el
    sample = f"{args.steps} SSP-RK3 steps of the blast on a 1024^2 grid per run (FP64 oracle)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "2-D corner blast (Sedov-type), sampled at 1024^2",
                   "grid": [n, n], "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
