#!/usr/bin/env python
"""Benchmark: IRK stage-system solves per second at rtol 1e-8.

One step = one full stage-system solve (irk_factor + irk_solve, Sec. 4: the
preconditioner is rebuilt once per linear solve) for each dt in
{0.01, 0.1, 1} of the 2D workload T=20000 triangles (periodic 100x100 split
grid, r=3), p=3 (m=40), Radau IIA s=3, synthetic seeded DG-shaped blocks.
Solver: FGMRES(30), double-float Krylov arithmetic on the FP32 pipe, shifted
stage-uncoupled block ILU(0) with FP32 factors in two-colour element order,
all stages per launch.

Reported beside it: the plain FP64 GPU path (FP64 factors and Krylov, one
request at a time; in the input order and in the same two-colour order),
per-phase device times with roofline fractions, the end-to-end number
through host buffers, every precision variant's iterations, time and error
against the FP64 oracle, and the FP64 oracle itself on the host cores:
complete solves, timed, serial (one core) and multi-core (OpenMP build of
the same source).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run: every rank solves its own
independent systems (replicas, no collective on the data path).
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DTS = (0.01, 0.1, 1.0)
RTOL = 1e-8
METRIC = "IRK stage-system solves/s at rtol 1e-8"
UNIT = "solves/s"
TIME_EVERY = 4  # per-kernel CUDA events on every 4th timed step
WORKLOAD = ("2D periodic 100x100 split grid, T=20000 triangles, r=3, p=3 (m=40), Radau IIA s=3, "
            "dt in {0.01,0.1,1}, FGMRES(30) rtol 1e-8, shifted uncoupled block ILU(0)")
SOLVER = ("double-float Krylov, FP32 factors, shifted uncoupled block ILU(0) in two-colour order "
          "(all stages per launch; the preconditioner in two launches)")


def algorithmic_bytes(T, m, r, s):
    """Per-launch algorithmic bytes of the operator product (K1) and of one
    preconditioner application (K3, FP32 factors, upper blocks shared by the
    stages), and of one Gram-Schmidt step pair per basis vector."""
    n = T * m
    k1 = 8 * (r + 1) * m * m * T + 8 * m * m * T + 16 * s * n
    k3 = 4 * (s * (r / 2) * m * m * T + s * m * m * T + (r / 2) * m * m * T) + 32 * s * n
    return k1, k3


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return None


MEASURED_BF16 = measured_bf16()


def traffic_record(kernel):
    """DRAM bytes of one unit of a kernel (matvec: one launch; sweep_fwd /
    sweep_bwd: the launches of one application; factor_*: the launches of one
    factorisation) from the committed ncu summary, or None when absent or
    taken on a different source of the kernel."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_c1.txt")
    if not os.path.exists(path):
        return None
    src = os.path.join(ROOT, "paper_1701_07181_gb300", "csrc")
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel:
            h = hashlib.sha256(open(os.path.join(src, f[2]), "rb").read()).hexdigest()[:12]
            return float(f[1]) if h == f[3] else None
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 7:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def replica_aggregate(local_ms, local_solves, dist=None, device=None):
    """Whole-job throughput of independent replicas: solves of all ranks
    divided by the slowest rank's time (max over ranks).  Returns
    (value, max_ms, total_solves)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_solves / (local_ms / 1000.0), local_ms, local_solves
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(local_solves)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    max_ms, total = float(t.item()), float(n.item())
    return total / (max_ms / 1000.0), max_ms, total


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def arm_config(world):
    """The workload of a bench line; the same object on both arms."""
    return {"workload": WORKLOAD, "solver": SOLVER, "solves_per_step": len(DTS),
            "l2": "inputs larger than L2 (J alone 1.0 GB per rank)", "parallelism": "replicas x%d" % world}


def cpu_info():
    """(model, cores usable by this process) of the host."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model", "Hardware") and v.strip():
                    model = v.strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count()
    return model or "unknown", cores


def oracle_solves(P, dts, omp):
    """Complete oracle solves (FP64, uncoupled shifted block ILU(0) built for
    each dt, FGMRES(30) to rtol 1e-8), one per dt, each timed on its own.
    Returns (seconds per solve, iterations, threads used)."""
    import oracle
    threads = oracle.threads() if omp else 1
    ref = oracle.Problem(P.s, P.T, P.m, P.row_ptr, P.col_idx, P.J, P.M, omp=omp)
    secs, its = [], []
    for dt in dts:
        t0 = time.perf_counter()
        out = ref.solve(P.R, dt, rtol=RTOL)
        secs.append(time.perf_counter() - t0)
        its.append(out["iters"])
        if out["rc"] != 0 or not out["relres"] <= RTOL:
            raise RuntimeError("oracle solve did not converge at dt=%g" % dt)
    return secs, its, threads


def run_reference(args):
    """The oracle on the host cores: every step one complete solve of the
    full workload (multi-core build), at dt 0.01, 0.1, 1, 0.01, ... in turn."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1701_07181_gb300 import inputs
    P = inputs.config("c1", seed=0)
    for k in range(args.warmup):
        oracle_solves(P, [DTS[k % len(DTS)]], omp=True)
    t0 = time.perf_counter()
    its, threads = [], 1
    for k in range(args.steps):
        _, it, threads = oracle_solves(P, [DTS[k % len(DTS)]], omp=True)
        its += it
    total = time.perf_counter() - t0
    value = args.steps / total
    model, cores = cpu_info()
    sample = ("%d complete oracle solves of the full workload (one per step, dt cycling 0.01/0.1/1), timed "
              "end to end: multi-core build of the oracle's C source (OpenMP over block rows, the stages' "
              "factorisations and sweeps, inner products), %d threads on %s" % (args.steps, threads, model))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": arm_config(world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu_model": model, "host_cores": cores},
            "solves_per_step": 1,  # one complete solve per step (the GPU arm's step has one per dt)
            "iters_per_solve": its[: len(DTS)],
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def oracle_samples():
    """Samples of the oracle's W at rtol 1e-12 (tests/golden/oracle_w_c1.txt,
    written by tests/golden/make_oracle_w_c1.py, which calls only the
    oracle): {dt: dict(N, norm2, amax, idx, val)}."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_w_c1.txt")
    out, cur = {}, None
    if not os.path.exists(path):
        return out
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "dt":
            kv = dict(zip(f[0::2], f[1::2]))
            cur = {"N": int(kv["N"]), "norm2": float(kv["norm2"]), "amax": float(kv["amax"]), "idx": [],
                   "val": [], "iters": int(kv["iters"])}
            out[float(kv["dt"])] = cur
        else:
            cur["idx"].append(int(f[0]))
            cur["val"].append(float(f[1]))
    for v in out.values():
        v["idx"] = np.array(v["idx"], dtype=np.int64)
        v["val"] = np.array(v["val"])
    return out


def sampled_error(W, gold):
    """Error of W against the oracle on its stored samples: element-wise
    max_i |W_i - ref_i| / max|ref| (the full vector's maximum) and an
    estimate of ||W - ref|| / ||ref|| from the samples' mean square."""
    d = W[gold["idx"]] - gold["val"]
    return {"max_rel": float(np.max(np.abs(d)) / gold["amax"]),
            "norm_rel_est": float(np.sqrt(np.mean(d * d) * gold["N"]) / gold["norm2"]),
            "samples": int(d.size)}


def precision_variants(dev):
    """Per factor precision and Krylov arithmetic, on the benchmark workload
    (two-colour order, every dt) and on the 48000-tetrahedra workload
    (dt = 0.1): iterations, time of one factorisation + solve (CUDA events,
    after a warm-up solve at another dt), and W's error against the FP64
    oracle solved to 1e-12 (benchmark workload: on the stored oracle samples;
    tetrahedra: against this run's binary64 GPU path, which the tests pin to
    the oracle)."""
    import torch
    from paper_1701_07181_gb300 import inputs, irk
    # fp64-dfop: binary64 Krylov vectors, Gram-Schmidt and residual, the
    # operator product alone in double-float
    variants = (("fp64", "fp64"), ("fp32", "fp64"), ("fp32", "fp64-dfop"), ("fp32", "df64"), ("bf16", "df64"))
    gold = oracle_samples()
    out = {}
    for name, dts in (("c1", DTS), ("c2", (0.1,))):
        P = inputs.config(name, seed=0)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        rp, ci, J, M, R = t(P.row_ptr), t(P.col_idx), t(P.J), t(P.M), t(P.R)
        res, ref = {}, {}
        for fprec, kry in variants:
            key = "%s_factors_%s_krylov" % (fprec, kry.replace("-", "_"))
            rows = {}
            with irk.Solver(P.s, P.T, P.m, rp, ci, J, M, precond="uncoupled", factor_prec=fprec, krylov=kry,
                            ordering="multicolor") as S:
                for dt in dts:
                    S.solve(R, 3.7 * dt, rtol=RTOL)  # warm-up (and autotuning); the timed solve refactors
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    W, it, rr, rc = S.solve(R, dt, rtol=RTOL)
                    e1.record()
                    torch.cuda.synchronize()
                    Wn = W.cpu().numpy()
                    row = {"iters": it, "relres": rr, "ms": e0.elapsed_time(e1)}
                    if name == "c1" and dt in gold:
                        row["error_vs_oracle"] = sampled_error(Wn, gold[dt])
                    elif fprec == "fp64":
                        ref[dt] = Wn
                    else:
                        row["rel_diff_from_fp64_gpu"] = float(np.linalg.norm(Wn - ref[dt]) / np.linalg.norm(ref[dt]))
                    rows[str(dt)] = row
            ms = sum(r["ms"] for r in rows.values())
            res[key] = {"per_dt": rows, "solves_per_s": len(dts) / (ms / 1000.0)}
        out[name] = {"T": P.T, "m": P.m, "s": P.s, "dts": list(dts), **res}
        del rp, ci, J, M, R
    nsamp = len(gold[DTS[0]]["idx"]) if gold else 0
    out["note"] = ("c1 errors: on %d stored samples of the oracle's W (tests/golden/oracle_w_c1.txt); the "
                   "full-vector bars are in tests/test_gpu_fullsize.py" % nsamp)
    return out


def ortho_compare(P, dev, rp, ci, J, M, R, steps=2):
    """The benchmark configuration with modified Gram-Schmidt and with CGS2
    orthogonalisation: solves/s over `steps` steps of the three dt, the
    Arnoldi device time per solve (CUDA events on every kernel of those
    steps) and the iteration counts."""
    import torch
    from paper_1701_07181_gb300 import irk
    out = {}
    for ortho in ("mgs", "cgs2"):
        with irk.Solver(P.s, P.T, P.m, rp, ci, J, M, precond="uncoupled", factor_prec="fp32", krylov="df64",
                        ordering="multicolor", orthogonalization=ortho) as S:
            for dt in DTS:
                S.solve(R, dt, rtol=RTOL)  # warm-up
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            its = []
            e0.record()
            for _ in range(steps):
                for dt in DTS:
                    its.append(S.solve(R, dt, rtol=RTOL)[1])
            e1.record()
            torch.cuda.synchronize()
            wall = e0.elapsed_time(e1)
            S.set_timing(2)
            S.stats()
            for dt in DTS:
                S.solve(R, dt, rtol=RTOL)
            st = S.stats()
        out[ortho] = {"solves_per_s": steps * len(DTS) / (wall / 1000.0), "iters_per_solve": its[: len(DTS)],
                      "arnoldi_ms_per_solve": st["ortho_ms"] / len(DTS),
                      "arnoldi_ms_per_iteration": st["ortho_ms"] / max(1, st["n_ortho"])}
    out["note"] = ("benchmark configuration (FP32 factors, double-float Krylov, two-colour order); Arnoldi "
                   "times from per-kernel CUDA events on one step of the three dt after the timed steps")
    return out


def dirk_comparison(P, dev, rp, ci, J, M, dt=0.1, reps=3):
    """Equal-order IRK vs DIRK steps of M u' = J u on the benchmark mesh
    (Sec. 5's comparison): RADAU23 vs DIRK33 and RADAU35 vs ESDIRK65.  One
    step = the factorisation(s) and all stage solves; equivalent
    multiplications = iterations x s (coupled system) or the sum of the
    stages' iterations (DIRK)."""
    import torch
    from paper_1701_07181_gb300 import irk, tableaux
    T, m = P.T, P.m
    u0 = torch.as_tensor(np.random.default_rng(17).standard_normal(T * m), device=dev)
    # J u0 by block gather (input preparation, untimed)
    rows = torch.repeat_interleave(torch.arange(T, device=dev), torch.diff(rp.long()))
    Ju0 = torch.zeros(T, m, dtype=torch.float64, device=dev)
    Ju0.index_add_(0, rows, torch.bmm(J.view(-1, m, m), u0.view(T, m)[ci.long()].unsqueeze(-1)).squeeze(-1))
    Ju0 = Ju0.reshape(-1)
    out = {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, s in (("RADAU23", 2), ("RADAU35", 3)):
        S = irk.Solver(s, T, m, rp, ci, J, M, precond="uncoupled", factor_prec="fp32", krylov="df64",
                       ordering="multicolor")
        R = (dt * Ju0).repeat(s)
        times, its = [], 0
        for rep in range(reps + 1):
            S.factor(2.0 * dt)  # invalidate the cached factor: every step refactors
            torch.cuda.synchronize()
            ev0.record()
            W, its, rr, rc = S.solve(R, dt, rtol=RTOL)
            ev1.record()
            torch.cuda.synchronize()
            if rep:
                times.append(ev0.elapsed_time(ev1))
        S.close()
        out[name] = {"stages": s, "iters": its, "equivalent_multiplications": its * s,
                     "ms_per_step": float(np.median(times))}
    for name, fn in (("DIRK33", tableaux.dirk33), ("ESDIRK65", tableaux.esdirk65)):
        A, b, _ = fn()
        D = irk.Dirk(A, b, T, m, rp, ci, J, M, factor_prec="fp32", krylov="df64", ordering="multicolor")
        times, its = [], []
        for rep in range(reps + 1):
            D.step(u0, 2.0 * dt, rtol=RTOL)  # so that the timed step refactors
            torch.cuda.synchronize()
            ev0.record()
            u1, _, its, rr, rc = D.step(u0, dt, rtol=RTOL)
            ev1.record()
            torch.cuda.synchronize()
            if rep:
                times.append(ev0.elapsed_time(ev1))
        D.close()
        out[name] = {"stages": len(b), "implicit_stages": int(np.count_nonzero(np.diag(A))), "iters": its,
                     "equivalent_multiplications": int(sum(its)), "ms_per_step": float(np.median(times))}
    out["dt"] = dt
    out["note"] = ("one step of M u' = J u on the benchmark mesh and blocks, each scheme refactored per step; "
                   "FP32 factors, double-float Krylov, two-colour order, rtol 1e-8 per solve")
    return out


# FP64 FMA units: 2 per SM per clock on GB300 (1.26 TFLOP/s at the 2.07 GHz
# maximum SM clock), the bound of the binary64 operator product
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def fp64_matvec_roofline(P, r, total_ms, n):
    """Binary64 operator product: algorithmic flops 2s(r+1)m^2T + 2sm^2T +
    2s^2 n per product over its measured time, against the FP64-pipe peak."""
    s, T, m = P.s, P.T, P.m
    flops = 2 * s * (r + 1) * m * m * T + 2 * s * m * m * T + 2 * s * s * T * m
    avg = total_ms / max(1, n)
    ach = flops / (avg * 1e9) if avg > 0 else None
    return {"bound": "alu", "pipe": "fp64", "avg_ms": avg, "units": n, "alg_flops": flops, "achieved": ach,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS if ach else None,
            "peak_source": "FP64 FMA unit count and max SM clock (152 x 2 x 2 x 2.07 GHz)"}


def persistent_sweep_roofline(P, r, total_ms, n, fbytes, levels):
    """The input-order preconditioner application (one persistent launch
    running both sweeps over every level, rows synchronised through published
    values): algorithmic bytes of the level form (lower blocks per stage,
    upper blocks once, D^-1 per stage, v in, z out, y through memory) per
    application over its measured time."""
    s, T, m = P.s, P.T, P.m
    n_ = T * m
    lower = (P.nnzb - T) // 2
    alg = fbytes * (s * lower * m * m + lower * m * m + s * T * m * m) + 8 * s * n_ + 8 * s * n_ + 16 * s * n_
    avg = total_ms / max(1, n)
    peak, kind = peaks()
    ach = alg / (avg * 1e6) if avg > 0 else None
    return {"kernel": "k_sweep_staged", "levels_per_sweep": "%d lower, %d upper (input order)" % levels, "avg_ms": avg, "units": n,
            "alg_bytes": alg, "achieved_gbs": ach, "frac": ach / peak if ach else None,
            "bound": "latency of the level chain: each level waits for the rows of the previous one"}


def c2_rooflines(dev, hbm_peak, peak_kind, solves=3):
    """Per-kernel times and rooflines on the 48000-tetrahedra workload (r = 4,
    m = 50, s = 3; FP32 factors, double-float Krylov, four-colour order: the
    preconditioner runs as level sweeps), from CUDA events over `solves`
    solves after a warm-up."""
    import torch
    from paper_1701_07181_gb300 import inputs, irk
    P = inputs.config("c2", seed=0)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    rp, ci, J, M, R = t(P.row_ptr), t(P.col_idx), t(P.J), t(P.M), t(P.R)
    acc = dict(iters=[], n_factor=solves)
    with irk.Solver(P.s, P.T, P.m, rp, ci, J, M, precond="uncoupled", factor_prec="fp32", krylov="df64",
                    ordering="multicolor", timing=2) as S:
        S.solve(R, 0.37, rtol=RTOL)  # warm-up and autotuning
        S.stats()
        for k in range(solves):
            _, it, rr, rc = S.solve(R, 0.1 * (k + 1), rtol=RTOL)
            acc["iters"].append(it)
        st = S.stats()
    for k in ("matvec_ms", "precond_ms", "ortho_ms", "factor_assemble_ms", "factor_products_ms",
              "factor_inverse_ms", "sweep_fwd_ms", "sweep_bwd_ms", "n_matvec", "n_precond", "n_ortho"):
        acc[k] = st[k]
    acc["factor_ms"] = st["factor_assemble_ms"] + st["factor_products_ms"] + st["factor_inverse_ms"]
    roof, kern = kernel_rooflines(P, 4, acc, hbm_peak, peak_kind, two_colour=st["sweep_two_colour"] == 1)
    del rp, ci, J, M, R
    return {"workload": "3D periodic 20^3 Kuhn grid, T=48000 tetrahedra, r=4, p=2 (m=50), s=3, dt 0.1/0.2/0.3",
            "iters_per_solve": acc["iters"], "dominant": roof, "kernels": kern,
            "sweep_form": "two-colour" if st["sweep_two_colour"] == 1 else "level sweeps (four colours)"}


def kernel_rooflines(P, r, acc, hbm_peak, peak_kind, two_colour=False):
    """Per-kernel measured time (CUDA events, irk_options.timing) over the
    timed solves, algorithmic bytes or flops per unit, and the roofline of
    the kernel with the largest total time."""
    s, T, m = P.s, P.T, P.m
    n = T * m
    mm = m * m
    nnzb = P.nnzb
    lower = (nnzb - T) // 2  # lower blocks per stage (symmetric pattern)
    alu_peak = 152 * 128 * 2 * 2.070e9 / 1e12  # FP32 FMA lanes x 2 flops x max SM clock
    tf32_peak = MEASURED_BF16 * 1.1 / 2.25 if MEASURED_BF16 else 1100.0  # nominal tf32 / bf16 ratio
    napp = max(1, acc["n_precond"])
    nfac = max(1, acc.get("n_factor", len(acc["iters"])))
    if two_colour:
        # first launch: forward rows of the second colour (nb elements, each
        # with its r neighbours below it) and their D^-1 products; second
        # launch: backward rows of the first colour, upper blocks once for
        # all stages; binary32 blocks, double-float v and z, binary32 y
        nb = lower // r
        na = T - nb
        fwd = 4 * s * lower * mm + 4 * s * nb * mm + 8 * s * n + 12 * s * nb * m
        bwd = 4 * lower * mm + 4 * s * na * mm + 8 * s * na * m + 4 * s * nb * m + 12 * s * na * m
    else:
        fwd = 4 * s * lower * mm + 8 * s * n + 4 * s * n
        bwd = 4 * lower * mm + 4 * s * mm * T + 16 * s * n
    rows = {
        # name: (total ms, units, algorithmic amount per unit, kind)
        "matvec": (acc["matvec_ms"], acc["n_matvec"], 8 * (r + 1) * mm * T + 8 * mm * T + 16 * s * n, "hbm"),
        "sweep_fwd": (acc.get("sweep_fwd_ms", 0.0), napp, fwd, "hbm"),
        "sweep_bwd": (acc.get("sweep_bwd_ms", 0.0), napp, bwd, "hbm"),
        "factor_assemble": (acc.get("factor_assemble_ms", 0.0), nfac,
                            8 * nnzb * mm + 8 * mm * T + 4 * s * nnzb * mm, "hbm"),
        "factor_products": (acc.get("factor_products_ms", 0.0), nfac, 4.0 * s * lower * m ** 3, "tensor"),
        "factor_inverse": (acc.get("factor_inverse_ms", 0.0), nfac, 2.0 * s * T * m ** 3, "alu"),
    }
    kernels = {}
    for name, (tot, units, amount, kind) in rows.items():
        avg = tot / max(1, units)
        entry = {"total_ms": tot, "units": units, "avg_ms": avg}
        if kind == "hbm":
            entry["alg_bytes"] = amount
            entry["achieved_gbs"] = amount / (avg * 1e6) if avg > 0 else None
        else:
            entry["alg_flops"] = amount
            entry["achieved_tflops"] = amount / (avg * 1e9) if avg > 0 else None
        kernels[name] = entry
    kernels["arnoldi_total_ms"] = acc["ortho_ms"]
    kernels["factor_total_ms"] = acc["factor_ms"]
    kernels["precond_total_ms"] = acc["precond_ms"]
    dominant = max(rows, key=lambda k: rows[k][0])
    dk, kind = kernels[dominant], rows[dominant][3]
    if kind == "hbm":
        roofline = {"bound": "hbm", "kernel": dominant, "achieved": dk["achieved_gbs"], "peak": hbm_peak,
                    "unit": "GB/s", "frac": dk["achieved_gbs"] / hbm_peak if dk["achieved_gbs"] else None,
                    "peak_source": peak_kind + " hbm_gbs", "traffic": traffic_record(dominant)}
    else:
        pk = tf32_peak if kind == "tensor" else alu_peak
        src = ("measured bf16 x nominal tf32/bf16 ratio (1.1/2.25)" if kind == "tensor" else
               "FP32 CUDA-core peak from unit counts and max clock (152 x 128 x 2 x 2.07 GHz)")
        roofline = {"bound": kind if kind == "alu" else "tensor", "kernel": dominant,
                    "achieved": dk["achieved_tflops"], "peak": pk, "unit": "TFLOP/s",
                    "frac": dk["achieved_tflops"] / pk if dk["achieved_tflops"] else None, "peak_source": src,
                    "traffic": traffic_record(dominant)}
    return roofline, kernels


def batched_uneven(n, dev):
    """Config-3 shape: n independent 2D meshes of 500-5000 triangles, p 1..3
    (m 12/24/40), s 2..3, dt 0.1, all submitted at once (a backlog served by
    continuous batching), against the same requests one at a time in plain
    binary64 and in the same mixed precision."""
    import torch
    from paper_1701_07181_gb300 import inputs, serve
    ub = inputs.batched_uneven(n, seed=5)
    for q in ub:
        q["arrival"] = 0.0
    probs = serve.prepare(ub, dev)
    torch.cuda.synchronize()
    recs_b, sb = serve.run_stream(ub, probs, budget_bytes=120 << 30, max_wall_s=300)
    recs_m, sm = serve.run_fifo(ub, probs, factor_prec="fp32", krylov="df64", ordering="multicolor")
    recs_f, sf = serve.run_fifo(ub, probs)
    out = {"requests": sb.n, "meshes": "2D periodic, 500-5000 triangles, p 1..3 (m 12/24/40), s 2..3, dt 0.1",
           "batched": {"solves_per_s": sb.solves_per_s, "wall_s": sb.wall_s, "groups": sb.extra["groups"],
                       "all_converged": all(r.status == 0 for r in recs_b)},
           "fifo_mixed": {"solves_per_s": sm.solves_per_s, "wall_s": sm.wall_s,
                          "solver": "same precision and order as the batched arm, one request at a time",
                          "all_converged": all(r.status == 0 for r in recs_m)},
           "fifo_plain_fp64": {"solves_per_s": sf.solves_per_s, "wall_s": sf.wall_s,
                               "all_converged": all(r.status == 0 for r in recs_f)}}
    del probs
    return out


def serving(n, dev, fifo_requests=10, rate=200.0, loads=(0.5, 1.0, 2.0), curve_requests=60):
    """Config-4 shape: a Poisson stream (mean 200/s) of 2D/3D requests of
    1k-40k elements, p 1..3, s 2..3, dt log-uniform [1e-3, 1], each request's
    data generated on the device at admission (inside its latency).  The
    first n requests of the 2000-request stream; FIFO arms (plain binary64,
    and the batched arm's mixed precision one request at a time) on its first
    fifo_requests; a load curve: the first curve_requests at offered loads of
    0.5, 1 and 2 times the batched arm's measured service rate."""
    from paper_1701_07181_gb300 import inputs, serve
    full = inputs.serving_stream(2000, rate=rate, seed=11, elements=(1000, 40000), degrees=(1, 2, 3),
                                 stages=(2, 3))
    stream = full[:n]
    recs_b, sb = serve.run_stream(stream, None, budget_bytes=120 << 30, max_wall_s=600 + 2 * n)
    head = stream[:fifo_requests]
    recs_m, sm = serve.run_fifo(head, None, factor_prec="fp32", krylov="df64", ordering="multicolor")
    recs_f, sf = serve.run_fifo(head, None)
    curve = serve.load_curve(stream[:curve_requests], loads, sb.solves_per_s, budget_bytes=120 << 30,
                             max_wall_s=300)
    return {"requests": sb.n, "of_stream": len(full), "arrival_rate_per_s": rate,
            "stream": "2D/3D periodic meshes of 1k-40k elements, p 1..3 (m 12..100), s 2..3, dt log-uniform "
                      "[1e-3, 1]; data generated on the device at admission",
            "batched": {"solves_per_s": sb.solves_per_s, "p50_ms": sb.p50_ms, "p99_ms": sb.p99_ms,
                        "groups": sb.extra["groups"], "all_converged": all(r.status == 0 for r in recs_b)},
            "fifo_mixed": {"requests": sm.n, "solves_per_s": sm.solves_per_s, "p50_ms": sm.p50_ms,
                           "p99_ms": sm.p99_ms, "all_converged": all(r.status == 0 for r in recs_m)},
            "fifo_plain_fp64": {"requests": sf.n, "solves_per_s": sf.solves_per_s, "p50_ms": sf.p50_ms,
                                "p99_ms": sf.p99_ms, "all_converged": all(r.status == 0 for r in recs_f)},
            "load_curve": curve}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-dirk", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--uneven-requests", type=int, default=512)
    ap.add_argument("--serving-requests", type=int, default=120)
    ap.add_argument("--fifo-requests", type=int, default=10)
    ap.add_argument("--matvec-variant", type=int, default=-1,
                    help="pin the headline solver's operator-product launch variant (-1: autotuned); the "
                         "autotuner's timings are distorted under a profiler, so launch lists pin the variant "
                         "the plain run picked")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving measurement (with --serving-requests up to 2000) and print it")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(3, args.warmup)
    if args.serving_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"serving": serving(args.serving_requests, torch.device("cuda", 0),
                                             fifo_requests=args.fifo_requests)}))
        return 0

    import torch
    from paper_1701_07181_gb300 import inputs, irk

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    P = inputs.config("c1", seed=rank)
    r = 3
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    rp, ci, J, M, R = t(P.row_ptr), t(P.col_idx), t(P.J), t(P.M), t(P.R)
    W = torch.empty_like(R)
    # per-kernel CUDA events on the solver's stream, read back only when the
    # stats are asked for (timing 2): once after the timed region, so no event
    # query sits between two solves of the measurement
    S = irk.Solver(P.s, P.T, P.m, rp, ci, J, M, precond="uncoupled", factor_prec="fp32", krylov="df64",
                   timing=2, ordering="multicolor", kernel_options={"matvec_variant": args.matvec_variant})

    def step(solver, acc=None, per_solve_stats=True):
        for dt in DTS:
            _, it, rr, rc = solver.solve(R, dt, rtol=RTOL, out=W)
            if rc != 0 or not rr <= RTOL:
                raise RuntimeError("solve did not converge: rc=%d relres=%g" % (rc, rr))
            if acc is not None and not per_solve_stats:
                acc["iters"].append(it)
            elif acc is not None:
                st = solver.stats()
                acc["launches"] += st["kernel_launches"]
                acc["iters"].append(it)
                for k in ("matvec_ms", "precond_ms", "ortho_ms", "factor_ms", "solve_ms", "factor_assemble_ms",
                          "factor_products_ms", "factor_inverse_ms", "sweep_fwd_ms", "sweep_bwd_ms"):
                    acc[k] = acc.get(k, 0.0) + st[k]
                for k in ("n_matvec", "n_precond", "n_ortho"):
                    acc[k] += st[k]
                acc["two_colour"] = acc.get("two_colour", True) and st["sweep_two_colour"] == 1

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if dist is None:
            return x
        v = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        return float(v.item())

    for _ in range(args.warmup):
        step(S)
    S.stats()  # releases the warm-up's timing marks
    # per-kernel events on every TIME_EVERY-th timed step only: an event
    # between two kernels costs about 2 % of the wall time of a solve
    acc = dict(launches=0, iters=[], matvec_ms=0.0, precond_ms=0.0, ortho_ms=0.0, factor_ms=0.0,
               solve_ms=0.0, n_matvec=0, n_precond=0, n_ortho=0)
    clocks = Clocks(local)
    barrier()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        S.set_timing(2 if k % TIME_EVERY == 0 else 0)
        step(S, acc, per_solve_stats=False)
    e1.record()
    barrier()
    clk = clocks.stop()
    S.set_timing(2)
    tot = S.stats()  # totals over the timed region (kernel times: the sampled steps)
    acc["launches"] = tot["kernel_launches"]
    acc["timed_steps"] = len(range(0, args.steps, TIME_EVERY))
    acc["n_factor"] = acc["timed_steps"] * len(DTS)  # every solve changes dt: one factorisation each
    for k in ("matvec_ms", "precond_ms", "ortho_ms", "factor_assemble_ms", "factor_products_ms",
              "factor_inverse_ms", "sweep_fwd_ms", "sweep_bwd_ms", "n_matvec", "n_precond", "n_ortho"):
        acc[k] = tot[k]
    acc["factor_ms"] = tot["factor_assemble_ms"] + tot["factor_products_ms"] + tot["factor_inverse_ms"]
    acc["two_colour"] = tot["sweep_two_colour"] == 1
    value, ms, solves = replica_aggregate(e0.elapsed_time(e1), args.steps * len(DTS), dist, dev)

    # end to end through host buffers (pinned), inputs copied in and the
    # result copied out on every solve
    Rh = torch.empty(R.numel(), dtype=torch.float64, pin_memory=True)
    Rh.copy_(R.cpu())
    Wh = torch.empty(R.numel(), dtype=torch.float64, pin_memory=True)
    Rn, Wn = Rh.numpy(), Wh.numpy()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for dt in DTS:
            S.solve(Rn, dt, rtol=RTOL, out=Wn)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": solves / e2e_s, "unit": UNIT, "h2d_bytes_per_step": len(DTS) * R.numel() * 8,
           "d2h_bytes_per_step": len(DTS) * R.numel() * 8}
    st_last = S.stats()
    S.close()

    # the same mixed path with the ILU(0) in the input (natural) element order
    Sn = irk.Solver(P.s, P.T, P.m, rp, ci, J, M, precond="uncoupled", factor_prec="fp32", krylov="df64")
    step(Sn)  # warm-up
    nat_acc = dict(launches=0, iters=[], matvec_ms=0.0, precond_ms=0.0, ortho_ms=0.0, factor_ms=0.0,
                   solve_ms=0.0, n_matvec=0, n_precond=0, n_ortho=0)
    barrier()
    n0, n1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0.record()
    for _ in range(args.plain_steps):
        step(Sn, nat_acc)
    n1.record()
    barrier()
    nat_ms = max_over_ranks(n0.elapsed_time(n1))
    nat_value = world * args.plain_steps * len(DTS) / (nat_ms / 1000.0)
    # the persistent (one-launch) sweep of the input order: per-kernel events
    # on one more step
    Sn.set_timing(2)
    Sn.stats()
    step(Sn)
    st = Sn.stats()
    nat_sweep = persistent_sweep_roofline(P, 3, st["precond_ms"], st["n_precond"], 4,
                                          (st["levels_lower"], st["levels_upper"]))
    Sn.close()

    # plain FP64 GPU path, one request at a time: in the input (natural)
    # element order, and in the benchmark's two-colour order (the speed-up
    # of precision alone)
    plain = {}
    fp64_mv = None
    for order in ("natural", "multicolor"):
        Sp = irk.Solver(P.s, P.T, P.m, rp, ci, J, M, precond="uncoupled", factor_prec="fp64", krylov="fp64",
                        ordering=order)
        step(Sp)  # warm-up
        plain_acc = dict(launches=0, iters=[], matvec_ms=0.0, precond_ms=0.0, ortho_ms=0.0, factor_ms=0.0,
                         solve_ms=0.0, n_matvec=0, n_precond=0, n_ortho=0)
        barrier()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record()
        for _ in range(args.plain_steps):
            step(Sp, plain_acc)
        p1.record()
        barrier()
        plain_ms = max_over_ranks(p0.elapsed_time(p1))
        plain[order] = (world * args.plain_steps * len(DTS) / (plain_ms / 1000.0), plain_acc["iters"])
        if order == "multicolor":
            # the binary64 operator product's FP64-pipe fraction: one more
            # step with per-kernel events (after the timed one)
            Sp.set_timing(2)
            Sp.stats()
            step(Sp)
            st = Sp.stats()
            fp64_mv = fp64_matvec_roofline(P, 3, st["matvec_ms"], st["n_matvec"])
        Sp.close()
    plain_value = plain["natural"][0]

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peak, peak_kind = peaks()
    roofline, kernels = kernel_rooflines(P, r, acc, peak, peak_kind, two_colour=acc.get("two_colour", False))
    kernels["event_sample"] = ("CUDA events around every kernel on every %dth timed step (%d of %d steps, %d solves); "
                               "the other steps run without them" % (TIME_EVERY, acc["timed_steps"], args.steps,
                                                                     acc["n_factor"]))
    kernels["matvec_variant"] = st_last["matvec_variant"]
    kernels["sweep_form"] = ("two-colour: forward rows of the second colour with their D^-1 products, then the "
                             "first colour's backward rows" if acc.get("two_colour") else "level sweeps")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "df64 Krylov / f32 factors",
            "data": "synthetic",
            "config": arm_config(world), "iters_per_solve": acc["iters"][: len(DTS)],
            "plain_fp64_gpu": {"value": plain_value, "unit": UNIT, "iters_per_solve": plain["natural"][1],
                               "solver": "binary64 Krylov and factors, natural order",
                               "speedup_of_value": value / plain_value,
                               "two_colour_order": {"value": plain["multicolor"][0],
                                                    "iters_per_solve": plain["multicolor"][1],
                                                    "speedup_of_value": value / plain["multicolor"][0]},
                               "fp64_matvec": fp64_mv},
            "natural_order_mixed": {"value": nat_value, "unit": UNIT, "iters_per_solve": nat_acc["iters"],
                                    "persistent_sweep": nat_sweep},
            "roofline": roofline, "kernels": kernels, "e2e": e2e,
            "gpu_launches": acc["launches"], "clocks": clk,
            "last_solve": {"iters": st_last["iters"], "relres": st_last["relres"]}}
    if not args.no_dirk and world == 1:
        line["dirk_comparison"] = dirk_comparison(P, dev, rp, ci, J, M)
        line["orthogonalization"] = ortho_compare(P, dev, rp, ci, J, M, R)
    if not args.no_variants and world == 1:
        line["precision_variants"] = precision_variants(dev)
        line["c2_kernels"] = c2_rooflines(dev, peak, peak_kind)
    if not args.no_serving and world == 1 and args.uneven_requests > 0:
        line["batched_uneven"] = batched_uneven(args.uneven_requests, dev)
    if not args.no_serving and world == 1:
        line["serving"] = serving(args.serving_requests, dev, fifo_requests=args.fifo_requests)
    if not args.no_cpu_baseline and world == 1:
        # the oracle as it stands, complete solves of the full workload, timed:
        # serial (one core) at dt = 0.01 (its cheapest solve: a bounded
        # sample), and the multi-core build at every dt
        model, host_cores = cpu_info()
        secs, its, _ = oracle_solves(P, [DTS[0]], omp=False)
        line["cpu_baseline"] = {"value": 1.0 / secs[0], "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "one complete serial oracle solve (C, FP64) of the full workload at "
                                          "dt=0.01 (%d iterations, %.1f s), timed end to end on %s"
                                          % (its[0], secs[0], model),
                                "cpu_model": model, "host_cores": host_cores}
        secs, its, threads = oracle_solves(P, DTS, omp=True)
        line["cpu_baseline_all_cores"] = {
            "value": len(DTS) / sum(secs), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "complete oracle solves of the full workload at dt 0.01, 0.1, 1 (%s iterations; %s s), "
                      "multi-core build of the same C source (OpenMP over block rows, the stages' "
                      "factorisations and sweeps, inner products), %d threads on %s"
                      % ("/".join(map(str, its)), "/".join("%.1f" % x for x in secs), threads, model),
            "cpu_model": model}
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
