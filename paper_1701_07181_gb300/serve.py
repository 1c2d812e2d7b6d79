"""Serving loop: continuous batching of IRK stage-system solves on one GPU.

Requests (a mesh, block size m = basis x variables, s stages, dt) arrive over
time.  Each is admitted, in arrival order, into the multi-request engine of
its class (one ``irk.Group`` per (m, s), created on first use with a share of
the HBM budget) as soon as it has arrived and its group's pools can hold it;
its factors and Krylov basis then stay on the device until it finishes.  Every
round steps each group once (one FGMRES iteration of all of its requests, one
launch per phase), so requests that arrive while others are being solved
join the running work, and finished requests are collected immediately,
freeing their pools for the queue.

``run_stream`` serves a request list and returns per-request records and a
summary (p50 / p99 latency from arrival to result, solves/s); ``run_fifo``
serves the same list one request at a time with a fresh single-request
context per request (the plain path used for comparison).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs, irk


def bytes_per_element(m, s, r, restart=30, factor_bytes=4):
    """Device bytes one element of a request occupies in a group (pools)."""
    krylov = (2 * restart + 3) * s * m * 8
    jac = (r + 1) * m * m * 8 + m * m * 8
    factors = s * (r + 1) * m * m * factor_bytes + s * m * m * factor_bytes
    words = 2 * s * m * 8 * (2 if factor_bytes == 8 else 1)
    return krylov + jac + factors + words


@dataclass
class Record:
    idx: int
    arrival: float
    m: int
    s: int
    elements: int
    admitted: float = -1.0
    finished: float = -1.0
    iters: int = 0
    relres: float = 0.0
    status: int = 0
    result: object = None

    @property
    def latency(self):
        return self.finished - self.arrival


@dataclass
class Summary:
    n: int
    wall_s: float
    solves_per_s: float
    p50_ms: float
    p99_ms: float
    mean_iters: float
    extra: dict = field(default_factory=dict)


def _summ(recs, wall):
    lat = np.array([r.latency for r in recs]) * 1000.0
    return Summary(len(recs), wall, len(recs) / wall, float(np.percentile(lat, 50)),
                   float(np.percentile(lat, 99)), float(np.mean([r.iters for r in recs])))


def prepare(stream, device, seed_offset=0):
    """Pattern and device data of each request (generated before the clock
    starts: the serving loop measures solving, not data generation)."""
    probs = []
    for k, q in enumerate(stream):
        nbrs = inputs.mesh_for_elements(q["elements"], q["dim"])
        sigma = 4.0 if q["dim"] == 2 else 6.0
        probs.append(inputs.make_problem_device(nbrs, q["m"], q["s"], q["dt"], sigma,
                                                q["seed"] + seed_offset, device))
    return probs


def run_stream(stream, probs, budget_bytes=120 << 30, group_elements=None, restart=30, factor_prec="fp32",
               krylov="df64", ordering="multicolor", keep_results=False, time_scale=1.0):
    """Serve ``stream`` (dicts with arrival times, from inputs.serving_stream)
    whose data are ``probs`` (from prepare).  time_scale multiplies the
    arrival times (1 = real time)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(max_workers=16)
    groups = {}
    used = 0
    fb = 8 if factor_prec == "fp64" else 4
    recs = [Record(k, q["arrival"] * time_scale, q["m"], q["s"], probs[k].T) for k, q in enumerate(stream)]
    order = list(range(len(stream)))
    active = []  # (group key, slot, idx)
    t0 = time.perf_counter()
    nxt = 0
    done = 0
    while done < len(stream):
        now = time.perf_counter() - t0
        # admission, in arrival order; the head of the queue blocks the rest
        while nxt < len(order) and recs[order[nxt]].arrival <= now:
            k = order[nxt]
            P = probs[k]
            key = (P.m, P.s)
            if key not in groups:
                r = 4 if stream[k]["dim"] == 3 else 3
                cap_e = group_elements or max(4 * P.T, 20000)
                need = bytes_per_element(P.m, P.s, r, restart, fb) * cap_e
                if used + need > budget_bytes:
                    cap_e = int(max(0, budget_bytes - used) // bytes_per_element(P.m, P.s, r, restart, fb))
                if cap_e < P.T:
                    break  # no room for a group of this class now
                G = irk.Group(P.s, P.m, cap_e, cap_e * (r + 1), 64, restart=restart, factor_prec=factor_prec,
                              krylov=krylov, ordering=ordering)
                used += G.device_bytes()
                groups[key] = G
            G = groups[key]
            slot = G.submit(P.T, torch.as_tensor(P.row_ptr).cuda(), torch.as_tensor(P.col_idx).cuda(), P.J, P.M,
                            P.R, P.dt, 1e-8)
            if slot is None:
                break
            recs[k].admitted = time.perf_counter() - t0
            active.append((key, slot, k))
            nxt += 1
        if not active:
            if nxt < len(order):
                wait = recs[order[nxt]].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.01))
            continue
        # step every group that has work; each group has its own stream and
        # the calls release the interpreter lock, so the groups' kernels
        # overlap on the device
        keys = sorted({a[0] for a in active})
        if len(keys) == 1:
            groups[keys[0]].step()
        else:
            list(pool.map(lambda kk: groups[kk].step(), keys))
        still = []
        for key, slot, k in active:
            running, iters, relres, status = groups[key].query(slot)
            if running:
                still.append((key, slot, k))
                continue
            W = groups[key].collect(slot, device="cuda")
            rec = recs[k]
            rec.finished = time.perf_counter() - t0
            rec.iters, rec.relres, rec.status = iters, relres, status
            if keep_results:
                rec.result = W
            done += 1
        active = still
    wall = time.perf_counter() - t0
    pool.shutdown()
    for G in groups.values():
        G.close()
    s = _summ(recs, wall)
    s.extra["groups"] = len(groups)
    s.extra["device_bytes"] = used
    return recs, s


def run_fifo(stream, probs, factor_prec="fp64", krylov="fp64", ordering="natural", time_scale=1.0,
             keep_results=False):
    """The same stream served one request at a time, in arrival order, each
    with its own single-request context (set-up, factorisation, solve)."""
    import torch
    recs = [Record(k, q["arrival"] * time_scale, q["m"], q["s"], probs[k].T) for k, q in enumerate(stream)]
    t0 = time.perf_counter()
    for k, q in enumerate(stream):
        now = time.perf_counter() - t0
        if recs[k].arrival > now:
            time.sleep(recs[k].arrival - now)
        P = probs[k]
        recs[k].admitted = time.perf_counter() - t0
        try:
            with irk.Solver(P.s, P.T, P.m, torch.as_tensor(P.row_ptr).cuda(), torch.as_tensor(P.col_idx).cuda(),
                            P.J, P.M, factor_prec=factor_prec, krylov=krylov, ordering=ordering) as S:
                W, iters, relres, rc = S.solve(P.R, P.dt, rtol=1e-8)
        except irk.IrkError as exc:
            W, iters, relres, rc = None, 0, float("nan"), exc.code
        recs[k].finished = time.perf_counter() - t0
        recs[k].iters, recs[k].relres, recs[k].status = iters, relres, rc
        if keep_results:
            recs[k].result = W
    wall = time.perf_counter() - t0
    return recs, _summ(recs, wall)
