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
context per request (the plain path used for comparison, in binary64 or in
the same mixed precision).  Request data either come prepared (``prepare``,
generated before the clock starts) or are generated on the device when the
request is admitted (``probs=None``: the generation, on its own stream, is
part of the request's latency, as a transfer of its data would be), which
keeps a long stream of large requests within device memory.  ``load_curve``
serves the same requests at several offered loads.
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


def make_request(q, device, seed_offset=0):
    """Pattern and device data of one request descriptor (inputs.serving_stream)."""
    pat = inputs.pattern_for_elements(q["elements"], q["dim"])
    sigma = 4.0 if q["dim"] == 2 else 6.0
    return inputs.make_problem_device(pat, q["m"], q["s"], q["dt"], sigma, q["seed"] + seed_offset, device)


def prepare(stream, device, seed_offset=0):
    """Pattern and device data of each request (generated before the clock
    starts: the serving loop then measures solving, not data generation)."""
    return [make_request(q, device, seed_offset) for q in stream]


def request_elements(q):
    """Element count of a request descriptor's mesh (without building it)."""
    return int(inputs.pattern_for_elements(q["elements"], q["dim"])[0].size - 1)


def run_stream(stream, probs, budget_bytes=120 << 30, group_elements=None, restart=30, factor_prec="fp32",
               krylov="df64", ordering="multicolor", keep_results=False, time_scale=1.0, device="cuda",
               max_wall_s=None):
    """Serve ``stream`` (dicts with arrival times, from inputs.serving_stream)
    whose data are ``probs`` (from prepare), or, with probs=None, generated
    on the device at admission.  time_scale multiplies the arrival times
    (1 = real time).  Groups (one per (m, s) class) share the HBM budget; a
    class that finds no room closes groups that hold no request, and a
    request larger than its class's group is admitted once that group is idle
    and has been rebuilt for it.  max_wall_s: raise RuntimeError past this
    wall time."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(max_workers=16)
    groups = {}
    gbytes = {}
    gcap = {}  # elements a group's pools hold
    used = 0
    fb = 8 if factor_prec == "fp64" else 4
    elems = [probs[k].T if probs is not None else request_elements(q) for k, q in enumerate(stream)]
    recs = [Record(k, q["arrival"] * time_scale, q["m"], q["s"], elems[k]) for k, q in enumerate(stream)]
    order = list(range(len(stream)))
    active = []  # (group key, slot, idx)
    gen_stream = torch.cuda.Stream(device=device) if probs is None else None
    staged = {}  # idx -> generated request awaiting admission
    t0 = time.perf_counter()
    nxt = 0
    done = 0
    evicted = 0
    while done < len(stream):
        now = time.perf_counter() - t0
        if max_wall_s is not None and now > max_wall_s:
            pool.shutdown()
            for G in groups.values():
                G.close()
            raise RuntimeError("serving stream exceeded %.0f s (%d of %d done)" % (max_wall_s, done, len(stream)))
        # admission, in arrival order; the head of the queue blocks the rest
        while nxt < len(order) and recs[order[nxt]].arrival <= now:
            k = order[nxt]
            q = stream[k]
            key = (q["m"], q["s"])
            T = elems[k]
            r = 4 if q["dim"] == 3 else 3
            if key in groups and T > gcap[key]:
                # larger than its class's pools: rebuild the group once idle
                if any(a[0] == key for a in active):
                    break
                groups.pop(key).close()
                used -= gbytes.pop(key)
                gcap.pop(key)
            if key not in groups:
                per = bytes_per_element(q["m"], q["s"], r, restart, fb)
                # room for four requests like this one (at least 20000
                # elements), but no more than a quarter of the budget unless
                # the request itself needs it
                cap_e = group_elements or max(T, min(max(4 * T, 20000), budget_bytes // (4 * per)))
                if per * T > budget_bytes:
                    raise ValueError("request %d (%d elements, m %d) exceeds the HBM budget" % (k, T, q["m"]))
                if used + per * cap_e > budget_bytes:
                    # close idle groups (no request in them) to make room
                    busy = {a[0] for a in active}
                    for kk in [kk for kk in groups if kk not in busy]:
                        groups.pop(kk).close()
                        used -= gbytes.pop(kk)
                        gcap.pop(kk)
                        evicted += 1
                        if used + per * cap_e <= budget_bytes:
                            break
                if used + per * cap_e > budget_bytes:
                    cap_e = int(max(0, budget_bytes - used) // per)
                if cap_e < T:
                    break  # no room for a group of this class now
                try:
                    G = irk.Group(q["s"], q["m"], cap_e, cap_e * (r + 1), 64, restart=restart,
                                  factor_prec=factor_prec, krylov=krylov, ordering=ordering)
                except irk.IrkError as exc:
                    if exc.code != -2:
                        raise
                    # device memory held by torch's cache of freed request
                    # data: release it and try once more
                    torch.cuda.empty_cache()
                    G = irk.Group(q["s"], q["m"], cap_e, cap_e * (r + 1), 64, restart=restart,
                                  factor_prec=factor_prec, krylov=krylov, ordering=ordering)
                gbytes[key] = G.device_bytes()
                gcap[key] = cap_e
                used += gbytes[key]
                groups[key] = G
            G = groups[key]
            if probs is not None:
                P = probs[k]
            else:
                if k not in staged:
                    with torch.cuda.stream(gen_stream):
                        staged[k] = make_request(q, device)
                    gen_stream.synchronize()
                P = staged[k]
            slot = G.submit(P.T, torch.as_tensor(P.row_ptr).cuda(), torch.as_tensor(P.col_idx).cuda(), P.J, P.M,
                            P.R, P.dt, 1e-8)
            if slot is None:
                if not any(a[0] == key for a in active):
                    # an idle group that cannot take it (fragmented pools):
                    # rebuild the group for this request
                    groups.pop(key).close()
                    used -= gbytes.pop(key)
                    gcap.pop(key)
                    continue
                break
            staged.pop(k, None)  # the group holds its own copy now
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
    peak_groups = len(groups)
    for G in groups.values():
        G.close()
    staged.clear()
    torch.cuda.empty_cache()
    s = _summ(recs, wall)
    s.extra["groups"] = peak_groups + evicted
    s.extra["groups_closed_for_room"] = evicted
    s.extra["device_bytes"] = used
    return recs, s


def run_fifo(stream, probs, factor_prec="fp64", krylov="fp64", ordering="natural", time_scale=1.0,
             keep_results=False, device="cuda"):
    """The same stream served one request at a time, in arrival order, each
    with its own single-request context (set-up, factorisation, solve);
    probs=None: each request's data generated on the device when it is
    served (inside its latency, as in run_stream)."""
    import torch
    elems = [probs[k].T if probs is not None else request_elements(q) for k, q in enumerate(stream)]
    recs = [Record(k, q["arrival"] * time_scale, q["m"], q["s"], elems[k]) for k, q in enumerate(stream)]
    t0 = time.perf_counter()
    for k, q in enumerate(stream):
        now = time.perf_counter() - t0
        if recs[k].arrival > now:
            time.sleep(recs[k].arrival - now)
        P = probs[k] if probs is not None else make_request(q, device)
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
        del P
    wall = time.perf_counter() - t0
    torch.cuda.empty_cache()
    return recs, _summ(recs, wall)


def load_curve(stream, loads, service_rate, **kw):
    """Serve the same requests at several offered loads: the arrival times of
    ``stream`` rescaled so that its mean rate is load x service_rate.
    Returns one summary per load (p50 / p99 latency, solves/s)."""
    base = len(stream) / max(stream[-1]["arrival"], 1e-9)
    out = []
    for ld in loads:
        scale = base / (ld * service_rate)
        recs, summ = run_stream(stream, None, time_scale=scale, **kw)
        out.append({"offered_load": ld, "offered_per_s": ld * service_rate, "solves_per_s": summ.solves_per_s,
                    "p50_ms": summ.p50_ms, "p99_ms": summ.p99_ms, "requests": summ.n,
                    "all_converged": all(r.status == 0 for r in recs)})
    return out
