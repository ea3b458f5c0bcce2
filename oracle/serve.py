"""TEST INFRASTRUCTURE ONLY: plain Python restatement of the serving loop.

Only tests, `__graft_entry__.smoke()` and bench.py's reference leg may use it;
the engine's serving loop (C++, in the CUDA library) shares no code with it.

What it computes (Section III-C's setting, with the serving extensions):
  * arrivals are given as events per poll tick; tick t covers
    [t*poll, (t+1)*poll) and is visible from its end on; event j of a tick
    with n events arrives at t*poll + (j + 0.5)*poll/n;
  * a dataset (Alg. 1's unit) is the not yet processed part of one tick;
  * policies: fixed size (exactly N events once N are buffered), fixed trigger
    (everything buffered, every T ms), and Alg. 1 (oracle.control.Admission)
    with the latency bound as target, using Eq. 5 or a processing-time
    predictor; once every tick has arrived the rest is flushed;
  * memory admission: a batch is cut to the backend's admissible row count;
    the datasets left over are offered to Alg. 1 again;
  * the clock advances by the processing time of each batch; idle waits jump to
    the next tick end (or fixed-trigger instant);
  * per-event latency = batch completion - arrival (Eq. 4 per event); the
    quantile q is the ceil(q*N)-th smallest latency.
Serving latency numbers themselves have no printed values in the paper (parity
unpinned numerically); the loop is pinned by closed forms in the tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, List, Optional

import numpy as np

from oracle import control as oc

FIXED_SIZE, FIXED_TRIGGER, ANALYTIC, LEARNED = 0, 1, 2, 3


@dataclass
class Piece:
    t0: float
    w: float
    n_total: int
    jb: int
    je: int
    fed: bool = False

    def arrivals(self) -> np.ndarray:
        j = np.arange(self.jb, self.je, dtype=np.float64)
        return self.t0 + (j + 0.5) * self.w / self.n_total


@dataclass
class BatchRecord:
    admit_ms: float
    n_events: int
    proc_ms: float
    maxlat_ms: float
    est_ms: float
    forced: bool


def kth_smallest(lat: np.ndarray, q: float) -> float:
    k = max(1, int(math.ceil(q * len(lat))))
    return float(np.sort(lat)[k - 1])


def run(tick_counts, *, poll_ms: float, policy: int, bound_ms: float,
        process: Callable[[List[Piece], int], float], fixed_rows: int = 0,
        trigger_ms: float = 0.0, bytes_per_event: float = 16.0, admit_rule: str = "guarded",
        predictor: Optional[Callable[[float, int], float]] = None,
        admissible: Optional[Callable[[], int]] = None, q_hi: float = 0.99):
    counts = [int(c) for c in tick_counts]
    pending: List[Piece] = []
    tick, now = 0, 0.0
    next_fire = trigger_ms
    adm = None
    if policy in (ANALYTIC, LEARNED):
        adm = oc.Admission(slide_ms=bound_ms, policy=admit_rule, poll_ms=poll_ms)
    lat_parts, log = [], []
    while True:
        while tick < len(counts) and (tick + 1) * poll_ms <= now + 1e-9:
            if counts[tick] > 0:
                pending.append(Piece(tick * poll_ms, poll_ms, counts[tick], 0, counts[tick]))
            tick += 1
        all_arrived = tick == len(counts)
        if not pending:
            if all_arrived:
                break
            now = (tick + 1) * poll_ms
            continue
        n_pend = sum(p.je - p.jb for p in pending)
        take, via_alg1, forced, est = 0, False, False, 0.0
        if policy == FIXED_SIZE:
            if n_pend >= fixed_rows:
                take = fixed_rows
            elif all_arrived:
                take, forced = n_pend, True
        elif policy == FIXED_TRIGGER:
            if now >= next_fire - 1e-9 or all_arrived:
                forced = now < next_fire - 1e-9
                take = n_pend
                next_fire = (math.floor(now / trigger_ms + 1e-9) + 1.0) * trigger_ms
        else:
            new = []
            for p in pending:
                if not p.fed:
                    new.append(oc.Dataset(p.t0 + (p.jb + 0.5) * p.w / p.n_total,
                                          (p.je - p.jb) * bytes_per_event))
                    p.fed = True
            if policy == LEARNED:
                ok = _poll_with_predictor(adm, now, new, predictor)
            else:
                ok = adm.poll(now, new)
            est = adm.last_est
            if ok:
                take, via_alg1 = n_pend, True
            elif all_arrived:
                take, forced = n_pend, True
        if take > 0 and admissible is not None:
            cap = int(admissible())
            if cap > 0 and take > cap:
                take, forced = cap, True
        if take == 0:
            nxt = (tick + 1) * poll_ms if tick < len(counts) else now + poll_ms
            if policy == FIXED_TRIGGER and next_fire > now:
                nxt = min(nxt, next_fire)
            now = max(now, nxt)
            continue
        batch, left, split = [], take, False
        while left > 0:
            p = pending[0]
            use = min(p.je - p.jb, left)
            batch.append(Piece(p.t0, p.w, p.n_total, p.jb, p.jb + use))
            left -= use
            if use == p.je - p.jb:
                pending.pop(0)
            else:
                p.jb += use
                p.fed = False
                split = True
        if via_alg1 and pending:
            for p in pending:
                p.fed = False
            last = batch[-1]
            adm.truncate(len(batch), (last.je - last.jb) * bytes_per_event if split else 0.0)
        proc = float(process(batch, take))
        if via_alg1:
            adm.complete(proc)
        arrivals = np.concatenate([p.arrivals() for p in batch])
        now += proc
        lat_parts.append(now - arrivals)
        log.append(BatchRecord(now - proc, take, proc, now - float(arrivals.min()), est, forced))
    lat = np.concatenate(lat_parts) if lat_parts else np.zeros(0)
    res = dict(offered=sum(counts), processed=int(lat.size), batches=len(log))
    if lat.size:
        res.update(p50=kth_smallest(lat, 0.5), p_hi=kth_smallest(lat, q_hi),
                   mean=float(lat.mean()), max=float(lat.max()))
        res["met_bound"] = res["p_hi"] <= bound_ms
    return res, log, lat


def _poll_with_predictor(adm: oc.Admission, now: float, new, predictor) -> bool:
    """Alg. 1 with Eq. 5's bytes / AvgThPut term replaced by a predictor of the
    processing time (the learned policy)."""
    if not new and (adm.policy == "paper" or not adm.buffered):
        return False
    tmp = list(adm.buffered) + sorted(new, key=lambda d: d.arrival_ms)
    buff = [now - d.arrival_ms for d in tmp]
    total = float(sum(d.nbytes for d in tmp))
    if not adm.proc_hist:
        admit = True
        adm.last_est = float(max(buff))
    else:
        est = float(max(buff)) + float(predictor(total, len(tmp)))
        adm.last_est = est
        target = oc.latency_target(adm.slide_ms, adm.maxlat_hist)
        admit = est + adm.poll_ms >= target if adm.policy == "guarded" else est >= target
    if admit:
        adm.buffered, adm.admitted, adm.admitted_at = [], tmp, now
        return True
    adm.buffered = tmp
    return False
