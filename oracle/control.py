"""TEST INFRASTRUCTURE ONLY: plain Python restatement of LMStream's control plane.

Only tests, `__graft_entry__.smoke()` and bench.py's reference leg may use it;
the engine's own implementation (C++, in the CUDA library) shares no code with
it.  Each function follows the paper's definition in its notation:

  Eq. 3   AvgThPut_i  = (sum over past micro-batches and partitions of Part)
                        / (sum over past micro-batches of Proc)
  Eq. 4   MaxLat_i    = max_j Buff_(i,j) + Proc_i
  Eq. 5   EstMaxLat_i = max_j Buff_(i,j) + (sum_j Part_(i,j)) / AvgThPut_(i-1)
  Eq. 1/2 target: SlideTime (sliding) or the mean of past MaxLat (tumbling)
  Alg. 1  ConstructMicroBatch: admit buffered + new datasets once the
          estimate reaches the target, otherwise keep buffering
  Eqs. 6-8 CPU = baseCost*Part/InfPT, GPU = baseCost*InfPT/Part,
           Trans = baseTransCost*Part/InfPT
  Alg. 2  MapDevice over a chain of operators
  Eq. 9   InfPT = b0 + b1*Throughput + b2*Latency, least squares over history,
          evaluated at target throughput = max past throughput and target
          latency = SlideTime (sliding) or the mean past latency (tumbling)

Readings where the paper is ambiguous (same as the engine's):
  * Eq. 2 divides a sum of i terms by i-1: read as the mean of the past MaxLat.
  * Eq. 3 sums j = 0..NumCores (one too many): read as all partitions.
  * AvgThPut_(-1) is undefined: the first non-empty micro-batch is admitted.
  * Alg. 1 returns at once when no new data arrived (policy "paper"); policy
    "guarded" also re-evaluates buffered data on every poll and admits when
    EstMaxLat + poll period reaches the target.
  * Eq. 9 is fitted on centred inputs (the same least-squares solution); with
    fewer than 3 samples, a constant input or collinear inputs (1 - r^2 below
    1e-12) it falls back to b = (mean InfPT, 0, 0).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Table II: base cost of each query operation (and its initial preference).
BASE_COST = {
    "aggregation": 1.0,  # hash aggregation, initial preference CPU
    "filter": 1.0,       # CPU
    "shuffle": 1.0,      # CPU
    "project": 0.9,      # neutral
    "join": 0.9,         # neutral
    "expand": 0.9,       # neutral
    "scan": 0.8,         # GPU (CSV scan)
    "sort": 0.8,         # GPU
}
OP_CODES = ["aggregation", "filter", "shuffle", "project", "join", "expand", "scan", "sort"]
BASE_TRANS_COST = 0.1        # Section III-D, initial baseTransCost
INFPT0_BYTES = 150 * 1024    # Section III-D, initial inflection point 150 KB
POLL_MS = 10.0               # Section III-C, ConstructMicroBatch polling period


def avg_thput(parts_per_batch: Sequence[float], procs: Sequence[float]) -> float:
    """Eq. 3 over micro-batches 0..i: total partition bytes / total processing time."""
    return float(np.sum(parts_per_batch)) / float(np.sum(procs))


def max_lat(buff: Sequence[float], proc: float) -> float:
    """Eq. 4: the longest buffering time among the batch's datasets plus Proc_i."""
    return float(max(buff)) + float(proc)


def est_max_lat(buff: Sequence[float], parts: Sequence[float], avg_thput_prev: float) -> float:
    """Eq. 5: the longest buffering time plus the batch size at the average throughput."""
    return float(max(buff)) + float(np.sum(parts)) / float(avg_thput_prev)


def latency_target(slide_ms: float, past_max_lat: Sequence[float]) -> Optional[float]:
    """Eq. 1 (sliding) / Eq. 2 (tumbling, mean of past MaxLat; None without history)."""
    if slide_ms > 0:
        return float(slide_ms)
    if len(past_max_lat) == 0:
        return None
    return float(np.mean(past_max_lat))


@dataclass
class Dataset:
    arrival_ms: float
    nbytes: float


@dataclass
class Admission:
    """Alg. 1 state: buffered datasets, history of Proc, Part and MaxLat."""

    slide_ms: float
    policy: str = "paper"  # or "guarded"
    poll_ms: float = POLL_MS
    buffered: List[Dataset] = field(default_factory=list)
    parts_hist: List[float] = field(default_factory=list)
    proc_hist: List[float] = field(default_factory=list)
    maxlat_hist: List[float] = field(default_factory=list)
    last_est: float = 0.0
    admitted: List[Dataset] = field(default_factory=list)
    admitted_at: float = 0.0

    def poll(self, now_ms: float, new: Sequence[Dataset]) -> bool:
        """One call of ConstructMicroBatch (Alg. 1); True = admitted."""
        if not new and (self.policy == "paper" or not self.buffered):
            return False
        tmp = list(self.buffered) + sorted(new, key=lambda d: d.arrival_ms)
        buff = [now_ms - d.arrival_ms for d in tmp]
        parts = [d.nbytes for d in tmp]
        if not self.proc_hist:  # AvgThPut_(-1) undefined: admit the first batch
            admit = True
            self.last_est = float(max(buff))
        else:
            thp = avg_thput(self.parts_hist, self.proc_hist)
            est = est_max_lat(buff, parts, thp)
            self.last_est = est
            target = latency_target(self.slide_ms, self.maxlat_hist)
            if target is None:
                admit = True
            elif self.policy == "guarded":
                admit = est + self.poll_ms >= target
            else:
                admit = est >= target
        if admit:
            self.buffered = []
            self.admitted = tmp
            self.admitted_at = now_ms
            return True
        self.buffered = tmp
        return False

    def truncate(self, n_keep: int, last_bytes: float = 0.0) -> None:
        """Memory admission of the serving loop (not in the paper): keep the
        first n_keep admitted datasets; the caller re-offers the rest."""
        assert self.admitted and 1 <= n_keep <= len(self.admitted)
        self.admitted = self.admitted[:n_keep]
        if last_bytes > 0:
            self.admitted[-1] = Dataset(self.admitted[-1].arrival_ms, float(last_bytes))

    def complete(self, proc_ms: float) -> float:
        """Records Proc_i of the last admitted batch; returns MaxLat_i (Eq. 4)."""
        buff = [self.admitted_at - d.arrival_ms for d in self.admitted]
        ml = max_lat(buff, proc_ms)
        self.parts_hist.append(float(sum(d.nbytes for d in self.admitted)))
        self.proc_hist.append(float(proc_ms))
        self.maxlat_hist.append(ml)
        return ml


def device_costs(op: str, part: float, infpt: float) -> Tuple[float, float, float]:
    """Eqs. 6-8: (CPU cost, GPU cost, transition cost) of one operation."""
    b = BASE_COST[op]
    return b * part / infpt, b * infpt / part, BASE_TRANS_COST * part / infpt


def map_device(ops: Sequence[str], batch_bytes: float, num_cores: int, infpt: float):
    """Alg. 2 over a chain of operations (first = leaf).  Returns per-op
    ("GPU"|"CPU", CPU cost, GPU cost) after the transition cost is added."""
    part = batch_bytes / num_cores
    plan = ["GPU"] * len(ops)
    out = []
    for o, op in enumerate(ops):
        cpu, gpu, trans = device_costs(op, part, infpt)
        if o == 0 or o == len(ops) - 1 or plan[o - 1] == "CPU":
            gpu += trans
        else:
            cpu += trans
        if gpu > cpu:
            plan[o] = "CPU"
        out.append((plan[o], cpu, gpu))
    return out


def regress_infpt(thput: Sequence[float], lat: Sequence[float], infpt: Sequence[float],
                  target_thput: float, target_lat: float) -> Tuple[np.ndarray, float]:
    """Eq. 9 by ordinary least squares with an intercept, solved on centred
    inputs.  Returns (beta, predicted InfPT at the targets)."""
    t = np.asarray(thput, float)
    l = np.asarray(lat, float)
    y = np.asarray(infpt, float)
    if len(y) == 0:
        beta = np.array([float(INFPT0_BYTES), 0.0, 0.0])
    else:
        tc, lc, yc = t - t.mean(), l - l.mean(), y - y.mean()
        stt, sll, stl = float(tc @ tc), float(lc @ lc), float(tc @ lc)
        degenerate = len(y) < 3 or stt == 0.0 or sll == 0.0 or 1.0 - stl * stl / (stt * sll) < 1e-12
        if degenerate:
            beta = np.array([float(y.mean()), 0.0, 0.0])
        else:
            b12 = np.linalg.solve(np.array([[stt, stl], [stl, sll]]),
                                  np.array([float(tc @ yc), float(lc @ yc)]))
            beta = np.array([float(y.mean() - b12[0] * t.mean() - b12[1] * l.mean()),
                             float(b12[0]), float(b12[1])])
    return beta, float(beta[0] + beta[1] * target_thput + beta[2] * target_lat)


class VariantAnalytic:
    """Alg. 2 re-read as the choice between the fused pass's two variants, with
    Eq. 9 refitting the inflection point (the reading is the engine's; the
    paper places operations on a CPU or a GPU).

    Variant 1 takes the place of the CPU in Eqs. 6-8 and variant 2 that of the
    GPU; Part = batch bytes / partitions.  Each variant is first tried
    `explore` times (the less sampled one first).  After a pass of `rows` rows
    taking `ms`: each variant's cost is fitted as ln ms = a + b ln rows over
    its latest `window` passes (least squares); where the two fits cross (kept
    within [1/2 smallest, 2 x largest] size seen; the far end on the cheaper
    side if they do not cross there) is the observed inflection point, in bytes
    per partition; Eq. 9 is refitted on (rows/ms, ms, observed InfPT) and
    evaluated at (largest throughput seen, mean latency) for the next pass."""

    def __init__(self, partitions: int, bytes_per_row: float, infpt0: float = INFPT0_BYTES,
                 history: int = 0, explore: int = 2, window: int = 16):
        self.partitions, self.bpr, self.infpt = partitions, float(bytes_per_row), float(infpt0)
        self.history, self.explore, self.window = history, explore, window
        self.obs = {1: [], 2: []}  # (ln rows, ln ms)
        self.hist = []  # (throughput, latency, observed InfPT)
        self.max_thput, self.sum_lat, self.n = 0.0, 0.0, 0
        self.picks = {1: 0, 2: 0}

    def choose(self, rows: int) -> int:
        if len(self.obs[1]) < self.explore or len(self.obs[2]) < self.explore:
            pick = 1 if len(self.obs[1]) <= len(self.obs[2]) else 2
        else:
            plan = map_device(["aggregation"], max(rows, 1) * self.bpr, self.partitions,
                              self.infpt)
            pick = 1 if plan[0][0] == "CPU" else 2
        self.picks[pick] += 1
        return pick

    def _fit(self, v):
        o = self.obs[v]
        x = np.array([p[0] for p in o])
        if len(o) < 2 or np.sum((x - x.mean()) ** 2) <= 1e-12:
            return None
        b, a = np.polyfit(x, np.array([p[1] for p in o]), 1)  # ln ms = a + b ln rows
        return a, b

    def predict(self, rows: int, v: int) -> float:
        f = self._fit(v)
        return -1.0 if f is None else float(np.exp(f[0] + f[1] * np.log(rows)))

    def observe(self, rows: int, v: int, ms: float) -> None:
        self.obs[v].append((np.log(rows), np.log(ms)))
        self.obs[v] = self.obs[v][-self.window:]
        self.max_thput = max(self.max_thput, rows / ms)
        self.sum_lat += ms
        self.n += 1
        f1, f2 = self._fit(1), self._fit(2)
        if f1 is None or f2 is None:
            return
        xs = [p[0] for v_ in (1, 2) for p in self.obs[v_]]
        lo, hi = min(xs) - np.log(2.0), max(xs) + np.log(2.0)
        (a1, b1), (a2, b2) = f1, f2
        x = (a1 - a2) / (b2 - b1) if b1 != b2 else (hi if a1 < a2 else lo)
        if x < lo or x > hi:
            x = hi if a1 + b1 * hi < a2 + b2 * hi else lo
        self.hist.append((rows / ms, ms, float(np.exp(x)) * self.bpr / self.partitions))
        h = self.hist[-self.history:] if self.history else self.hist
        _, inf = regress_infpt([p[0] for p in h], [p[1] for p in h], [p[2] for p in h],
                               self.max_thput, self.sum_lat / self.n)
        if inf > 0:
            self.infpt = inf
