"""Seeded synthetic stream generators (input data only).

This module produces columnar micro-batches — event time `ts` (int64 ms), group
key `key` (uint32), `value` (int32 or float32) and `type` (uint8) — with the
shapes and value distributions of the workloads the engine is measured on.  It
holds none of the method's arithmetic (no filtering, windowing or aggregation),
so the engine and the CPU oracle can both be fed from it.

The paper evaluates on the Linear Road and Google cluster-monitoring streams,
which are not available here; these synthetic streams stand in for them:

* tiny (integer) stream: ts monotone with uniform integer gaps of 0..5 ms,
  key uniform over 1,024 keys, value uniform int32 in [0, 1000), type uniform
  in {0, 1, 2};
* large (float) stream: same ts, key Zipf(s=1.1) over 1,000,000 keys (rank r
  gets key r-1), value float32 lognormal(0, 1);
* a jittered variant of either, whose ts are out of order by up to `jitter` ms.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

BASE_SEED = 2111_04289


@dataclass
class Batch:
    ts: np.ndarray  # int64, ms
    key: np.ndarray  # uint32
    value: np.ndarray  # int32 or float32
    type: Optional[np.ndarray] = None  # uint8 or None

    def __len__(self) -> int:
        return int(self.ts.shape[0])

    def slice(self, a: int, b: int) -> "Batch":
        return Batch(
            self.ts[a:b], self.key[a:b], self.value[a:b],
            None if self.type is None else self.type[a:b],
        )


def monotone_ts(rng: np.random.Generator, n: int, start_ms: int, max_gap: int = 5) -> np.ndarray:
    """ts[i] = ts[i-1] + U{0..max_gap}; ts[0] = start_ms + U{0..max_gap}."""
    gaps = rng.integers(0, max_gap + 1, size=n, dtype=np.int64)
    return start_ms + np.cumsum(gaps, dtype=np.int64)


def jitter_ts(rng: np.random.Generator, ts: np.ndarray, jitter: int) -> np.ndarray:
    """Adds U{0..jitter} ms to each timestamp (makes the stream out of order)."""
    return ts + rng.integers(0, jitter + 1, size=ts.shape[0], dtype=np.int64)


class ZipfKeys:
    """Inverse-CDF sampler of Zipf(s) ranks over `card` keys; rank r -> key r-1."""

    def __init__(self, card: int, s: float):
        w = np.arange(1, card + 1, dtype=np.float64) ** (-float(s))
        c = np.cumsum(w)
        self.cdf = c / c[-1]
        self.card = card
        self.s = s

    def sample(self, rng: np.random.Generator, n: int) -> np.ndarray:
        u = rng.random(n)
        r = np.searchsorted(self.cdf, u, side="right")
        return np.minimum(r, self.card - 1).astype(np.uint32)


def uniform_keys(rng: np.random.Generator, n: int, card: int) -> np.ndarray:
    return rng.integers(0, card, size=n, dtype=np.int64).astype(np.uint32)


def lognormal_values(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.lognormal(0.0, 1.0, size=n).astype(np.float32)


def int_values(rng: np.random.Generator, n: int, lo: int = 0, hi: int = 1000) -> np.ndarray:
    return rng.integers(lo, hi, size=n, dtype=np.int64).astype(np.int32)


def type_column(rng: np.random.Generator, n: int, ntypes: int = 3) -> np.ndarray:
    return rng.integers(0, ntypes, size=n, dtype=np.int64).astype(np.uint8)


class TinyIntStream:
    """Micro-batches of the tiny integer workload (uniform keys, int values, type)."""

    def __init__(self, seed: int = BASE_SEED + 1, card: int = 1024, start_ms: int = 0,
                 max_gap: int = 5):
        self.rng = np.random.default_rng(seed)
        self.card = card
        self.next_ms = start_ms
        self.max_gap = max_gap

    def next_batch(self, n: int) -> Batch:
        ts = monotone_ts(self.rng, n, self.next_ms, self.max_gap)
        if n:
            self.next_ms = int(ts[-1])
        return Batch(
            ts, uniform_keys(self.rng, n, self.card), int_values(self.rng, n),
            type_column(self.rng, n),
        )


class LargeFloatStream:
    """Micro-batches of the large float workload (Zipf keys, lognormal values)."""

    def __init__(self, seed: int = BASE_SEED + 2, card: int = 1_000_000, s: float = 1.1,
                 start_ms: int = 0, max_gap: int = 5, with_type: bool = False,
                 uniform: bool = False):
        self.rng = np.random.default_rng(seed)
        self.zipf = None if uniform else ZipfKeys(card, s)
        self.card = card
        self.next_ms = start_ms
        self.max_gap = max_gap
        self.with_type = with_type

    def next_batch(self, n: int) -> Batch:
        ts = monotone_ts(self.rng, n, self.next_ms, self.max_gap)
        if n:
            self.next_ms = int(ts[-1])
        keys = (uniform_keys(self.rng, n, self.card) if self.zipf is None
                else self.zipf.sample(self.rng, n))
        return Batch(
            ts, keys, lognormal_values(self.rng, n),
            type_column(self.rng, n) if self.with_type else None,
        )


def device_large_float_batches(torch, nbatches: int, n: int, seed: int, device,
                               card: int = 1_000_000, s: float = 1.1, start_ms: int = 0,
                               max_gap: int = 5):
    """Generates the large float workload directly in device memory with torch.

    Same distributions as `LargeFloatStream` (a different random stream); used
    where the host would take too long to produce gigabytes of input.  Returns a
    list of dicts of device tensors {ts, key, value}.
    """
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    w = torch.arange(1, card + 1, dtype=torch.float64, device=device) ** (-float(s))
    cdf = torch.cumsum(w, 0)
    cdf = cdf / cdf[-1]
    out = []
    t0 = int(start_ms)
    for _ in range(nbatches):
        gaps = torch.randint(0, max_gap + 1, (n,), generator=g, device=device, dtype=torch.int64)
        ts = t0 + torch.cumsum(gaps, 0)
        t0 = int(ts[-1].item())
        u = torch.rand(n, generator=g, device=device, dtype=torch.float64)
        r = torch.searchsorted(cdf, u, right=True).clamp_(max=card - 1)
        key = r.to(torch.int32)
        val = torch.exp(torch.randn(n, generator=g, device=device, dtype=torch.float32))
        out.append({"ts": ts.contiguous(), "key": key.contiguous(), "value": val.contiguous()})
    return out


@dataclass
class ServingLoad:
    """Arrival process of the serving workload: Poisson arrivals whose rate
    follows a sinusoid between rate_min and rate_max events/s (period
    period_ms, starting at the minimum), times rate_scale, with one burst per
    period of burst_factor times the rate lasting burst_ms at a seeded phase.
    Produces events per poll tick (the serving loop's input)."""

    rate_min: float = 1e6
    rate_max: float = 200e6
    period_ms: float = 20_000.0
    burst_factor: float = 5.0
    burst_ms: float = 500.0
    rate_scale: float = 1.0

    def rate(self, t_ms: np.ndarray, burst_starts: np.ndarray) -> np.ndarray:
        phase = 2.0 * np.pi * t_ms / self.period_ms
        r = self.rate_min + (self.rate_max - self.rate_min) * 0.5 * (1.0 - np.cos(phase))
        k = np.floor(t_ms / self.period_ms).astype(np.int64)
        b0 = burst_starts[np.clip(k, 0, len(burst_starts) - 1)]
        in_burst = (t_ms >= b0) & (t_ms < b0 + self.burst_ms)
        return self.rate_scale * r * np.where(in_burst, self.burst_factor, 1.0)

    def mean_rate(self) -> float:
        """Mean offered events/s over whole periods (bursts included)."""
        base = 0.5 * (self.rate_min + self.rate_max)
        # each burst adds (factor - 1) x the rate integrated over the burst; its
        # phase is random, so on average that is the mean rate
        extra = (self.burst_factor - 1.0) * base * self.burst_ms / self.period_ms
        return self.rate_scale * (base + extra)

    def ticks(self, seed: int, duration_ms: float, poll_ms: float = 10.0) -> np.ndarray:
        rng = np.random.default_rng(seed)
        n_periods = int(np.ceil(duration_ms / self.period_ms))
        burst_starts = (np.arange(n_periods) * self.period_ms +
                        rng.uniform(0.0, self.period_ms - self.burst_ms, n_periods))
        n_ticks = int(round(duration_ms / poll_ms))
        # expected events per tick by the midpoint rule on 8 sub-steps
        sub = (np.arange(n_ticks)[:, None] + (np.arange(8)[None, :] + 0.5) / 8.0) * poll_ms
        lam = self.rate(sub, burst_starts).mean(axis=1) * poll_ms * 1e-3
        return rng.poisson(lam).astype(np.int64)
