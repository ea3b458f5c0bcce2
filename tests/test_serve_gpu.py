"""The serving loop on the GPU backend.

* The load generator writes what its definition says (ts = floor of the
  arrival time, keys in range, positive values, Zipf head share) and depends
  only on each event's stream-wide index (the same events however the ticks
  are cut into batches).
* Every row the engine emitted during a serving run (Alg. 1 choosing uneven
  batch sizes, memory admission on) equals the oracle's rows for the same
  events cut at the same batch boundaries.
* Admission by memory keeps every batch within what the stream's state cap
  allows, and the run completes without running out of device memory."""
import numpy as np
import pytest

from paper_2111_04289_b300 import lmstream as lm
from tests.engine_helpers import assert_rows_match, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QUERIES = [dict(size=400, slide=100, col="value", op="gt", value=0.5),
           dict(size=250, slide=250)]


class _Events:
    def __init__(self, ts, key, value):
        self.ts, self.key, self.value, self.type = ts, key, value, None


def _generate_all(g, chunks, max_rows):
    """The events of all chunks, made in pieces the backend accepts."""
    parts, cur, n = [], [], 0
    for c in chunks:
        m = c[4] - c[3]
        if cur and n + m > max_rows:
            parts.append(g.generate(cur))
            cur, n = [], 0
        cur.append(c)
        n += m
    if cur:
        parts.append(g.generate(cur))
    return [np.concatenate([p[i] for p in parts]) for i in range(3)]


def _chunks_for(ticks, poll):
    out, first = [], 0
    for t, c in enumerate(ticks):
        if c:
            out.append((t * poll, poll, int(c), 0, int(c), first))
            first += int(c)
    return out


def test_generator_definition_and_split_invariance():
    g = lm.ServeGpu(QUERIES, seed=7, n_keys=1_000_000, max_batch_rows=1 << 20)
    ticks = np.random.default_rng(1).poisson(20_000, 40)
    ch = _chunks_for(ticks, 10.0)
    ts, key, val = g.generate(ch)
    arr = np.concatenate([t0 + (np.arange(n) + 0.5) * w / n for (t0, w, n, _, _, _) in ch])
    np.testing.assert_array_equal(ts, np.floor(arr).astype(np.int64))
    assert key.max() < 1_000_000 and np.all(val > 0)
    # rank 1 of Zipf(1.1) over 1e6 keys has probability 1 / H(1e6, 1.1)
    h = np.sum(np.arange(1, 1_000_001, dtype=np.float64) ** -1.1)
    share = np.mean(key == 0)
    assert abs(share - 1.0 / h) < 0.01
    assert abs(np.median(np.log(val.astype(np.float64)))) < 0.02  # lognormal(0, 1)
    # cut every tick in two pieces: same events
    half = []
    for (t0, w, n, jb, je, f) in ch:
        m = n // 3
        half += [(t0, w, n, 0, m, f), (t0, w, n, m, n, f)]
    ts2, key2, val2 = g.generate(half)
    np.testing.assert_array_equal(ts2, ts)
    np.testing.assert_array_equal(key2, key)
    np.testing.assert_array_equal(val2.view(np.uint32), val.view(np.uint32))
    g.close()


@pytest.mark.parametrize("policy,device_input,ingest", [(lm.POLICY_ANALYTIC, False, False),
                                                        (lm.POLICY_FIXED_SIZE, False, False),
                                                        (lm.POLICY_ANALYTIC, True, False),
                                                        (lm.POLICY_ANALYTIC, False, True),
                                                        (lm.POLICY_FIXED_SIZE, False, True)])
def test_serving_rows_match_oracle(policy, device_input, ingest):
    """Ingest mode: ticks go to the device through the ingest ring as they
    arrive (overlapped with buffering and compute); the rows must not change."""
    ticks = np.random.default_rng(3).poisson(np.linspace(500, 6000, 260)).astype(np.int64)
    g = lm.ServeGpu(QUERIES, seed=11, n_keys=20_000, max_batch_rows=1 << 18, keep_rows=True,
                    device_input=device_input, ingest=ingest)
    res, log = lm.serve_run(ticks, poll_ms=10.0, policy=policy, bound_ms=60.0,
                            backend=g.backend(), fixed_rows=17_000)
    assert res["processed_events"] == ticks.sum() and res["completed"] == 1
    sizes = [r["n_events"] for r in log]
    if policy == lm.POLICY_ANALYTIC:
        assert len(set(sizes)) > 3  # Alg. 1 picks uneven batch sizes
    ts, key, val = _generate_all(g, _chunks_for(ticks, 10.0), 1 << 18)
    bounds = np.concatenate([[0], np.cumsum(sizes)])
    batches = [_Events(ts[a:b], key[a:b], val[a:b]) for a, b in zip(bounds[:-1], bounds[1:])]
    orc, _ = run_oracle(batches, QUERIES, True, eos=False)
    for j in range(len(QUERIES)):
        eng = g.kept_rows(j)
        assert len(eng) > 100
        assert_rows_match(eng, orc[j], True, ctx=f"query {j}")
    g.close()


def test_memory_admission_bounds_batches():
    cap = 320 << 20
    g = lm.ServeGpu(QUERIES[:1], seed=5, n_keys=100_000, max_batch_rows=1 << 22,
                    state_cap_bytes=cap)
    adm0 = g.admissible_rows()
    assert 0 < adm0 < 1 << 22
    ticks = np.full(60, 400_000, dtype=np.int64)  # far more than one batch may hold
    res, log = lm.serve_run(ticks, poll_ms=10.0, policy=lm.POLICY_FIXED_TRIGGER, bound_ms=1e6,
                            trigger_ms=200.0, backend=g.backend())
    assert res["processed_events"] == ticks.sum()
    assert max(r["n_events"] for r in log) <= adm0
    assert any(r["forced"] for r in log)
    assert g.stats()["device_bytes"] <= cap
    g.close()
