"""GPU parity at the kernel step's sizes.

* 2^24 events of the large float stream (key Zipf(1.1) over 1M keys, value
  lognormal(0, 1), ts +U{0..5} ms; query value > 0.5, sliding 60 s / 5 s, all
  five aggregates) in one micro-batch with end of stream: every row against
  the CPU oracle (counts, min, max exact; sums and averages within 1e-9
  relative).
* 2^26 events (the benchmark's micro-batch) in one push: the rows are streamed
  back in pieces and checked by properties that hold at any size (order,
  Σ count = K x surviving events) and, for a random sample of rows, against
  their definition recomputed from the events (math.fsum for the sums) plus,
  for sampled windows, the number of distinct keys.
"""
import math

import numpy as np
import pytest

from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import synth
from tests.engine_helpers import assert_rows_match, run_engine, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZE, SLIDE, THETA = 60_000, 5_000, 0.5
K = SIZE // SLIDE


def test_bench_workload_2p24_against_the_oracle():
    b = synth.LargeFloatStream(seed=synth.BASE_SEED + 500).next_batch(1 << 24)
    q = [dict(size=SIZE, slide=SLIDE, col="value", op="gt", value=THETA)]
    eng, st = run_engine([b], q, True, device_input=True, torch=torch)
    orc, late = run_oracle([b], q, True)
    assert len(eng[0]) > 40_000_000
    step = 1 << 22
    for a in range(0, len(orc[0]), step):
        assert_rows_match(eng[0][a:a + step], orc[0][a:a + step], True, ctx=f"rows {a}..")
    assert len(eng[0]) == len(orc[0])
    assert st["late_rows"] == sum(late) == 0


def _brute_force_row(ts, key, val, ws, k):
    a, z = np.searchsorted(ts, [ws, ws + SIZE])
    sel = (key[a:z] == k) & (val[a:z] > np.float32(THETA))
    v = val[a:z][sel].astype(np.float64)
    return len(v), math.fsum(v), v.min() if len(v) else None, v.max() if len(v) else None


def test_bench_workload_2p26_sampled_rows_and_invariants():
    rng = np.random.default_rng(synth.BASE_SEED + 501)
    b = synth.LargeFloatStream(seed=synth.BASE_SEED + 502).next_batch(1 << 26)
    ts, key, val = b.ts, b.key, b.value
    survivors = int(np.count_nonzero(val > np.float32(THETA)))
    # windows whose rows are counted: starts drawn inside the batch's span
    first = (int(ts[0]) // SLIDE + K) * SLIDE
    last = (int(ts[-1]) // SLIDE - K) * SLIDE
    wsel = np.sort(rng.choice(np.arange(first, last, SLIDE), 6, replace=False))
    wrows = dict.fromkeys(wsel.tolist(), 0)
    s = lm.Stream("float32")
    qid = s.register_query(SIZE, SLIDE, "value", "gt", THETA)
    cols = [torch.from_numpy(c).cuda() for c in (ts, key, val)]
    s.push(*cols, eos=True)
    del cols
    n_rows = s.pending(qid)
    assert n_rows > 150_000_000
    sample = np.sort(rng.choice(n_rows, 400, replace=False))
    piece = 1 << 22
    h = torch.empty(piece * 48, dtype=torch.uint8, pin_memory=True)
    got_rows, total_count, prev = 0, 0, None
    picked = []
    while True:
        m = s.poll_into(qid, h.data_ptr(), piece)
        if m == 0:
            break
        r = h[: m * 48].numpy().view(s.row_dtype)
        ws, k = r["window_start"], r["key"]
        # (window_start, key) strictly increasing, also across pieces
        same = ws[1:] == ws[:-1]
        assert np.all((ws[1:] > ws[:-1]) | (same & (k[1:] > k[:-1])))
        if prev is not None:
            assert (int(ws[0]), int(k[0])) > prev
        prev = (int(ws[-1]), int(k[-1]))
        assert np.all(r["count"] > 0) and np.all(ws % SLIDE == 0)
        total_count += int(r["count"].sum())
        for w in wrows:
            wrows[w] += int(np.count_nonzero(ws == w))
        lo, hi = np.searchsorted(sample, [got_rows, got_rows + m])
        picked.append(r[sample[lo:hi] - got_rows].copy())
        got_rows += m
    s.close()
    assert got_rows == n_rows
    # every surviving event lands in exactly K windows
    assert total_count == K * survivors
    for row in np.concatenate(picked):
        cnt, fsum, mn, mx = _brute_force_row(ts, key, val, int(row["window_start"]),
                                             int(row["key"]))
        assert cnt == int(row["count"])
        assert abs(float(row["sum"]) - fsum) <= 1e-9 * abs(fsum)
        assert abs(float(row["avg"]) - fsum / cnt) <= 1e-9 * abs(fsum / cnt)
        assert np.float32(row["min"]) == np.float32(mn) and np.float32(row["max"]) == np.float32(mx)
    # a window's rows are its distinct surviving keys
    for w, n in wrows.items():
        a, z = np.searchsorted(ts, [w, w + SIZE])
        assert n == len(np.unique(key[a:z][val[a:z] > np.float32(THETA)])) > 1000
