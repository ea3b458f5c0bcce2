"""GPU parity: the CUDA engine (through the C ABI) against the CPU oracle on the
same seeded micro-batches.  Counts, integer sums, min and max are compared
bit-exactly; float sums and averages within 1e-9 relative of the oracle's
sequential FP64 sums (engine_helpers.FLOAT_REL_TOL)."""
import json
import os

import numpy as np
import pytest

from paper_2111_04289_b300 import synth
from tests.engine_helpers import assert_rows_match, run_engine, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "window_semantics.json")


def _check(batches, queries, is_float, lateness=0, **kw):
    eng, st = run_engine(batches, queries, is_float, lateness, torch=torch, **kw)
    orc, late = run_oracle(batches, queries, is_float, lateness)
    for j in range(len(queries)):
        assert_rows_match(eng[j], orc[j], is_float, ctx=f"query {j}: {queries[j]}")
    assert st["late_rows"] == sum(late)
    return eng, st


def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_golden_micro_streams(case):
    """Hand-worked streams, push by push, through the engine."""
    is_float = case["value_type"] == "float32"
    from paper_2111_04289_b300 import lmstream as lm
    s = lm.Stream("float32" if is_float else "int32", has_type=True,
                  allowed_lateness_ms=case["lateness"])
    q = case["query"]
    qid = s.register_query(q["size"], q["slide"], q["filter_col"], q["filter_op"], q["filter"])
    for push in case["pushes"]:
        rows = push["rows"]
        ts = np.array([r[0] for r in rows], dtype=np.int64)
        key = np.array([r[1] for r in rows], dtype=np.uint32)
        val = np.array([r[2] for r in rows], dtype=np.float32 if is_float else np.int32)
        typ = np.array([r[3] for r in rows], dtype=np.uint8)
        s.push(ts, key, val, typ, eos=push["eos"])
        got = s.poll(qid)
        exp = push["expect"]
        assert len(got) == len(exp), (case["name"], got, exp)
        for g, e in zip(got, exp):
            assert (int(g["window_start"]), int(g["window_start"]) + q["size"], int(g["key"]),
                    int(g["count"])) == tuple(e[:4])
            assert g["sum"] == e[4] and g["avg"] == e[7]
            if is_float:
                assert np.float32(g["min"]).tobytes() == np.float32(e[5]).tobytes()
                assert np.float32(g["max"]).tobytes() == np.float32(e[6]).tobytes()
            else:
                assert (int(g["min"]), int(g["max"])) == (e[5], e[6])
        assert s.stats()["late_rows"] == push["late"]
    s.close()


def test_tiny_int_workload():
    """Uniform 1,024 keys, int values, filter type == 0, tumbling 10 s, count + sum."""
    s = synth.TinyIntStream()
    batches = [s.next_batch(65_536) for _ in range(12)]
    _check(batches, [dict(size=10_000, col="type", op="eq", value=0)], False)


@pytest.mark.parametrize("sizes", [[2**14, 3, 2**16 + 123, 0, 2**15], [2**17]])
def test_large_float_sliding(sizes):
    """Zipf(1.1) over 1M keys, lognormal values, value > 0.5, sliding 60 s / 5 s."""
    s = synth.LargeFloatStream()
    batches = [s.next_batch(n) for n in sizes]
    _check(batches, [dict(size=60_000, slide=5_000, col="value", op="gt", value=0.5)], True)


@pytest.mark.parametrize("n", [1, 2, 2047, 2048, 2049, 4095, 4097, 12_345])
def test_ragged_batch_sizes(n):
    s = synth.TinyIntStream(seed=31, card=97)
    batches = [s.next_batch(n), s.next_batch(0), s.next_batch(n // 2 + 1)]
    _check(batches, [dict(size=1_000, slide=250), dict(size=700)], False)


def _gapped(n, gap, seed, card=50):
    """One batch whose events sit every `gap` ms: windows anchored at absent
    panes do not exist, so a range's window ids are not consecutive."""
    b = synth.TinyIntStream(seed=seed, card=card).next_batch(n)
    b.ts = np.arange(n, dtype=np.int64) * gap
    return b


def test_gapped_panes_few_windows_per_range():
    """Non-consecutive window ids, few per range (searched in shared memory)."""
    b = _gapped(40_000, 3, seed=61)
    _check([b], [dict(size=2, slide=1), dict(size=4, slide=2)], False)


def test_gapped_panes_many_windows_per_range():
    """Non-consecutive window ids, more per range than are staged (searched in
    global memory): over 512 windows for each of the kernel's ranges."""
    b = _gapped(1_300_000, 2, seed=67)
    _check([b], [dict(size=1)], False)


def test_float_avg_counts_around_2p24():
    """One tumbling window whose keys hold 2^24 - 1 and 2^24 + 1 events (the
    two ways an average is divided: below 2^24 counts a float32-built
    reciprocal, from 2^24 on a refined one), plus 3 and 2^20 events; the hot
    keys' partial groups form runs far longer than a tile."""
    rng = np.random.default_rng(71)
    sizes = {5: (1 << 24) - 1, 9: (1 << 24) + 1, 11: 3, 13: 1 << 20}
    key = np.concatenate([np.full(c, k, np.uint32) for k, c in sizes.items()])
    rng.shuffle(key)
    n = len(key)
    ts = np.sort(rng.integers(0, 1000, n)).astype(np.int64)
    val = rng.lognormal(0.0, 1.0, n).astype(np.float32)
    eng, _ = _check([synth.Batch(ts, key, val)], [dict(size=1000)], True)
    assert sorted(zip(eng[0]["key"].tolist(), eng[0]["count"].tolist())) == sorted(sizes.items())


def test_special_float_values():
    """Subnormal values, values near the float maximum (sums far beyond it),
    negative values, signed zeros (min and max in total order: -0.0 < +0.0),
    and keys holding one +Inf or one -Inf: counts, min and max exact, finite
    sums and averages within the tolerance, infinite ones equal."""
    rng = np.random.default_rng(73)
    v5 = rng.lognormal(0.0, 1.0, 3000)
    v5[1234] = np.inf
    v6 = -rng.lognormal(0.0, 1.0, 3000)
    v6[77] = -np.inf
    vals = {1: rng.uniform(1e-45, 1e-38, 3000), 2: rng.uniform(1e37, 3.4e38, 3000),
            3: -rng.lognormal(0.0, 1.0, 3000), 4: np.where(rng.random(3000) < 0.5, -0.0, 0.0),
            5: v5, 6: v6}
    key = np.concatenate([np.full(len(v), k, np.uint32) for k, v in vals.items()])
    val = np.concatenate([np.asarray(v, np.float32) for v in vals.values()])
    perm = rng.permutation(len(key))
    key, val = key[perm], val[perm]
    ts = np.sort(rng.integers(0, 1000, len(key))).astype(np.int64)
    batches = [synth.Batch(ts, key, val)]
    q = [dict(size=1000)]
    eng, _ = run_engine(batches, q, True, torch=torch)
    orc, _ = run_oracle(batches, q, True)
    e, o = eng[0], orc[0]
    assert len(e) == len(o) == 6
    np.testing.assert_array_equal(e["key"], o["key"])
    np.testing.assert_array_equal(e["count"], o["count"])
    np.testing.assert_array_equal(e["min"].view(np.uint32), o["min_f"].view(np.uint32))
    np.testing.assert_array_equal(e["max"].view(np.uint32), o["max_f"].view(np.uint32))
    for f, of in (("sum", "sum_f"), ("avg", "avg")):
        fin = np.isfinite(o[of])
        assert np.array_equal(e[f][~fin], o[of][~fin]), (f, e[f], o[of])
        assert np.all(np.abs(e[f][fin] - o[of][fin]) <= 1e-9 * np.abs(o[of][fin]) + 1e-300), f


def test_int32_extreme_values():
    """Keys whose every value is INT32_MAX, INT32_MIN, alternating extremes or
    -1, several thousand events each (many per fused-pass tile): the packed
    count-and-sum words at their limits; all aggregates bit-exact."""
    rng = np.random.default_rng(79)
    imax, imin = np.iinfo(np.int32).max, np.iinfo(np.int32).min
    vals = {1: np.full(5000, imax), 2: np.full(5000, imin),
            3: np.where(np.arange(5000) % 2 == 0, imax, imin), 4: np.full(5000, -1)}
    key = np.concatenate([np.full(len(v), k, np.uint32) for k, v in vals.items()])
    val = np.concatenate([np.asarray(v, np.int32) for v in vals.values()])
    perm = rng.permutation(len(key))
    key, val = key[perm], val[perm]
    ts = np.sort(rng.integers(0, 1000, len(key))).astype(np.int64)
    eng, _ = _check([synth.Batch(ts, key, val)], [dict(size=1000), dict(size=400, slide=200)], False)
    assert len(eng[0]) == 4


def test_empty_stream_and_eos_only():
    b = synth.TinyIntStream().next_batch(0)
    eng, st = _check([b, b], [dict(size=1_000)], False)
    assert len(eng[0]) == 0 and st["rows_emitted"] == 0


def test_jittered_stream_with_lateness():
    rng = np.random.default_rng(7)
    s = synth.LargeFloatStream(seed=41, card=5000, s=1.3)
    batches = []
    for n in (3000, 5000, 4000, 1):
        b = s.next_batch(n)
        b.ts = synth.jitter_ts(rng, b.ts, 5)
        batches.append(b)
    _check(batches, [dict(size=2_000, slide=500)], True, lateness=5)
    # without the allowance some rows arrive late; both sides must agree on them
    _check(batches, [dict(size=2_000, slide=500), dict(size=300)], True, lateness=0)


def test_late_batch_rows_dropped_and_counted():
    s = synth.TinyIntStream(seed=43, card=20)
    b1 = s.next_batch(3000)
    b2 = s.next_batch(3000)
    late = synth.Batch(b1.ts[:500].copy(), b1.key[:500].copy(), b1.value[:500].copy(),
                       b1.type[:500].copy())
    _, st = _check([b1, b2, late, s.next_batch(100)], [dict(size=1_000, slide=200)], False)
    assert st["late_rows"] > 0


@pytest.mark.parametrize("col,op,value", [
    ("ts", "ge", 1000), ("ts", "lt", 3000), ("key", "eq", 5), ("key", "ne", 5),
    ("key", "le", 10), ("value", "gt", 500), ("value", "le", 100), ("type", "eq", 2),
    ("type", "ne", 0), ("type", "none", 0)])
def test_filter_columns_and_ops_int(col, op, value):
    s = synth.TinyIntStream(seed=51, card=30)
    batches = [s.next_batch(2500), s.next_batch(2500)]
    _check(batches, [dict(size=1_500, slide=500, col=col, op=op, value=value)], False)


@pytest.mark.parametrize("op,value", [("gt", 0.5), ("le", 1.0), ("eq", 0.0), ("ne", 1.5),
                                      ("ge", 10.24), ("lt", 0.2776)])
def test_filter_float_value(op, value):
    s = synth.LargeFloatStream(seed=52, card=1000)
    batches = [s.next_batch(3000), s.next_batch(3000)]
    _check(batches, [dict(size=1_000, slide=1_000, col="value", op=op, value=value)], True)


def test_big_windows_take_the_global_merge_path():
    """64 panes x ~1000 distinct keys per pane: windows exceed the shared buffer."""
    rng = np.random.default_rng(61)
    n = 140_000
    ts = np.sort(rng.integers(0, 64 * 100 * 2, size=n)).astype(np.int64)
    key = rng.integers(0, 5000, size=n).astype(np.uint32)
    val = rng.integers(-1000, 1000, size=n).astype(np.int32)
    b = synth.Batch(ts, key, val, None)
    eng, st = _check([b.slice(0, 70_000), b.slice(70_000, n)], [dict(size=6_400, slide=100)],
                     False)
    assert len(eng[0]) > 0


def test_max_panes_per_window():
    s = synth.TinyIntStream(seed=62, card=7)
    batches = [s.next_batch(150), s.next_batch(150)]
    _check(batches, [dict(size=4096 * 3, slide=3)], False)


def test_negative_and_epoch_timestamps():
    rng = np.random.default_rng(63)
    for start in (-50_000, 1_700_000_000_000):
        s = synth.TinyIntStream(seed=64, card=40, start_ms=start)
        batches = [s.next_batch(4000), s.next_batch(4000)]
        _check(batches, [dict(size=3_000, slide=1_000), dict(size=777)], False)
    del rng


def test_eight_fused_queries_equal_each_alone():
    s = synth.LargeFloatStream(seed=71, card=10_000, s=1.3, with_type=True)
    batches = [s.next_batch(20_000), s.next_batch(7), s.next_batch(30_000)]
    queries = [dict(size=1_000), dict(size=10_000), dict(size=30_000, slide=1_000),
               dict(size=1_000, col="value", op="gt", value=10.24),
               dict(size=10_000, col="value", op="gt", value=3.602),
               dict(size=30_000, slide=1_000, col="value", op="gt", value=1.0),
               dict(size=1_000, col="value", op="gt", value=0.2776),
               dict(size=60_000, slide=5_000, col="type", op="eq", value=1)]
    fused, _ = run_engine(batches, queries, True, torch=torch)
    orc, _ = run_oracle(batches, queries, True)
    for j, q in enumerate(queries):
        alone, _ = run_engine(batches, [q], True, torch=torch)
        assert_rows_match(fused[j], orc[j], True, ctx=f"fused {q}")
        assert_rows_match(alone[0], orc[j], True, ctx=f"alone {q}")
        for f in ("window_start", "key", "count", "sum", "min", "max"):
            np.testing.assert_array_equal(fused[j][f], alone[0][f])


def test_device_input_equals_host_input():
    s = synth.LargeFloatStream(seed=72)
    batches = [s.next_batch(50_000), s.next_batch(20_000)]
    q = [dict(size=60_000, slide=5_000, col="value", op="gt", value=0.5)]
    host, _ = run_engine(batches, q, True, torch=torch)
    dev, _ = run_engine(batches, q, True, torch=torch, device_input=True)
    for f in ("window_start", "key", "count", "min", "max"):
        np.testing.assert_array_equal(host[0][f], dev[0][f])
    np.testing.assert_allclose(host[0]["sum"], dev[0]["sum"], rtol=1e-12)


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_k1_variants_agree(variant):
    """Every variant of the fused pass (1024 / 2048-event tiles, with and
    without warp aggregation), float and int values, ragged batch ends."""
    s = synth.LargeFloatStream(seed=73, card=100, s=1.3)
    batches = [s.next_batch(40_000), s.next_batch(2049), s.next_batch(70_001)]
    _check(batches, [dict(size=5_000, slide=1_000), dict(size=900, col="value", op="gt",
                                                         value=1.0)], True, k1_variant=variant)
    t = synth.TinyIntStream(seed=74, card=300)
    _check([t.next_batch(33_333), t.next_batch(4097)],
           [dict(size=2_000, slide=500, col="type", op="eq", value=1)], False, k1_variant=variant)


def test_autotuner_samples_every_variant_then_settles():
    """Seven int queries on 2^15-row batches (a size class no other test uses):
    each of the four variants is timed three times (the first as warm-up),
    then the fastest is kept; the rows match the oracle throughout."""
    t = synth.TinyIntStream(seed=75, card=2_000)
    batches = [t.next_batch(1 << 15) for _ in range(15)]
    q = [dict(size=1_000 * (j + 1), slide=500 * (j + 1) if j % 2 else 0) for j in range(7)]
    eng, st = _check(batches, q, False, k1_variant=0)
    assert st["autotune_samples"] == 12
    assert st["k1_tile_events"] in (1024, 2048)


@pytest.mark.parametrize("timing", [False, True])
def test_graph_replay_equals_plain_launches(timing):
    """The tail of a push (watermark, sort/reduce, pane index, emission, carry)
    replayed from a CUDA graph gives the rows of plain launches."""
    t = synth.TinyIntStream(seed=82, card=700)
    batches = [t.next_batch(n) for n in [6000] * 10 + [9000] * 4 + [20]]
    q = [dict(size=3_000, slide=1_000), dict(size=2_000, col="type", op="eq", value=0)]
    plain, st0 = run_engine(batches, q, False, graph_mode=1, enable_timing=timing)
    graph, st1 = run_engine(batches, q, False, graph_mode=2, enable_timing=timing)
    orc, _ = run_oracle(batches, q, False)
    for j in range(len(q)):
        assert_rows_match(graph[j], orc[j], False, ctx=f"graph q{j}")
        assert graph[j].tobytes() == plain[j].tobytes()
    assert st0["graph_launches"] == 0
    assert st1["graph_launches"] >= 8 and st1["graph_captures"] >= 1


def test_batching_invariance_on_gpu():
    s = synth.TinyIntStream(seed=74, card=300)
    full = s.next_batch(60_000)
    q = [dict(size=20_000, slide=2_000)]
    ref, _ = run_engine([full], q, False, torch=torch)
    cuts = [full.slice(0, 1), full.slice(1, 30_000), full.slice(30_000, 30_000),
            full.slice(30_000, 60_000)]
    got, _ = run_engine(cuts, q, False, torch=torch)
    for f in ("window_start", "key", "count", "sum", "min", "max", "avg"):
        np.testing.assert_array_equal(ref[0][f], got[0][f])


@pytest.mark.parametrize("is_float", [False, True])
def test_hot_key_runs_longer_than_a_tile(is_float):
    """Event time barely moves (a serving-like stream): one key takes 60 % of
    the events of a pane, so its partial groups from hundreds of K1 tiles form
    one long run that the cooperative reduce combines."""
    rng = np.random.default_rng(21)
    n = 600_000
    ts = np.sort(rng.integers(0, 900, n)).astype(np.int64)
    key = np.where(rng.random(n) < 0.6, 7, rng.integers(0, 5000, n)).astype(np.uint32)
    val = (rng.lognormal(0, 1, n).astype(np.float32) if is_float
           else rng.integers(-1000, 1000, n).astype(np.int32))
    batches = [synth.Batch(ts[a:a + 200_000], key[a:a + 200_000], val[a:a + 200_000])
               for a in range(0, n, 200_000)]
    _check(batches, [dict(size=1000, slide=250), dict(size=300, slide=300)], is_float)


def test_run_longer_than_the_cooperative_threshold():
    """4.6M events in one pane with one key in 90 % of them: that key's partial
    groups (one per K1 tile, > 4096) form a run that crosses many reduce
    chunks and goes to the cooperative reduce."""
    rng = np.random.default_rng(23)
    n = 4_600_000
    ts = np.sort(rng.integers(0, 900, n)).astype(np.int64)
    key = np.where(rng.random(n) < 0.9, 7, rng.integers(0, 300, n)).astype(np.uint32)
    val = rng.integers(-1000, 1000, n).astype(np.int32)
    _check([synth.Batch(ts, key, val)], [dict(size=1000)], False)
