"""Key sharding's host logic on the CPU: the native split (lms_shard_of /
lms_shard_split), and ShardedStream / DistShardedStream (two gloo ranks) over
oracle-backed shards against one unsharded oracle stream.

What makes sharding exact: a group (window, key) is built from its key's rows
only, and every shard is given the whole micro-batch's max event time, so every
shard's watermark, and the set of windows it closes, is the single stream's
(Section II-A's event-time windows).  Rows of a key keep their input order in
the split, so even float sums come out bit-identical when one process splits."""
import os
import socket

import numpy as np
import pytest

from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import sharded
from paper_2111_04289_b300 import synth
from tests.shard_helpers import OracleShard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fmix32(h):
    h = np.asarray(h, np.uint64) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x85EBCA6B)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0xC2B2AE35)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    return h


def _shard_ref(key, mask, g):
    return ((_fmix32(np.asarray(key, np.uint64) & np.uint64(mask)) * np.uint64(g))
            >> np.uint64(32)).astype(np.uint32)


def test_shard_of_is_the_stated_hash():
    rng = np.random.default_rng(5)
    keys = np.concatenate([rng.integers(0, 1 << 32, 3000, dtype=np.uint64).astype(np.uint32),
                           np.array([0, 1, 0xFFFFFFFF], np.uint32)])
    for g in (1, 2, 3, 7, 8):
        for mask in (0xFFFFFFFF, 0xFF):
            np.testing.assert_array_equal(sharded.shard_of(keys, mask, g),
                                          _shard_ref(keys, mask, g))
    # fmix32's known value on 0 is 0 and the split is close to uniform
    assert int(sharded.shard_of(np.array([0], np.uint32), 0xFFFFFFFF, 4)[0]) == 0
    c = np.bincount(sharded.shard_of(np.arange(40000, dtype=np.uint32), 0xFFFFFFFF, 4),
                    minlength=4)
    assert c.min() > 9000


@pytest.mark.parametrize("n,g", [(0, 3), (1, 1), (5000, 3), (5000, 8), ((1 << 20) + 7, 5)])
def test_shard_split_is_a_stable_partition(n, g):
    rng = np.random.default_rng(n + g)
    ts = rng.integers(-10_000, 10_000, n).astype(np.int64)
    key = rng.integers(0, 1 << 20, n).astype(np.uint32)
    val = rng.standard_normal(n).astype(np.float32)
    typ = rng.integers(0, 4, n).astype(np.uint8)
    mask = 0x0FFFF
    parts, mx = sharded.shard_split(ts, key, val, typ, g, mask)
    assert len(parts) == g
    assert mx == (None if n == 0 else int(ts.max()))
    sh = _shard_ref(key, mask, g)
    for s, (t, k, v, y) in enumerate(parts):
        sel = np.flatnonzero(sh == s)
        np.testing.assert_array_equal(t, ts[sel])
        np.testing.assert_array_equal(k, key[sel])
        np.testing.assert_array_equal(v.view(np.uint32), val[sel].view(np.uint32))
        np.testing.assert_array_equal(y, typ[sel])
    assert sum(len(p[0]) for p in parts) == n


def _batches(seed, nb=6, n=4000, card=300, lateness_jitter=0, float_values=False):
    rng = np.random.default_rng(seed)
    out, t0 = [], 0
    for _ in range(nb):
        ts = synth.monotone_ts(rng, n, t0, max_gap=3)
        if lateness_jitter:
            ts = synth.jitter_ts(rng, ts, lateness_jitter)
        t0 = int(ts.max()) + 1
        key = synth.uniform_keys(rng, n, card)
        # packed fields: field 0 (8 bits) = key % 256, field 1 (8 bits) = key // 256 % 4
        key = (key % 256) | (((key // 7) % 4) << 8)
        val = (synth.lognormal_values(rng, n) if float_values
               else synth.int_values(rng, n, -500, 500))
        out.append(synth.Batch(ts.astype(np.int64), key.astype(np.uint32), val,
                               synth.type_column(rng, n)))
    # an empty batch in the middle
    out.insert(3, synth.Batch(np.zeros(0, np.int64), np.zeros(0, np.uint32),
                              out[0].value[:0], np.zeros(0, np.uint8)))
    return out


QUERIES = [
    dict(size_ms=1000),
    dict(size_ms=800, slide_ms=200, filter_col="value", filter_op="gt", filter_value=0),
    dict(size_ms=600, slide_ms=300, group_fields=1, having=("count", "ge", 3),
         order_by=("sum", True)),
    dict(size_ms=500, filter_col="type", filter_op="ne", filter_value=1, order_by=("avg", False)),
]


def _run(stream, batches, queries, join=True):
    qids = [stream.register_query(**q) for q in queries]
    jid = stream.register_join(400, 200, ("type", "eq", 0), ("type", "ne", 0)) if join else None
    rows = [[] for _ in qids]
    jrows = []
    for i, b in enumerate(batches):
        stream.push(b.ts, b.key, b.value, b.type, eos=(i == len(batches) - 1))
        for j, q in enumerate(qids):
            rows[j].append(stream.poll(q))
        if join:
            jrows.append(stream.poll_join(jid))
    return rows, jrows


@pytest.mark.parametrize("g", [1, 2, 3, 5])
@pytest.mark.parametrize("float_values", [False, True])
def test_sharded_stream_equals_one_stream(g, float_values):
    vt = "float32" if float_values else "int32"
    batches = _batches(11 + g, float_values=float_values, lateness_jitter=40)
    kw = dict(value_type=vt, allowed_lateness_ms=25, key_fields=(8, 8))
    ref_rows, ref_join = _run(OracleShard(**kw), batches, QUERIES)
    # every query groups by field 0 at least, so shard by field 0's bits
    sh = sharded.ShardedStream([OracleShard(**kw) for _ in range(g)], key_mask=0xFF)
    got_rows, got_join = _run(sh, batches, QUERIES)
    total = 0
    for q in range(len(QUERIES)):
        for b, (a, e) in enumerate(zip(got_rows[q], ref_rows[q])):
            assert a.tobytes() == e.tobytes(), (q, b)
            total += len(e)
    assert total > 1000
    for a, e in zip(got_join, ref_join):
        assert a.tobytes() == e.tobytes()
    assert sum(len(e) for e in ref_join) > 100


def _dist_worker(rank, world, port, q, float_values):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        vt = "float32" if float_values else "int32"
        kw = dict(value_type=vt, allowed_lateness_ms=25, key_fields=(8, 8))
        batches = _batches(29, float_values=float_values, lateness_jitter=40)
        ds = sharded.DistShardedStream(OracleShard(**kw), key_mask=0xFF)
        qids = [ds.register_query(**qq) for qq in QUERIES]
        got = [[] for _ in qids]
        recv = 0
        for i, b in enumerate(batches):
            # each rank's source holds every other row (rank 1 gets nothing of batch 1)
            sel = np.arange(len(b.ts)) % world == rank
            if i == 1:
                sel[:] = rank == 0
            recv += ds.push(b.ts[sel], b.key[sel], b.value[sel], b.type[sel],
                            eos=(i == len(batches) - 1))
            for j, qid in enumerate(qids):
                got[j].append(ds.gather(qid))
        q.put((rank, recv, got if rank == 0 else None))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("float_values", [False, True])
def test_two_gloo_ranks_shard_like_one_stream(float_values):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    procs = [ctx.Process(target=_dist_worker, args=(r, 2, port, q, float_values))
             for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in procs], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    batches = _batches(29, float_values=float_values, lateness_jitter=40)
    assert res[0][1] + res[1][1] == sum(len(b.ts) for b in batches)
    assert min(res[0][1], res[1][1]) > 0
    vt = "float32" if float_values else "int32"
    ref, _ = _run(OracleShard(value_type=vt, allowed_lateness_ms=25, key_fields=(8, 8)),
                  batches, QUERIES, join=False)
    got = res[0][2]
    for qi in range(len(QUERIES)):
        for b in range(len(batches)):
            a, e = got[qi][b], ref[qi][b]
            assert len(a) == len(e), (qi, b)
            for f in ("window_start", "key", "count", "min", "max"):
                np.testing.assert_array_equal(a[f], e[f])
            if float_values:
                # the exchange reorders a key's rows (rank 0's source first), so
                # float sums may differ by rounding: values are positive here
                np.testing.assert_allclose(a["sum"], e["sum"], rtol=1e-12)
                np.testing.assert_allclose(a["avg"], e["avg"], rtol=1e-12)
            else:
                np.testing.assert_array_equal(a["sum"], e["sum"])
                np.testing.assert_array_equal(a["avg"], e["avg"])


def test_restore_rejects_a_buffer_that_is_not_a_snapshot():
    # the header is checked before any device call
    for blob in (b"", b"LMSSNAP\0" + b"\0" * 8, b"x" * 4096):
        with pytest.raises(lm.LmsError) as e:
            lm.Stream.restore(blob)
        assert e.value.status == lm.LMS_EINVAL
