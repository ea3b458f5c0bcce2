"""The ingest ring (lms_ingest / lms_push_ingested): datasets copied to the
device on a side stream as they arrive, then pushed as micro-batches.  The rows
equal the oracle's for the same batch boundaries whatever the dataset sizes,
with the rings wrapping around and growing while rows are held, for datasets
copied through the library's pinned ring and for stable pinned ones; misuse
is rejected."""
import numpy as np
import pytest

from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import synth
from tests.engine_helpers import assert_rows_match, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = [dict(size=2_000, slide=500, col="value", op="gt", value=0.5), dict(size=700)]


def _datasets(seed, n_sets):
    rng = np.random.default_rng(seed)
    s = synth.LargeFloatStream(seed=seed + 1, card=5_000, s=1.2)
    return [s.next_batch(int(rng.integers(1, 9000))) for _ in range(n_sets)]


def _run_ingested(sets, cuts, stable):
    s = lm.Stream("float32")
    for q in Q:
        s.register_query(q["size"], q.get("slide", 0), q.get("col", "ts"), q.get("op", "none"),
                         q.get("value", 0))
    out = [[] for _ in Q]
    held = []  # pinned copies for stable ingests
    i = 0
    for k, c in enumerate(cuts):  # c datasets per micro-batch
        n = 0
        for b in sets[i:i + c]:
            if stable:
                cols = [torch.from_numpy(x).pin_memory() for x in (b.ts, b.key, b.value)]
                held.append(cols)
                s.ingest(*cols, stable=True)
            else:
                s.ingest(b.ts, b.key, b.value)
            n += len(b)
        i += c
        assert s.ingest_pending() == n
        s.push_ingested(n, eos=k == len(cuts) - 1)
        for j in range(len(Q)):
            out[j].append(s.poll(j))
    st = s.stats()
    s.close()
    return [np.concatenate(r) for r in out], st


@pytest.mark.parametrize("stable", [False, True])
def test_ingested_batches_equal_the_oracle(stable):
    sets = _datasets(91, 60)
    rng = np.random.default_rng(92)
    cuts = []
    left = len(sets)
    while left:
        c = int(min(left, rng.integers(1, 9)))
        cuts.append(c)
        left -= c
    eng, st = _run_ingested(sets, cuts, stable)
    bounds = np.concatenate([[0], np.cumsum(cuts)])
    batches = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        part = sets[a:b]
        batches.append(synth.Batch(np.concatenate([p.ts for p in part]),
                                   np.concatenate([p.key for p in part]),
                                   np.concatenate([p.value for p in part])))
    orc, late = run_oracle(batches, Q, True)
    for j in range(len(Q)):
        assert_rows_match(eng[j], orc[j], True, ctx=f"query {j}")
    assert st["late_rows"] == sum(late)


def test_ring_wraps_and_grows_while_rows_are_held():
    """Datasets ingested ahead of the pushes (the ring holds several batches),
    sizes chosen so that batches straddle the ring's end and the ring grows
    with rows in it."""
    sets = _datasets(93, 40)
    s = lm.Stream("float32")
    s.register_query(2_000, 500, "value", "gt", 0.5)
    pushed = []
    queue = []
    for k, b in enumerate(sets):
        s.ingest(b.ts, b.key, b.value)
        queue.append(len(b))
        if len(queue) >= 3 and k % 2 == 0:  # push two datasets, keep the rest held
            n = queue.pop(0) + queue.pop(0)
            s.push_ingested(n)
            pushed.append(n)
    rest = sum(queue)
    s.push_ingested(rest, eos=True)
    pushed.append(rest)
    eng = s.poll(0)
    s.close()
    allb = synth.Batch(np.concatenate([b.ts for b in sets]), np.concatenate([b.key for b in sets]),
                       np.concatenate([b.value for b in sets]))
    bounds = np.concatenate([[0], np.cumsum(pushed)])
    batches = [allb.slice(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:])]
    orc, _ = run_oracle(batches, Q[:1], True)
    assert_rows_match(eng, orc[0], True)


def test_ingest_misuse_is_rejected():
    s = lm.Stream("int32")
    s.register_query(1000)
    b = synth.TinyIntStream(seed=94).next_batch(500)
    s.ingest(b.ts, b.key, b.value)
    with pytest.raises(lm.LmsError) as ei:
        s.push(b.ts, b.key, b.value)  # ingested rows pending
    assert ei.value.status == lm.LMS_EINVAL
    with pytest.raises(lm.LmsError) as ei:
        s.push_ingested(501)
    assert ei.value.status == lm.LMS_EINVAL
    s.push_ingested(500, eos=True)
    with pytest.raises(lm.LmsError) as ei:
        s.ingest(b.ts, b.key, b.value)
    assert ei.value.status == lm.LMS_ECLOSED
    s.close()
