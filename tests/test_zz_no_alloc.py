"""GPU test of lms_aggregate_batch_static, the entry point for callers that may
not allocate device memory (e.g. a plug-in whose host process owns the device
memory budget).  It must give the same rows as the stream API — one
push_microbatch with end-of-stream, then poll_results — on two calls in a row
(the second call runs on the fixed scratch the first one left behind).

This file is collected last on purpose: it needs nothing from the other tests,
passes alone in a fresh process, and runs after them in a full `-m gpu` run."""
import numpy as np
import pytest

from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import synth
from tests.engine_helpers import FLOAT_REL_TOL, assert_rows_match, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "float_sliding": dict(value_type="float32", size_ms=60_000, slide_ms=5_000,
                          filter_col="value", filter_op="gt", filter_value=0.5),
    "int_tumbling": dict(value_type="int32", size_ms=10_000, slide_ms=0,
                         filter_col="type", filter_op="eq", filter_value=0),
}


def _batches(name):
    if name == "float_sliding":
        g = synth.LargeFloatStream(seed=synth.BASE_SEED + 301)
        return [g.next_batch(60_000), g.next_batch(90_001)]
    g = synth.TinyIntStream(seed=synth.BASE_SEED + 302)
    return [g.next_batch(65_536), g.next_batch(12_345)]


def _via_stream(b, spec):
    s = lm.Stream(spec["value_type"], has_type=b.type is not None)
    qid = s.register_query(spec["size_ms"], spec["slide_ms"], spec["filter_col"],
                           spec["filter_op"], spec["filter_value"])
    s.push(b.ts, b.key, b.value, b.type, eos=True)
    rows = s.poll(qid)
    s.close()
    return rows


def _via_static(b, spec, side_stream=None):
    k = spec["size_ms"] // (spec["slide_ms"] or spec["size_ms"])
    cap = len(b) * k
    if side_stream is None:
        out = torch.zeros(cap * 48, dtype=torch.uint8, device="cuda")
        cols = [None if c is None else torch.from_numpy(np.ascontiguousarray(c)).cuda()
                for c in (b.ts, b.key, b.value, b.type)]
        n = lm.aggregate_batch_static(*cols, **spec, rows_ptr=out.data_ptr(), rows_cap=cap)
    else:
        # the columns are produced on a non-blocking side stream just before
        # the call, which is given that stream: the call must read them after
        # the copies that produce them
        with torch.cuda.stream(side_stream):
            out = torch.zeros(cap * 48, dtype=torch.uint8, device="cuda")
            host = [None if c is None else torch.from_numpy(np.ascontiguousarray(c)).pin_memory()
                    for c in (b.ts, b.key, b.value, b.type)]
            cols = [None if c is None else c.to("cuda", non_blocking=True) for c in host]
            n = lm.aggregate_batch_static(*cols, **spec, rows_ptr=out.data_ptr(), rows_cap=cap,
                                          cuda_stream=side_stream.cuda_stream)
        side_stream.synchronize()
    dt = lm.ROW_DTYPE_FLOAT if spec["value_type"] == "float32" else lm.ROW_DTYPE_INT
    return out[: n * 48].cpu().numpy().view(dt)


def _oracle_rows(b, spec):
    q = dict(size=spec["size_ms"], slide=spec["slide_ms"], col=spec["filter_col"],
             op=spec["filter_op"], value=spec["filter_value"])
    return run_oracle([b], [q], spec["value_type"] == "float32")[0][0]


@pytest.mark.parametrize("name", list(CASES))
def test_static_scratch_entry_point_matches_stream_api(name):
    spec = CASES[name]
    for b in _batches(name):  # two calls in a row
        ref = _via_stream(b, spec)
        got = _via_static(b, spec)
        assert_rows_match(got, _oracle_rows(b, spec), spec["value_type"] == "float32")
        assert len(got) == len(ref) > 0
        for f in ("window_start", "key", "count", "query_id"):
            np.testing.assert_array_equal(got[f], ref[f], err_msg=f)
        if spec["value_type"] == "float32":
            for f in ("min", "max"):
                np.testing.assert_array_equal(got[f].view(np.uint32), ref[f].view(np.uint32))
            for f in ("sum", "avg"):
                assert np.all(np.abs(got[f] - ref[f]) <= FLOAT_REL_TOL * np.abs(ref[f]))
        else:
            for f in ("sum", "min", "max", "avg"):
                np.testing.assert_array_equal(got[f], ref[f], err_msg=f)


@pytest.mark.parametrize("name", list(CASES))
def test_static_scratch_entry_point_on_a_non_blocking_stream(name):
    spec = CASES[name]
    side = torch.cuda.Stream()
    for b in _batches(name):  # two calls in a row
        got = _via_static(b, spec, side_stream=side)
        assert_rows_match(got, _oracle_rows(b, spec), spec["value_type"] == "float32")


def test_static_scratch_rejects_oversized_batch():
    n = lm.STATIC_MAX_ROWS + 1
    cols = [torch.zeros(n, dtype=t, device="cuda") for t in (torch.int64, torch.int32,
                                                            torch.int32)]
    out = torch.zeros(48, dtype=torch.uint8, device="cuda")
    with pytest.raises(lm.LmsError) as ei:
        lm.aggregate_batch_static(*cols, value_type="int32", size_ms=1000,
                                  rows_ptr=out.data_ptr(), rows_cap=1)
    assert ei.value.status == lm.LMS_EINVAL
