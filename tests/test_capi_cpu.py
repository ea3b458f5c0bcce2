"""CPU-only checks of the C ABI library: it builds, loads, exports every
function include/lmstream.h declares, its struct layouts match the header,
host-side helpers work, and opening a stream without a GPU fails cleanly."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2111_04289_b300 import build as lbuild
from paper_2111_04289_b300 import lmstream as lm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "lmstream.h")


def _declared_functions():
    inc = os.path.dirname(HEADER)
    src = "\n".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                    if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#ifdef __cplusplus.*?#endif", "", src, flags=re.S)  # extern "C" { and }
    src = re.sub(r"\{[^{}]*\}", "{}", src)  # struct bodies (function-pointer members)
    src = "\n".join(l for l in src.splitlines() if not l.lstrip().startswith("typedef"))
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_and_exports_all_declared_symbols():
    lbuild.build()
    lib = ctypes.CDLL(lbuild.LIB)
    decl = _declared_functions()
    assert {"stream_open", "query_register", "push_microbatch", "poll_results",
            "stream_close"} <= set(decl)
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) == set(lm.EXPORTED_SYMBOLS)


def test_struct_layouts_match_header():
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "lmstream.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(lms_stream_config), sizeof(lms_query_spec),
         sizeof(lms_batch), sizeof(lms_result_row), sizeof(lms_stats));
  printf("%zu %zu %zu %zu\n", offsetof(lms_result_row, avg), offsetof(lms_result_row, key),
         offsetof(lms_result_row, query_id), offsetof(lms_stream_config, cuda_stream));
  printf("%zu %zu %zu %zu %zu\n", sizeof(lms_serve_chunk), sizeof(lms_serve_batch),
         sizeof(lms_serve_backend), sizeof(lms_serve_config), sizeof(lms_serve_result));
  printf("%zu %zu %zu\n", offsetof(lms_serve_batch, h2d_ms), offsetof(lms_serve_config, quantile_hi),
         offsetof(lms_serve_result, max_backlog_events));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), "-o", exe, c])
        out = subprocess.check_output([exe]).decode().split()
    sizes = list(map(int, out))
    assert sizes[:5] == [ctypes.sizeof(lm.StreamConfig), ctypes.sizeof(lm.QuerySpec),
                         ctypes.sizeof(lm.BatchC), lm.ROW_DTYPE_INT.itemsize,
                         ctypes.sizeof(lm.StatsC)]
    assert sizes[3] == 48
    assert sizes[5:9] == [lm.ROW_DTYPE_INT.fields["avg"][1], lm.ROW_DTYPE_INT.fields["key"][1],
                          lm.ROW_DTYPE_INT.fields["query_id"][1],
                          lm.StreamConfig.cuda_stream.offset]
    assert sizes[9:14] == [ctypes.sizeof(x) for x in (lm.ServeChunk, lm.ServeBatch,
                                                      lm.ServeBackend, lm.ServeConfig,
                                                      lm.ServeResult)]
    assert sizes[14:] == [lm.ServeBatch.h2d_ms.offset, lm.ServeConfig.quantile_hi.offset,
                          lm.ServeResult.max_backlog_events.offset]


def test_invariant_division_matches_integer_division():
    rng = np.random.default_rng(5)
    ds = [1, 2, 3, 5, 7, 10, 1000, 1024, 5000, 60000, 86_400_000, 2**31 - 1, 2**32 - 1]
    ns = [0, 1, 2, 2**31, 2**32 - 1, 2**62, 2**63 - 1, 2**64 - 1] + [
        int(x) for x in rng.integers(0, 2**63 - 1, size=200, dtype=np.int64)]
    for d in ds + [int(x) for x in rng.integers(1, 2**32, size=30)]:
        for n in ns:
            assert lm.udiv_invariant(n, d) == n // d, (n, d)


def test_open_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lm.LmsError) as ei:
        lm.Stream("int32")
    assert ei.value.status == lm.LMS_ECUDA
