"""TEST INFRASTRUCTURE ONLY: CPU oracles for the LMStream hot path.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package.  The engine (`paper_2111_04289_b300`) never imports it
and shares no code with it.

Contents
  window_agg   per-event windowed group-by aggregation (C++, built with g++)
  control      the paper's cost models and algorithms (Eqs. 3-9, Alg. 1, Alg. 2)
  mlp          fp64 forward/backward of the learned latency model
"""
