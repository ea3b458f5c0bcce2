"""Fused-pass variant choice on the GPU (Alg. 2 and Eq. 9 re-read, and the
learned chooser): on the fused eight-query mix over uneven batch sizes, every
policy (static variant 1 or 2, the timing autotuner, the analytic chooser, the
learned chooser) gives the oracle's rows; the choosers see every pass and
their picks cover both variants."""
import numpy as np
import pytest

from paper_2111_04289_b300 import lmstream as lm
from paper_2111_04289_b300 import synth
from tests.engine_helpers import assert_rows_match, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

QUERIES = [dict(size=1_000), dict(size=10_000), dict(size=30_000, slide=1_000),
           dict(size=1_000, col="value", op="gt", value=10.24),
           dict(size=10_000, col="value", op="gt", value=3.602),
           dict(size=30_000, slide=1_000, col="value", op="gt", value=1.0),
           dict(size=1_000, col="value", op="gt", value=0.2776),
           dict(size=60_000, slide=5_000, col="value", op="gt", value=0.5)]


def _batches():
    rng = np.random.default_rng(301)
    s = synth.LargeFloatStream(seed=302, card=10_000, s=1.3, max_gap=1)
    return [s.next_batch(int(2 ** rng.uniform(12, 18))) for _ in range(14)]


def _run(batches, policy):
    s = lm.Stream("float32", enable_timing=True,
                  k1_variant={"static1": 1, "static2": 2}.get(policy, 0))
    for q in QUERIES:
        s.register_query(q["size"], q.get("slide", 0), q.get("col", "ts"), q.get("op", "none"),
                         q.get("value", 0))
    chooser = None
    if policy == "analytic":
        chooser = lm.VariantAnalytic(148, 16.0, explore=2)
    elif policy == "learned":
        judge = lm.VariantAnalytic(148, 16.0, explore=2)
        net = lm.Mlp(lm.mlp_init_params(7))
        chooser = lm.VariantLearned(net, judge, key_card=10_000, selectivity=0.5, panes=12,
                                    n_queries=8)
        chooser.set_online(refit_every=4, refit_steps=50)
        chooser._keep = (judge, net)
    if chooser is not None:
        s.set_variant_chooser(chooser)
    out = [[] for _ in QUERIES]
    for i, b in enumerate(batches):
        s.push(b.ts, b.key, b.value, eos=i == len(batches) - 1)
        for j in range(len(QUERIES)):
            out[j].append(s.poll(j))
    st = s.stats()
    s.close()
    return [np.concatenate(r) for r in out], st, chooser


@pytest.mark.parametrize("policy", ["static1", "static2", "autotune", "analytic", "learned"])
def test_every_variant_policy_gives_the_oracle_rows(policy):
    batches = _batches()
    eng, st, chooser = _run(batches, policy)
    orc, _ = run_oracle(batches, QUERIES, True)
    for j in range(len(QUERIES)):
        assert_rows_match(eng[j], orc[j], True, ctx=f"{policy} query {j}")
    if policy == "analytic":
        picks = chooser.state()["picks"]
        assert sum(picks) == st["k1_launches"] and min(picks) >= 2  # both explored
        assert chooser.state()["infpt_bytes"] > 0
    if policy == "learned":
        sts = chooser.stats()
        assert sum(sts["picks"]) == st["k1_launches"] and min(sts["picks"]) >= 1
        assert sts["uses_net"] + sts["uses_analytic"] == st["k1_launches"]
        assert sts["uses_net"] > 0  # the network was trained online and answered
