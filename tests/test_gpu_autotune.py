"""The autotuner measures (nb, schedule) candidates and caches the choice."""
import json
import time

import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,cands", [("fp64", {32, 64, 128, 256, 512, 1024}), ("fp32", {128, 256, 512})])
def test_autotune_picks_a_candidate_and_caches(tmp_path, prec, cands):
    import paper_2606_11937_gb300 as chol
    path = str(tmp_path / "tune.json")
    o = chol.chol_autotune(1536, prec, path, budget_s=20.0)
    assert o.nb in cands and o.schedule in (chol.CHOL_SCHED_DATAFLOW, chol.CHOL_SCHED_FORK_JOIN)
    t = time.perf_counter()
    o2 = chol.chol_autotune(1536, prec, path, budget_s=20.0)
    assert time.perf_counter() - t < 0.5          # served from the cache
    assert (o2.nb, o2.schedule) == (o.nb, o.schedule)
    data = json.load(open(path))
    assert any(e["nb"] == o.nb for e in data["entries"])
