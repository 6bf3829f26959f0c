"""Per-iteration logs of the weight iteration (the convergence traces of App. A): the
JSON lines written through the iteration observer carry one record per iteration whose
flatness measure of the chosen stop rule equals the stop metric the iteration used, and
the schedule's attempt counts."""
import json

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def muca_mod():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca
    return muca


@pytest.mark.parametrize("rule,key,thr", [(0, "min_over_mean", 0.8), (1, "d_k", 0.01), (2, "d_c", 0.3)])
def test_iteration_log_lines(muca_mod, tmp_path, rule, key, thr):
    M = muca_mod
    L, W = 8, 128
    N = L * L
    p = M.make_params(stop_rule=rule, flat_threshold=thr, therm_sweeps=31, sweeps_per_iter=100, max_iterations=400)
    path = str(tmp_path / "trace.jsonl")
    with M.Muca(L, W, 4) as m:
        log = M.IterationLog(path, L, W)
        m.set_iteration_observer(log)
        st = m.iterate_until_flat(p)
        m.set_iteration_observer(None)
        log.close()
    recs = [json.loads(line) for line in open(path)]
    assert st.converged and len(recs) == st.iterations
    assert [r["iteration"] for r in recs] == list(range(1, st.iterations + 1))
    assert all(r["stop_metric"] == r[key] for r in recs)
    assert all(r["n_therm"] == 31 * N and r["n_updates"] == 100 * N for r in recs)
    assert all(0 < r["w"] <= N + 1 and r["attempts_per_s"] > 0 for r in recs)
    flat = (lambda v: v >= thr) if rule == 0 else (lambda v: v < thr)
    assert flat(recs[-1][key]) and not any(flat(r[key]) for r in recs[:-1])
    assert recs[-1]["w"] >= 10
