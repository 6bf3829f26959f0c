"""Serving with continuous batching: requests of different L and walker counts arrive
while others run, are admitted under a memory budget and iterated together; each result
must equal the same request run alone (muca_iterate_until_flat), bit for bit, and the
oracle's weight iteration of the same request (Sec. 2.2, Eq. 4)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import muca
    return muca


SPECS = [(8, 128, 1, 100), (16, 1024, 2, 40), (8, 256, 3, 100), (24, 2048, 4, 20), (16, 512, 5, 60),
         (32, 4096, 6, 10)]


def params(M, S):
    return M.make_params(therm_sweeps=31, sweeps_per_iter=S, max_iterations=400)


def test_requests_alone_and_in_the_mix_agree(M, orc):
    alone = []
    for L, W, seed, S in SPECS:
        with M.Muca(L, W, seed) as m:
            st = m.iterate_until_flat(params(M, S))
            alone.append((st, m.get_weights()))
    # the L = 32 request (4.24 MB on the device) fits this budget only once the L = 24
    # request (1.2 MB) has left, so it arrives while others run and has to wait
    budget = 4_300_000
    with M.Server(budget) as srv:
        ids = []
        arrivals = {0: [0, 1], 2: [2], 3: [3, 4], 6: [5]}   # step -> requests arriving before it
        step = 0
        max_queue = 0
        while True:
            for k in arrivals.get(step, []):
                L, W, seed, S = SPECS[k]
                ids.append((k, srv.submit(L, W, seed, params(M, S))))
            active, queued = srv.step()
            max_queue = max(max_queue, queued)
            step += 1
            if step > 7 and active == 0 and queued == 0:
                break
            assert step < 5000
        assert max_queue >= 1                           # admission really waited for memory
        for k, rid in ids:
            L, W, seed, S = SPECS[k]
            st = srv.status(rid)
            assert st.state == M.C.MUCA_REQ_DONE
            ref, lnW = alone[k]
            assert st.stats.iterations == ref.iterations
            assert bool(st.stats.converged) == ref.converged
            assert st.stats.last_metric == ref.last_metric
            assert np.array_equal(srv.weights(rid, L * L + 1), lnW)
            assert st.seconds_total >= st.seconds_queued >= 0.0
        att, sec, steps, used = srv.totals()
        assert used == 0 and att > 0
        # two served requests of different L against the oracle's iteration: iteration
        # count, last stop metric and final ln W bit for bit
        for k in (0, 4):
            L, W, seed, S = SPECS[k]
            rid = dict(ids)[k]
            s, e = orc.init(L, seed, W)
            lnW = np.zeros(L * L + 1)
            p = orc.make_params(schedule=0, stop_rule=0, flat_threshold=0.8, therm_sweeps=31,
                                sweeps_per_iter=S, max_iterations=400)
            res, _, _, _ = orc.iterate(L, seed, s, e, lnW, 0, p)
            st = srv.status(rid)
            assert st.stats.iterations == res.iterations and bool(st.stats.converged) == bool(res.converged)
            assert st.stats.last_metric == res.last_metric
            assert np.array_equal(srv.weights(rid, L * L + 1), lnW), (L, W)


def test_paper_schedule_requests_alone_and_in_the_mix(M):
    """Requests with the Eq. (7) schedule (each member grows its own update counts) are
    served together and each equals the same request run alone, bit for bit."""
    specs = [(8, 64, 31), (16, 256, 32), (24, 512, 33), (8, 128, 34)]
    p = M.make_params(schedule=M.MUCA_SCHEDULE_PAPER, stop_rule=M.MUCA_STOP_MIN_MEAN, flat_threshold=0.8,
                      max_iterations=500)
    alone = []
    for L, W, seed in specs:
        with M.Muca(L, W, seed) as m:
            st = m.iterate_until_flat(p)
            alone.append((st, m.get_weights()))
    with M.Server(1 << 30) as srv:
        ids = [srv.submit(L, W, seed, p) for L, W, seed in specs[:2]]
        active, _ = srv.step()
        ids += [srv.submit(L, W, seed, p) for L, W, seed in specs[2:]]   # arrive while others run
        for _ in range(5000):
            active, queued = srv.step()
            if active == 0 and queued == 0:
                break
        for k, rid in enumerate(ids):
            L, W, seed = specs[k]
            st = srv.status(rid)
            ref, lnW = alone[k]
            assert st.state == M.C.MUCA_REQ_DONE and st.stats.converged == ref.converged
            assert st.stats.iterations == ref.iterations and st.stats.last_metric == ref.last_metric
            assert st.stats.attempts_per_walker == ref.attempts_per_walker
            assert np.array_equal(srv.weights(rid, L * L + 1), lnW)


def test_server_rejects_bad_requests(M):
    with M.Server(1 << 20) as srv:
        with pytest.raises(M.MucaError):
            srv.submit(12, 64, 1, params(M, 10))                  # no whole-sweep kernel
        with pytest.raises(M.MucaError) as ex:
            srv.submit(64, 1 << 20, 1, params(M, 1))              # larger than the budget
        assert ex.value.code == M.C.MUCA_ENOMEM
