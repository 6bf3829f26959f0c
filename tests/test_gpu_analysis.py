"""Production statistics on the GPU path: the jackknife chunks equal the oracle's, the
jackknife errors equal the oracle's analysis of the same chunks, and at L = 16 the
production estimate and its canonical reweighting agree with the exact result."""
import numpy as np
import pytest

from conftest import load_exact_ln_dos

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


def test_jackknife_chunks_and_errors_match_oracle(M, orc):
    L, W, seed = 8, 128, 1
    N = L * L
    lg = load_exact_ln_dos(L)
    lnW = np.where(np.isfinite(lg), -lg, 0.0) + 0.01 * np.arange(N + 1)
    with M.Muca(L, W, seed) as m:
        m.set_weights(lnW)
        Hc, g, err = m.production_jackknife(31, 10, 20)
    s, e = orc.init(L, seed, W)
    T = orc.build_table(L, lnW)
    orc.run(L, seed, s, e, T, 0, 31 * N, False)
    ref = []
    for c in range(10):
        ref.append(orc.run(L, seed, s, e, T, (31 + 20 * c) * N, 20 * N, True))
    ref = np.array(ref)
    assert np.array_equal(Hc, ref)
    g_o, err_o = orc.jackknife(L, lnW, ref)
    fin = np.isfinite(g_o)
    assert np.array_equal(np.isfinite(g), fin)
    assert np.allclose(g[fin], g_o[fin], rtol=0, atol=1e-12)
    ok = np.isfinite(err_o)
    assert np.array_equal(np.isfinite(err), ok)
    assert np.allclose(err[ok], err_o[ok], rtol=1e-10, atol=1e-14)


def test_L16_production_errors_and_reweighting(M):
    L, W = 16, 4096
    N = L * L
    ex = load_exact_ln_dos(L)
    acc = np.isfinite(ex)
    with M.Muca(L, W, 1) as m:
        st = m.iterate_until_flat(M.make_params(therm_sweeps=31, sweeps_per_iter=20, max_iterations=500))
        assert st.converged
        Hc, g, err = m.production_jackknife(31, 20, 100)
    dev = np.abs(g[acc] - ex[acc])
    assert dev.max() < 0.05
    # the jackknife errors describe the actual deviations
    assert np.all(np.isfinite(err[acc]))
    assert 0.3 < np.median(err[acc]) / np.median(dev) < 3.0
    betas = [0.2, 0.3, 0.4406868, 0.5, 0.7]
    e_est, c_est = M.muca_reweight(L, g, betas)
    e_ex, c_ex = M.muca_reweight(L, ex, betas)
    assert np.max(np.abs(e_est - e_ex)) < 0.005
    assert np.max(np.abs(c_est - c_ex) / c_ex) < 0.03
