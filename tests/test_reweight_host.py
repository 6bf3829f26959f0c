"""muca_reweight is host-only arithmetic in the product library: it must agree with the
oracle's reweighting (itself pinned against enumeration) on exact and perturbed ln g."""
import numpy as np
import pytest

from conftest import load_exact_ln_dos


@pytest.fixture(scope="module")
def M():
    from paper_1707_00919_gb300 import build
    build.build()
    from paper_1707_00919_gb300 import muca
    return muca


@pytest.mark.parametrize("L", [4, 8, 16, 32, 64])
def test_reweight_matches_oracle(M, orc, L):
    lg = load_exact_ln_dos(L)
    rng = np.random.default_rng(L)
    noisy = np.where(np.isfinite(lg), lg + rng.normal(0, 0.05, lg.size), -np.inf)
    betas = np.array([0.0, 0.1, 0.3, 0.4406868, 0.6, 1.0])
    for g in (lg, noisy):
        e, c = M.muca_reweight(L, g, betas)
        for i, b in enumerate(betas):
            eo, co = orc.canonical(L, g, b)
            assert e[i] == pytest.approx(eo, rel=1e-12, abs=1e-14)
            assert c[i] == pytest.approx(co, rel=1e-10, abs=1e-14)


def test_reweight_rejects_bad_input(M):
    with pytest.raises(M.MucaError):
        M.muca_reweight(8, np.zeros(10), [0.1])
    with pytest.raises(M.MucaError):
        M.muca_reweight(4, np.full(17, -np.inf), [0.1])
