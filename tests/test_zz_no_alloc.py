"""The allocation-free batched sweep (muca_batch_sweep_noalloc), for callers that must
not allocate device memory while they run: it works on device buffers the caller owns
and keeps its own scratch in a fixed device array.  Its results must equal those of the
ordinary batched sweep (muca_batch_sweep) on the same state, exactly (integer work), over
two calls in a row.  Collected last so that a failure here comes after every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1707_00919_gb300 import _lib, muca
    return torch, muca, _lib


def to_layout(lat, L, layout):
    """int8 spins [walker][site] -> the device layout of include/muca.h."""
    if layout == 0:
        return np.ascontiguousarray(lat.T)                       # [site][walker]
    W = lat.shape[0]
    bits = (lat.reshape(W, L, L) < 0).astype(np.uint64)          # [walker][y][x]
    rows = (bits << np.arange(L, dtype=np.uint64)).sum(axis=2)   # [walker][y]
    rows = np.ascontiguousarray(rows.T)                          # [y][walker]
    return rows.astype(np.uint32) if L <= 32 else rows


def from_layout(buf, L, layout, W):
    if layout == 0:
        return np.ascontiguousarray(buf.reshape(L * L, W).T)
    rows = buf.reshape(L, W).astype(np.uint64).T                 # [walker][y]
    bits = (rows[:, :, None] >> np.arange(L, dtype=np.uint64)) & 1
    return np.where(bits.reshape(W, L * L) == 1, -1, 1).astype(np.int8)


def weights(L, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.normal(0.0, 0.4, L * L + 1))


def raw_copy(torch, C, m, L, W, layout, seed):
    """Caller-owned device buffers holding the same state as instance m."""
    dev = "cuda"
    host = to_layout(m.get_lattice(), L, layout)
    if host.dtype == np.uint64:
        host = host.view(np.int64)
    elif host.dtype == np.uint32:
        host = host.view(np.int32)
    bufs = {
        "lattice": torch.from_numpy(host).to(dev),
        "energy": torch.from_numpy(m.get_energies()).to(dev),
        "table": torch.from_numpy(m.get_table().view(np.int32)).to(dev),
        "hist": torch.zeros(L * L + 1, dtype=torch.int64, device=dev),
        "err": torch.zeros(1, dtype=torch.int32, device=dev),
    }
    r = C.muca_raw_instance(L, layout, W, seed, 0, bufs["lattice"].data_ptr(), bufs["energy"].data_ptr(),
                            bufs["table"].data_ptr(), bufs["hist"].data_ptr(), bufs["err"].data_ptr())
    return r, bufs


def test_noalloc_matches_batched_sweep(env):
    torch, M, C = env
    specs = [(8, 33, 1), (16, 100, 0), (32, 257, 1), (48, 40, 0), (64, 70, 1)]
    inst, raws, bufs = [], [], []
    for i, (L, W, lay) in enumerate(specs):
        m = M.Muca(L, W, 500 + i, layout=lay)
        m.set_weights(weights(L, i))
        r, b = raw_copy(torch, C, m, L, W, lay, 500 + i)
        inst.append(m)
        raws.append(r)
        bufs.append(b)
    torch.cuda.synchronize()
    with M.Batch(inst) as batch:
        for n_sweeps, record in [(1, False), (2, True)]:       # two calls in a row, both paths
            if record:
                for m in inst:
                    m.reset_histogram()
            batch.sweep(n_sweeps, record)
            M.muca_batch_sweep_noalloc(raws, n_sweeps, record)
            for (L, W, lay), r in zip(specs, raws):
                r.t0 += n_sweeps * L * L
        torch.cuda.synchronize()
        for (L, W, lay), m, r, b in zip(specs, inst, raws, bufs):
            assert m.attempt_counter == r.t0
            buf = b["lattice"].cpu().numpy()
            if lay == 1:
                buf = buf.view(np.uint32 if L <= 32 else np.uint64)
            assert np.array_equal(from_layout(buf, L, lay, W), m.get_lattice()), (L, W, lay)
            assert np.array_equal(b["energy"].cpu().numpy(), m.get_energies()), (L, W, lay)
            assert np.array_equal(b["hist"].cpu().numpy().view(np.uint64), m.get_histogram()), (L, W, lay)
            assert int(b["err"].item()) == 0
    for m in inst:
        m.close()


def test_noalloc_rejects_sizes_beyond_its_limits(env):
    torch, M, C = env
    L, W = 16, 64
    with M.Muca(L, W, 9) as m:
        r, b = raw_copy(torch, C, m, L, W, 0, 9)
        with pytest.raises(M.MucaError) as ex:
            M.muca_batch_sweep_noalloc([r] * (C.MUCA_NOALLOC_MAX_INSTANCES + 1), 1, False)
        assert ex.value.code == C.MUCA_EINVAL
        with pytest.raises(M.MucaError) as ex:
            M.muca_batch_sweep_noalloc([r], 0xFFFFFFFF // 256 // (L * L) + 1, True)
        assert ex.value.code == C.MUCA_EINVAL
        with pytest.raises(M.MucaError) as ex:       # the same buffers twice in one call
            M.muca_batch_sweep_noalloc([r, r], 1, False)
        assert ex.value.code == C.MUCA_EINVAL
        r.t0 = 5
        with pytest.raises(M.MucaError):
            M.muca_batch_sweep_noalloc([r], 1, False)


def test_noalloc_flags_an_energy_off_the_grid(env):
    """A walker whose stored energy index lies outside 0..L*L sets the error word's
    energy bit and is left untouched (no table read, lattice and energy kept); the
    instance's other walkers and the other instances sweep exactly as before."""
    torch, M, C = env
    specs = [(16, 64, 0, 5, -1), (32, 100, 1, 99, 32 * 32 + 1), (24, 100, 0, 97, 10 ** 6), (8, 33, 0, None, 0)]
    inst, raws, bufs, before = [], [], [], []
    for i, (L, W, lay, bad, val) in enumerate(specs):
        m = M.Muca(L, W, 800 + i, layout=lay)
        m.set_weights(weights(L, 10 + i))
        r, b = raw_copy(torch, C, m, L, W, lay, 800 + i)
        if bad is not None:
            b["energy"][bad] = val
        before.append((b["lattice"].cpu().numpy().copy(), b["energy"].cpu().numpy().copy()))
        inst.append(m)
        raws.append(r)
        bufs.append(b)
    torch.cuda.synchronize()
    with M.Batch(inst) as batch:
        for m in inst:
            m.reset_histogram()
        batch.sweep(2, True)
        M.muca_batch_sweep_noalloc(raws, 2, True)
        torch.cuda.synchronize()
        for (L, W, lay, bad, val), m, b, (lat0, en0) in zip(specs, inst, bufs, before):
            buf = b["lattice"].cpu().numpy()
            view = (lambda x: x.view(np.uint32 if L <= 32 else np.uint64)) if lay == 1 else (lambda x: x)
            got, ref = from_layout(view(buf), L, lay, W), m.get_lattice()
            en = b["energy"].cpu().numpy()
            err = int(b["err"].item())
            keep = np.ones(W, bool)
            if bad is None:
                assert err == 0
                assert np.array_equal(b["hist"].cpu().numpy().view(np.uint64), m.get_histogram())
            else:
                assert err == 1, (L, err)
                keep[bad] = False
                assert np.array_equal(got[bad], from_layout(view(lat0), L, lay, W)[bad])
                assert en[bad] == en0[bad] == val
                assert not np.array_equal(got[keep], from_layout(view(lat0), L, lay, W)[keep])
            assert np.array_equal(got[keep], ref[keep]), (L, W, lay)
            assert np.array_equal(en[keep], m.get_energies()[keep]), (L, W, lay)
    for m in inst:
        m.close()


def test_noalloc_energies_that_do_not_match_the_lattices(env, orc):
    """Caller-owned energies inside 0..L*L that do not match the lattices (the ground and
    top energies, shifted ones): the sweep keeps every threshold load inside the table
    (the candidates of a decision lie within two rows of the current energy, and the
    table has zero rows around the grid), flips that would leave the grid are rejected,
    and lattices, energies and histogram equal the oracle's run on the same inputs."""
    torch, M, C = env
    for L, W, lay, seed in [(16, 64, 0, 31), (32, 100, 1, 32), (24, 40, 0, 33), (8, 50, 0, 34), (64, 40, 1, 35)]:
        N = L * L
        with M.Muca(L, W, seed, layout=lay) as m:
            m.set_weights(weights(L, seed))
            m.sweep(1, False)
            r, b = raw_copy(torch, C, m, L, W, lay, seed)
            r.t0 = N
            e_true = m.get_energies()
            bad = np.where(np.arange(W) % 3 == 0, 0, np.where(np.arange(W) % 3 == 1, N, (e_true + 37) % (N + 1)))
            bad = bad.astype(np.int32)
            b["energy"].copy_(torch.from_numpy(bad))
            s, T = m.get_lattice(), m.get_table()
            torch.cuda.synchronize()
            M.muca_batch_sweep_noalloc([r], 2, True)
            torch.cuda.synchronize()
            buf = b["lattice"].cpu().numpy()
            if lay == 1:
                buf = buf.view(np.uint32 if L <= 32 else np.uint64)
            got = from_layout(buf, L, lay, W)
        eo = bad.copy()
        Ho = orc.run(L, seed, s, eo, T, N, 2 * N, True)
        assert int(b["err"].item()) == 0
        assert np.array_equal(got, s), L
        assert np.array_equal(b["energy"].cpu().numpy(), eo), L
        assert np.array_equal(b["hist"].cpu().numpy().view(np.uint64), Ho), L
