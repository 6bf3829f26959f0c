"""The C ABI library builds, loads, and exports every symbol include/muca.h declares
(no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "muca.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(muca_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1707_00919_gb300 import build
    build.build()
    from paper_1707_00919_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_every_symbol():
    from paper_1707_00919_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_symbols()


def test_default_params_and_errors_without_gpu(lib):
    from paper_1707_00919_gb300 import _lib
    p = _lib.muca_params()
    assert lib.muca_default_params(ctypes.byref(p)) == 0
    assert p.flat_threshold == 0.8 and p.f_therm == 30.0 and p.z == 2.25 and p.growth == 1.1
    assert lib.muca_default_params(None) == _lib.MUCA_EINVAL
    assert b"NULL" in lib.muca_last_error()
    # argument validation happens before any device call
    h = ctypes.c_void_p()
    assert lib.muca_create(6, 10, 1, ctypes.byref(h)) == _lib.MUCA_EINVAL
    assert lib.muca_create(68, 10, 1, ctypes.byref(h)) == _lib.MUCA_EINVAL
    assert lib.muca_create(8, 0, 1, ctypes.byref(h)) == _lib.MUCA_EINVAL
    assert lib.muca_create(8, -2, 1, ctypes.byref(h)) == _lib.MUCA_EINVAL
    assert lib.muca_sweep(None, 1, 0) == _lib.MUCA_EINVAL
    n, wpb = ctypes.c_int64(), ctypes.c_int32()
    assert lib.muca_optimal_walkers(6, 0, ctypes.byref(n), ctypes.byref(wpb)) == _lib.MUCA_EINVAL
    assert lib.muca_optimal_walkers(32, _lib.MUCA_LAYOUT_AUTO, ctypes.byref(n), None) == _lib.MUCA_EINVAL
    assert lib.muca_optimal_walkers(32, 0, None, None) == _lib.MUCA_EINVAL


def test_checkpoint_files_are_checked_without_gpu(lib, tmp_path):
    """muca_load reads and checks the file before it touches the device."""
    import ctypes
    from paper_1707_00919_gb300 import _lib
    h = ctypes.c_void_p()
    missing = str(tmp_path / "none.muca").encode()
    assert lib.muca_load(missing, ctypes.byref(h)) == _lib.MUCA_EIO
    junk = tmp_path / "junk.muca"
    junk.write_bytes(b"NOTMUCA!" + bytes(64))
    assert lib.muca_load(str(junk).encode(), ctypes.byref(h)) == _lib.MUCA_EIO
    short = tmp_path / "short.muca"
    short.write_bytes(b"MUCACKP1" + bytes(10))
    assert lib.muca_load(str(short).encode(), ctypes.byref(h)) == _lib.MUCA_EIO
    bad_l = tmp_path / "bad_l.muca"
    import struct
    bad_l.write_bytes(b"MUCACKP1" + struct.pack("<iiqQiiQq", 6, 0, 10, 1, 0, 0, 0, 0))
    assert lib.muca_load(str(bad_l).encode(), ctypes.byref(h)) == _lib.MUCA_EIO
    # the current format carries the iteration state after first_walker
    head = b"MUCACKP2" + struct.pack("<iiqQiiQq", 8, 0, 2, 1, 32, 0, 0, 0)
    for state, ok in [((0, -1, -1, 0), True), ((65, 0, 64, 1), True), ((3, 5, 4, 0), False),
                      ((2, 64, 65, 0), False), ((4, 1, 2, 0), False), ((3, 0, 2, 2), False)]:
        f = tmp_path / "v2.muca"
        f.write_bytes(head + struct.pack("<iiiiQ", *state, 7) + bytes(16))   # body cut short
        rc = lib.muca_load(str(f).encode(), ctypes.byref(h))
        assert rc == _lib.MUCA_EIO, state
        assert ("truncated" in lib.muca_last_error().decode()) == ok, state
    assert lib.muca_load(None, ctypes.byref(h)) == _lib.MUCA_EINVAL
    assert not h.value


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1707_00919_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()
