"""Host-side pieces of bench.py that need no GPU: the DRAM traffic read from a profile
summary is reported only while the summary's kernel-source hash matches the built
source, and the workload description names the measured configuration."""
import os

import bench


def _write_profile(path, digest, value):
    with open(path, "w") as f:
        f.write("# summary\n\n")
        f.write(f"- kernel_source_sha256_16: `{digest}`\n")
        f.write(f"- dram_bytes_per_step_launch: `{value}`\n")


def test_profiled_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    p = tmp_path / "profile.md"
    _write_profile(p, bench.kernel_source_hash(), 16950741)
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(p))
    assert bench.profiled_traffic() == 16950741.0
    _write_profile(p, "0000000000000000", 16950741)       # captured on other source
    assert bench.profiled_traffic() is None
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(tmp_path / "missing.md"))
    assert bench.profiled_traffic() is None


def test_kernel_source_hash_is_stable_and_short():
    h = bench.kernel_source_hash()
    assert h == bench.kernel_source_hash()
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)


def test_workload_names_the_headline_configuration():
    c = bench.config_dict()
    assert c["workload"] == "muca2d_ising_L32_W16384_int8_therm31_rec10"
    assert (c["L"], c["walkers"], c["therm_sweeps"], c["sweeps_per_iter"]) == (32, 16384, 31, 10)
    assert c["energy_bins"] == 32 * 32 + 1
    assert os.path.isfile(bench.TRAFFIC_PROFILE)
