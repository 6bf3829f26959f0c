"""Pins the oracle's Philox4x32-10 (Sec. 2.3: counter-based generator of Salmon et al.)
to an independent implementation: PyTorch's header-only at::philox_engine, compiled here
as a small host program.  Also pins the counter layout of the stream reading: key = seed,
counter = (attempt block, walker, tag), word = t & 3."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HARNESS = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cinttypes>
int main() {
  unsigned long long seed, subseq, offset; int skip;
  while (std::scanf("%llu %llu %llu %d", &seed, &subseq, &offset, &skip) == 4) {
    at::philox_engine eng(seed, subseq, offset);
    for (int i = 0; i < skip; ++i) eng();
    unsigned a = eng(), b = eng(), c = eng(), d = eng();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def aten_philox(tmp_path_factory):
    try:
        import torch
    except ImportError:
        pytest.skip("torch not importable")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")) or not shutil.which("g++"):
        pytest.skip("ATen Philox header or g++ unavailable")
    d = tmp_path_factory.mktemp("aten_philox")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, str(src), "-o", str(exe)], check=True)

    def call(queries):
        inp = "".join(f"{s} {q} {o} {k}\n" for s, q, o, k in queries)
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
        return [list(map(int, line.split())) for line in out.strip().splitlines()]

    return call


def test_philox_block_matches_aten(orc, aten_philox):
    rng = np.random.default_rng(7)
    queries, mine = [], []
    for _ in range(200):
        seed = int(rng.integers(0, 2**64, dtype=np.uint64))
        walker = int(rng.integers(0, 2**32, dtype=np.uint64))
        tag = int(rng.integers(0, 4))
        block = int(rng.integers(0, 2**40, dtype=np.uint64))
        ctr = [block & 0xFFFFFFFF, block >> 32, walker, tag]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        mine.append([int(x) for x in orc.philox4x32_10(ctr, key)])
        queries.append((seed, walker | (tag << 32), block, 0))
    assert aten_philox(queries) == mine


def test_philox_extreme_counters(orc, aten_philox):
    cases = [(0, 0, 0), (2**64 - 1, 2**64 - 1, 2**64 - 1), (1, 2**32 - 1, 2**32 - 1), (2**63, 5, 2**32)]
    queries, mine = [], []
    for seed, subseq, block in cases:
        ctr = [block & 0xFFFFFFFF, block >> 32, subseq & 0xFFFFFFFF, subseq >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        mine.append([int(x) for x in orc.philox4x32_10(ctr, key)])
        queries.append((seed, subseq, block, 0))
    assert aten_philox(queries) == mine


def test_random_word_stream_layout(orc, aten_philox):
    """orc_random_word(seed, walker, tag, t) is word t&3 of block t>>2 of the
    sub-stream (walker, tag)."""
    seed, walker, tag = 0x0123456789ABCDEF, 77, 0
    queries, mine = [], []
    for t in [0, 1, 2, 3, 4, 5, 1023, 1024, 10**9 + 3, 2**34 + 2]:
        queries.append((seed, walker | (tag << 32), t >> 2, t & 3))
        mine.append(orc.random_word(seed, walker, tag, t))
    got = [row[0] for row in aten_philox(queries)]
    assert got == mine


def test_philox_words_are_uniform(orc):
    """Weak statistical sanity: 4096 words from one stream have mean ~ 2^31 and a top
    bit that is set about half of the time."""
    w = np.array([orc.random_word(5, 3, 0, t) for t in range(4096)], dtype=np.float64)
    assert abs(w.mean() / 2**32 - 0.5) < 0.02
    top = (w >= 2**31).mean()
    assert abs(top - 0.5) < 0.04
