"""The pins catch plausible mistakes in the oracle: each case plants one mistake in a copy
of the oracle's C source (a flipped sign, a wrong energy step, a dropped neighbour, the
histogram recorded before the decision, the recursion's sign, the Kullback-Leibler
reference and its support, a Philox constant, the exp series, the tag of the random-order
site stream, the energy step of a random-order flip, the Eq. (7) schedule's width and its
switch to the growth rule), builds it, and runs the existing pin tests
against it; at least one must fail.  A planted mistake can drive an index off the grid,
so the pins of each copy run in a child process: a failed assertion or a crash both
count as caught.  The unmodified copy passes the same pins through the same path."""
import os
import subprocess
import sys

import pytest

import test_oracle_philox as ophilox

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE = os.path.join(ROOT, "oracle")

# pin sets: (module, test functions taking the oracle binding)
PINS = {
    "chain": ("test_oracle_chain", ["test_all_accept_limit", "test_quench_limit",
                                    "test_tracked_energy_matches_recomputed",
                                    "test_detailed_balance_against_exact_dos", "test_table_rule"]),
    "recursion": ("test_oracle_chain", ["test_weight_update", "test_flatness_metrics"]),
    "math": ("test_oracle_math", ["test_exp_against_libm", "test_exp_special_values"]),
    "random": ("test_oracle_random_order", ["test_site_definition", "test_all_accept_limit", "test_quench_limit",
                                            "test_splits_compose_and_energy_tracked"]),
    "schedule": ("test_oracle_chain", ["test_kl_support_hand_made", "test_kl_measure_nonnegative_and_zero_when_flat",
                                       "test_paper_schedule_first_iteration_counts", "test_paper_schedule_trace"]),
}

_RANDOM_TAIL = "            }\n            if (record)\n                H[ew] += 1u;\n        }\n        e[w] = ew;\n    }\n}\n\n/* Updates in the order"
_TYPEWRITER_TAIL = "\n        }\n        e[w] = ew;\n    }\n}\n\n/* Site of attempt t in random order"

MUTATIONS = [
    ("sign of the weight difference", "double dw = lnW[ep] - lnW[e];", "double dw = lnW[e] - lnW[ep];", "chain"),
    ("energy step of an accepted flip", "                ew += 2 - k;\n            }\n            if (record)\n                H[ew] += 1u;" + _TYPEWRITER_TAIL,
     "                ew += k - 2;\n            }\n            if (record)\n                H[ew] += 1u;" + _TYPEWRITER_TAIL, "chain"),
    ("a dropped neighbour", "    k += s[orc_site(L, x, y - 1)] != si;\n", "", "chain"),
    ("histogram of the pre-decision energy",
     "            if (orc_accept(r, T[ew * 5 + k])) {\n                s[i] = (int8_t)(-s[i]);\n                ew += 2 - k;\n"
     "            }\n            if (record)\n                H[ew] += 1u;" + _TYPEWRITER_TAIL,
     "            if (record)\n                H[ew] += 1u;\n            if (orc_accept(r, T[ew * 5 + k])) {\n"
     "                s[i] = (int8_t)(-s[i]);\n                ew += 2 - k;\n            }" + _TYPEWRITER_TAIL, "chain"),
    ("sign of the recursion", "            lnW[e] -= orc_log((double)H[e]);", "            lnW[e] += orc_log((double)H[e]);",
     "recursion"),
    ("Kullback-Leibler reference", "        dk += P * orc_log(P * q);", "        dk += P * orc_log(P / q);", "recursion"),
    ("a term of the exp series", "1.0 / 120.0,", "1.0 / 121.0,", "math"),
    ("tag of the random-order site stream", "orc_random_word(seed, ORC_SHARED_STREAM, ORC_TAG_SITE, t);",
     "orc_random_word(seed, ORC_SHARED_STREAM, ORC_TAG_METROPOLIS, t);", "random"),
    ("energy step of a random-order flip", "                ew += 2 - k;\n" + _RANDOM_TAIL,
     "                ew += k - 2;\n" + _RANDOM_TAIL, "random"),
    ("Kullback-Leibler support from the previous range only",
     "            if (lo < 0 || e < lo)\n                lo = e;\n            if (hi < 0 || e > hi)\n                hi = e;",
     "            ;", "schedule"),
    ("growth rule one iteration early", "            if (full) {", "            if (full || prev_width == N + 1) {",
     "schedule"),
    ("schedule width as the accessible count", "        prev_width = orc_width(L, H);",
     "        prev_width = orc_accessible_in_range(L, H);", "schedule"),
]


def run_pins_in_child(lib: str, pins: str) -> int:
    """Runs one pin set against the oracle library `lib` in a fresh interpreter; returns
    its exit status (0: every pin held)."""
    module, names = PINS[pins]
    code = (
        "import sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        f"sys.path.insert(0, {HERE!r})\n"
        "from oracle import oracle as orc\n"
        f"import {module} as m\n"
        f"with orc.using({lib!r}):\n"
        f"    for name in {names!r}:\n"
        "        getattr(m, name)(orc)\n"
    )
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=HERE)
    return r.returncode


@pytest.fixture(scope="module")
def source():
    return {name: open(os.path.join(ORACLE, name)).read() for name in ("muca_oracle.c", "exact_dos.c")}


def _build(orc, tmp_path, src, exact, name):
    (tmp_path / "muca_oracle.c").write_text(src)
    (tmp_path / "exact_dos.c").write_text(exact)
    return orc.build_variant([str(tmp_path / "muca_oracle.c"), str(tmp_path / "exact_dos.c")], str(tmp_path / name))


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(orc, source, tmp_path, name, old, new, pins):
    src = source["muca_oracle.c"]
    assert src.count(old) == 1, name
    lib = _build(orc, tmp_path, src.replace(old, new), source["exact_dos.c"], "libmutant.so")
    assert run_pins_in_child(lib, pins) != 0, name


def test_planted_philox_mistake_is_caught(orc, source, tmp_path, aten_philox):
    """A wrong multiplier in the generator fails the comparison with PyTorch's Philox."""
    src = source["muca_oracle.c"]
    i = src.index("void orc_philox4x32_10(")
    body = src[i:]
    mutated_body = body.replace("0xD2511F53u", "0xD2511F55u", 1)
    assert mutated_body != body
    lib = _build(orc, tmp_path, src[:i] + mutated_body, source["exact_dos.c"], "libmutant.so")
    with orc.using(lib):
        with pytest.raises(AssertionError):
            ophilox.test_philox_block_matches_aten(orc, aten_philox)


aten_philox = ophilox.aten_philox


def test_unmodified_copy_passes_the_same_pins(orc, source, tmp_path):
    """Control: the same build and child-process path with the unmodified source passes
    every pin set."""
    lib = _build(orc, tmp_path, source["muca_oracle.c"], source["exact_dos.c"], "libcopy.so")
    for pins in PINS:
        assert run_pins_in_child(lib, pins) == 0, pins
