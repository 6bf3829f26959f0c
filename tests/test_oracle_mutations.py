"""The pins catch plausible mistakes in the oracle: each case plants one mistake in a copy
of the oracle's C source (a flipped sign, a wrong energy step, a dropped neighbour, the
histogram recorded before the decision, the recursion's sign, the Kullback-Leibler
reference, a Philox constant, the exp series), builds it, and runs the existing pin
tests against it; at least one must fail.  The unmodified oracle passes them (the rest
of the suite)."""
import os

import numpy as np
import pytest

import test_oracle_chain as chain
import test_oracle_math as omath
import test_oracle_philox as ophilox

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(HERE), "oracle")


def _pins_chain(orc):
    chain.test_all_accept_limit(orc)
    chain.test_quench_limit(orc)
    chain.test_tracked_energy_matches_recomputed(orc)
    chain.test_detailed_balance_against_exact_dos(orc)
    chain.test_table_rule(orc)


def _pins_recursion_and_metrics(orc):
    chain.test_weight_update(orc)
    chain.test_flatness_metrics(orc)


def _pins_math(orc):
    omath.test_exp_against_libm(orc)
    omath.test_exp_special_values(orc)


MUTATIONS = [
    ("sign of the weight difference", "double dw = lnW[ep] - lnW[e];", "double dw = lnW[e] - lnW[ep];",
     _pins_chain),
    ("energy step of an accepted flip", "                ew += 2 - k;\n            }\n            if (record)",
     "                ew += k - 2;\n            }\n            if (record)", _pins_chain),
    ("a dropped neighbour", "    k += s[orc_site(L, x, y - 1)] != si;\n", "", _pins_chain),
    ("histogram of the pre-decision energy",
     "            if (orc_accept(r, T[ew * 5 + k])) {\n                s[i] = (int8_t)(-s[i]);\n                ew += 2 - k;\n"
     "            }\n            if (record)\n                H[ew] += 1u;",
     "            if (record)\n                H[ew] += 1u;\n            if (orc_accept(r, T[ew * 5 + k])) {\n"
     "                s[i] = (int8_t)(-s[i]);\n                ew += 2 - k;\n            }", _pins_chain),
    ("sign of the recursion", "            lnW[e] -= orc_log((double)H[e]);", "            lnW[e] += orc_log((double)H[e]);",
     _pins_recursion_and_metrics),
    ("Kullback-Leibler reference", "        dk += P * orc_log(P * q);", "        dk += P * orc_log(P / q);",
     _pins_recursion_and_metrics),
    ("a term of the exp series", "1.0 / 120.0,", "1.0 / 121.0,", _pins_math),
]


@pytest.fixture(scope="module")
def source():
    return {name: open(os.path.join(ORACLE, name)).read() for name in ("muca_oracle.c", "exact_dos.c")}


@pytest.mark.parametrize("name,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(orc, source, tmp_path, name, old, new, pins):
    src = source["muca_oracle.c"]
    assert src.count(old) >= 1, name
    mutated = tmp_path / "muca_oracle.c"
    mutated.write_text(src.replace(old, new, 1))
    (tmp_path / "exact_dos.c").write_text(source["exact_dos.c"])
    lib = orc.build_variant([str(mutated), str(tmp_path / "exact_dos.c")], str(tmp_path / "libmutant.so"))
    with orc.using(lib):
        with pytest.raises(AssertionError):
            pins(orc)


def test_planted_philox_mistake_is_caught(orc, source, tmp_path, aten_philox):
    """A wrong multiplier in the generator fails the comparison with PyTorch's Philox."""
    src = source["muca_oracle.c"]
    i = src.index("void orc_philox4x32_10(")
    body = src[i:]
    mutated_body = body.replace("0xD2511F53u", "0xD2511F55u", 1)
    assert mutated_body != body
    mutated = tmp_path / "muca_oracle.c"
    mutated.write_text(src[:i] + mutated_body)
    (tmp_path / "exact_dos.c").write_text(source["exact_dos.c"])
    lib = orc.build_variant([str(mutated), str(tmp_path / "exact_dos.c")], str(tmp_path / "libmutant.so"))
    with orc.using(lib):
        with pytest.raises(AssertionError):
            ophilox.test_philox_block_matches_aten(orc, aten_philox)


aten_philox = ophilox.aten_philox


def test_unmodified_copy_passes_the_same_pins(orc, source, tmp_path):
    """Control: the same build path with the unmodified source passes every pin set."""
    (tmp_path / "muca_oracle.c").write_text(source["muca_oracle.c"])
    (tmp_path / "exact_dos.c").write_text(source["exact_dos.c"])
    lib = orc.build_variant([str(tmp_path / "muca_oracle.c"), str(tmp_path / "exact_dos.c")],
                            str(tmp_path / "libcopy.so"))
    with orc.using(lib):
        for pins in {id(m[3]): m[3] for m in MUTATIONS}.values():
            pins(orc)
