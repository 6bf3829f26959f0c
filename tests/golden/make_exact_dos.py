"""Writes the exact density-of-states fixtures used by the tests.

Every value comes from the oracle (oracle/exact_dos.c, oracle/kaufman.py), which the
tests pin against brute-force enumeration and the exact transfer matrix.  The paper
(arXiv:1707.00919, Sec. 3.3) compares its estimates with this exact finite-lattice
density of states of the model of Eq. (5).

    python tests/golden/make_exact_dos.py            # L = 4, 6, 8, 16, 32
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import kaufman, oracle  # noqa: E402


def write(L: int, g: list[int], method: str, integers: bool) -> None:
    path = os.path.join(HERE, f"exact_dos_L{L}.txt")
    lng = kaufman.ln_dos_from_integers(g)
    with open(path, "w") as f:
        f.write(f"# exact density of states of the periodic {L}x{L} Ising model (J = 1)\n")
        f.write(f"# e = (E + 2N)/4, N = {L * L}; method: {method}; written by make_exact_dos.py\n")
        f.write("# columns: e  ln_g" + ("  g" if integers else "") + "\n")
        for e, (x, lx) in enumerate(zip(g, lng)):
            if integers:
                f.write(f"{e} {lx!r} {x}\n")
            else:
                f.write(f"{e} {lx!r}\n")


def main(sizes=(4, 6, 8, 16, 32)) -> None:
    for L in sizes:
        if L <= 4:
            g, method = oracle.dos_bruteforce(L), "brute-force enumeration"
        elif L <= 8:
            g, method = oracle.dos_transfer(L), "exact transfer matrix"
        else:
            g, method = kaufman.exact_dos(L), "Kaufman closed form, high precision"
        write(L, g, method, integers=L <= 16)
        print("wrote L =", L)


if __name__ == "__main__":
    main(tuple(int(a) for a in sys.argv[1:]) or (4, 6, 8, 16, 32))
