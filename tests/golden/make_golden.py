"""Writes the stored exact values under tests/golden/.  Calls oracle/ only.

    python tests/golden/make_golden.py

ising_L32_exact_dos.txt: exact g(E) of the 32 x 32 periodic Ising model from
Kaufman's partition function expanded as a polynomial (Beale, PRL 76, 78
(1996)), computed by oracle.exact_dos.ising_dos_kaufman (about a minute).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact_dos  # noqa: E402


def main():
    E, g = exact_dos.ising_dos_kaufman(32)
    with open(os.path.join(HERE, "ising_L32_exact_dos.txt"), "w") as f:
        f.write("# exact g(E), 2D Ising 32x32 periodic, J=1; columns: E count\n")
        f.write("# written by tests/golden/make_golden.py via oracle.exact_dos.ising_dos_kaufman\n")
        for e, c in zip(E, g):
            f.write("%d %d\n" % (e, c))


if __name__ == "__main__":
    main()
