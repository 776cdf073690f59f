"""Writes the stored exact values under tests/golden/.  Calls oracle/ only.

    python tests/golden/make_golden.py

ising_L32_exact_dos.txt, ising_L8_exact_dos.txt: exact g(E) of the 32 x 32
and 8 x 8 periodic Ising models from Kaufman's partition function expanded as
a polynomial (Beale, PRL 76, 78 (1996)), computed by
oracle.exact_dos.ising_dos_kaufman (about a minute for L = 32).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact_dos  # noqa: E402


def write_ising(L):
    E, g = exact_dos.ising_dos_kaufman(L)
    with open(os.path.join(HERE, "ising_L%d_exact_dos.txt" % L), "w") as f:
        f.write("# exact g(E), 2D Ising %dx%d periodic, J=1; columns: E count\n" % (L, L))
        f.write("# written by tests/golden/make_golden.py via oracle.exact_dos.ising_dos_kaufman\n")
        for e, c in zip(E, g):
            f.write("%d %d\n" % (e, c))


def main():
    for L in (8, 32):
        write_ising(L)


if __name__ == "__main__":
    main()
