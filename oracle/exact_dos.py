"""Exact densities of states of small and medium 2D lattices (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

These are the plain definitions that the converged WL output must reproduce
(paper, Ising paragraph: deviations from the exact results are of the order of
the statistical error).  Three independent routes, each pinned against the
others and against closed-form counts in tests/test_exact_dos.py:

  * ``enumerate_dos``   -- brute force over all q^N configurations (N <= 16
                           for q = 2; q^N <= 2e6 for Potts);
  * ``transfer_dos``    -- site-by-site transfer matrix on the torus with the
                           first row held fixed, exact integer counts;
  * ``ising_dos_kaufman`` -- Kaufman's (1949) partition function of the L x L
                           torus expanded as a polynomial in y = exp(-2K)
                           (the route of P. D. Beale, PRL 76, 78 (1996)),
                           evaluated in fixed-point integer arithmetic and
                           rounded to exact integer counts.

Energies: Ising and +-J E = -sum_<ij> J_ij s_i s_j over the 2N bonds of the
periodic lattice (right and down of each site); Potts E = -sum delta(s_i,s_j).
Every function returns (E values, exact counts as Python ints).
"""
import math
from itertools import product

import numpy as np


def _bonds(L):
    N = L * L
    right = np.array([(i // L) * L + (i % L + 1) % L for i in range(N)])
    down = np.array([((i // L + 1) % L) * L + i % L for i in range(N)])
    return right, down


def _bonds3(L):
    """Right, down and behind neighbours on the periodic L x L x L cube, site
    i = (z L + y) L + x."""
    N = L ** 3
    i = np.arange(N)
    x, y, z = i % L, (i // L) % L, i // (L * L)
    at = lambda a, b, c: (c * L + b) * L + a
    return at((x + 1) % L, y, z), at(x, (y + 1) % L, z), at(x, y, (z + 1) % L)


def enumerate_dos(L, model="ising", q=2, couplings=None):
    """Brute force over all configurations.  couplings: 2N values +-1 (right,
    down of each site) for the +-J model, 3N (right, down, behind) for the
    3D +-J model "ea3d" on the L x L x L cube."""
    if model == "ea3d":
        N = L ** 3
        if N > 20:
            raise ValueError("too many configurations")
        nb = _bonds3(L)
        c = np.ones((N, 3), np.int64) if couplings is None else np.asarray(couplings, np.int64).reshape(N, 3)
        idx = np.arange(1 << N, dtype=np.int64)
        spin = lambda i: 1 - 2 * ((idx >> i) & 1)
        E = np.zeros(1 << N, np.int64)
        for i in range(N):
            for d in range(3):
                E -= c[i, d] * spin(i) * spin(int(nb[d][i]))
        vals, counts = np.unique(E, return_counts=True)
        return [int(v) for v in vals], [int(c) for c in counts]
    N = L * L
    right, down = _bonds(L)
    if model == "potts":
        total = q ** N
        if total > 3_000_000:
            raise ValueError("too many configurations")
        idx = np.arange(total, dtype=np.int64)
        s = np.zeros((total, N), np.int8)
        for i in range(N):
            s[:, i] = idx % q
            idx //= q
        E = -((s == s[:, right]).sum(1) + (s == s[:, down]).sum(1))
    else:
        if N > 20:
            raise ValueError("too many configurations")
        Jr = np.ones(N, np.int64)
        Jd = np.ones(N, np.int64)
        if couplings is not None:
            c = np.asarray(couplings).reshape(N, 2)
            Jr, Jd = c[:, 0].astype(np.int64), c[:, 1].astype(np.int64)
        E = np.zeros(1 << N, np.int64)
        idx = np.arange(1 << N, dtype=np.int64)
        spin = lambda i: 1 - 2 * ((idx >> i) & 1)
        for i in range(N):
            si = spin(i)
            E -= Jr[i] * si * spin(right[i]) + Jd[i] * si * spin(down[i])
    vals, counts = np.unique(E, return_counts=True)
    return [int(v) for v in vals], [int(c) for c in counts]


def transfer_dos(L, model="ising", q=2, couplings=None):
    """Site-by-site transfer matrix on the L x L torus.  The first row is
    fixed (for Potts, one representative per colour pattern of the row,
    weighted by the number of colourings with that pattern); the remaining
    sites are added one at a time with the last L placed spins as the state.
    The state carries a count per number of unsatisfied bonds."""
    N = L * L
    nb = 2 * N
    if model != "potts":
        q = 2
    Jr = np.ones(N, np.int64)
    Jd = np.ones(N, np.int64)
    if couplings is not None:
        c = np.asarray(couplings).reshape(N, 2)
        Jr, Jd = c[:, 0].astype(np.int64), c[:, 1].astype(np.int64)

    def unsat(i, j, a, b, J):
        # 1 if the bond (i,j) with spins a,b is unsatisfied
        if model == "potts":
            return (a != b).astype(np.int64) if isinstance(a, np.ndarray) else int(a != b)
        # Ising / +-J: satisfied iff J s_a s_b = +1, s = 1 - 2b
        sa = 1 - 2 * a
        sb = 1 - 2 * b
        v = J * sa * sb
        return (v < 0).astype(np.int64) if isinstance(v, np.ndarray) else int(v < 0)

    # first-row representatives and weights
    if model == "potts":
        reps = []

        def rec(prefix, used):
            if len(prefix) == L:
                reps.append(tuple(prefix))
                return
            for c_ in range(min(used + 1, q)):
                rec(prefix + [c_], max(used, c_ + 1))

        rec([], 0)
        weights = []
        for r in reps:
            k = len(set(r))
            w_ = 1
            for t in range(k):
                w_ *= (q - t)
            weights.append(w_)
    else:
        reps = list(product(range(2), repeat=L))
        weights = [1] * len(reps)

    S = q ** L
    # state index: spins of the last L placed sites, oldest = most significant digit
    digits = np.array([[(s // q ** (L - 1 - k)) % q for k in range(L)] for s in range(S)], np.int64)
    total = [0] * (nb + 1)
    for rep, wt in zip(reps, weights):
        row0 = list(rep)
        u0 = 0
        for x in range(L):  # horizontal bonds inside the first row (periodic)
            u0 += unsat(x, (x + 1) % L, row0[x], row0[(x + 1) % L], Jr[x])
        st0 = 0
        for k in range(L):
            st0 = st0 * q + row0[k]
        V = np.zeros((S, nb + 1), np.int64)
        V[st0, u0] = 1
        for i in range(L, N):
            x, y = i % L, i // L
            newV = np.zeros_like(V)
            oldest = digits[:, 0]            # spin at (x, y-1)
            newest = digits[:, L - 1]        # spin at (x-1, y)
            first_of_row = digits[:, L - x] if x > 0 else None  # spin at (0, y) when x = L-1
            for v in range(q):
                du = unsat(0, 0, oldest, np.full(S, v), Jd[(y - 1) * L + x])  # vertical bond to (x, y-1)
                if x > 0:
                    du = du + unsat(0, 0, newest, np.full(S, v), Jr[y * L + x - 1])  # bond to (x-1, y)
                if x == L - 1:
                    du = du + unsat(0, 0, np.full(S, v), first_of_row, Jr[y * L + x])  # periodic bond to (0, y)
                if y == L - 1:
                    du = du + unsat(0, 0, np.full(S, v), np.full(S, row0[x]), Jd[y * L + x])  # to (x, 0)
                nxt = (np.arange(S) % (q ** (L - 1))) * q + v
                for d in np.unique(du):
                    sel = np.nonzero(du == d)[0]
                    if d == 0:
                        np.add.at(newV, nxt[sel], V[sel])
                    else:
                        np.add.at(newV, nxt[sel], np.pad(V[sel][:, :-d], ((0, 0), (d, 0))))
            V = newV
        col = V.sum(0)
        for u in range(nb + 1):
            total[u] += int(col[u]) * wt
    if model == "potts":
        Es = [u - nb for u in range(nb + 1)]
    else:
        Es = [2 * u - nb for u in range(nb + 1)]
    pairs = [(e, c) for e, c in zip(Es, total) if c]
    return [p[0] for p in pairs], [p[1] for p in pairs]


# ---------------------------------------------------------------------------
# Kaufman / Beale closed form for the ferromagnetic Ising model on the L x L
# torus.  With K = beta J and y = exp(-2K), y^N Z = sum_k g(-2N + 4k) y^(2k).
# Kaufman: Z = 1/2 (2 sinh 2K)^(N/2) (Z1 + Z2 + Z3 + Z4), products over
# 2cosh / 2sinh of (L gamma_l / 2) with cosh gamma_l = cosh 2K coth 2K -
# cos(pi l / L).  Pairing l with 2L - l turns each pair into 2(T_L(c_l) +- 1)
# (T_L a Chebyshev polynomial), and the two unpaired terms l = 0, L have
# exp(gamma_0) = (1-y)/(y(1+y)), exp(gamma_L) = (1+y)/(y(1-y)), so every factor
# is a polynomial in y after clearing the common denominator
# (2y(1-y^2))^(N/2) against the prefactor.
# ---------------------------------------------------------------------------
def _pmul(a, b):
    """Product of integer-coefficient polynomials (lists, lowest degree first)."""
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x == 0:
            continue
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _padd(a, b, sa=1, sb=1):
    n = max(len(a), len(b))
    return [sa * (a[i] if i < len(a) else 0) + sb * (b[i] if i < len(b) else 0) for i in range(n)]


def _ppow(a, k):
    out = [1]
    for _ in range(k):
        out = _pmul(out, a)
    return out


def ising_dos_kaufman(L, extra_bits=256):
    """Exact g(E) of the L x L periodic Ising model (L even) from Kaufman's
    partition function, in fixed-point integer arithmetic with P fraction bits
    and a final rounding to integers (checked: all counts integral within
    2^-32, odd powers of y vanish, sum = 2^N)."""
    import mpmath

    if L % 2 or L < 4:
        raise ValueError("L must be even and >= 4")
    m = n = L
    N = L * L
    P = 2 * N + extra_bits
    one = 1 << P
    mpmath.mp.prec = P + 64

    def fx(x):
        return int(mpmath.nint(x * mpmath.mpf(2) ** P))

    def fmul(a, b):  # fixed x fixed -> fixed
        prod_ = _pmul(a, b)
        return [v >> P if v >= 0 else -((-v) >> P) for v in prod_]

    D = [0, 2, 0, -2]            # 2y(1 - y^2), exact integers
    D2 = _pmul(D, D)
    A_ = [1, 0, 2, 0, 1]          # (1 + y^2)^2

    def Q(l, sign):
        c = fx(mpmath.cos(mpmath.pi * l / n))
        num = [a * one - c * d for a, d in zip(A_, D + [0])]  # (1+y^2)^2 - D cos, fixed
        S_prev = [one]            # D^0 T_0
        S_cur = num               # D^1 T_1
        for _ in range(1, m):     # S_{k+1} = 2 num S_k - D^2 S_{k-1}
            S_next = _padd(fmul(num, S_cur), [v * 1 for v in _pmul(D2, S_prev)], 2, -1)
            S_prev, S_cur = S_cur, S_next
        Dm = [v * one for v in _ppow(D, m)]
        return _padd(S_cur, Dm, 1, sign)

    def prod_Q(ls, sign):
        out = [one]
        for l in ls:
            out = fmul(out, Q(l, sign))
        return out

    odd = [l for l in range(1, n, 2)]
    even = [l for l in range(2, n - 1, 2)]
    P1 = prod_Q(odd, +1)
    P2 = prod_Q(odd, -1)
    P3 = prod_Q(even, +1)
    P4 = prod_Q(even, -1)
    omy2 = [1, 0, -1]
    a_m = _ppow(omy2, m)
    u_a = _padd(a_m, [0] * (2 * m) + a_m)                     # (1-y^2)^m (1 + y^(2m))
    u_b = _padd([0] * m + _ppow([1, -1], 2 * m), [0] * m + _ppow([1, 1], 2 * m))  # y^m[(1-y)^2m + (1+y)^2m]
    U3 = _padd(u_a, u_b, 1, 1)
    U4 = _padd(u_a, u_b, 1, -1)
    T12 = _padd(P1, P2)
    T34 = _padd(_pmul(U3, P3), _pmul(U4, P4))
    e12 = n // 2 - N // 2 - 1
    e34 = m + n // 2 - N // 2 - 2
    # total = 2^e12 T12 + 2^e34 T34, all in fixed point with P fraction bits
    deg = max(len(T12), len(T34))
    coeffs = []
    for k in range(deg):
        t12 = T12[k] if k < len(T12) else 0
        t34 = T34[k] if k < len(T34) else 0
        v = _shift(t12, e12) + _shift(t34, e34)       # fixed point
        r = (v + (one >> 1)) >> P if v >= 0 else -((-v + (one >> 1)) >> P)
        if abs(v - r * one) > (one >> 32):
            raise ArithmeticError("coefficient %d not integral" % k)
        coeffs.append(r)
    if any(coeffs[k] for k in range(1, len(coeffs), 2)):
        raise ArithmeticError("odd powers of y present")
    g = [coeffs[2 * k] if 2 * k < len(coeffs) else 0 for k in range(N + 1)]
    if sum(g) != 2 ** N or any(c < 0 for c in g):
        raise ArithmeticError("counts do not sum to 2^N")
    pairs = [(-2 * N + 4 * k, c) for k, c in enumerate(g) if c]
    return [p[0] for p in pairs], [p[1] for p in pairs]


def _shift(v, e):
    if e >= 0:
        return v << e
    return v >> (-e) if v >= 0 else -((-v) >> (-e))


def ln_counts(counts):
    """Natural log of exact (possibly huge) integer counts."""
    out = []
    for c in counts:
        if c <= 0:
            out.append(-math.inf)
            continue
        b = c.bit_length()
        if b > 1000:
            out.append(math.log(c >> (b - 60)) + (b - 60) * math.log(2.0))
        else:
            out.append(math.log(c))
    return np.array(out)
