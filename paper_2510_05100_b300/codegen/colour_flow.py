"""Exact SU(N) colour algebra for one quark line and n gluons (code generator).

The colour-flow basis for q q~ + n gluons is the set of ordered generator
products (t^{a_s1} t^{a_s2} ... t^{a_sn})_{i j}, one per permutation s of the
gluons (i = quark, j = antiquark).  The flow colour matrix

    C_{s s'} = sum over a_1..a_n, i, j of conj((t^s)_{ij}) (t^s')_{ij}
             = sum_a tr(t^{s_n} ... t^{s_1} t^{s'_1} ... t^{s'_n})

is computed exactly with rationals by eliminating one repeated adjoint index
at a time with the SU(N) Fierz identity (t^a normalised as tr(t^a t^b) = delta/2):

    sum_a tr(t^a X t^a Y)       = 1/2 tr(X) tr(Y) - 1/(2N) tr(X Y)
    sum_a tr(t^a X) tr(t^a Y)   = 1/2 tr(X Y)     - 1/(2N) tr(X) tr(Y)

with tr() = N and tr(t^a) = 0.
"""
from __future__ import annotations

import itertools
from fractions import Fraction
from math import lcm

NC = 3


def _reduce(coef: Fraction, traces: tuple, n: int) -> Fraction:
    """Fully reduce coef * prod(traces) (each index appearing exactly twice)."""
    # find the first trace holding an index
    for ti, tr in enumerate(traces):
        if tr:
            break
    else:
        return coef * Fraction(n) ** len(traces)
    a = tr[0]
    others = traces[:ti] + traces[ti + 1:]
    rest = tr[1:]
    if a in rest:
        k = rest.index(a)
        x, y = rest[:k], rest[k + 1:]              # tr(t^a X t^a Y)
        t1 = _reduce(coef * Fraction(1, 2), others + (x, y), n)
        t2 = _reduce(coef * Fraction(-1, 2 * n), others + (x + y,), n)
        return t1 + t2
    for oi, other in enumerate(others):
        if a in other:
            k = other.index(a)
            y = other[k + 1:] + other[:k]           # tr(t^a Y) after cyclic rotation
            rem = others[:oi] + others[oi + 1:]
            t1 = _reduce(coef * Fraction(1, 2), rem + (rest + y,), n)
            t2 = _reduce(coef * Fraction(-1, 2 * n), rem + (rest, y), n)
            return t1 + t2
    return Fraction(0)                               # tr(t^a) = 0


def trace_sum(word: tuple, n: int = NC) -> Fraction:
    """sum over repeated adjoint indices of tr(t^{w_1} ... t^{w_k})."""
    return _reduce(Fraction(1), (tuple(word),), n)


def flow_basis(ngluon: int) -> list:
    return list(itertools.permutations(range(ngluon)))


def flow_colour_matrix(ngluon: int, n: int = NC) -> list:
    flows = flow_basis(ngluon)
    return [[trace_sum(tuple(reversed(s)) + tuple(sp), n) for sp in flows] for s in flows]


def integer_colour_matrix(ngluon: int) -> tuple:
    """(integer matrix, denominator) with C = M / den exactly."""
    c = flow_colour_matrix(ngluon)
    den = 1
    for row in c:
        for v in row:
            den = lcm(den, v.denominator)
    return [[int(v * den) for v in row] for row in c], den
