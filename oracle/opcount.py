"""Leading operation counts of one RCCSDT iteration.  TEST INFRASTRUCTURE ONLY.

Counts multiply-add pairs (FMA), the paper's unit (Sec. II.C).  ``compact_fma``
enumerates the representative contractions per stored block, as tabulated in
the appendix operation-count table:
* pp-ladder: 3 terms of v^2 (ab) x v (c) outputs over v^2 (de)  -> 3 v^5;
* ring: 3 (2<3, spin-summed) + 3 (2<3, two unpacked blocks summed first)
        + 6 (all permutations) terms of v^3 outputs over o v (ld) -> 12 o v^4;
* hh-ladder: 3 terms of v^3 outputs over o^2 (lm) -> 3 o^2 v^3.
``full_fma`` is o^3 v^5 + 3 o^4 v^4 + o^5 v^3 (Sec. II.C.3).
"""
from __future__ import annotations


def n3(o: int) -> int:
    return o * (o + 1) * (o + 2) // 6


def compact_fma_enumerated(o: int, v: int) -> int:
    total = 0
    for k in range(o):
        for j in range(k + 1):
            for i in range(j + 1):
                total += 3 * (v * v) * v * (v * v)       # pp: 3 GEMMs M=v^2, N=v, K=v^2
                total += (3 + 3 + 6) * (v ** 3) * (o * v)  # ring: 12 GEMMs M*N=v^3, K=o v
                total += 3 * (v ** 3) * (o * o)          # hh: 3 GEMMs M*N=v^3, K=o^2
    return total


def compact_fma(o: int, v: int) -> int:
    return n3(o) * (3 * v ** 5 + 12 * o * v ** 4 + 3 * o * o * v ** 3)


def full_fma(o: int, v: int) -> int:
    return o ** 3 * v ** 5 + 3 * o ** 4 * v ** 4 + o ** 5 * v ** 3


def compact_asymptotic(o: float, v: float) -> float:
    return 0.5 * o ** 3 * v ** 5 + 2 * o ** 4 * v ** 4 + 0.5 * o ** 5 * v ** 3


def flop_per_iteration(o: int, v: int) -> int:
    """Algorithmic flop (2 per FMA) of the leading compact contractions."""
    return 2 * compact_fma(o, v)


def t3_bytes(o: int, v: int, itemsize: int = 8) -> int:
    return n3(o) * v ** 3 * itemsize
