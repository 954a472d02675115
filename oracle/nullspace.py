"""Spin-free overlap metric of appendix B.  TEST INFRASTRUCTURE ONLY.

For the n! spin-free operators obtained by permuting the virtual labels, the
overlap depends only on the relative permutation rho:
m(rho) = sgn(rho) * 2^{c(rho)}, c = number of cycles including 1-cycles
(Eq. spinfree_overlap_class_function).  The projector that removes the
redundant fully symmetric sector for triples is 1 - Pi_[3] with
Pi_[3] = (1/6) sum_pi P_pi (Eq. r3_null_constraint and the line after it).
"""
from __future__ import annotations

import itertools

import numpy as np


def cycles(perm) -> int:
    seen, c = set(), 0
    for s in range(len(perm)):
        if s in seen:
            continue
        c += 1
        x = s
        while x not in seen:
            seen.add(x)
            x = perm[x]
    return c


def sign(perm) -> int:
    return -1 if (len(perm) - cycles(perm)) % 2 else 1


def compose(p, q):
    """(p o q)(x) = p(q(x))."""
    return tuple(p[q[x]] for x in range(len(q)))


def inverse(p):
    inv = [0] * len(p)
    for i, x in enumerate(p):
        inv[x] = i
    return tuple(inv)


def overlap_matrix(n: int) -> np.ndarray:
    """M[pi, tau] = m(pi^-1 tau) over all permutations of n virtual labels."""
    perms = list(itertools.permutations(range(n)))
    M = np.empty((len(perms), len(perms)))
    for a, p in enumerate(perms):
        for b, q in enumerate(perms):
            rho = compose(inverse(p), q)
            M[a, b] = sign(rho) * 2.0 ** cycles(rho)
    return M


def projector_triples() -> np.ndarray:
    """Matrix of 1 - (1/6) sum_pi P_pi acting on the 6 virtual orderings of one triple."""
    return np.eye(6) - np.full((6, 6), 1.0 / 6.0)
