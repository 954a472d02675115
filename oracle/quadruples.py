"""Compact T4 (RCCSDTQ) pieces, FP64, numpy.  TEST INFRASTRUCTURE ONLY.

Written from Sec. II.C.4 ("RCCSDTQ contractions"), Sec. II.D (symmetrisation,
purification and orthogonalisation of R4) and appendix B (the quadruples overlap
metric, its null space [4] + 3[3,1] and the polynomial form of the projector
1 - Pi_[4] - Pi_[3,1], Eq. T4ortho).

Storage: ``t4c[blk, a, b, c, d]`` for occupied quadruples i <= j <= k <= l in colex
order, ``blk(i,j,k,l) = C(l+3,4) + C(k+2,3) + C(j+1,2) + i`` (the order of the triples
extended by one index; the paper fixes none), each block a contiguous v^4 array.
Full tensors are ``t4[i, j, k, l, a, b, c, d]`` with the column-pair symmetry
t_{pi(ijkl)}^{pi(abcd)} = t_{ijkl}^{abcd}.  ``W[a, b, e, f] = W^{ab}_{ef}`` with the
pair-exchange symmetry W^{ab}_{ef} = W^{ba}_{fe}.

Readings (the paper is silent or brief here):
* the symmetrisation "r <- P_(ia)(jb) r" of a block with two equal occupied
  indices is the average 1/2 (r + P r), as for R3 (a plain sum would double it);
  a block i = j < k = l takes both its rules (they act on disjoint columns);
* purification zeroes every block with three equal occupied indices
  (i = j = k <= l and i <= j = k = l);
* the projector acts on the virtual labels of every stored block.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np

from . import nullspace

einsum = lambda *a: np.einsum(*a, optimize=True)  # noqa: E731

PERMS4 = list(itertools.permutations(range(4)))


def n4(o: int) -> int:
    return o * (o + 1) * (o + 2) * (o + 3) // 24


def blk4(i: int, j: int, k: int, l: int) -> int:
    assert i <= j <= k <= l
    return comb(l + 3, 4) + comb(k + 2, 3) + comb(j + 1, 2) + i


def quads(o: int):
    """Occupied quadruples i <= j <= k <= l in storage order."""
    out = [None] * n4(o)
    for l in range(o):
        for k in range(l + 1):
            for j in range(k + 1):
                for i in range(j + 1):
                    out[blk4(i, j, k, l)] = (i, j, k, l)
    return out


def pack4(t4: np.ndarray) -> np.ndarray:
    o = t4.shape[0]
    return np.ascontiguousarray(np.stack([t4[q] for q in quads(o)]))


def unpack4(t4c: np.ndarray, o: int) -> np.ndarray:
    """The full tensor: t_{lmnp}^{x} from the stored block of sorted(l, m, n, p), its
    virtual axes permuted by the same sort (the column-pair symmetry)."""
    v = t4c.shape[1]
    t4 = np.empty((o,) * 4 + (v,) * 4)
    for occ in itertools.product(range(o), repeat=4):
        s = sorted(range(4), key=lambda q: occ[q])
        B = t4c[blk4(*[occ[q] for q in s])]
        t4[occ] = np.transpose(B, np.argsort(s))
    return t4


def perm_pairs4(x):
    """P_(ia)(jb)(kc)(ld) x: the 24 joint permutations of the column pairs (Eq. rcc-perm-op)."""
    out = np.zeros_like(x)
    for p in PERMS4:
        out += x.transpose(p[0], p[1], p[2], p[3], 4 + p[0], 4 + p[1], 4 + p[2], 4 + p[3])
    return out


def pp_ladder_full(W: np.ndarray, t4: np.ndarray) -> np.ndarray:
    """The W^vv_vv * T4 term on full storage (Sec. II.C.4):
    r_ijkl^abcd <- P_(ia)(jb)(kc)(ld) 1/4 sum_ef W^{ab}_{ef} t_ijkl^{efcd}."""
    return perm_pairs4(0.25 * einsum("abef,ijklefcd->ijklabcd", W, t4))


def pp_ladder_compact(W: np.ndarray, t4c: np.ndarray, o: int) -> np.ndarray:
    """The same term on compact storage by direct traversal: for every stored block
    the six terms of Sec. II.C.4, each read from the same stored block after
    relabelling the paired columns:
      W^{ab}_{ef} t_ijkl^{efcd} + W^{ac}_{ef} t_ikjl^{efbd} + W^{ad}_{ef} t_iljk^{efbc}
    + W^{bc}_{ef} t_jkil^{efad} + W^{bd}_{ef} t_jlik^{efac} + W^{cd}_{ef} t_klij^{efab}."""
    R = np.zeros_like(t4c)
    for b in range(len(t4c)):
        T = t4c[b]                                          # T[a, b, c, d] = t_ijkl^{abcd}
        r = einsum("abef,efcd->abcd", W, T)                 # t_ijkl^{efcd}
        r += einsum("acef,ebfd->abcd", W, T)                # t_ikjl^{efbd} = t_ijkl^{ebfd}
        r += einsum("adef,ebcf->abcd", W, T)                # t_iljk^{efbc} = t_ijkl^{ebcf}
        r += einsum("bcef,aefd->abcd", W, T)                # t_jkil^{efad} = t_ijkl^{aefd}
        r += einsum("bdef,aecf->abcd", W, T)                # t_jlik^{efac} = t_ijkl^{aecf}
        r += einsum("cdef,abef->abcd", W, T)                # t_klij^{efab} = t_ijkl^{abef}
        R[b] = r
    return R


def _vperm(B, p):
    """out[x0..x3] = B[x_p0, .., x_p3] on a v^4 block."""
    return np.transpose(B, np.argsort(p))


def symmetrise4(r4c: np.ndarray, o: int) -> np.ndarray:
    """Blocks with two equal occupied indices (Sec. II.D.1): i = j < k <= l averages
    over the swap of columns 1, 2; i < j = k < l over columns 2, 3; i <= j < k = l
    over columns 3, 4."""
    out = r4c.copy()
    for b, (i, j, k, l) in enumerate(quads(o)):
        B = out[b]
        if i == j < k <= l:
            B = 0.5 * (B + _vperm(B, (1, 0, 2, 3)))
        if i < j == k < l:
            B = 0.5 * (B + _vperm(B, (0, 2, 1, 3)))
        if i <= j < k == l:
            B = 0.5 * (B + _vperm(B, (0, 1, 3, 2)))
        out[b] = B
    return out


def purify4(r4c: np.ndarray, o: int) -> np.ndarray:
    """Zero the blocks with three or four equal occupied indices (Sec. II.D.2)."""
    out = r4c.copy()
    for b, (i, j, k, l) in enumerate(quads(o)):
        if i == j == k or j == k == l:
            out[b] = 0.0
    return out


def omega(B: np.ndarray) -> np.ndarray:
    """Omega = the sum of the six transpositions of the virtual labels (appendix B)."""
    out = np.zeros_like(B)
    for x, y in itertools.combinations(range(4), 2):
        p = [0, 1, 2, 3]
        p[x], p[y] = p[y], p[x]
        out += _vperm(B, tuple(p))
    return out


def orthogonalise4_block(B: np.ndarray) -> np.ndarray:
    """(Omega - 6)(Omega - 2)(2 Omega^2 + 19 Omega + 48) / 576 applied to one v^4 block
    (Eq. T4ortho, the polynomial form)."""
    x = 2.0 * omega(omega(B)) + 19.0 * omega(B) + 48.0 * B
    x = omega(x) - 2.0 * x
    x = omega(x) - 6.0 * x
    return x / 576.0


def postprocess4(r4c: np.ndarray, o: int) -> np.ndarray:
    """Symmetrise, purify, orthogonalise (the order of Sec. II.D)."""
    out = purify4(symmetrise4(r4c, o), o)
    return np.stack([orthogonalise4_block(B) for B in out]) if len(out) else out


def projector_from_characters() -> np.ndarray:
    """1 - Pi_[4] - Pi_[3,1] as a 24 x 24 matrix on the virtual orderings: Pi_[4] =
    1/24 sum_pi P_pi and Pi_[3,1] = 3/24 sum_pi chi_[3,1](pi) P_pi with the character
    chi_[3,1](pi) = (fixed points of pi) - 1 (appendix B's table)."""
    perms = PERMS4
    index = {p: n for n, p in enumerate(perms)}
    M = np.eye(24)
    for pi in perms:
        chi = sum(1 for x in range(4) if pi[x] == x) - 1
        coef = 1.0 / 24.0 + 3.0 / 24.0 * chi
        for a, tau in enumerate(perms):
            M[index[nullspace.compose(pi, tau)], a] -= coef
    return M


def projector_polynomial() -> np.ndarray:
    """The polynomial form as a 24 x 24 matrix (Omega on the orderings)."""
    perms = PERMS4
    index = {p: n for n, p in enumerate(perms)}
    Om = np.zeros((24, 24))
    for x, y in itertools.combinations(range(4), 2):
        t = [0, 1, 2, 3]
        t[x], t[y] = t[y], t[x]
        for a, tau in enumerate(perms):
            Om[index[nullspace.compose(tuple(t), tau)], a] += 1.0
    I = np.eye(24)
    return (Om - 6 * I) @ (Om - 2 * I) @ (2 * Om @ Om + 19 * Om + 48 * I) / 576.0


def multiplicity4(i, j, k, l) -> int:
    """Number of distinct occupied quadruples that map onto the stored block."""
    return len(set(itertools.permutations((i, j, k, l))))


def residual_norm4(r4c: np.ndarray, o: int) -> float:
    """Full-tensor norm of a compact R4: sum over stored blocks of multiplicity x |block|^2."""
    w = np.array([multiplicity4(*q) for q in quads(o)], dtype=np.float64)
    return float(np.sqrt(np.sum(w * np.sum(r4c.reshape(len(w), -1) ** 2, axis=1))))
