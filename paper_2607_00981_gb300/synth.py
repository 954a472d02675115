"""Seeded synthetic closed-shell Hamiltonians shaped like the paper's workloads.

This module only draws random numbers; it holds none of the coupled-cluster
arithmetic, so both the CPU oracle (through the tests) and the CUDA path can
be fed from it.  numpy's ``default_rng`` (PCG64) is used, with this fixed
draw order for one instance:

1. ``A = standard_normal((naux, n, n))`` with ``n = o + v``;
2. ``L = 0.5 * (A + A^T) * scale * exp(-|p - q| / 4)``  (symmetric in p,q);
3. occupied orbital energies ``sort(uniform(-2.0, -0.5, o))``;
4. virtual orbital energies ``sort(uniform(0.2, 5.0, v))``.

The ERIs are the low-rank product ``(pq|rs) = sum_P L[P,p,q] L[P,r,s]`` and the
Fock matrix is diagonal (canonical orbitals, occupied first).  The batched
workload draws ``o`` in [3, 8] and ``v`` in [20, 60] from seed 0 and gives
instance ``i`` the seed ``1000 + i`` with ``naux = 4 (o + v)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Instance:
    """One synthetic problem: spatial orbital counts, factors and Fock diagonal."""

    o: int
    v: int
    naux: int
    seed: int
    L: np.ndarray          # [naux][n][n] float64, symmetric in the last two axes
    fock_diag: np.ndarray  # [n] float64, occupied first

    @property
    def n(self) -> int:
        return self.o + self.v


def make_instance(o: int, v: int, naux: int, seed: int = 0, scale: float = 0.3) -> Instance:
    """Draw one seeded instance with the recipe in the module docstring."""
    if o < 1 or v < 1 or naux < 1:
        raise ValueError("o, v and naux must be positive")
    n = o + v
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((naux, n, n))
    p = np.arange(n)
    envelope = scale * np.exp(-np.abs(p[:, None] - p[None, :]) / 4.0)
    L = 0.5 * (A + A.transpose(0, 2, 1)) * envelope[None, :, :]
    e_occ = np.sort(rng.uniform(-2.0, -0.5, o))
    e_vir = np.sort(rng.uniform(0.2, 5.0, v))
    return Instance(o=o, v=v, naux=naux, seed=seed, L=np.ascontiguousarray(L),
                    fock_diag=np.concatenate([e_occ, e_vir]))


# The five workloads, by size.  naux follows the stated ranks.
WORKLOADS = {
    "o3v12": dict(o=3, v=12, naux=40, seed=0),
    "o8v80": dict(o=8, v=80, naux=320, seed=0),
    "o12v120": dict(o=12, v=120, naux=480, seed=0),
    "o16v160": dict(o=16, v=160, naux=640, seed=0),
}


# Weakly coupled instances for runs that must converge.  With the per-entry scale
# fixed at 0.3 the ERIs grow with the rank and the iteration stalls or diverges at
# these sizes; here the scale is 0.6 * 0.3 * sqrt(40 / naux) (rank-normalised,
# then reduced).
CONVERGENCE = {
    "o6v48w": dict(o=6, v=48, naux=216, seed=7, scale=0.6 * 0.3 * (40 / 216) ** 0.5),
    "o8v80w": dict(o=8, v=80, naux=320, seed=0, scale=0.6 * 0.3 * (40 / 320) ** 0.5),
    "o12v120w": dict(o=12, v=120, naux=480, seed=0, scale=0.6 * 0.3 * (40 / 480) ** 0.5),
    "o16v160w": dict(o=16, v=160, naux=640, seed=0, scale=0.6 * 0.3 * (40 / 640) ** 0.5),
}


def workload(name: str) -> Instance:
    spec = WORKLOADS.get(name) or CONVERGENCE[name]
    return make_instance(**spec)


def batch_shapes(count: int = 64, seed: int = 0):
    """(o, v, naux, seed) of the batched uneven-instance workload."""
    rng = np.random.default_rng(seed)
    o = rng.integers(3, 9, size=count)
    v = rng.integers(20, 61, size=count)
    return [(int(oi), int(vi), int(4 * (oi + vi)), 1000 + i) for i, (oi, vi) in enumerate(zip(o, v))]


def batch_instances(count: int = 64, seed: int = 0, weak: bool = True):
    """The batched uneven-instance workload: ``batch_shapes`` with each instance's
    factors drawn by ``make_instance``.  With ``weak`` the per-entry scale is the
    rank-normalised, reduced ``0.6 * 0.3 * sqrt(40 / naux)`` of ``CONVERGENCE`` (the
    scale 0.3 of the other workloads makes these ranks strongly coupled)."""
    out = []
    for o, v, naux, sd in batch_shapes(count, seed):
        scale = 0.6 * 0.3 * (40 / naux) ** 0.5 if weak else 0.3
        out.append(make_instance(o, v, naux, sd, scale=scale))
    return out


def _orbit_copy(y: np.ndarray, perms) -> np.ndarray:
    """Copy one drawn value to every image of its orbit under the axis permutations
    ``perms`` (a group, identity included): each element takes the value of the
    image with the smallest flat index.  Values keep all 53 bits; the symmetries
    hold bit for bit because equal positions read the same draw."""
    idx = np.arange(y.size).reshape(y.shape)
    rep = idx
    for p in perms:
        rep = np.minimum(rep, idx.transpose(p))
    return y.reshape(-1)[rep]


_T2_PERMS = [(0, 1, 2, 3), (1, 0, 3, 2)]
_S3 = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
_T3_PERMS = [p + tuple(3 + q for q in p) for p in _S3]


def random_amplitudes(o: int, v: int, seed: int, scale: float = 0.05):
    """Seeded (t1, t2, t3) with the spin-free column symmetries, for parity tests.

    t2[i,j,a,b] = t2[j,i,b,a]; t3 is full [o,o,o,v,v,v] and invariant under the six
    simultaneous permutations of its (occupied, virtual) column pairs.  One normal
    draw per orbit of those permutations is copied to every image, so the values
    carry full 53-bit mantissas (FP32 storage of T3 rounds them).  These are plain
    random numbers, not solutions of any equation.
    """
    rng = np.random.default_rng(seed)
    t1 = scale * rng.standard_normal((o, v))
    t2 = _orbit_copy(scale * rng.standard_normal((o, o, v, v)), _T2_PERMS)
    t3 = _orbit_copy(scale * rng.standard_normal((o, o, o, v, v, v)), _T3_PERMS)
    return t1, t2, t3


def random_amplitudes_compact(o: int, v: int, seed: int, scale: float = 0.05):
    """As ``random_amplitudes`` with T3 drawn directly in compact storage
    ``t3c[n3][v][v][v]`` (colex blocks i <= j <= k, the library's layout), for sizes
    whose full o^3 v^3 tensor is too large to draw.  Inside a stored block the
    column symmetries that map the block onto itself are imposed by the same orbit
    copy: a <-> b for i = j < k, b <-> c for i < j = k, all six orders of abc for
    i = j = k."""
    rng = np.random.default_rng(seed)
    t1 = scale * rng.standard_normal((o, v))
    t2 = _orbit_copy(scale * rng.standard_normal((o, o, v, v)), _T2_PERMS)
    blocks = []
    for k in range(o):
        for j in range(k + 1):
            for i in range(j + 1):
                y = scale * rng.standard_normal((v, v, v))
                if i == j == k:
                    y = _orbit_copy(y, _S3)
                elif i == j:
                    y = _orbit_copy(y, [(0, 1, 2), (1, 0, 2)])
                elif j == k:
                    y = _orbit_copy(y, [(0, 1, 2), (0, 2, 1)])
                blocks.append(y)
    return t1, t2, np.ascontiguousarray(np.stack(blocks))


_S4 = [(0, 1, 2, 3), (0, 1, 3, 2), (0, 2, 1, 3), (0, 2, 3, 1), (0, 3, 1, 2), (0, 3, 2, 1),
       (1, 0, 2, 3), (1, 0, 3, 2), (1, 2, 0, 3), (1, 2, 3, 0), (1, 3, 0, 2), (1, 3, 2, 0),
       (2, 0, 1, 3), (2, 0, 3, 1), (2, 1, 0, 3), (2, 1, 3, 0), (2, 3, 0, 1), (2, 3, 1, 0),
       (3, 0, 1, 2), (3, 0, 2, 1), (3, 1, 0, 2), (3, 1, 2, 0), (3, 2, 0, 1), (3, 2, 1, 0)]


def random_t4(o: int, v: int, seed: int, scale: float = 0.05):
    """Seeded full quadruples tensor t4[i,j,k,l,a,b,c,d] invariant under the 24 joint
    permutations of its (occupied, virtual) column pairs (one full-precision draw per
    orbit, copied to every image), for small sizes."""
    rng = np.random.default_rng(seed)
    perms = [p + tuple(4 + q for q in p) for p in _S4]
    return _orbit_copy(scale * rng.standard_normal((o,) * 4 + (v,) * 4), perms)


def random_pair_symmetric(v: int, seed: int, scale: float = 0.1):
    """Seeded W[a,b,e,f] with the pair-exchange symmetry W[a,b,e,f] = W[b,a,f,e] (the
    symmetry of the particle-particle ladder intermediate), full-precision values."""
    rng = np.random.default_rng(seed)
    return _orbit_copy(scale * rng.standard_normal((v, v, v, v)), [(0, 1, 2, 3), (1, 0, 3, 2)])
