"""RCCSDT(Q) perturbative quadruples energy correction, full storage, FP64, numpy.
TEST INFRASTRUCTURE ONLY (never imported by the library's product path).

Written from the paper's appendix on the (Q) energy correction (Eqs. ener-pt-q,
resi-pt-q, q_t3_terms, q_w_vvv_voo, q_w_vvo_ooo, the alternative intermediates of
q_w_alter) with the spin summations of Eq. quadruples-spin-sum, the paired-index
permutation operator of Eq. rcc-perm-op and the orbital-energy denominators of
Eq. orb-energy-deno.  Conventions as in ``oracle.rccsdt``: occupied orbitals first,
``v[p, q, r, s] = v^{pq}_{rs} = (pr|qs)`` from the BARE factors (the (Q) correction
uses undressed integrals), spin-free ``t2[i, j, a, b]``, ``t3[i, j, k, a, b, c]``;
quadruples arrays ``x[i, j, k, l, a, b, c, d]`` (lower indices first).

Pinned in ``tests/test_oracle_pins.py`` against the determinant-space spin-orbital
CCSDT(Q) energy (``oracle.detcc``) built from its own converged CCSDT amplitudes:
    E(Q) = sum_Q <Q|V (T2 + T3)|0> <Q|V T3 + 1/2 [[V, T2], T2]|0> / D_Q.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import rccsdt as full

einsum = lambda *a: np.einsum(*a, optimize=True)  # noqa: E731

PERMS4 = list(itertools.permutations(range(4)))


def perm_pairs4(x):
    """P_{(ia)(jb)(kc)(ld)} x: the sum over the 24 simultaneous permutations of the
    paired occupied-virtual columns (Eq. rcc-perm-op)."""
    out = np.zeros_like(x)
    for p in PERMS4:
        out += x.transpose(p[0], p[1], p[2], p[3], 4 + p[0], 4 + p[1], 4 + p[2], 4 + p[3])
    return out


def _vswap(x, a, b):
    """P_a^b on the virtual labels (positions 4..7) of a quadruples array."""
    axes = list(range(8))
    axes[4 + a], axes[4 + b] = axes[4 + b], axes[4 + a]
    return x.transpose(axes)


def spin_sum_t4_full(t4):
    """The fully spin-summed quadruples amplitude of Eq. quadruples-spin-sum and the
    (Q) appendix: check on the first column (2 - P_a^b - P_a^c - P_a^d), then on the
    second (2 - P_b^c - P_b^d), then on the third (2 - P_c^d), and the fourth check
    a factor of 2."""
    s1 = 2.0 * t4 - _vswap(t4, 0, 1) - _vswap(t4, 0, 2) - _vswap(t4, 0, 3)
    s2 = 2.0 * s1 - _vswap(s1, 1, 2) - _vswap(s1, 1, 3)
    s3 = 2.0 * s2 - _vswap(s2, 2, 3)
    return 2.0 * s3


def denom4(e, o):
    """eps_{ijkl}^{abcd} = e_i + e_j + e_k + e_l - e_a - e_b - e_c - e_d."""
    eo, ev = e[:o], e[o:]
    return (eo[:, None, None, None, None, None, None, None] + eo[None, :, None, None, None, None, None, None]
            + eo[None, None, :, None, None, None, None, None] + eo[None, None, None, :, None, None, None, None]
            - ev[None, None, None, None, :, None, None, None] - ev[None, None, None, None, None, :, None, None]
            - ev[None, None, None, None, None, None, :, None] - ev[None, None, None, None, None, None, None, :])


def wbar_vvvo(v, t2, o, alternative=False):
    """Wbar_{ejk}^{abc} as [e, j, k, a, b, c] (Eq. q_w_vvv_voo): P_{(jb)(kc)} of
    1/2 sum_f v^{ab}_{ef} t_{jk}^{fc}; the alternative form (Eq. q_w_alter) adds
    - sum_m v^{mb}_{ej} t_{mk}^{ac} - sum_m v^{ma}_{je} t_{mk}^{bc} inside P."""
    O, V = slice(0, o), slice(o, None)
    a = 0.5 * einsum("abef,jkfc->ejkabc", v[V, V, V, V], t2)
    if alternative:
        a = a - einsum("mbej,mkac->ejkabc", v[O, V, V, O], t2)
        a = a - einsum("maje,mkbc->ejkabc", v[O, V, O, V], t2)
    return a + a.transpose(0, 2, 1, 3, 5, 4)


def wbar_vvoo(v, t2, o, alternative=False):
    """Wbar_{ijk}^{abm} as [i, j, k, a, b, m] (Eq. q_w_vvo_ooo): P_{(ia)(jb)} of
    sum_e v^{ma}_{ei} t_{jk}^{be} + sum_e v^{ma}_{ke} t_{ji}^{be} - 1/2 sum_n v^{mn}_{ki} t_{nj}^{ab};
    the alternative form (Eq. q_w_alter) keeps only the last term."""
    O, V = slice(0, o), slice(o, None)
    b = -0.5 * einsum("mnki,njab->ijkabm", v[O, O, O, O], t2)
    if not alternative:
        b = b + einsum("maei,jkbe->ijkabm", v[O, V, V, O], t2)
        b = b + einsum("make,jibe->ijkabm", v[O, V, O, V], t2)
    return b + b.transpose(1, 0, 2, 4, 3, 5)


def q_intermediates(v, t2, t3, o, alternative=False):
    """X, Y and V of Eqs. q_t3_terms / resi-pt-q, each [i, j, k, l, a, b, c, d]."""
    O, V = slice(0, o), slice(o, None)
    X = (0.5 * einsum("abej,iklecd->ijklabcd", v[V, V, V, O], t3)
         - 0.5 * einsum("amij,mklbcd->ijklabcd", v[V, O, O, O], t3))
    w1 = wbar_vvvo(v, t2, o, alternative)
    w2 = wbar_vvoo(v, t2, o, alternative)
    Y = 0.5 * einsum("ejkabc,iled->ijklabcd", w1, t2) - 0.5 * einsum("ijkabm,mlcd->ijklabcd", w2, t2)
    Vq = 0.25 * einsum("abij,klcd->ijklabcd", v[V, V, O, O], t2)
    return X, Y, Vq


def energy_q(L, fock_diag, t2, t3, o, alternative=False):
    """E_(Q) = 1/24 sum z t-fully-spin-summed with t = r / eps, r = P(X + Y),
    z = P(X + V) (Eq. ener-pt-q), from converged spin-free t2 and t3 and the bare
    Hamiltonian (L, fock_diag).  T1 does not enter."""
    e = np.asarray(fock_diag, dtype=np.float64)
    n = len(e)
    eri = full.Eri(np.asarray(L, dtype=np.float64), o)
    # the whole v^{pq}_{rs} (small systems only)
    v = np.zeros((n, n, n, n))
    for s in itertools.product("ov", repeat=4):
        sl = [slice(0, o) if c == "o" else slice(o, None) for c in s]
        v[sl[0], sl[1], sl[2], sl[3]] = eri("".join(s))
    X, Y, Vq = q_intermediates(v, t2, t3, o, alternative)
    r = perm_pairs4(X + Y)
    z = perm_pairs4(X + Vq)
    t4 = r / denom4(e, o)
    return float(np.sum(z * spin_sum_t4_full(t4)) / 24.0)


def degeneracy4(n):
    """f_{pqrs} of the triangular (Q) sums: 24 for p < q < r < s, 12 for one equal
    adjacent pair, 6 for p = q < r = s, 0 for every other tuple (unordered, or three
    or four equal labels: no quadruple excitation puts three electrons in one spatial
    orbital)."""
    f = np.zeros((n, n, n, n))
    for p, q, r, s in itertools.product(range(n), repeat=4):
        if not (p <= q <= r <= s):
            continue
        eq = (p == q) + (q == r) + (r == s)
        if eq == 0:
            f[p, q, r, s] = 24.0
        elif eq == 1:
            f[p, q, r, s] = 12.0
        elif eq == 2 and p == q and r == s:
            f[p, q, r, s] = 6.0
    return f


def energy_q_triangular(L, fock_diag, t2, t3, o, over="occ"):
    """E_(Q) restricted to i <= j <= k <= l (the IJK-based order) or a <= b <= c <= d
    (the ABC-based order, Eq. ener-pt-q-abc), each tuple weighted by its degeneracy
    factor f; equal to energy_q."""
    e = np.asarray(fock_diag, dtype=np.float64)
    n = len(e)
    eri = full.Eri(np.asarray(L, dtype=np.float64), o)
    v = np.zeros((n, n, n, n))
    for s in itertools.product("ov", repeat=4):
        sl = [slice(0, o) if c == "o" else slice(o, None) for c in s]
        v[sl[0], sl[1], sl[2], sl[3]] = eri("".join(s))
    X, Y, Vq = q_intermediates(v, t2, t3, o)
    r = perm_pairs4(X + Y)
    z = perm_pairs4(X + Vq)
    prod = z * spin_sum_t4_full(r / denom4(e, o))
    if over == "occ":
        return float(einsum("ijklabcd,ijkl->", prod, degeneracy4(o)) / 24.0)
    return float(einsum("ijklabcd,abcd->", prod, degeneracy4(n - o)) / 24.0)


def pack_virtual_triangular(t3c, o):
    """The one-time transposition before the ABC-based (Q) evaluation (Sec. II.E.2,
    Fig. q_operation_counts(a)): compact T3 stored by occupied
    triples i <= j <= k, each a v^3 block over abc, becomes T3 stored by virtual
    triples a <= b <= c (colex order, as the occupied blocks), each an o^3 block over
    ijk: out[blk(a, b, c)][i, j, k] = t_{ijk}^{abc}."""
    from . import compact as cmp
    v = t3c.shape[1]
    t3 = cmp.unpack_full(np.asarray(t3c), o)
    return np.ascontiguousarray(np.stack([t3[:, :, :, a, b, c] for (a, b, c) in cmp.triples(v)]))


def unpack_virtual_triangular(t3v, o, v):
    """The full t_{ijk}^{abc} from the virtual-triangular layout, reading the stored
    (a, b, c) block of sorted(a, b, c) with the occupied axes permuted by the same
    sort (the column-permutation symmetry, as for the occupied-triangular layout)."""
    from . import compact as cmp
    t3 = np.empty((o, o, o, v, v, v))
    for a, b, c in itertools.product(range(v), repeat=3):
        lab = (a, b, c)
        s = sorted(range(3), key=lambda q: lab[q])
        blk = t3v[cmp.blk_index(lab[s[0]], lab[s[1]], lab[s[2]])]   # blk[y0, y1, y2]: occupied of sorted labels
        t3[:, :, :, a, b, c] = np.transpose(blk, np.argsort(s))
    return t3
