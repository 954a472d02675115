"""RCCSDT on compact ``i <= j <= k`` storage, FP64, numpy.  TEST INFRASTRUCTURE ONLY.

Follows Sec. II.B.1 (only the i<=j<=k blocks of T3/R3 are stored, each a
contiguous v^3 array over abc), Sec. II.C (residual contributions evaluated per
stored output block: the direct traversal of the pp-ladder, unpacking of
off-triangle blocks for the hh-ladder, F_oo and ring terms, the representative
contractions of the operation-count table of appendix B) and Sec. II.D
(symmetrisation of degenerate blocks, purification, orthogonalisation).

Storage: ``t3c[blk, a, b, c]`` with the colex block index
``blk(i<=j<=k) = C(k+2, 3) + C(j+1, 2) + i`` (the paper does not fix an order).

Unpacking (Fig. t3_perm): for any occupied triple (l, m, n), sort it with a
permutation s, read the stored block of the sorted triple and apply the same
permutation to the virtual axes, using t_{lmn}^{abc} = t_{s(lmn)}^{s(abc)}
(Eq. rccsdt-amps-symm).

The T3 contributions to R1, R2, W^{ab}_{dj} and W^{al}_{ij} (step (iii) of
Sec. III.A.2) are summed here over all o^3 occupied triples of unpacked
blocks, i.e. straight from their definitions in appendix A.5.
"""
from __future__ import annotations

import itertools
from math import comb

import numpy as np

from . import rccsdt as full

einsum = full.einsum


def n3(o: int) -> int:
    return o * (o + 1) * (o + 2) // 6


def blk_index(i: int, j: int, k: int) -> int:
    assert i <= j <= k
    return comb(k + 2, 3) + comb(j + 1, 2) + i


def triples(o: int):
    """Ordered triples in storage order."""
    out = [None] * n3(o)
    for k in range(o):
        for j in range(k + 1):
            for i in range(j + 1):
                out[blk_index(i, j, k)] = (i, j, k)
    return out


def multiplicity(i, j, k) -> int:
    """Number of distinct occupied triples that map onto the stored block."""
    return len(set(itertools.permutations((i, j, k))))


def pack(t3: np.ndarray) -> np.ndarray:
    o = t3.shape[0]
    return np.ascontiguousarray(np.stack([t3[i, j, k] for (i, j, k) in triples(o)]))


def unpack_block(t3c: np.ndarray, l: int, m: int, n: int) -> np.ndarray:
    """U[x0, x1, x2] = t_{lmn}^{x0 x1 x2} from the stored block of sorted(l, m, n)."""
    occ = (l, m, n)
    s = sorted(range(3), key=lambda q: occ[q])        # occ[s[0]] <= occ[s[1]] <= occ[s[2]]
    B = t3c[blk_index(occ[s[0]], occ[s[1]], occ[s[2]])]
    # t_{lmn}^{x} = B[x[s0], x[s1], x[s2]]; B axis q holds output axis s[q]
    return np.transpose(B, np.argsort(s))


def unpack_full(t3c: np.ndarray, o: int) -> np.ndarray:
    v = t3c.shape[1]
    t3 = np.empty((o, o, o, v, v, v))
    for l, m, n in itertools.product(range(o), repeat=3):
        t3[l, m, n] = unpack_block(t3c, l, m, n)
    return t3


def _vp(U, perm):
    """u[x0,x1,x2] = U[x_perm0, x_perm1, x_perm2] for a v^3 block."""
    return np.transpose(U, np.argsort(perm))


def single_check(U):
    """(2 - P_a^b - P_a^c) on a v^3 block (first column checked)."""
    return 2.0 * U - _vp(U, (1, 0, 2)) - _vp(U, (2, 1, 0))


def double_check(U):
    """(2 - P_b^c)(2 - P_a^b - P_a^c) on a v^3 block (first two columns checked)."""
    return (4.0 * U - 2.0 * _vp(U, (1, 0, 2)) - 2.0 * _vp(U, (2, 1, 0))
            - 2.0 * _vp(U, (0, 2, 1)) + _vp(U, (2, 0, 1)) + _vp(U, (1, 2, 0)))


# ---------------------------------------------------------------------------
# Step (iii): T3 contributions to R1, R2 and the RCCSDT intermediates
# ---------------------------------------------------------------------------

def t3_contributions(eri, ft, t3c, o):
    """Returns (dR1, dX2, dWvvvo, dWvooo) summed over all o^3 unpacked blocks.

    dR1[i,a]       += 1/2 sum_jkbc v~^{jk}_{bc} t_{j^k^i}^{b^c^a}
    dX2[i,j,a,b]   += 1/2 sum_kc f~^k_c t_{k^ij}^{c^ab} + sum_kcd v~^{bk}_{cd} t_{k^ij}^{d^ac}
                      - sum_klc v~^{kl}_{jc} t_{l^ik}^{c^ab}       (before P_{(ia)(jb)})
    dWvvvo[a,b,d,j] -= sum_lme v~^{lm}_{de} t_{m^jl}^{e^ba}
    dWvooo[a,l,i,j] += sum_mde v~^{lm}_{de} t_{m^ij}^{e^ad}
    """
    v = t3c.shape[1]
    O, V = slice(0, o), slice(o, None)
    oovv, vovv, ooov = eri("oovv"), eri("vovv"), eri("ooov")
    dR1 = np.zeros((o, v))
    dX2 = np.zeros((o, o, v, v))
    dWvvvo = np.zeros((v, v, v, o))
    dWvooo = np.zeros((v, o, o, o))
    for x, y, z in itertools.product(range(o), repeat=3):
        U = unpack_block(t3c, x, y, z)          # t_{xyz}
        S = single_check(U)                      # t_{x^yz}
        D = double_check(U)                      # t_{x^y^z}
        # R1: (j,k,i) = (x,y,z)
        dR1[z] += 0.5 * einsum("bc,bca->a", oovv[x, y], D)
        # R2 term 1: (k,i,j) = (x,y,z)
        dX2[y, z] += 0.5 * einsum("c,cab->ab", ft[O, V][x], S)
        # R2 term 2: (k,i,j) = (x,y,z): v~^{bk}_{cd} t_{k^ij}^{d^ac}
        dX2[y, z] += einsum("bcd,dac->ab", vovv[:, x], S)
        # R2 term 3: (l,i,k) = (x,y,z): -sum_{kc} v~^{kl}_{jc} t_{l^ik}^{c^ab}, k = z, l = x
        dX2[y] -= einsum("jc,cab->jab", ooov[z, x], S)
        # W^{ab}_{dj}: (m,j,l) = (x,y,z): -v~^{lm}_{de} t_{m^jl}^{e^ba}
        dWvvvo[:, :, :, y] -= einsum("de,eba->abd", oovv[z, x], S)
        # W^{al}_{ij}: (m,i,j) = (x,y,z): +v~^{lm}_{de} t_{m^ij}^{e^ad}
        dWvooo[:, :, y, z] += einsum("lde,ead->al", oovv[:, x], S)
    return dR1, dX2, dWvvvo, dWvooo


def intermediates_compact(Lt, ft, t2, t3c, o):
    """RCCSD and RCCSDT intermediates, with the T3 terms of W^{ab}_{dj} and
    W^{al}_{ij} taken from compact T3.  Also returns the T3 parts of R1 and R2."""
    eri = full.Eri(Lt, o)
    I = full.intermediates(Lt, ft, t2, None, triples=True)
    dR1, dX2, dWvvvo, dWvooo = t3_contributions(eri, ft, t3c, o)
    I["Wvvvo"] = I["Wvvvo"] + dWvvvo
    I["Wvooo"] = I["Wvooo"] + dWvooo
    return I, eri, dR1, dX2


# ---------------------------------------------------------------------------
# R3 on compact storage (Sec. II.C, operation-count table)
# ---------------------------------------------------------------------------

def r3_block(I, t2, t3c, i, j, k):
    """Raw residual block r_{ijk}^{abc} for one stored i <= j <= k.

    Terms, with ``U(l,m,n)`` the unpacked block t_{lmn}:
    * T2 terms, all 6 column permutations of
      X(p1;p2;p3) = sum_d W^{a1 a2}_{d i2} t_{i1 i3}^{d a3} - sum_l W^{a1 l}_{i1 i2} t_{l i3}^{a2 a3};
    * F_vv (direct): F^a_d t^{dbc} + F^b_d t^{adc} + F^c_d t^{abd};
    * F_oo (unpacked): -(F^l_i t_{ljk}^{abc} + F^l_j t_{lik}^{bac} + F^l_k t_{lij}^{cab});
    * pp-ladder (direct traversal, three terms from the same block):
      W^{ab}_{de} t_{ijk}^{dec} + W^{ac}_{de} t_{ikj}^{deb} + W^{bc}_{de} t_{jki}^{dea};
    * hh-ladder (unpacked): W^{lm}_{ij} t_{lmk}^{abc} + W^{lm}_{ik} t_{lmj}^{acb} + W^{lm}_{jk} t_{lmi}^{bca};
    * ring, 1/2 P_{2<3}[Wbar^{la}_{di} t_{l^jk}^{d^bc}];
    * ring, -1/2 P_{2<3}[Wbar^{la}_{id}(t_{jlk}^{dbc} + t_{klj}^{dcb})];
    * ring, -P[Wbar^{lb}_{id} t_{jlk}^{dac}] (all 6).
    """
    o = t2.shape[0]
    T = t3c[blk_index(i, j, k)]
    pairs = ((i, 0), (j, 1), (k, 2))        # (occupied index, virtual axis of the output)
    Wvvvo, Wvooo = I["Wvvvo"], I["Wvooo"]
    Fvv, Foo, Woooo, Wvvvv = I["Fvv"], I["Foo"], I["Woooo"], I["Wvvvv"]
    Wb_vo, Wb_ov = I["Wbar_ovvo"], I["Wbar_ovov"]
    labels = "abc"
    R = np.zeros_like(T)

    # -- T2-driven terms, all 6 permutations
    for (i1, x1), (i2, x2), (i3, x3) in itertools.permutations(pairs):
        s1, s2, s3 = labels[x1], labels[x2], labels[x3]
        R += einsum(f"{s1}{s2}d,d{s3}->abc", Wvvvo[:, :, :, i2], t2[i1, i3])
        R -= einsum(f"{s1}l,l{s2}{s3}->abc", Wvooo[:, :, i1, i2], t2[:, i3])

    # -- F_vv, direct
    R += einsum("ad,dbc->abc", Fvv, T) + einsum("bd,adc->abc", Fvv, T) + einsum("cd,abd->abc", Fvv, T)

    # -- F_oo, unpacked: positions p1 = (i,a),(j,b),(k,c) in turn
    for (i1, x1), (i2, x2), (i3, x3) in ((pairs[0], pairs[1], pairs[2]),
                                          (pairs[1], pairs[0], pairs[2]),
                                          (pairs[2], pairs[0], pairs[1])):
        for l in range(o):
            U = unpack_block(t3c, l, i2, i3)
            R -= Foo[l, i1] * einsum(f"{labels[x1]}{labels[x2]}{labels[x3]}->abc", U)

    # -- pp-ladder, direct traversal of the one stored block
    R += einsum("abde,dec->abc", Wvvvv, T)          # W^{ab}_{de} t_ijk^{dec}
    R += einsum("acde,dbe->abc", Wvvvv, T)          # W^{ac}_{de} t_ikj^{deb} = t_ijk^{dbe}
    R += einsum("bcde,ade->abc", Wvvvv, T)          # W^{bc}_{de} t_jki^{dea} = t_ijk^{ade}

    # -- hh-ladder, unpacked: P_{1<2}
    for (i1, x1), (i2, x2), (i3, x3) in ((pairs[0], pairs[1], pairs[2]),
                                          (pairs[0], pairs[2], pairs[1]),
                                          (pairs[1], pairs[2], pairs[0])):
        for l in range(o):
            for m in range(o):
                U = unpack_block(t3c, l, m, i3)
                R += Woooo[l, m, i1, i2] * einsum(f"{labels[x1]}{labels[x2]}{labels[x3]}->abc", U)

    # -- ring terms with P_{2<3}
    for (i1, x1), (i2, x2), (i3, x3) in ((pairs[0], pairs[1], pairs[2]),
                                          (pairs[1], pairs[0], pairs[2]),
                                          (pairs[2], pairs[0], pairs[1])):
        s1, s2, s3 = labels[x1], labels[x2], labels[x3]
        for l in range(o):
            # 1/2 Wbar^{l a1}_{d i1} t_{l^ i2 i3}^{d^ a2 a3}
            S = single_check(unpack_block(t3c, l, i2, i3))
            R += 0.5 * einsum(f"{s1}d,d{s2}{s3}->abc", Wb_vo[l, :, :, i1], S)
            # -1/2 Wbar^{l a1}_{i1 d} (t_{i2 l i3}^{d a2 a3} + t_{i3 l i2}^{d a3 a2})
            U1 = unpack_block(t3c, i2, l, i3)
            U2 = unpack_block(t3c, i3, l, i2)
            R -= 0.5 * einsum(f"{s1}d,d{s2}{s3}->abc", Wb_ov[l, :, i1, :], U1)
            R -= 0.5 * einsum(f"{s1}d,d{s3}{s2}->abc", Wb_ov[l, :, i1, :], U2)

    # -- ring term, all 6 permutations: -Wbar^{l a2}_{i1 d} t_{i2 l i3}^{d a1 a3}
    for (i1, x1), (i2, x2), (i3, x3) in itertools.permutations(pairs):
        s1, s2, s3 = labels[x1], labels[x2], labels[x3]
        for l in range(o):
            U = unpack_block(t3c, i2, l, i3)
            R -= einsum(f"{s2}d,d{s1}{s3}->abc", Wb_ov[l, :, i1, :], U)
    return R


def residuals_compact(L, fock_diag, t1, t2, t3c, return_intermediates=False):
    """Raw (r1, r2, r3c) with compact T3 in and out; no post-processing."""
    o, v = t1.shape
    O, V = slice(0, o), slice(o, None)
    Lt, ft = full.dress(L, fock_diag, t1)
    I, eri, dR1, dX2 = intermediates_compact(Lt, ft, t2, t3c, o)
    ts2 = full.spin_sum_t2(t2)
    r1 = (ft[V, O].T.copy()
          + einsum("kc,ikac->ia", ft[O, V], ts2)
          + einsum("akcd,ikcd->ia", eri("vovv"), ts2)
          - einsum("klic,klac->ia", eri("ooov"), ts2)
          + dR1)
    X2 = (0.5 * eri("vvoo").transpose(2, 3, 0, 1)
          + einsum("bc,ijac->ijab", I["Fvv"], t2)
          - einsum("kj,ikab->ijab", I["Foo"], t2)
          + 0.5 * einsum("abcd,ijcd->ijab", eri("vvvv"), t2)
          + 0.5 * einsum("klij,klab->ijab", I["Woooo"], t2)
          + 0.5 * einsum("kaci,kjcb->ijab", I["Wovvo"], ts2)
          - 0.5 * einsum("kaic,jkcb->ijab", I["Wovov"], t2)
          - einsum("kbic,jkca->ijab", I["Wovov"], t2)
          + dX2)
    r2 = full.perm_op2(X2)
    r3c = np.stack([r3_block(I, t2, t3c, i, j, k) for (i, j, k) in triples(o)])
    if return_intermediates:
        return r1, r2, r3c, I
    return r1, r2, r3c


# ---------------------------------------------------------------------------
# Post-processing and update on compact storage (Sec. II.D, A.1)
# ---------------------------------------------------------------------------

def symmetrise(r3c, o):
    """i = j < k: r <- 1/2 (r^{abc} + r^{bac});  i < j = k: r <- 1/2 (r^{abc} + r^{acb})."""
    out = r3c.copy()
    for b, (i, j, k) in enumerate(triples(o)):
        if i == j and j < k:
            out[b] = 0.5 * (r3c[b] + r3c[b].transpose(1, 0, 2))
        elif i < j and j == k:
            out[b] = 0.5 * (r3c[b] + r3c[b].transpose(0, 2, 1))
    return out


def purify(r3c, o):
    out = r3c.copy()
    for b, (i, j, k) in enumerate(triples(o)):
        if i == j == k:
            out[b] = 0.0
    return out


def orthogonalise(r3c):
    """r <- r - 1/6 sum_{pi in S3} r^{pi(abc)} on every stored block."""
    mean = sum(np.transpose(r3c, (0,) + tuple(1 + np.argsort(p))) for p in full.PERMS3) / 6.0
    return r3c - mean


def postprocess(r3c, o):
    """Symmetrise, purify, orthogonalise (paper order, Sec. II.D)."""
    return orthogonalise(purify(symmetrise(r3c, o), o))


def denom3c(e, o):
    ev = e[o:]
    dv = ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
    return np.stack([(e[i] + e[j] + e[k]) - dv for (i, j, k) in triples(o)])


def weights(o):
    return np.array([multiplicity(*t) for t in triples(o)], dtype=np.float64)


def residual_norm(r1, r2, r3c, o):
    """sqrt(|r1|^2 + |r2|^2 + sum_blk m(blk) |r3_blk|^2): the full-tensor norm."""
    w = weights(o)
    return float(np.sqrt(np.sum(r1 ** 2) + np.sum(r2 ** 2)
                         + np.sum(w * np.sum(r3c.reshape(len(w), -1) ** 2, axis=1))))


def solve_compact(L, fock_diag, o, tol=1e-10, max_iter=200, diis_space=8, diis_start=2,
                  verbose=False, callback=None, diis_t3_nvir=None):
    """RCCSDT iterations on compact storage from t1 = 0, t2 = MP2, t3 = 0.

    Each iteration: raw residuals, post-processing of R3, norm, energy, Jacobi
    step, DIIS over (t1, t2, sqrt(m) t3c).  With ``diis_t3_nvir = ns`` the T3 part of
    the DIIS vectors keeps only the components with all three virtual labels below
    ns (the DIIS in a reduced virtual subspace of Sec. III.A.5); the other T3
    components keep their Jacobi step.  Returns (E, t1, t2, t3c, iters, history).
    """
    e = np.asarray(fock_diag, dtype=np.float64)
    v = len(e) - o
    t1 = np.zeros((o, v))
    t2 = full.mp2_t2(L, e, o)
    t3c = np.zeros((n3(o), v, v, v))
    d1, d2, d3 = full.denom1(e, o), full.denom2(e, o), denom3c(e, o)
    sw = np.sqrt(weights(o))[:, None, None, None]
    ns = v if diis_t3_nvir is None or not 0 < diis_t3_nvir < v else diis_t3_nvir
    diis = full.Diis(diis_space)
    hist = []
    for it in range(1, max_iter + 1):
        r1, r2, r3c = residuals_compact(L, e, t1, t2, t3c)
        r3c = postprocess(r3c, o)
        norm = residual_norm(r1, r2, r3c, o)
        E = full.energy(L, e, t1, t2)
        hist.append((it, E, norm))
        if verbose:
            print(f"iter {it:3d}  E = {E:.14f}  |R| = {norm:.3e}", flush=True)
        if callback is not None:
            callback(it, E, norm)
        if norm <= tol:
            return E, t1, t2, t3c, it, hist
        n1, n2, n3c = t1 + r1 / d1, t2 + r2 / d2, t3c + r3c / d3
        sub = (slice(None), slice(0, ns), slice(0, ns), slice(0, ns))
        vec = np.concatenate([n1.ravel(), n2.ravel(), (sw * n3c)[sub].ravel()])
        old = np.concatenate([t1.ravel(), t2.ravel(), (sw * t3c)[sub].ravel()])
        diis.push(vec, vec - old)
        if it >= diis_start:
            vec = diis.extrapolate()
        t1 = vec[: o * v].reshape(o, v)
        t2 = vec[o * v: o * v + (o * v) ** 2].reshape(o, o, v, v)
        t3c = n3c.copy()
        t3c[sub] = vec[o * v + (o * v) ** 2:].reshape(len(t3c), ns, ns, ns) / sw
    raise RuntimeError(f"RCCSDT (compact) did not converge in {max_iter} iterations")
