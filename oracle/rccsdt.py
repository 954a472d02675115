"""RCCSD / RCCSDT on full storage, FP64, numpy.  TEST INFRASTRUCTURE ONLY.

Written from the paper's appendix A (notation of A.2, Hamiltonian of A.3,
T1-dressing of A.4, working equations of A.5 "RCCSD" and "RCCSDT") and the
DIIS of Sec. III.A.5.  Array conventions (all row-major numpy):

* orbitals are ordered occupied first, ``n = o + v``;
* ``L[P, p, q]`` factorises the chemists' ERIs, ``(pq|rs) = sum_P L[P,p,q] L[P,r,s]``;
* physicists' integrals ``v[p, q, r, s] = v^{pq}_{rs} = (pr|qs)``;
* ``t1[i, a]``, ``t2[i, j, a, b]``, ``t3[i, j, k, a, b, c]`` are the spin-free
  amplitudes (upper = virtual, lower = occupied);
* intermediates keep the paper's index order, upper indices first:
  ``Fvv[a, d] = F^a_d``, ``Foo[l, i] = F^l_i``, ``Woooo[k, l, i, j] = W^{kl}_{ij}``,
  ``Wovvo[k, a, c, i] = W^{ka}_{ci}``, ``Wovov[k, a, i, c] = W^{ka}_{ic}``,
  ``Wvvvo[a, b, d, j] = W^{ab}_{dj}``, ``Wvooo[a, l, i, j] = W^{al}_{ij}``,
  ``Wvvvv[a, b, d, e] = W^{ab}_{de}``.

Readings of the paper used here (each is listed with its reason in the design
notes): the energy uses the bare ``v`` and ``f``; the R2 term with ``f^k_c`` sums
over ``k, c``; the Fock-like terms of R3 use the RCCSD intermediates ``F``; the
denominators use the bare Fock diagonal; the post-processing order is
symmetrise, purify, orthogonalise; the DIIS error vector is the Jacobi step.
"""
from __future__ import annotations

import itertools

import numpy as np

PERMS3 = list(itertools.permutations(range(3)))

einsum = lambda *a: np.einsum(*a, optimize=True)  # noqa: E731


# ---------------------------------------------------------------------------
# Hamiltonian and T1-dressing (appendix A.3, A.4)
# ---------------------------------------------------------------------------

def bare_fock(fock_diag: np.ndarray) -> np.ndarray:
    return np.diag(np.asarray(fock_diag, dtype=np.float64))


def dress(L: np.ndarray, fock_diag: np.ndarray, t1: np.ndarray):
    """T1-dressed factors and Fock matrix (appendix A.4).

    ``t1`` embeds into the (n x n) matrix whose vo block is ``t_i^a`` (row a,
    column i); ``x = I - t1``, ``y = I + t1^T``.  The dressed integrals are
    ``v~^{pq}_{rs} = sum x_pt x_qu v^{tu}_{vw} y_rv y_sw``; with
    ``v^{tu}_{vw} = sum_P L[P,t,v] L[P,u,w]`` this is
    ``v~^{pq}_{rs} = sum_P Lt[P,p,r] Lt[P,q,s]`` with ``Lt[P] = x L[P] y^T``.
    The dressed Fock matrix is ``f~ = x [f + G(t1)] y^T`` with
    ``G_rs = sum_ia (2 v^{ri}_{sa} - v^{ri}_{as}) t_i^a``.
    Returns ``(Lt, ft)`` with ``ft[p, q] = f~^p_q``.
    """
    o, v = t1.shape
    n = o + v
    T = np.zeros((n, n))
    T[o:, :o] = t1.T
    x = np.eye(n) - T
    y = np.eye(n) + T.T
    Lt = einsum("pt,Ptv,rv->Ppr", x, L, y)
    # v^{ri}_{sa} = (rs|ia);  v^{ri}_{as} = (ra|is)
    J = einsum("Prs,Pia,ia->rs", L, L[:, :o, o:], t1)
    K = einsum("Pra,Pis,ia->rs", L[:, :, o:], L[:, :o, :], t1)
    F = bare_fock(fock_diag) + 2.0 * J - K
    ft = x @ F @ y.T
    return Lt, ft


class Eri:
    """Blocks of ``v^{pq}_{rs} = sum_P Lt[P,p,r] Lt[P,q,s]`` by orbital space."""

    def __init__(self, Lt: np.ndarray, o: int):
        self.Lt = Lt
        self.o = o
        self._cache = {}

    def _sl(self, c):
        return slice(0, self.o) if c == "o" else slice(self.o, None)

    def __call__(self, spaces: str) -> np.ndarray:
        if spaces not in self._cache:
            p, q, r, s = (self._sl(c) for c in spaces)
            A = self.Lt[:, p, r]
            B = self.Lt[:, q, s]
            P = A.shape[0]
            M = A.reshape(P, -1).T @ B.reshape(P, -1)
            M = M.reshape(A.shape[1], A.shape[2], B.shape[1], B.shape[2])
            self._cache[spaces] = np.ascontiguousarray(M.transpose(0, 2, 1, 3))
        return self._cache[spaces]


# ---------------------------------------------------------------------------
# Spin summation (appendix A.5, "check" notation)
# ---------------------------------------------------------------------------

def spin_sum_t2(t2):
    """t_{i^j}^{a^b} = (2 - P_a^b) t_ij^ab = 2 t_ij^ab - t_ij^ba."""
    return 2.0 * t2 - t2.transpose(0, 1, 3, 2)


def vperm(t3, perm):
    """Array u with u[i,j,k,x0,x1,x2] = t3[i,j,k, x_perm[0], x_perm[1], x_perm[2]]."""
    inv = np.argsort(perm)
    return t3.transpose(0, 1, 2, 3 + inv[0], 3 + inv[1], 3 + inv[2])


def spin_sum_t3_single(t3):
    """Check on the first column: (2 - P_a^b - P_a^c) t^{abc} = 2t^{abc} - t^{bac} - t^{cba}."""
    return 2.0 * t3 - vperm(t3, (1, 0, 2)) - vperm(t3, (2, 1, 0))


def spin_sum_t3_double(t3):
    """Checks on the first two columns, Eq. triples-spin-sum:
    (2 - P_b^c)(2 - P_a^b - P_a^c) t^{abc}
      = 4t^{abc} - 2t^{bac} - 2t^{cba} - 2t^{acb} + t^{cab} + t^{bca}."""
    return (4.0 * t3 - 2.0 * vperm(t3, (1, 0, 2)) - 2.0 * vperm(t3, (2, 1, 0))
            - 2.0 * vperm(t3, (0, 2, 1)) + vperm(t3, (2, 0, 1)) + vperm(t3, (1, 2, 0)))


def perm_op2(X):
    """P_{(ia)(jb)} X_ij^ab = X_ij^ab + X_ji^ba (Eq. rcc-perm-op, n = 2)."""
    return X + X.transpose(1, 0, 3, 2)


def perm_op3(X):
    """P_{(ia)(jb)(kc)}: the sum over the 6 simultaneous column permutations."""
    out = np.zeros_like(X)
    for p in PERMS3:
        out += X.transpose(p[0], p[1], p[2], 3 + p[0], 3 + p[1], 3 + p[2])
    return out


# ---------------------------------------------------------------------------
# Residuals
# ---------------------------------------------------------------------------

def intermediates(Lt, ft, t2, t3=None, triples=None):
    """RCCSD intermediates (A.5 RCCSD) and, if ``triples`` (default: ``t3`` given),
    the RCCSDT ones.  The T3 terms of W^{ab}_{dj} and W^{al}_{ij} are added only
    when ``t3`` (full storage) is passed."""
    if triples is None:
        triples = t3 is not None
    o = t2.shape[0]
    eri = Eri(Lt, o)
    O, V = slice(0, o), slice(o, None)
    oovv = eri("oovv")
    vs_oovv = 2.0 * oovv - oovv.transpose(0, 1, 3, 2)   # v^{k^l}_{d^c} at [k,l,d,c]
    ts2 = spin_sum_t2(t2)
    I = {}
    # F^b_c = f~^b_c - sum_kld v^{k^l}_{d^c} t_kl^db
    I["Fvv"] = ft[V, V] - einsum("kldc,kldb->bc", vs_oovv, t2)
    # F^k_j = f~^k_j + sum_lcd v^{l^k}_{c^d} t_lj^cd
    I["Foo"] = ft[O, O] + einsum("lkcd,ljcd->kj", vs_oovv, t2)
    # W^{kl}_{ij} = v~^{kl}_{ij} + sum_cd v~^{kl}_{cd} t_ij^cd
    I["Woooo"] = eri("oooo") + einsum("klcd,ijcd->klij", oovv, t2)
    # W^{ka}_{ci} = v~^{k^a}_{c^i} + 1/2 sum_ld v~^{l^k}_{d^c} t_{l^i}^{d^a}
    ovvo = eri("ovvo")
    ovov = eri("ovov")
    I["Wovvo"] = (2.0 * ovvo - ovov.transpose(0, 1, 3, 2)
                  + 0.5 * einsum("lkdc,lida->kaci", vs_oovv, ts2))
    # W^{ka}_{ic} = v~^{ka}_{ic} - 1/2 sum_ld v~^{lk}_{cd} t_il^da
    I["Wovov"] = ovov - 0.5 * einsum("lkcd,ilda->kaic", oovv, t2)
    if not triples:
        return I
    ovvv = eri("ovvv")
    oovo = eri("oovo")
    ooov = eri("ooov")
    vs_ovvv = 2.0 * ovvv - ovvv.transpose(0, 1, 3, 2)   # v~^{l^a}_{e^d} at [l,a,e,d]
    # W^{ab}_{dj}
    I["Wvvvo"] = (eri("vvvo")
                  + 0.5 * einsum("laed,ljeb->abdj", vs_ovvv, ts2)
                  - 0.5 * einsum("lade,jleb->abdj", ovvv, t2)
                  - einsum("lbde,jlea->abdj", ovvv, t2)
                  + einsum("lmdj,lmab->abdj", oovo, t2))
    # W^{al}_{ij}
    vs_oovo = 2.0 * oovo - ooov.transpose(0, 1, 3, 2)   # v~^{m^l}_{d^j} at [m,l,d,j]
    I["Wvooo"] = (eri("vooo")
                  + einsum("ld,ijad->alij", ft[O, V], t2)
                  + 0.5 * einsum("mldj,mida->alij", vs_oovo, ts2)
                  - 0.5 * einsum("mljd,imda->alij", ooov, t2)
                  - einsum("mlid,jmda->alij", ooov, t2)
                  + einsum("alde,ijde->alij", eri("vovv"), t2))
    if t3 is not None:
        ss3 = spin_sum_t3_single(t3)
        I["Wvvvo"] = I["Wvvvo"] - einsum("lmde,mjleba->abdj", oovv, ss3)
        I["Wvooo"] = I["Wvooo"] + einsum("lmde,mijead->alij", oovv, ss3)
    # Wbar^{la}_{di} = W^{la}_{di} + 1/2 sum_me v~^{m^l}_{e^d} t_{m^i}^{e^a}
    I["Wbar_ovvo"] = I["Wovvo"] + 0.5 * einsum("mled,miea->ladi", vs_oovv, ts2)
    # Wbar^{la}_{id} = W^{la}_{id} - 1/2 sum_me v~^{ml}_{de} t_im^ea
    I["Wbar_ovov"] = I["Wovov"] - 0.5 * einsum("mlde,imea->laid", oovv, t2)
    # W^{ab}_{de} = v~^{ab}_{de} + sum_lm v~^{lm}_{de} t_lm^ab
    I["Wvvvv"] = eri("vvvv") + einsum("lmde,lmab->abde", oovv, t2)
    return I


def residuals(L, fock_diag, t1, t2, t3=None, return_intermediates=False):
    """Raw RCCSD (``t3 is None``) or RCCSDT residuals on full storage.

    R1 and R2 follow Eqs. ccsd_r1 / ccsd_r2 plus the T3 corrections of A.5
    RCCSDT; R3 is Eq. resi-rccsdt with the 6-term permutation operator written
    out.  No post-processing is applied here.
    """
    o, v = t1.shape
    O, V = slice(0, o), slice(o, None)
    Lt, ft = dress(L, fock_diag, t1)
    eri = Eri(Lt, o)
    I = intermediates(Lt, ft, t2, t3)
    ts2 = spin_sum_t2(t2)

    # ---- R1 (Eq. ccsd_r1)
    r1 = (ft[V, O].T.copy()
          + einsum("kc,ikac->ia", ft[O, V], ts2)
          + einsum("akcd,ikcd->ia", eri("vovv"), ts2)
          - einsum("klic,klac->ia", eri("ooov"), ts2))

    # ---- R2 (Eq. ccsd_r2), term order as printed
    X2 = (0.5 * eri("vvoo").transpose(2, 3, 0, 1)
          + einsum("bc,ijac->ijab", I["Fvv"], t2)
          - einsum("kj,ikab->ijab", I["Foo"], t2)
          + 0.5 * einsum("abcd,ijcd->ijab", eri("vvvv"), t2)
          + 0.5 * einsum("klij,klab->ijab", I["Woooo"], t2)
          + 0.5 * einsum("kaci,kjcb->ijab", I["Wovvo"], ts2)
          - 0.5 * einsum("kaic,jkcb->ijab", I["Wovov"], t2)
          - einsum("kbic,jkca->ijab", I["Wovov"], t2))

    r3 = None
    if t3 is not None:
        ss3 = spin_sum_t3_single(t3)
        ds3 = spin_sum_t3_double(t3)
        # R1 += 1/2 sum_jkbc v~^{jk}_{bc} t_{j^k^i}^{b^c^a}
        r1 = r1 + 0.5 * einsum("jkbc,jkibca->ia", eri("oovv"), ds3)
        # R2 += P( 1/2 f~^k_c t_{k^ij}^{c^ab} + v~^{bk}_{cd} t_{k^ij}^{d^ac} - v~^{kl}_{jc} t_{l^ik}^{c^ab} )
        X2 = (X2
              + 0.5 * einsum("kc,kijcab->ijab", ft[O, V], ss3)
              + einsum("bkcd,kijdac->ijab", eri("vovv"), ss3)
              - einsum("kljc,likcab->ijab", eri("ooov"), ss3))
        # R3 (Eq. resi-rccsdt), the bracket before the permutation operator
        X3 = (einsum("abdj,ikdc->ijkabc", I["Wvvvo"], t2)
              - einsum("alij,lkbc->ijkabc", I["Wvooo"], t2)
              + 0.5 * einsum("ad,ijkdbc->ijkabc", I["Fvv"], t3)
              - 0.5 * einsum("li,ljkabc->ijkabc", I["Foo"], t3)
              + 0.25 * einsum("ladi,ljkdbc->ijkabc", I["Wbar_ovvo"], ss3)
              - 0.5 * einsum("laid,jlkdbc->ijkabc", I["Wbar_ovov"], t3)
              - einsum("lbid,jlkdac->ijkabc", I["Wbar_ovov"], t3)
              + 0.5 * einsum("lmij,lmkabc->ijkabc", I["Woooo"], t3)
              + 0.5 * einsum("abde,ijkdec->ijkabc", I["Wvvvv"], t3))
        r3 = perm_op3(X3)
    r2 = perm_op2(X2)
    if return_intermediates:
        return r1, r2, r3, I
    return r1, r2, r3


def energy(L, fock_diag, t1, t2):
    """E = sum v^{i^j}_{a^b}(t_ij^ab + t_i^a t_j^b) + 2 sum f^i_a t_i^a, bare v and f (A.5)."""
    o = t1.shape[0]
    ovov = einsum("Pia,Pjb->iajb", L[:, :o, o:], L[:, :o, o:])  # (ia|jb) = v^{ij}_{ab}
    v_ijab = ovov.transpose(0, 2, 1, 3)
    vs = 2.0 * v_ijab - v_ijab.transpose(0, 1, 3, 2)
    tau = t2 + einsum("ia,jb->ijab", t1, t1)
    f_ov = bare_fock(fock_diag)[:o, o:]
    return float(einsum("ijab,ijab->", vs, tau) + 2.0 * einsum("ia,ia->", f_ov, t1))


def mp2_t2(L, fock_diag, o):
    """First-order doubles t_ij^ab = v^{ab}_{ij} / (e_i + e_j - e_a - e_b) (A.1 denominators)."""
    e = np.asarray(fock_diag)
    ovov = einsum("Pia,Pjb->iajb", L[:, :o, o:], L[:, :o, o:])
    num = ovov.transpose(0, 2, 1, 3)  # v^{ij}_{ab} = v^{ab}_{ij} for real orbitals
    return num / denom2(e, o)


def mp2_energy_closed_form(L, fock_diag, o):
    """E_MP2 = sum_ijab (ia|jb) [2 (ia|jb) - (ib|ja)] / (e_i + e_j - e_a - e_b)."""
    e = np.asarray(fock_diag)
    iajb = np.einsum("Pia,Pjb->iajb", L[:, :o, o:], L[:, :o, o:])
    E = 0.0
    for i, a, j, b in itertools.product(range(o), range(len(e) - o), range(o), range(len(e) - o)):
        d = e[i] + e[j] - e[o + a] - e[o + b]
        E += iajb[i, a, j, b] * (2.0 * iajb[i, a, j, b] - iajb[i, b, j, a]) / d
    return E


# ---------------------------------------------------------------------------
# Denominators, post-processing, update (A.1, Sec. II.D)
# ---------------------------------------------------------------------------

def denom1(e, o):
    return e[:o, None] - e[None, o:]


def denom2(e, o):
    eo, ev = e[:o], e[o:]
    return (eo[:, None, None, None] + eo[None, :, None, None]
            - ev[None, None, :, None] - ev[None, None, None, :])


def denom3(e, o):
    eo, ev = e[:o], e[o:]
    d_occ = eo[:, None, None] + eo[None, :, None] + eo[None, None, :]
    d_vir = ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
    return d_occ[:, :, :, None, None, None] - d_vir[None, None, None, :, :, :]


def orthogonalise_full(r3):
    """r <- r - (1/6) sum_{pi in S3} r^{pi(abc)} at every (i,j,k) (Sec. II.D.3)."""
    mean = sum(vperm(r3, p) for p in PERMS3) / 6.0
    return r3 - mean


def purify_full(r3):
    """Zero the i = j = k components (Sec. II.D.2)."""
    out = r3.copy()
    for i in range(r3.shape[0]):
        out[i, i, i] = 0.0
    return out


def postprocess_full(r3):
    """Full storage is already column-symmetric; purify, then orthogonalise."""
    return orthogonalise_full(purify_full(r3))


class Diis:
    """DIIS of Sec. III.A.5: B_mn = e_m . e_n, bordered solve, t = sum c_m t_m.

    Vectors are flat float64 arrays.  Keeps the last ``space`` pairs.  The
    bordered system is solved by least squares (pseudo-inverse), which also
    covers a singular B.
    """

    def __init__(self, space: int = 8):
        self.space = space
        self.ts: list[np.ndarray] = []
        self.es: list[np.ndarray] = []

    def push(self, t: np.ndarray, e: np.ndarray):
        self.ts.append(t.copy())
        self.es.append(e.copy())
        if len(self.ts) > self.space:
            self.ts.pop(0)
            self.es.pop(0)

    def coefficients(self) -> np.ndarray:
        m = len(self.es)
        B = np.empty((m + 1, m + 1))
        for a in range(m):
            for b in range(m):
                B[a, b] = float(np.dot(self.es[a], self.es[b]))
        B[m, :m] = 1.0
        B[:m, m] = 1.0
        B[m, m] = 0.0
        rhs = np.zeros(m + 1)
        rhs[m] = 1.0
        sol = np.linalg.lstsq(B, rhs, rcond=None)[0]
        return sol[:m]

    def extrapolate(self) -> np.ndarray:
        c = self.coefficients()
        return sum(ci * ti for ci, ti in zip(c, self.ts))


def solve_full(L, fock_diag, o, triples=True, tol=1e-10, max_iter=200,
               diis_space=8, diis_start=2, t3_frozen_zero=False, verbose=False):
    """Iterate RCCSD or RCCSDT on full storage from t1 = 0, t2 = MP2, t3 = 0.

    Jacobi update ``t += r / eps`` (A.1) with the post-processed R3, DIIS on
    (t1, t2, t3), convergence when the full-tensor residual norm is <= tol.
    Returns (E_corr, t1, t2, t3, iterations, history).
    """
    e = np.asarray(fock_diag, dtype=np.float64)
    v = len(e) - o
    t1 = np.zeros((o, v))
    t2 = mp2_t2(L, e, o)
    t3 = np.zeros((o, o, o, v, v, v)) if triples else None
    d1, d2 = denom1(e, o), denom2(e, o)
    d3 = denom3(e, o) if triples else None
    diis = Diis(diis_space)
    hist = []
    for it in range(1, max_iter + 1):
        r1, r2, r3 = residuals(L, e, t1, t2, t3 if triples else None)
        if triples:
            r3 = postprocess_full(r3)
            if t3_frozen_zero:
                r3 = np.zeros_like(r3)
        norm = np.sqrt(np.sum(r1 ** 2) + np.sum(r2 ** 2) + (np.sum(r3 ** 2) if triples else 0.0))
        E = energy(L, e, t1, t2)
        hist.append((it, E, norm))
        if verbose:
            print(f"iter {it:3d}  E = {E:.14f}  |R| = {norm:.3e}")
        if norm <= tol:
            return E, t1, t2, t3, it, hist
        n1 = t1 + r1 / d1
        n2 = t2 + r2 / d2
        parts_new = [n1.ravel(), n2.ravel()]
        parts_old = [t1.ravel(), t2.ravel()]
        if triples:
            n3 = t3 + r3 / d3
            parts_new.append(n3.ravel())
            parts_old.append(t3.ravel())
        vec = np.concatenate(parts_new)
        diis.push(vec, vec - np.concatenate(parts_old))
        if it >= diis_start:
            vec = diis.extrapolate()
        t1 = vec[: o * v].reshape(o, v)
        t2 = vec[o * v: o * v + (o * v) ** 2].reshape(o, o, v, v)
        if triples:
            t3 = vec[o * v + (o * v) ** 2:].reshape(o, o, o, v, v, v)
    raise RuntimeError(f"RCC did not converge in {max_iter} iterations (|R| = {hist[-1][2]:.3e})")
