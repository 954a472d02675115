"""Brute-force FCI and determinant-space spin-orbital CC.  TEST INFRASTRUCTURE ONLY.

Written from the definitions of appendix A.1, with no working equations: the
wavefunction is a vector over Slater determinants of fixed (N_alpha, N_beta);
``T = sum_mu t_mu X_mu`` with ``X_mu = a+_{a1}..a+_{an} a_{in}..a_{i1}`` over the
unique spin-orbital excitations up to rank N; the residual is
``r_mu = <Phi_mu| e^{-T} H e^{T} |Phi_0>`` and the energy
``<Phi_0| e^{-T} H e^{T} |Phi_0>``; the amplitudes are found with the Jacobi
update ``t += r / eps`` (spin-orbital Fock diagonal of the reference) and DIIS.
``e^{+-T}`` is a terminating Taylor series because T only raises the
excitation level.

The Hamiltonian is the second-quantised spin-free form of A.3,
``H = sum h_pq E_pq + 1/2 sum (pr|qs) (E_pr E_qs - delta_qr E_ps)``, with
``E_pq = sum_sigma a+_{p sigma} a_{q sigma}``, built as sparse matrices from
Jordan-Wigner signs on bit strings.  Spin orbital ``2p + s`` is spatial
orbital ``p`` with spin ``s`` (0 = alpha, 1 = beta).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def _popcount(x: int) -> int:
    return bin(x).count("1")


def apply_ops(det: int, ops):
    """Apply a string of (spin-orbital, is_creation) operators, rightmost first.

    Returns (sign, new_det) or None if the result vanishes.
    """
    sign = 1
    for so, create in reversed(ops):
        bit = 1 << so
        occupied = bool(det & bit)
        if create == occupied:
            return None
        if _popcount(det & (bit - 1)) % 2:
            sign = -sign
        det ^= bit
    return sign, det


class DetSpace:
    """Determinants with ``na`` alpha and ``nb`` beta electrons in ``n`` spatial orbitals."""

    def __init__(self, n: int, na: int, nb: int):
        self.n, self.na, self.nb = n, na, nb
        dets = []
        for a_occ in itertools.combinations(range(n), na):
            for b_occ in itertools.combinations(range(n), nb):
                d = 0
                for p in a_occ:
                    d |= 1 << (2 * p)
                for p in b_occ:
                    d |= 1 << (2 * p + 1)
                dets.append(d)
        self.dets = sorted(dets)
        self.index = {d: i for i, d in enumerate(self.dets)}
        self.dim = len(self.dets)

    def operator(self, ops) -> sp.csr_matrix:
        rows, cols, vals = [], [], []
        for j, d in enumerate(self.dets):
            res = apply_ops(d, ops)
            if res is None:
                continue
            s, nd = res
            i = self.index.get(nd)
            if i is None:
                continue
            rows.append(i)
            cols.append(j)
            vals.append(float(s))
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.dim, self.dim))


def hamiltonian(space: DetSpace, h: np.ndarray, eri_chem: np.ndarray) -> sp.csr_matrix:
    """Sparse H over ``space`` from one-electron ``h`` and chemists' ``(pq|rs)``."""
    n = space.n
    E = [[None] * n for _ in range(n)]
    for p in range(n):
        for q in range(n):
            E[p][q] = (space.operator([(2 * p, True), (2 * q, False)])
                       + space.operator([(2 * p + 1, True), (2 * q + 1, False)]))
    H = sp.csr_matrix((space.dim, space.dim))
    for p in range(n):
        for q in range(n):
            H = H + h[p, q] * E[p][q]
    for p in range(n):
        for r in range(n):
            G = sp.csr_matrix((space.dim, space.dim))
            for q in range(n):
                for s in range(n):
                    if eri_chem[p, r, q, s] != 0.0:
                        G = G + eri_chem[p, r, q, s] * E[q][s]
            H = H + 0.5 * (E[p][r] @ G)
    for p in range(n):
        for s in range(n):
            c = sum(eri_chem[p, q, q, s] for q in range(n))
            H = H - 0.5 * c * E[p][s]
    return H.tocsr()


def core_hamiltonian(fock_diag: np.ndarray, eri_chem: np.ndarray, o: int) -> np.ndarray:
    """h_pq = f_pq - sum_i [2 (pq|ii) - (pi|iq)] so that the closed-shell Fock
    matrix of A.3 (``f = h + sum_i (2 v^{pi}_{qi} - v^{pi}_{iq})``) is ``diag(fock_diag)``."""
    f = np.diag(fock_diag)
    J = np.einsum("pqii->pq", eri_chem[:, :, :o, :o])
    K = np.einsum("piiq->pq", eri_chem[:, :o, :o, :])
    return f - 2.0 * J + K


def eri_from_factors(L: np.ndarray) -> np.ndarray:
    return np.einsum("Ppq,Prs->pqrs", L, L)


class DetCC:
    """Spin-orbital CC of truncation rank ``rank`` about the determinant ``ref``."""

    def __init__(self, space: DetSpace, H: sp.csr_matrix, ref: int, rank: int,
                 fock_so_diag: np.ndarray):
        self.space, self.H, self.ref, self.rank = space, H, ref, rank
        n_so = 2 * space.n
        occ = [p for p in range(n_so) if ref >> p & 1]
        vir = [p for p in range(n_so) if not ref >> p & 1]
        self.excitations = []   # (occ tuple, vir tuple)
        self.X = []             # sparse X_mu
        self.targets = []       # (index of X_mu |ref>, sign)
        self.eps = []
        for nexc in range(1, rank + 1):
            for I in itertools.combinations(occ, nexc):
                for A in itertools.combinations(vir, nexc):
                    # spin conservation: same number of beta orbitals removed and added
                    if sum(i % 2 for i in I) != sum(a % 2 for a in A):
                        continue
                    ops = [(a, True) for a in A] + [(i, False) for i in reversed(I)]
                    res = apply_ops(ref, ops)
                    if res is None or res[1] not in space.index:
                        continue
                    self.excitations.append((I, A))
                    self.X.append(space.operator(ops))
                    self.targets.append((space.index[res[1]], res[0]))
                    self.eps.append(sum(fock_so_diag[i] for i in I) - sum(fock_so_diag[a] for a in A))
        self.eps = np.array(self.eps)
        self.phi0 = np.zeros(space.dim)
        self.phi0[space.index[ref]] = 1.0

    def T_matrix(self, t: np.ndarray) -> sp.csr_matrix:
        T = sp.csr_matrix((self.space.dim, self.space.dim))
        for tm, X in zip(t, self.X):
            if tm != 0.0:
                T = T + tm * X
        return T

    @staticmethod
    def _expm_apply(T, vec, sign):
        out = vec.copy()
        term = vec.copy()
        for k in range(1, 64):
            term = sign * (T @ term) / k
            if not np.any(term):
                break
            out = out + term
        return out

    def psi(self, t):
        return self._expm_apply(self.T_matrix(t), self.phi0, 1.0)

    def residual(self, t):
        """(E_total, r) with r_mu = <Phi_mu| e^{-T} H e^{T} |Phi_0>."""
        T = self.T_matrix(t)
        psi = self._expm_apply(T, self.phi0, 1.0)
        phi = self._expm_apply(T, self.H @ psi, -1.0)
        r = np.array([s * phi[i] for i, s in self.targets])
        return float(phi @ self.phi0), r

    def solve(self, tol=1e-11, max_iter=500, diis_space=8):
        t = np.zeros(len(self.excitations))
        ts, es = [], []
        for it in range(1, max_iter + 1):
            E, r = self.residual(t)
            if np.linalg.norm(r) <= tol:
                return E, t, it
            tn = t + r / self.eps
            ts.append(tn)
            es.append(tn - t)
            ts, es = ts[-diis_space:], es[-diis_space:]
            if len(ts) >= 2:
                m = len(es)
                B = np.zeros((m + 1, m + 1))
                for a in range(m):
                    for b in range(m):
                        B[a, b] = es[a] @ es[b]
                B[m, :m] = B[:m, m] = 1.0
                rhs = np.zeros(m + 1)
                rhs[m] = 1.0
                c = np.linalg.lstsq(B, rhs, rcond=None)[0][:m]
                tn = sum(ci * ti for ci, ti in zip(c, ts))
            t = tn
        raise RuntimeError("determinant CC did not converge")


def fock_spin_orbital_diag(h, eri_chem, ref: int, n: int) -> np.ndarray:
    """Diagonal of the spin-orbital Fock operator of determinant ``ref``:
    f_pp = h_pp + sum_{j in ref} [(pp|jj) - delta_spin (pj|jp)]."""
    out = np.empty(2 * n)
    occ = [p for p in range(2 * n) if ref >> p & 1]
    for P in range(2 * n):
        p, s = divmod(P, 2)
        val = h[p, p]
        for J in occ:
            j, sj = divmod(J, 2)
            val += eri_chem[p, p, j, j]
            if s == sj:
                val -= eri_chem[p, j, j, p]
        out[P] = val
    return out


def reference_det(n_alpha_occ: int, n_beta_occ: int) -> int:
    d = 0
    for p in range(n_alpha_occ):
        d |= 1 << (2 * p)
    for p in range(n_beta_occ):
        d |= 1 << (2 * p + 1)
    return d


def setup(L: np.ndarray, fock_diag: np.ndarray, o_closed: int, na: int, nb: int):
    """Space, H and reference for the Hamiltonian defined by (L, closed-shell Fock
    diagonal with ``o_closed`` doubly occupied orbitals), with ``na``/``nb`` electrons."""
    n = L.shape[1]
    eri = eri_from_factors(L)
    h = core_hamiltonian(np.asarray(fock_diag), eri, o_closed)
    space = DetSpace(n, na, nb)
    H = hamiltonian(space, h, eri)
    ref = reference_det(na, nb)
    f_so = fock_spin_orbital_diag(h, eri, ref, n)
    return space, H, ref, f_so, h, eri


def fci_energies(H: sp.csr_matrix) -> np.ndarray:
    return np.linalg.eigvalsh(H.toarray())


def ccsdt_q_energy(cc: "DetCC", t: np.ndarray, fock_so_diag: np.ndarray) -> float:
    """Spin-orbital CCSDT(Q) correction in determinant space from converged CCSDT
    amplitudes ``t`` of ``cc`` (rank 3), the standard second-order quadruples
    estimate and its fourth- and fifth-order energy (T1 left out):

        R_Q = <Q| H T3 + 1/2 [[H, T2], T2] |0>,  L_Q = <Q| H (T2 + T3) |0>,
        E(Q) = sum_Q L_Q R_Q / D_Q,  D_Q = sum of the occupied minus the virtual
        spin-orbital energies of Q.

    With a canonical reference (no singles in H|0>) the double commutator keeps the
    connected H T2 T2 terms and the T3 term is connected by construction; L_Q is the
    <0|(T2^+ + T3^+) V|Q> projection.  Test infrastructure: a brute-force definition."""
    space, H = cc.space, cc.H
    ranks = np.array([len(I) for I, _ in cc.excitations])
    T2 = cc.T_matrix(np.where(ranks == 2, t, 0.0))
    T3 = cc.T_matrix(np.where(ranks == 3, t, 0.0))
    phi0 = cc.phi0
    v2, v3 = T2 @ phi0, T3 @ phi0
    R = H @ v3 + 0.5 * (H @ (T2 @ v2) - 2.0 * (T2 @ (H @ v2)) + T2 @ (T2 @ (H @ phi0)))
    Lv = H @ (v2 + v3)
    ref = cc.ref
    E = 0.0
    for det, idx in space.index.items():
        if _popcount(det & ~ref) != 4:
            continue
        removed = [p for p in range(2 * space.n) if (ref >> p & 1) and not (det >> p & 1)]
        added = [p for p in range(2 * space.n) if (det >> p & 1) and not (ref >> p & 1)]
        D = sum(fock_so_diag[p] for p in removed) - sum(fock_so_diag[p] for p in added)
        E += Lv[idx] * R[idx] / D
    return float(E)

