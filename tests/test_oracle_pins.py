"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these compare the oracle with itself: each checks it against brute
force (determinant-space CC / FCI), an exactness theorem, a closed form, an
invariant or a number printed in the paper.
"""
import itertools

import numpy as np
import pytest

from oracle import compact as C
from oracle import detcc, nullspace, opcount
from oracle import rccsdt as full
from paper_2607_00981_gb300.synth import make_instance, random_amplitudes


def _det_cc_energy(inst, o, rank, na=None, nb=None):
    na = o if na is None else na
    nb = o if nb is None else nb
    space, H, ref, fso, h, eri = detcc.setup(inst.L, inst.fock_diag, o, na, nb)
    cc = detcc.DetCC(space, H, ref, rank, fso)
    E, t, _ = cc.solve(tol=1e-11)
    return E, H[space.index[ref], space.index[ref]], cc, t, H


# ---------------------------------------------------------------- exactness (A.1)

@pytest.mark.parametrize("v", [2, 3])
def test_ccsdt_is_exact_for_three_electrons(v):
    """CC truncated at N = n_elec is exact: CCSDT on 3 electrons is an FCI eigenstate."""
    inst = make_instance(2, v, naux=10, seed=5)
    E, _, cc, t, H = _det_cc_energy(inst, 2, 3, na=2, nb=1)
    psi = cc.psi(t)
    assert np.linalg.norm(H @ psi - E * psi) / np.linalg.norm(psi) < 1e-8
    assert np.min(np.abs(detcc.fci_energies(H) - E)) < 1e-10


@pytest.mark.parametrize("v", [2, 3])
def test_ccsdtq_is_exact_for_four_electrons(v):
    inst = make_instance(2, v, naux=10, seed=5)
    E, _, cc, t, H = _det_cc_energy(inst, 2, 4)
    assert np.min(np.abs(detcc.fci_energies(H) - E)) < 1e-10


def test_ccsdt_is_not_exact_for_four_electrons():
    """Negative control: the exactness pin does distinguish a truncated method."""
    inst = make_instance(2, 3, naux=10, seed=5)
    E, _, cc, t, H = _det_cc_energy(inst, 2, 3)
    assert np.min(np.abs(detcc.fci_energies(H) - E)) > 1e-7


# ------------------------------------------- working equations vs brute force (A.5)

@pytest.mark.parametrize("o,v,seed", [(2, 3, 3), (3, 3, 3)])
def test_rccsd_equals_determinant_ccsd(o, v, seed):
    inst = make_instance(o, v, naux=12, seed=seed)
    E_det, E0, *_ = _det_cc_energy(inst, o, 2)
    E_rcc = full.solve_full(inst.L, inst.fock_diag, o, triples=False, tol=1e-10, max_iter=400)[0]
    assert abs((E_det - E0) - E_rcc) < 1e-10


@pytest.mark.parametrize("o,v,seed", [(2, 2, 3), (2, 3, 3), (3, 3, 3), (3, 4, 3)])
def test_rccsdt_equals_determinant_ccsdt(o, v, seed):
    """The printed RCCSDT equations (with T1 dressing) reproduce spin-orbital CCSDT."""
    inst = make_instance(o, v, naux=12, seed=seed)
    E_det, E0, *_ = _det_cc_energy(inst, o, 3)
    E_rcc = full.solve_full(inst.L, inst.fock_diag, o, triples=True, tol=1e-10, max_iter=400)[0]
    assert abs((E_det - E0) - E_rcc) < 1e-10


def test_two_electrons_rccsd_rccsdt_fci():
    """o = 1: the only T3 block is i = j = k (purified), so RCCSD = RCCSDT = FCI."""
    inst = make_instance(1, 4, naux=8, seed=2)
    space, H, ref, *_ = detcc.setup(inst.L, inst.fock_diag, 1, 1, 1)
    E0 = H[space.index[ref], space.index[ref]]
    e_fci = detcc.fci_energies(H)[0] - E0
    e_sd = full.solve_full(inst.L, inst.fock_diag, 1, triples=False)[0]
    e_sdt = C.solve_compact(inst.L, inst.fock_diag, 1)[0]
    assert abs(e_sd - e_fci) < 1e-10
    assert abs(e_sdt - e_fci) < 1e-10


# ------------------------------------------------------------ invariants (A.2, II.D)

def test_full_residual_has_column_symmetry():
    o, v = 3, 5
    inst = make_instance(o, v, naux=20, seed=1)
    t1, t2, t3 = random_amplitudes(o, v, seed=4)
    _, r2, r3 = full.residuals(inst.L, inst.fock_diag, t1, t2, t3)
    assert np.abs(r2 - r2.transpose(1, 0, 3, 2)).max() < 1e-12
    for p in full.PERMS3:
        rp = r3.transpose(p[0], p[1], p[2], 3 + p[0], 3 + p[1], 3 + p[2])
        assert np.abs(r3 - rp).max() < 1e-12 * max(1.0, np.abs(r3).max())


def test_compact_residual_equals_full_residual():
    """Compact expansions (direct traversal + unpacking) give the full residual."""
    o, v = 3, 12
    inst = make_instance(o, v, naux=40, seed=0)
    t1, t2, t3 = random_amplitudes(o, v, seed=7)
    r1f, r2f, r3f = full.residuals(inst.L, inst.fock_diag, t1, t2, t3)
    r1c, r2c, r3c = C.residuals_compact(inst.L, inst.fock_diag, t1, t2, C.pack(t3))
    scale = np.abs(r3f).max()
    assert np.abs(r1f - r1c).max() < 1e-12 * scale
    assert np.abs(r2f - r2c).max() < 1e-12 * scale
    assert np.abs(C.pack(r3f) - r3c).max() < 1e-12 * scale


@pytest.mark.parametrize("o,v", [(3, 5), (4, 4)])
def test_compact_residual_norm_equals_full_storage_norm(o, v):
    """The weighted compact norm (reading: |R|^2 = |r1|^2 + |r2|^2 + sum over stored
    blocks of m(blk) |r3_blk|^2, m = 6/3/1) is the norm of the post-processed residual
    on FULL storage, computed here from the full-storage equations alone.  Unit block
    weights, or the weights reversed (1/3/6), miss it."""
    inst = make_instance(o, v, naux=16, seed=o + 10 * v)
    t1, t2, t3 = random_amplitudes(o, v, seed=3 * o + v)
    r1, r2, r3f = full.residuals(inst.L, inst.fock_diag, t1, t2, t3)
    p3f = full.postprocess_full(r3f)
    ref = np.sqrt(np.sum(r1 ** 2) + np.sum(r2 ** 2) + np.sum(p3f ** 2))
    r1c, r2c, r3c = C.residuals_compact(inst.L, inst.fock_diag, t1, t2, C.pack(t3))
    p3c = C.postprocess(r3c, o)
    got = C.residual_norm(r1c, r2c, p3c, o)
    assert abs(got - ref) < 1e-12 * ref
    # negative controls: other block weights give other norms
    blk2 = np.sum(p3c.reshape(len(p3c), -1) ** 2, axis=1)
    base = np.sum(r1c ** 2) + np.sum(r2c ** 2)
    unit = np.sqrt(base + np.sum(blk2))
    w = C.weights(o)
    rev = np.sqrt(base + np.sum(np.where(w == 6, 1.0, np.where(w == 1, 6.0, 3.0)) * blk2))
    assert abs(unit - ref) > 1e-3 * ref
    assert abs(rev - ref) > 1e-3 * ref


def test_compact_converged_energy_equals_full():
    inst = make_instance(3, 6, naux=20, seed=11, scale=0.2)
    Ec, *_ = C.solve_compact(inst.L, inst.fock_diag, 3, tol=1e-10, max_iter=300)
    Ef, *_ = full.solve_full(inst.L, inst.fock_diag, 3, tol=1e-10, max_iter=300)
    assert abs(Ec - Ef) < 1e-11


def test_subspace_diis_reaches_the_same_fixed_point():
    """DIIS over a virtual subspace of T3 (Sec. III.A.5) changes the path, not the
    converged amplitudes: the energy equals the full-DIIS one; the whole space as the
    subspace is the full DIIS iteration for iteration."""
    inst = make_instance(3, 6, naux=20, seed=11, scale=0.2)
    Ef, *_, itf, hf = C.solve_compact(inst.L, inst.fock_diag, 3, tol=1e-10, max_iter=300)
    Es, *_, its, hs = C.solve_compact(inst.L, inst.fock_diag, 3, tol=1e-10, max_iter=300, diis_t3_nvir=3)
    Ea, *_, ita, ha = C.solve_compact(inst.L, inst.fock_diag, 3, tol=1e-10, max_iter=300, diis_t3_nvir=6)
    assert abs(Ef - Es) < 1e-11
    assert ha == hf
    assert hs[3][1] != hf[3][1]  # a different path


def test_frozen_zero_t3_reduces_to_rccsd():
    """T3 = 0 in the RCCSDT equations gives the RCCSD residuals and energy."""
    o, v = 3, 5
    inst = make_instance(o, v, naux=20, seed=1, scale=0.2)
    t1, t2, _ = random_amplitudes(o, v, seed=4)
    r1a, r2a, _ = full.residuals(inst.L, inst.fock_diag, t1, t2, None)
    r1b, r2b, _ = full.residuals(inst.L, inst.fock_diag, t1, t2, np.zeros((o,) * 3 + (v,) * 3))
    assert np.abs(r1a - r1b).max() < 1e-13 and np.abs(r2a - r2b).max() < 1e-13
    Ea = full.solve_full(inst.L, inst.fock_diag, o, triples=False)[0]
    Eb = full.solve_full(inst.L, inst.fock_diag, o, triples=True, t3_frozen_zero=True)[0]
    assert abs(Ea - Eb) < 1e-11


def test_unpack_reproduces_full_tensor():
    o, v = 4, 3
    _, _, t3 = random_amplitudes(o, v, seed=9)
    assert np.array_equal(C.unpack_full(C.pack(t3), o), t3)


def test_compact_block_index_is_a_bijection_in_colex_order():
    for o in range(1, 9):
        tr = C.triples(o)
        assert len(tr) == o * (o + 1) * (o + 2) // 6 == opcount.n3(o)
        assert len(set(tr)) == len(tr)
        assert tr == sorted(tr, key=lambda t: (t[2], t[1], t[0]))


def test_postprocessed_residual_is_in_the_nonredundant_subspace():
    o, v = 3, 5
    inst = make_instance(o, v, naux=20, seed=1)
    t1, t2, t3 = random_amplitudes(o, v, seed=4)
    _, _, r3c = C.residuals_compact(inst.L, inst.fock_diag, t1, t2, C.pack(t3))
    r = C.postprocess(r3c, o)
    s = sum(np.transpose(r, (0,) + tuple(1 + np.argsort(p))) for p in full.PERMS3)
    assert np.abs(s).max() < 1e-13
    for b, (i, j, k) in enumerate(C.triples(o)):
        if i == j == k:
            assert not np.any(r[b])
        if i == j:
            assert np.abs(r[b] - r[b].transpose(1, 0, 2)).max() < 1e-14
        if j == k:
            assert np.abs(r[b] - r[b].transpose(0, 2, 1)).max() < 1e-14


# --------------------------------------------------------------- closed forms

def test_first_energy_from_mp2_amplitudes_is_mp2_energy():
    o, v = 3, 6
    inst = make_instance(o, v, naux=20, seed=0)
    t2 = full.mp2_t2(inst.L, inst.fock_diag, o)
    E = full.energy(inst.L, inst.fock_diag, np.zeros((o, v)), t2)
    assert abs(E - full.mp2_energy_closed_form(inst.L, inst.fock_diag, o)) < 1e-12


def test_s3_overlap_eigenvalues_and_projector():
    M = nullspace.overlap_matrix(3)
    ev = np.sort(np.linalg.eigvalsh(M))
    assert np.allclose(ev, [0, 6, 6, 6, 6, 24], atol=1e-12)
    Pr = nullspace.projector_triples()
    assert np.allclose(Pr @ Pr, Pr)
    assert np.allclose(Pr @ np.ones(6), 0.0)
    # the null vector of M is the fully symmetric one
    w, U = np.linalg.eigh(M)
    null = U[:, np.argmin(np.abs(w))]
    assert np.allclose(np.abs(null), 1 / np.sqrt(6))


def test_s4_overlap_eigenvalues():
    ev = np.sort(np.linalg.eigvalsh(nullspace.overlap_matrix(4)))
    counts = {mu: int(np.sum(np.isclose(ev, mu))) for mu in (0, 12, 24, 120)}
    # [4] (1) + [3,1] (9) null; [2^2] 4, [2,1^2] 9, [1^4] 1
    assert counts == {0: 10, 12: 4, 24: 9, 120: 1}


def test_spin_free_overlap_matches_determinant_space():
    """<E^{pi(abc)}_{ijk} Phi | E^{tau(abc)}_{ijk} Phi> computed from determinants
    equals m(pi^-1 tau) = sgn 2^cycles (Eq. spinfree_overlap_class_function)."""
    o, v = 3, 3
    space = detcc.DetSpace(o + v, o, o)
    ref = detcc.reference_det(o, o)
    phi = np.zeros(space.dim)
    phi[space.index[ref]] = 1.0
    I, A = (0, 1, 2), (3, 4, 5)
    perms = list(itertools.permutations(range(3)))
    states = []
    for p in perms:
        vec = np.zeros(space.dim)
        for sig in itertools.product((0, 1), repeat=3):
            ops = ([(2 * A[p[q]] + sig[q], True) for q in range(3)]
                   + [(2 * I[q] + sig[q], False) for q in reversed(range(3))])
            vec += space.operator(ops) @ phi
        states.append(vec)
    S = np.array([[a @ b for b in states] for a in states])
    assert np.allclose(S, nullspace.overlap_matrix(3))


def test_operation_counts():
    for o, v in [(1, 1), (2, 3), (3, 4), (4, 2)]:
        assert opcount.compact_fma_enumerated(o, v) == opcount.compact_fma(o, v)
    # large-o limit of the compact count is 1/2 o^3 v^5 + 2 o^4 v^4 + 1/2 o^5 v^3
    o, v = 4000, 8000
    assert abs(opcount.compact_fma(o, v) / opcount.compact_asymptotic(o, v) - 1) < 1e-3
    # flop per iteration of the workloads (2 flop per FMA)
    assert f"{opcount.flop_per_iteration(3, 12):.3g}" == "3.08e+07"
    assert f"{opcount.flop_per_iteration(8, 80):.3g}" == "3.33e+12"
    assert f"{opcount.flop_per_iteration(16, 160):.3g}" == "7.24e+14"


def test_compact_memory_matches_paper_sizes():
    """n3 v^3 doubles, printed as 587 GB (o=40, v=190) and 623 GB (o=24, v=318)."""
    gib = lambda o, v: opcount.t3_bytes(o, v) / 2 ** 30  # noqa: E731
    assert round(gib(40, 190)) == 587
    assert round(gib(24, 318)) == 623
    assert round(opcount.t3_bytes(48, 292) / 2 ** 40, 1) == 3.6
    assert round(opcount.t3_bytes(52, 328) / 2 ** 40, 1) == 6.4


def test_diis_solves_a_linear_fixed_point():
    """DIIS on x <- A x + b converges to (I - A)^-1 b within dim + 1 steps."""
    rng = np.random.default_rng(0)
    n = 5
    A = 0.5 * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x = np.zeros(n)
    d = full.Diis(8)
    for _ in range(n + 2):
        xn = A @ x + b
        d.push(xn, xn - x)
        x = d.extrapolate()
    assert np.allclose(x, np.linalg.solve(np.eye(n) - A, b), atol=1e-10)


def test_pp_ladder_intermediate_is_pair_symmetric():
    """W^{ab}_{de} = W^{ba}_{ed} at generic (non-converged) amplitudes, and the sum /
    difference split over that exchange reproduces the plain pp-ladder view
    X^{xy}(w) = sum_de W^{xy}_{de} T(d, e, w) (Sec. II.C.1): the premise of the
    library's pair-symmetric pp-ladder GEMMs, checked on the oracle's intermediate."""
    o, v = 3, 7
    inst = make_instance(o, v, naux=20, seed=3)
    t1, t2, t3 = random_amplitudes(o, v, seed=5)
    *_, I = C.residuals_compact(inst.L, inst.fock_diag, t1, t2, C.pack(t3), return_intermediates=True)
    W = I["Wvvvv"]
    scale = max(1.0, np.abs(W).max())
    assert np.abs(W - W.transpose(1, 0, 3, 2)).max() < 1e-14 * scale
    T = np.random.default_rng(9).standard_normal((v, v, v))
    X = np.einsum("xyde,dew->xyw", W, T)
    du, eu = np.triu_indices(v)          # pairs d <= e
    dl, el = np.triu_indices(v, 1)       # pairs d < e
    Wp = W[:, :, du, eu] + np.where(du == eu, 0.0, 1.0) * W[:, :, eu, du]
    Tp = T[du, eu, :] + T[eu, du, :]
    Wm = W[:, :, dl, el] - W[:, :, el, dl]
    Tm = T[dl, el, :] - T[el, dl, :]
    Xp = np.einsum("xyk,kw->xyw", Wp, Tp)
    Xm = np.einsum("xyk,kw->xyw", Wm, Tm)
    Xs = X + X.transpose(1, 0, 2)
    Xd = X - X.transpose(1, 0, 2)
    assert np.abs(Xp - Xs).max() < 1e-12 * max(1.0, np.abs(Xs).max())
    assert np.abs(Xm - Xd).max() < 1e-12 * max(1.0, np.abs(Xd).max())
    # the recombination the epilogue performs: X^{xy} = (X+ + X-) / 2
    assert np.abs(0.5 * (Xp + Xm) - X).max() < 1e-12 * max(1.0, np.abs(X).max())


# ------------------------------------------------ (Q) correction (appendix, Eq. ener-pt-q)

from oracle import q_correction as Qc  # noqa: E402


def _q_pair(o, v, seed, scale=None):
    kw = {} if scale is None else {"scale": scale}
    inst = make_instance(o, v, naux=12, seed=seed, **kw)
    space, H, ref, fso, h, eri = detcc.setup(inst.L, inst.fock_diag, o, o, o)
    cc = detcc.DetCC(space, H, ref, 3, fso)
    _, t, _ = cc.solve(tol=1e-11, max_iter=800)
    e_det = detcc.ccsdt_q_energy(cc, t, fso)
    _, _, t2, t3, *_ = full.solve_full(inst.L, inst.fock_diag, o, triples=True, tol=1e-11, max_iter=800)
    return inst, e_det, t2, t3


@pytest.mark.parametrize("o,v,seed,scale", [(2, 2, 3, None), (2, 4, 7, 0.6), (3, 3, 3, None)])
def test_rccsdt_q_equals_determinant_ccsdt_q(o, v, seed, scale):
    """The spin-adapted (Q) energy of the paper's appendix, from converged RCCSDT
    amplitudes, equals the spin-orbital CCSDT(Q) correction computed by brute force
    in determinant space from the determinant CCSDT amplitudes (both without T1):
    E(Q) = sum_Q <Q|H(T2+T3)|0><Q|H T3 + [[H,T2],T2]/2|0> / D_Q.  Both intermediate
    forms the paper prints (Eq. q_w_alter) give it."""
    inst, e_det, t2, t3 = _q_pair(o, v, seed, scale)
    e_q = Qc.energy_q(inst.L, inst.fock_diag, t2, t3, o)
    e_alt = Qc.energy_q(inst.L, inst.fock_diag, t2, t3, o, alternative=True)
    assert abs(e_det) > 1e-7
    assert abs(e_q - e_det) < 1e-8 * abs(e_det)
    assert abs(e_alt - e_det) < 1e-8 * abs(e_det)


def test_q_pin_detects_planted_mistakes(monkeypatch):
    """Negative controls, planted in the oracle on the CPU: a missing factor in the
    quadruples spin summation, a dropped T2 T2 term of the residual, or the
    disconnected V term left out of the weights each move E(Q) far off."""
    o, v = 2, 4
    inst, e_det, t2, t3 = _q_pair(o, v, 7, 0.6)
    good = Qc.spin_sum_t4_full
    monkeypatch.setattr(Qc, "spin_sum_t4_full", lambda t4: 0.5 * good(t4))
    assert abs(Qc.energy_q(inst.L, inst.fock_diag, t2, t3, o) - e_det) > 0.1 * abs(e_det)
    monkeypatch.setattr(Qc, "spin_sum_t4_full", good)
    inter = Qc.q_intermediates
    monkeypatch.setattr(Qc, "q_intermediates", lambda *a, **k: (lambda X, Y, V: (X, 0 * Y, V))(*inter(*a, **k)))
    assert abs(Qc.energy_q(inst.L, inst.fock_diag, t2, t3, o) - e_det) > 0.1 * abs(e_det)
    monkeypatch.setattr(Qc, "q_intermediates", lambda *a, **k: (lambda X, Y, V: (X, Y, 0 * V))(*inter(*a, **k)))
    assert abs(Qc.energy_q(inst.L, inst.fock_diag, t2, t3, o) - e_det) > 0.1 * abs(e_det)


@pytest.mark.parametrize("over", ["occ", "vir"])
def test_q_triangular_sums_with_degeneracy_factors(over, monkeypatch):
    """The IJK- and ABC-ordered (Q) sums over i <= j <= k <= l or a <= b <= c <= d with
    the paper's degeneracy factors (24 / 12 / 6, and 0 for three equal labels) equal
    the full sum; weighting the three-equal tuples by their multiplicity 4 instead
    changes nothing either (their spin-summed products vanish), which pins the
    zeros as a property, not a truncation."""
    o, v = 3, 3
    inst, e_det, t2, t3 = _q_pair(o, v, 3)
    e_full = Qc.energy_q(inst.L, inst.fock_diag, t2, t3, o)
    e_tri = Qc.energy_q_triangular(inst.L, inst.fock_diag, t2, t3, o, over=over)
    assert abs(e_tri - e_full) < 1e-12 * max(1.0, abs(e_full)) + 1e-15
    good = Qc.degeneracy4

    def multiplicities(n):  # 4 for three equal labels, 1 for four
        f = good(n)
        for p, q, r, s in itertools.product(range(n), repeat=4):
            if p <= q <= r <= s and f[p, q, r, s] == 0.0:
                f[p, q, r, s] = 1.0 if p == s else 4.0
        return f

    monkeypatch.setattr(Qc, "degeneracy4", multiplicities)
    e_mult = Qc.energy_q_triangular(inst.L, inst.fock_diag, t2, t3, o, over=over)
    assert abs(e_mult - e_full) < 1e-12 * max(1.0, abs(e_full)) + 1e-15


def test_virtual_triangular_layout_is_a_bijection():
    """The ABC-based (Q) layout of T3 (stored by a <= b <= c, o^3 per block) holds the
    same tensor as the compact occupied-triangular one: unpacking either gives the
    full t_{ijk}^{abc}, bit for bit, for an amplitude with the column symmetry."""
    o, v = 3, 4
    _, _, t3 = random_amplitudes(o, v, seed=11)
    t3c = C.pack(t3)
    t3v = Qc.pack_virtual_triangular(t3c, o)
    assert t3v.shape == (v * (v + 1) * (v + 2) // 6, o, o, o)
    assert np.array_equal(Qc.unpack_virtual_triangular(t3v, o, v), t3)


# ---------------------------------------------------------------- compact T4 (Sec. II.C.4, II.D, appendix B)

def test_t4_compact_pp_ladder_equals_full_definition():
    """The six-term direct traversal of W^vv_vv * T4 on compact storage equals the
    full-storage definition P_(ia)(jb)(kc)(ld) 1/4 sum_ef W^{ab}_{ef} t^{efcd}_{ijkl}
    on every stored block (degenerate ones included); a dropped term fails."""
    from oracle import quadruples as Q
    from paper_2607_00981_gb300.synth import random_pair_symmetric, random_t4
    o, v = 3, 4
    W = random_pair_symmetric(v, seed=1)
    t4 = random_t4(o, v, seed=2)
    full = Q.pack4(Q.pp_ladder_full(W, t4))
    comp = Q.pp_ladder_compact(W, Q.pack4(t4), o)
    assert np.abs(full - comp).max() < 1e-13 * np.abs(full).max()
    assert np.array_equal(Q.unpack4(Q.pack4(t4), o), t4)
    # negative control: the last of the six terms left out
    T = Q.pack4(t4)
    partial = comp - np.stack([np.einsum("cdef,abef->abcd", W, T[b]) for b in range(len(T))])
    assert np.abs(full - partial).max() > 1e-3 * np.abs(full).max()


def test_t4_projector_polynomial_equals_character_projector():
    """(Omega - 6)(Omega - 2)(2 Omega^2 + 19 Omega + 48)/576 = 1 - Pi_[4] - Pi_[3,1]
    (appendix B): idempotent, rank 14, and its kernel is the null space of the
    spin-free overlap matrix of four virtual labels."""
    from oracle import quadruples as Q
    P = Q.projector_polynomial()
    assert np.abs(P - Q.projector_from_characters()).max() < 1e-13
    assert np.abs(P @ P - P).max() < 1e-13
    assert abs(np.trace(P) - 14.0) < 1e-12
    M = nullspace.overlap_matrix(4)
    assert np.abs(M @ (np.eye(24) - P)).max() < 1e-10   # the removed part is M's null space
    assert np.linalg.matrix_rank(M) == 14


def test_t4_block_projection_matches_the_matrix_on_distinct_labels():
    """orthogonalise4_block on a v^4 block acts, on the 24 orderings of four distinct
    labels, as the projector matrix; it annihilates a fully symmetric block."""
    from oracle import quadruples as Q
    rng = np.random.default_rng(3)
    B = rng.standard_normal((4, 4, 4, 4))
    out = Q.orthogonalise4_block(B)
    P = Q.projector_polynomial()
    vec = np.array([B[p] for p in Q.PERMS4])
    assert np.abs(np.array([out[p] for p in Q.PERMS4]) - P @ vec).max() < 1e-12
    S = sum(np.transpose(B, p) for p in Q.PERMS4)
    assert np.abs(Q.orthogonalise4_block(S)).max() < 1e-11


def test_t4_symmetrise_and_purify_on_column_symmetric_input():
    """A column-symmetric T4 is already symmetric inside its degenerate blocks
    (symmetrisation leaves it unchanged); purification zeroes exactly the blocks with
    three equal occupied indices."""
    from oracle import quadruples as Q
    from paper_2607_00981_gb300.synth import random_t4
    o, v = 4, 3
    t4c = Q.pack4(random_t4(o, v, seed=4))
    assert np.abs(Q.symmetrise4(t4c, o) - t4c).max() < 1e-15
    p = Q.purify4(t4c, o)
    for b, (i, j, k, l) in enumerate(Q.quads(o)):
        three = i == j == k or j == k == l
        assert (np.all(p[b] == 0.0)) == three or not np.any(t4c[b])
