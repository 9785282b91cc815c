"""Pins of the FP64 oracle against textbook physics, closed forms and invariants.

The paper prints no worked QEq example, so the oracle is pinned by what the
mathematics fixes (pins P1-P7):
  * the rock-salt Madelung constant (point-charge limit of the Ewald machinery);
  * the Ewald split equals the plain reciprocal-sum definition for any omega;
  * the single-Gaussian self term in a cubic box against the simple-cubic
    self-image constant xi (closed form);
  * Gaussian-minus-point energy against a direct, absolutely convergent erfc sum;
  * the large-box pair limit approaching erf(r/(sqrt2 gamma))/r of eq. (elec_energy);
  * N = 1 and N = 2 solves by hand, neutrality, the energy identity at the optimum,
    symmetry of perfect rock salt, translation and permutation invariance;
  * the large-cell C matrix-vector product against the dense matrix.
Each pin fails for a plausible slip (dropped self / width term, sign of mu,
transposed cell, wrong image range).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import erf, erfc

from oracle import qeq_oracle as O
from paper_2607_17978_b300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "lattice_constants.json")))
MADELUNG = GOLD["madelung_nacl_nn"]["value"]
XI_SC = GOLD["wigner_sc_xi"]["value"]


def _tri_cell():
    return np.array([[7.0, 0.3, 0.5], [0.0, 6.5, -0.4], [0.0, 0.0, 8.0]])


@pytest.mark.parametrize("ncell,omega", [(1, 1.2), (2, 1.5), (2, 2.5)])
def test_madelung_rocksalt_point_charges(ncell, omega):
    frac, spec = synth.rocksalt_sites(ncell, ncell, ncell)
    a = 5.64
    cell = np.eye(3) * ncell * a
    pos = frac @ cell
    q = np.where(spec == 0, 1.0, -1.0)
    A = O.coulomb_matrix(cell, pos, np.zeros(len(q)), omega=omega)
    E = 0.5 * q @ A @ q
    M = -E / (len(q) / 2) * (a / 2)
    assert abs(M - MADELUNG) < 1e-11


@pytest.mark.parametrize("omega", [0.8, 1.2, 2.0])
def test_madelung_constants_of_other_lattices_and_a_primitive_triclinic_cell(omega):
    """Rock salt on its two-atom primitive fcc cell (60-degree angles, so the reciprocal rows and the
    volume of a non-orthogonal cell enter), zinc blende on the same cell and caesium chloride on a
    simple cubic cell, each against its textbook Madelung constant."""
    a = 5.0
    fcc = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    cases = [(fcc, [0.5 * a, 0.0, 0.0], 0.5 * a, MADELUNG),
             (fcc, [0.25 * a] * 3, a * math.sqrt(3) / 4, GOLD["madelung_zincblende_nn"]["value"]),
             (np.eye(3) * a, [0.5 * a] * 3, a * math.sqrt(3) / 2, GOLD["madelung_cscl_nn"]["value"])]
    q = np.array([1.0, -1.0])
    for cell, second, r0, expect in cases:
        pos = np.array([[0.0, 0.0, 0.0], second])
        A = O.coulomb_matrix(cell, pos, np.zeros(2), omega=omega)
        M = -(0.5 * q @ A @ q) * r0
        assert abs(M - expect) < 1e-9, (expect, M)


def test_madelung_via_large_cell_matvec():
    frac, spec = synth.rocksalt_sites(2, 2, 2)
    a = 5.64
    cell = np.eye(3) * 2 * a
    pos = frac @ cell
    q = np.where(spec == 0, 1.0, -1.0)
    y = O.ewald_matvec(cell, pos, np.zeros(len(q)), q, omega=2.0)
    M = -(0.5 * q @ y) / (len(q) / 2) * (a / 2)
    assert abs(M - MADELUNG) < 1e-10


@pytest.mark.parametrize("omega", [0.8, 1.0, 2.0, 3.0])
def test_ewald_split_equals_definition(omega):
    rng = np.random.default_rng(11)
    cell = _tri_cell()
    pos = rng.random((5, 3)) @ cell
    sig = np.array([1.0, 1.8, 1.0, 1.8, 1.3])
    Ad = O.coulomb_matrix_definition(cell, pos, sig)
    Ae = O.coulomb_matrix(cell, pos, sig, omega=omega)
    assert np.abs(Ae - Ad).max() < 1e-12 * np.abs(Ad).max()
    assert np.abs(Ad - Ad.T).max() < 1e-14 * np.abs(Ad).max()


@pytest.mark.parametrize("sigma,L", [(1.0, 20.0), (1.3, 25.0), (0.7, 14.0)])
def test_single_gaussian_self_term_cubic_box(sigma, L):
    cell = np.eye(3) * L
    pos = np.array([[0.3, 1.1, -0.2]])
    expect = 1.0 / (sigma * math.sqrt(math.pi)) + XI_SC / L + 4 * math.pi * sigma ** 2 / L ** 3
    Ad = O.coulomb_matrix_definition(cell, pos, [sigma])
    Ae = O.coulomb_matrix(cell, pos, np.array([sigma]), omega=max(1.5, sigma * 1.6))
    assert abs(Ad[0, 0] - expect) < 1e-12
    assert abs(Ae[0, 0] - expect) < 1e-12


def _direct_erfc_sum(cell, pos, sigma, q, rmax=40.0):
    """sum over i, j, images n (excluding i = j, n = 0) of q_i q_j erfc(r/(sqrt2 gamma))/r, brute force."""
    n = len(pos)
    wd = O.plane_widths(cell)
    nm = [int(math.ceil(rmax / wd[d])) + 1 for d in range(3)]
    tot = 0.0
    for i in range(n):
        for j in range(n):
            g = math.sqrt(sigma[i] ** 2 + sigma[j] ** 2)
            for a in range(-nm[0], nm[0] + 1):
                for b in range(-nm[1], nm[1] + 1):
                    for c in range(-nm[2], nm[2] + 1):
                        if i == j and a == 0 and b == 0 and c == 0:
                            continue
                        d = pos[j] - pos[i] + a * cell[0] + b * cell[1] + c * cell[2]
                        r = float(np.linalg.norm(d))
                        if r < rmax:
                            tot += q[i] * q[j] * erfc(r / (math.sqrt(2) * g)) / r
    return tot


def test_gaussian_minus_point_energy_direct_sum():
    rng = np.random.default_rng(5)
    cell = _tri_cell()
    pos = rng.random((4, 3)) @ cell
    sig = np.array([1.0, 1.8, 0.9, 1.4])
    q = np.array([0.7, -0.3, -0.9, 0.5])       # neutral
    Eg = 0.5 * q @ O.coulomb_matrix_definition(cell, pos, sig) @ q
    Ep = 0.5 * q @ O.coulomb_matrix(cell, pos, np.zeros(4), omega=1.5) @ q
    rhs = np.sum(q ** 2 / (2 * sig * math.sqrt(math.pi))) - 0.5 * _direct_erfc_sum(cell, pos, sig, q)
    assert abs((Eg - Ep) - rhs) < 1e-12


def test_large_box_pair_limit():
    L, r, s1, s2 = 60.0, 1.7, 1.0, 1.8
    cell = np.eye(3) * L
    pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    A = O.coulomb_matrix(cell, pos, np.array([s1, s2]), omega=3.0)
    g = math.sqrt(s1 ** 2 + s2 ** 2)
    pair = erf(r / (math.sqrt(2) * g)) / r
    expect = pair + XI_SC / L + (2 * math.pi / 3) * r ** 2 / L ** 3 + 2 * math.pi * g ** 2 / L ** 3
    # neglected: the cubic-harmonic r^4/L^5 term of the periodic point potential
    assert abs(A[0, 1] - expect) < 5 * r ** 4 / L ** 5
    assert abs(A[0, 0] - (1 / (s1 * math.sqrt(math.pi)) + XI_SC / L + 4 * math.pi * s1 ** 2 / L ** 3)) < 1e-12


def test_solve_single_atom():
    cell = np.eye(3) * 9.0
    pos = np.array([[1.0, 2.0, 3.0]])
    A = O.coulomb_matrix(cell, pos, np.array([1.2]))
    q, mu = O.solve_bordered(A, np.array([1.7]), np.array([-0.4]), 1.0)
    assert abs(q[0] - 1.0) < 1e-14
    assert abs(mu - ((A[0, 0] + 1.7) * 1.0 - 0.4)) < 1e-12


def test_solve_two_atoms_by_hand():
    rng = np.random.default_rng(3)
    cell = _tri_cell()
    pos = rng.random((2, 3)) @ cell
    sig = np.array([1.0, 1.8])
    A = O.coulomb_matrix(cell, pos, sig)
    J = np.array([2.0, 1.5])
    chi = np.array([-1.1, 0.8])
    qt = 0.4
    H = A + np.diag(J)
    # eliminate q2 = qt - q1 from the stationarity condition (H q + chi) equal in both rows
    q1 = (qt * (H[1, 1] - H[0, 1]) + chi[1] - chi[0]) / (H[0, 0] + H[1, 1] - 2 * H[0, 1])
    q, mu = O.solve_bordered(A, J, chi, qt)
    assert abs(q[0] - q1) < 1e-13 and abs(q[1] - (qt - q1)) < 1e-13
    assert abs(mu - (H[0] @ q + chi[0])) < 1e-12


def test_neutrality_energy_identity_and_mu_sign():
    st = synth.rocksalt(1, 5.64, 0.2, synth.rng_for(99, 0))
    st.q_tot = 0.5
    A = O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=synth.COULOMB_K_EV_A)
    q, mu = O.solve_bordered(A, st.J, st.chi, st.q_tot)
    assert abs(q.sum() - st.q_tot) < 1e-12
    # stationarity (SI eq. qeq): (A + J) q + chi = mu 1
    r = A @ q + st.J * q + st.chi
    assert np.abs(r - mu).max() < 1e-11
    E, Ee = O.energies(A, st.J, st.chi, q)
    assert abs(E - (0.5 * st.chi @ q + 0.5 * mu * st.q_tot)) < 1e-11
    assert Ee >= 0


def test_coulomb_matrix_psd_on_random_cells():
    rng = np.random.default_rng(8)
    for _ in range(3):
        cell = _tri_cell() * rng.uniform(0.8, 1.3)
        pos = rng.random((12, 3)) @ cell
        sig = rng.uniform(0.8, 2.0, 12)
        A = O.coulomb_matrix(cell, pos, sig)
        assert np.linalg.eigvalsh(A).min() > -1e-12


def test_symmetry_perfect_rocksalt():
    frac, spec = synth.rocksalt_sites(1, 1, 1)
    a = 5.64
    cell = np.eye(3) * a
    pos = frac @ cell
    sig = np.where(spec == 0, 1.0, 1.8)
    A = O.coulomb_matrix_definition(cell, pos, sig)
    chiA, chiB, JA, JB = -2.0, 2.0, 2.0, 1.5
    chi = np.where(spec == 0, chiA, chiB)
    J = np.where(spec == 0, JA, JB)
    q, mu = O.solve_bordered(A, J, chi, 0.0)
    qa, qb = q[spec == 0], q[spec == 1]
    assert np.ptp(qa) < 1e-12 and np.ptp(qb) < 1e-12
    assert abs(qa[0] + qb[0]) < 1e-12
    s = np.where(spec == 0, 1.0, -1.0)
    cA = (A @ s)[spec == 0][0]
    cB = -(A @ s)[spec == 1][0]
    assert abs(qa[0] - (chiB - chiA) / (JA + JB + cA + cB)) < 1e-12


def test_translation_and_permutation_invariance():
    st = synth.rocksalt(1, 5.64, 0.2, synth.rng_for(98, 0))
    base = O.solve_structure(st, k_e=synth.COULOMB_K_EV_A)
    t = st.copy()
    t.pos = t.pos + np.array([1.234, -0.77, 3.1])
    tr = O.solve_structure(t, k_e=synth.COULOMB_K_EV_A)
    assert np.abs(tr.q - base.q).max() < 1e-12
    perm = np.random.default_rng(0).permutation(st.n)
    p = st.copy()
    p.pos, p.species, p.chi, p.J = st.pos[perm], st.species[perm], st.chi[perm], st.J[perm]
    pr = O.solve_structure(p, k_e=synth.COULOMB_K_EV_A)
    assert np.abs(pr.q - base.q[perm]).max() < 1e-12
    assert abs(pr.E_qeq - base.E_qeq) < 1e-10 * abs(base.E_qeq)


def test_large_cell_matvec_matches_dense():
    st = synth.rocksalt(2, 5.64, 0.15, synth.rng_for(97, 0), vacancy_frac=0.05, shear_deg=8.0)
    q = np.random.default_rng(2).normal(size=st.n)
    A = O.coulomb_matrix(st.cell, st.pos, st.sigma)
    y = O.ewald_matvec(st.cell, st.pos, st.sigma, q)
    assert np.abs(y - A @ q).max() < 1e-10 * np.abs(A @ q).max()
    rows = np.array([0, 5, st.n - 1])
    yr = O.ewald_matvec(st.cell, st.pos, st.sigma, q, rows=rows)
    assert np.abs(yr - (A @ q)[rows]).max() < 1e-10 * np.abs(A @ q).max()


def test_certified_bound_holds():
    st = synth.rocksalt(1, 5.64, 0.2, synth.rng_for(96, 0))
    A = O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=synth.COULOMB_K_EV_A)
    q, _ = O.solve_bordered(A, st.J, st.chi, 0.0)
    pert = np.random.default_rng(1).normal(size=st.n) * 1e-3
    pert -= pert.mean()
    qp = q + pert
    Pr, _ = O.projected_residual(A @ qp, st.J, st.chi, qp)
    assert np.linalg.norm(pert) <= O.certified_bound(Pr, st.J) * (1 + 1e-12)


# ---------------------------------------------------------------- forces of the force trick (SI eq. 4g_force_trick)

def test_forces_of_a_distant_gaussian_dimer_match_the_closed_form():
    """Two Gaussian charges +q, -q in a large cubic box: the force is the derivative of
    q1 q2 erf(r/(sqrt2 gamma))/r of eq. (elec_energy) plus the periodic sum's dipole term.
    With the G = 0 term dropped (tin-foil boundary), E = E_pair - (2 pi / 3V)|p|^2,
    p = q (R1 - R2), i.e. a force -4 pi q^2 r / (3V) along the bond; higher image terms
    fall off as 1/L^5."""
    L, r, s1, s2 = 80.0, 2.3, 1.0, 1.8
    cell = np.eye(3) * L
    pos = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
    q = np.array([0.8, -0.8])
    F = O.electrostatic_forces_fd(cell, pos, np.array([s1, s2]), q, k_e=1.0, h=1e-4)
    g = math.sqrt(s1 ** 2 + s2 ** 2)
    a = 1.0 / (math.sqrt(2.0) * g)
    dEdr = q[0] * q[1] * (2 * a / math.sqrt(math.pi) * math.exp(-(a * r) ** 2) / r - erf(a * r) / r ** 2)
    dEdr -= 4 * math.pi * q[0] ** 2 * r / (3 * L ** 3)
    # E depends on R2 - R1 = r x: F_1 = +dE/dr x, F_2 = -dE/dr x
    assert abs(F[0, 0] - dEdr) < 1e-5 * abs(dEdr)
    assert abs(F[1, 0] + dEdr) < 1e-5 * abs(dEdr)
    assert np.abs(F[:, 1:]).max() < 1e-7


def test_forces_sum_to_zero_and_follow_permutations_and_translations():
    rng = np.random.default_rng(17)
    cell = _tri_cell()
    pos = rng.random((5, 3)) @ cell
    sig = np.array([1.0, 1.8, 1.0, 1.8, 1.3])
    q = rng.normal(size=5)
    q -= q.mean()
    lam = rng.normal(size=5) * 0.3
    F = O.electrostatic_forces_fd(cell, pos, sig, q, lam)
    assert np.abs(F.sum(axis=0)).max() < 1e-7 * np.abs(F).max()
    perm = np.array([3, 0, 4, 1, 2])
    Fp = O.electrostatic_forces_fd(cell, pos[perm], sig[perm], q[perm], lam[perm])
    assert np.abs(Fp - F[perm]).max() < 1e-7 * np.abs(F).max()
    Ft = O.electrostatic_forces_fd(cell, pos + np.array([0.4, -1.3, 2.2]), sig, q, lam)
    assert np.abs(Ft - F).max() < 1e-7 * np.abs(F).max()


def test_force_trick_term_is_linear_in_lambda():
    """F(q, lam) = F(q, 0) + lam-term, the lam-term linear in lam: F(q, q/2) = 2 F(q, 0)
    (then (q/2 + lam)^T A q = q^T A q) and F(q, lam1 + lam2) = F(q, lam1) + F(q, lam2) - F(q, 0)."""
    rng = np.random.default_rng(21)
    cell = np.diag([9.0, 8.5, 10.0])
    pos = rng.random((4, 3)) @ cell
    sig = np.array([1.0, 1.5, 1.2, 0.9])
    q = rng.normal(size=4)
    l1, l2 = rng.normal(size=4), rng.normal(size=4)
    F0 = O.electrostatic_forces_fd(cell, pos, sig, q)
    assert np.abs(O.electrostatic_forces_fd(cell, pos, sig, q, 0.5 * q) - 2 * F0).max() < 1e-7 * np.abs(F0).max()
    F12 = O.electrostatic_forces_fd(cell, pos, sig, q, l1 + l2)
    F1 = O.electrostatic_forces_fd(cell, pos, sig, q, l1)
    F2 = O.electrostatic_forces_fd(cell, pos, sig, q, l2)
    assert np.abs(F12 - (F1 + F2 - F0)).max() < 1e-7 * np.abs(F12).max()


def test_element_potentials_sum_to_the_coulomb_potential():
    rng = np.random.default_rng(5)
    cell = _tri_cell()
    pos = rng.random((6, 3)) @ cell
    spc = np.array([0, 1, 2, 0, 1, 2])
    sig = np.array([1.0, 1.8, 1.3])[spc]
    q = rng.normal(size=6)
    A = O.coulomb_matrix(cell, pos, sig)
    G = O.element_potentials(A, spc, q, 3)
    assert np.abs(G.sum(axis=1) - A @ q).max() < 1e-13 * np.abs(A @ q).max()
    # a charge of element z only changes Gamma[:, z]
    q2 = q.copy()
    q2[1] += 0.7
    G2 = O.element_potentials(A, spc, q2, 3)
    assert np.abs(G2[:, [0, 2]] - G[:, [0, 2]]).max() == 0.0
    assert np.abs(G2[:, 1] - G[:, 1] - 0.7 * A[:, 1]).max() < 1e-14


@pytest.mark.parametrize("point", [False, True])
def test_analytic_ewald_gradient_matches_dense_central_differences(point):
    """The term-by-term position derivative of a row of the Ewald sum (large-cell force oracle)
    against central differences of the dense matrix, on a triclinic cell with two widths and
    with point charges (sigma = 0: textbook Ewald), with and without the lambda term."""
    rng = np.random.default_rng(33)
    cell = _tri_cell()
    n = 9
    pos = rng.random((n, 3)) @ cell
    sig = np.zeros(n) if point else np.where(np.arange(n) % 2 == 0, 1.0, 1.7)
    q = rng.normal(size=n)
    q -= q.mean()
    lam = rng.normal(size=n)
    rows = [0, 3, 8]
    for la in (None, lam):
        Ffd = O.electrostatic_forces_fd(cell, pos, sig, q, la, atoms=rows, omega=2.0 if point else None)
        Fan = O.electrostatic_forces_ewald(cell, pos, sig, q, rows, lam=la)
        assert np.abs(Fan - Ffd).max() < 1e-7 * np.abs(Ffd).max()


def test_analytic_ewald_forces_sum_to_zero():
    """Without the lambda term the forces are minus the gradient of a translation-invariant
    energy: they sum to zero over the cell (exactly, independent of the Ewald width)."""
    rng = np.random.default_rng(34)
    cell = _tri_cell()
    pos = rng.random((12, 3)) @ cell
    sig = rng.uniform(0.8, 1.8, size=12)
    q = rng.normal(size=12)
    F = O.electrostatic_forces_ewald(cell, pos, sig, q, np.arange(12))
    assert np.abs(F.sum(axis=0)).max() < 1e-10 * np.abs(F).max()
    F2 = O.electrostatic_forces_ewald(cell, pos, sig, q, np.arange(12), omega=3.0)
    assert np.abs(F2 - F).max() < 1e-9 * np.abs(F).max()


def test_force_trick_gives_the_total_derivative_through_the_solve():
    """SI eq. (4g_force_trick): for E(R) = 1/2 q*(R)^T A(R) q*(R) with q* the QEq charges,
    dE/dR_k = d/dR_k [(q/2 + lam)^T A q] at fixed q = q*, lam solving
    (A + J) lam = -dE/dq + nu 1 = -A q* + nu 1, sum lam = 0.  Checked against central
    differences of E with the charges re-solved at every displaced geometry."""
    rng = np.random.default_rng(41)
    cell = _tri_cell()
    n = 6
    pos = rng.random((n, 3)) @ cell
    sig = np.array([1.0, 1.6, 1.0, 1.6, 1.2, 1.2])
    J = rng.uniform(1.0, 3.0, size=n)
    chi = rng.normal(0.0, 1.0, size=n)
    q_tot = 1.0

    def energy(p):
        A = O.coulomb_matrix(cell, p, sig, omega=2.0)
        q, _ = O.solve_bordered(A, J, chi, q_tot)
        return 0.5 * q @ A @ q

    A = O.coulomb_matrix(cell, pos, sig, omega=2.0)
    q, _ = O.solve_bordered(A, J, chi, q_tot)
    lam, _ = O.solve_bordered(A, J, A @ q, 0.0)
    assert abs(lam.sum()) < 1e-12
    F = O.electrostatic_forces_fd(cell, pos, sig, q, lam, omega=2.0)
    h = 1e-4
    Ftot = np.zeros((n, 3))
    for k in range(n):
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[k, c] += h
            pm[k, c] -= h
            Ftot[k, c] = -(energy(pp) - energy(pm)) / (2 * h)
    assert np.abs(F - Ftot).max() < 1e-6 * np.abs(Ftot).max()
    # without lam the fixed-charge derivative is a different (wrong) total force here
    F0 = O.electrostatic_forces_fd(cell, pos, sig, q, omega=2.0)
    assert np.abs(F0 - Ftot).max() > 1e-3 * np.abs(Ftot).max()


@pytest.mark.parametrize("analytic", [False, True])
def test_strain_derivative_of_the_madelung_energy(analytic):
    """Perfect rock-salt of point charges +-1: W = 1/2 q^T A q = -(N/2) M / r0 (M the Madelung
    constant, r0 = a/2).  The energy is homogeneous of degree -1 in the lengths and the crystal
    is cubic, so dW/d eps = -W/3 times the identity."""
    frac, spec = synth.rocksalt_sites(2, 2, 2)
    a = 5.64
    cell = np.eye(3) * 2 * a
    pos = frac @ cell
    q = np.where(spec == 0, 1.0, -1.0)
    sig = np.zeros(len(q))
    W = -(len(q) / 2) * MADELUNG / (a / 2)
    if analytic:
        D = O.electrostatic_strain_derivative_ewald(cell, pos, sig, q, omega=2.0)
    else:
        D = O.electrostatic_strain_derivative_fd(cell, pos, sig, q, omega=2.0)
    assert np.abs(D - (-W / 3) * np.eye(3)).max() < 1e-7 * abs(W)


def test_strain_derivative_homogeneity_with_gaussian_widths():
    """W(s R, s h, s sigma) = W / s: trace(dW/d eps) + sum_s sigma_s dW/d sigma_s = -W, on a
    triclinic cell with three widths; the strain derivative is also symmetric (rotations
    leave W unchanged)."""
    rng = np.random.default_rng(51)
    cell = _tri_cell()
    n = 8
    pos = rng.random((n, 3)) @ cell
    spc = np.arange(n) % 3
    sig_s = np.array([1.0, 1.5, 1.9])
    q = rng.normal(size=n)
    lam = rng.normal(size=n)
    w = 0.5 * q + lam

    def W(s_s):
        return float(w @ O.coulomb_matrix(cell, pos, s_s[spc], omega=2.5) @ q)

    D = O.electrostatic_strain_derivative_fd(cell, pos, sig_s[spc], q, lam, omega=2.5)
    h = 1e-5
    dsig = 0.0
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        dsig += sig_s[k] * (W(sig_s + e) - W(sig_s - e)) / (2 * h)
    assert abs(np.trace(D) + dsig + W(sig_s)) < 1e-7 * np.abs(D).max()
    assert np.abs(D - D.T).max() < 1e-7 * np.abs(D).max()


@pytest.mark.parametrize("point", [False, True])
def test_analytic_strain_derivative_matches_dense_central_differences(point):
    rng = np.random.default_rng(52)
    cell = _tri_cell()
    n = 9
    pos = rng.random((n, 3)) @ cell
    sig = np.zeros(n) if point else np.where(np.arange(n) % 2 == 0, 0.9, 1.6)
    q = rng.normal(size=n)
    lam = rng.normal(size=n)
    for la in (None, lam):
        Dfd = O.electrostatic_strain_derivative_fd(cell, pos, sig, q, la, omega=2.0)
        Dan = O.electrostatic_strain_derivative_ewald(cell, pos, sig, q, la, omega=2.5)
        assert np.abs(Dan - Dfd).max() < 1e-7 * np.abs(Dfd).max()


# --------------------------------------------------------------------------- 4G charge training

def _train_case(n=7, seed=61):
    rng = np.random.default_rng(seed)
    cell = _tri_cell()
    pos = rng.random((n, 3)) @ cell
    sig = np.where(np.arange(n) % 2 == 0, 1.0, 1.6)
    A = O.coulomb_matrix(cell, pos, sig, omega=2.0)
    J = rng.uniform(1.0, 3.0, size=n)
    chi = rng.normal(size=n)
    return A, J, chi


def test_charges_from_the_cached_inverse_two_atoms_by_hand():
    """N = 2: q1 = (chi2 - chi1 + Q (a22 - a12)) / (a11 + a22 - 2 a12) with a = A + J, from
    eliminating q2 = Q - q1 in (A + J) q = -chi + mu 1."""
    a = np.array([[2.7, 0.4], [0.4, 1.9]])
    J = np.zeros(2)
    chi = np.array([0.3, -0.8])
    Q = 0.5
    Kinv = O.bordered_inverse(a, J)
    q, mu = O.charges_from_inverse(Kinv, chi, Q)
    q1 = (chi[1] - chi[0] + Q * (a[1, 1] - a[0, 1])) / (a[0, 0] + a[1, 1] - 2 * a[0, 1])
    assert abs(q[0] - q1) < 1e-14 and abs(q[1] - (Q - q1)) < 1e-14
    assert abs(a[0] @ q + chi[0] - mu) < 1e-14 and abs(a[1] @ q + chi[1] - mu) < 1e-14


def test_charge_training_gradients_match_central_differences():
    """dL/dchi and dL/dJ of L = 1/2 |q(chi, J) - q_ref|^2 through the re-inverted bordered
    matrix, against central differences; dL/dchi sums to zero (a uniform shift of chi only
    moves mu)."""
    A, J, chi = _train_case()
    q_ref = np.random.default_rng(3).normal(size=len(J)) * 0.2
    Q = -1.0

    def loss(c, j):
        q, _ = O.charges_from_inverse(O.bordered_inverse(A, j), c, Q)
        return 0.5 * float(np.sum((q - q_ref) ** 2))

    Kinv = O.bordered_inverse(A, J)
    q, _ = O.charges_from_inverse(Kinv, chi, Q)
    gchi, gJ = O.charges_backward(Kinv, q, q - q_ref)
    h = 1e-6
    for i in range(len(J)):
        e = np.zeros(len(J))
        e[i] = h
        assert abs((loss(chi + e, J) - loss(chi - e, J)) / (2 * h) - gchi[i]) < 1e-8
        assert abs((loss(chi, J + e) - loss(chi, J - e)) / (2 * h) - gJ[i]) < 1e-8
    assert abs(gchi.sum()) < 1e-12
    assert abs(q.sum() - Q) < 1e-12
