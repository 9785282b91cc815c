"""FP64 CPU oracle of the periodic QEq solve.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this module.  It
shares no code with the CUDA path (``paper_2607_17978_b300``): only the seeded
input generators are common to both.

What it computes (RuNNer 2.0 paper, Sec. 2.4 "Electrostatics and Charge
Equilibration" and SI "Fourth-Generation HDNNPs and Charge Equilibration"):

* the Coulomb kernel of normalised Gaussian charges, eq. (elec_energy):
  E_ii = 1/(sigma_i sqrt(pi)), E_ij = erf(r_ij / (sqrt(2) gamma_ij)) / r_ij,
  gamma_ij = sqrt(sigma_i^2 + sigma_j^2), summed over the periodic images of a
  cell with the G = 0 term of the density dropped (the neutralising
  background that the plane-wave kernel 4 pi / G^2 of eq. (matvec) implies):

      A_ij = k_e (4 pi / V) sum_{G != 0} exp(-G^2 gamma_ij^2 / 2) cos(G.(r_i - r_j)) / G^2

  (``coulomb_matrix_definition``; the Ewald-split assembly of SI "Ewald
  Summation" is ``coulomb_matrix``; both give the same matrix);
* the QEq energy E_QEq = 1/2 q^T (E + diag J) q + chi^T q, eq. (qeq_energy),
  reading the garbled "J^T I" as diag(J) as the SI energy expression states;
* the bordered (N+1) x (N+1) Lagrange system of eq. (4G_qeq_prime),
  [A 1; 1^T 0][q; lambda] = [-chi; q_tot], solved by dense LU; the SI form
  (A + J) q = -chi + mu 1 (eq. qeq) gives mu = -lambda;
* for cells too large for a dense matrix, the FP64 Ewald matrix-vector product
  (C, ``ewald_oracle.c``), the projected residual and the certified bound
  ||q - q*||_2 <= ||P (A q + chi)||_2 / J_min  (A >= diag(J) on the
  constraint plane because E_elec >= 0).

Units: the caller passes k_e (14.3996454784 eV*A/e^2 for eV, Angstrom, e;
1 for atomic units, which the paper uses internally).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np
from scipy.linalg import blas as _blas
from scipy.special import erfc as _erfc  # noqa: F401  (used by tests through this module)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_ewald_oracle.so")
_lib = None


def build_c(force: bool = False) -> str:
    """Compile ewald_oracle.c (plain C + OpenMP) next to this file."""
    src = os.path.join(_HERE, "ewald_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", _SO, src, "-lm"])
    return _SO


def _clib():
    global _lib
    if _lib is None:
        build_c()
        lib = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_realspace_dense.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_realspace_dense.restype = ctypes.c_int
        lib.oracle_ewald_matvec.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int, ip, dp]
        lib.oracle_ewald_matvec.restype = ctypes.c_int
        lib.oracle_ewald_potential_grad.argtypes = lib.oracle_ewald_matvec.argtypes
        lib.oracle_ewald_potential_grad.restype = ctypes.c_int
        lib.oracle_ewald_strain_derivative.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp, ctypes.c_double,
                                                       ctypes.c_double, ctypes.c_double, dp]
        lib.oracle_ewald_strain_derivative.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------- geometry

def volume(cell: np.ndarray) -> float:
    return abs(float(np.linalg.det(cell)))


def reciprocal_vectors(cell: np.ndarray) -> np.ndarray:
    """Rows b_k with a_j . b_k = delta_jk, so that G(m) = 2 pi m @ B."""
    return np.linalg.inv(cell).T


def plane_widths(cell: np.ndarray) -> np.ndarray:
    V = volume(cell)
    return np.array([V / np.linalg.norm(np.cross(cell[(d + 1) % 3], cell[(d + 2) % 3])) for d in range(3)])


def g_vectors_half(cell: np.ndarray, g_cut: float):
    """G = 2 pi m B for integer m in the half-space m > 0 (lexicographic), |G| <= g_cut."""
    B = reciprocal_vectors(cell)
    wd = plane_widths(cell)
    M = (np.floor(g_cut * wd / (2 * math.pi)) + 1).astype(int)
    r = [np.arange(-M[d], M[d] + 1) for d in range(3)]
    m = np.stack(np.meshgrid(*r, indexing="ij"), -1).reshape(-1, 3)
    half = (m[:, 0] > 0) | ((m[:, 0] == 0) & (m[:, 1] > 0)) | ((m[:, 0] == 0) & (m[:, 1] == 0) & (m[:, 2] > 0))
    m = m[half]
    G = 2 * math.pi * m @ B
    G2 = np.einsum("ij,ij->i", G, G)
    keep = G2 <= g_cut * g_cut
    return G[keep], G2[keep]


# --------------------------------------------------------------------------- Coulomb matrix

def coulomb_matrix_definition(cell, pos, sigma, k_e=1.0, tol=1e-17):
    """A without hardness, straight from the definition: the reciprocal sum with gamma_ij.

    Only for tiny cells (cost N^2 * n_G); sigma must be > 0.
    """
    sigma = np.asarray(sigma, float)
    assert np.all(sigma > 0)
    V = volume(cell)
    gmin = math.sqrt(2.0) * float(sigma.min())
    # exp(-G^2 gmin^2/2) < tol  ->  G_cut
    g_cut = math.sqrt(2.0 * math.log(1.0 / tol)) / gmin
    G, G2 = g_vectors_half(cell, g_cut)
    n = len(pos)
    A = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            gam2 = sigma[i] ** 2 + sigma[j] ** 2
            ph = G @ (pos[i] - pos[j])
            A[i, j] = 2.0 * (4 * math.pi / V) * np.sum(np.exp(-0.5 * G2 * gam2) * np.cos(ph) / G2)
    return k_e * A


def default_omega(cell, sigma) -> float:
    """Ewald width for the dense assembly (any value gives the same matrix)."""
    L = volume(cell) ** (1.0 / 3.0)
    return max(2.0, 0.05 * L, 0.5 * math.sqrt(2.0) * float(np.max(sigma)) if len(sigma) else 2.0)


def realspace_cut(omega: float, tol: float) -> float:
    """r with erfc(r/(sqrt2 omega)) <= tol (bisection on the monotone erfc)."""
    lo, hi = 0.0, 60.0 * omega
    from scipy.special import erfc
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if erfc(mid / (math.sqrt(2.0) * omega)) > tol:
            lo = mid
        else:
            hi = mid
    return hi


def recip_cut(omega: float, tol: float) -> float:
    """|G| with exp(-G^2 omega^2/2) <= tol."""
    return math.sqrt(2.0 * math.log(1.0 / tol)) / omega


def coulomb_matrix(cell, pos, sigma, k_e=1.0, omega=None, tol=1e-15):
    """A without hardness by the Ewald split (SI "Ewald Summation"), dense FP64.

    sigma may contain zeros (point charges; the divergent self energy is left
    out).  The reciprocal part is grouped by distinct pair width w_ij so that
    each group is one BLAS rank-k update over the structure-factor matrices.
    """
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    n = len(pos)
    if omega is None:
        omega = default_omega(cell, sigma)
    V = volume(cell)
    A = np.zeros((n, n))
    r_cut = realspace_cut(omega, tol * 1e-2)
    rc = _clib().oracle_realspace_dense(n, _dp(cell), _dp(pos), _dp(sigma), float(omega), float(r_cut), _dp(A))
    if rc != 0:
        raise MemoryError("oracle_realspace_dense failed")
    # reciprocal part: w_ij = max(gamma_ij, omega); group atoms by sigma
    uniq, inv = np.unique(sigma, return_inverse=True)
    gam = np.sqrt(uniq[:, None] ** 2 + uniq[None, :] ** 2)
    W = np.maximum(gam, omega)
    g_cut = recip_cut(float(W.min()), tol)
    G_all, G2_all = g_vectors_half(cell, g_cut)
    groups = [np.nonzero(inv == a)[0] for a in range(len(uniq))]
    chunk = max(256, int(2.0e8 // max(n, 1) // 8))
    for c0 in range(0, len(G2_all), chunk):
        G, G2 = G_all[c0:c0 + chunk], G2_all[c0:c0 + chunk]
        ph = pos @ G.T                                    # n x nG
        C, S = np.cos(ph), np.sin(ph)
        for a in range(len(uniq)):
            for b in range(a, len(uniq)):
                f = 2.0 * (4 * math.pi / V) * np.exp(-0.5 * G2 * W[a, b] ** 2) / G2
                sq = np.sqrt(f)
                ia, ib = groups[a], groups[b]
                Ca, Sa = C[ia] * sq, S[ia] * sq
                if a == b:
                    blk = _blas.dsyrk(1.0, np.asfortranarray(Ca)) + _blas.dsyrk(1.0, np.asfortranarray(Sa))
                    blk = np.triu(blk) + np.triu(blk, 1).T
                    A[np.ix_(ia, ia)] += blk
                else:
                    Cb, Sb = C[ib] * sq, S[ib] * sq
                    blk = Ca @ Cb.T + Sa @ Sb.T
                    A[np.ix_(ia, ib)] += blk
                    A[np.ix_(ib, ia)] += blk.T
    return k_e * A


# --------------------------------------------------------------------------- solve

@dataclass
class QEqSolution:
    q: np.ndarray
    mu: float
    E_qeq: float
    E_elec: float


def solve_bordered(A_elec, J, chi, q_tot) -> tuple[np.ndarray, float]:
    """Dense LU of the bordered system (eq. 4G_qeq_prime); returns q and mu = -lambda."""
    n = len(chi)
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = A_elec + np.diag(J)
    M[:n, n] = 1.0
    M[n, :n] = 1.0
    rhs = np.concatenate([-np.asarray(chi, float), [float(q_tot)]])
    x = np.linalg.solve(M, rhs)
    return x[:n], -float(x[n])


# --------------------------------------------------------------------------- 4G charge training

def bordered_inverse(A_elec, J):
    """Inverse of the bordered matrix A' = [[E + diag J, 1], [1^T, 0]] of eq. (4G_qeq_prime),
    the object Sec. "4G-HDNNP Charge Training" caches per training structure (re-inverted
    when the hardness J is learned)."""
    n = len(J)
    M = np.zeros((n + 1, n + 1))
    M[:n, :n] = np.asarray(A_elec, float) + np.diag(np.asarray(J, float))
    M[:n, n] = 1.0
    M[n, :n] = 1.0
    return np.linalg.inv(M)


def charges_from_inverse(Kinv, chi, q_tot):
    """q' = -A'^{-1} chi' with chi' = (chi, -q_tot): one matrix-vector product with the cached
    inverse (Sec. "4G-HDNNP Charge Training").  Returns q and mu (= -lambda)."""
    n = len(chi)
    x = Kinv @ np.concatenate([-np.asarray(chi, float), [float(q_tot)]])
    return x[:n], -float(x[n])


def charges_backward(Kinv, q, gq):
    """Gradients of a loss L(q) with respect to chi and J through the bordered solve: A' is
    symmetric, so with (lam, nu) = A'^{-1} (dL/dq, 0),
        dL/dchi = -lam,    dL/dJ_i = -lam_i q_i   (dA'/dJ_i = e_i e_i^T)."""
    n = len(q)
    x = Kinv @ np.concatenate([np.asarray(gq, float), [0.0]])
    lam = x[:n]
    return -lam, -lam * np.asarray(q, float)


def energies(A_elec, J, chi, q) -> tuple[float, float]:
    """E_QEq = chi.q + 1/2 q.(E + diag J) q (eq. qeq_energy) and E_elec = 1/2 q.E q (eq. elec_energy)."""
    Eq = A_elec @ q
    E_elec = 0.5 * float(q @ Eq)
    return float(chi @ q) + 0.5 * float(np.sum(J * q * q)) + E_elec, E_elec


def solve_structure(st, k_e=1.0, omega=None) -> QEqSolution:
    """Oracle solve of a ``synth.Structure``."""
    A = coulomb_matrix(st.cell, st.pos, st.sigma, k_e=k_e, omega=omega)
    q, mu = solve_bordered(A, st.J, st.chi, st.q_tot)
    E, Ee = energies(A, st.J, st.chi, q)
    return QEqSolution(q, mu, E, Ee)


# --------------------------------------------------------------------------- large cells

def _ewald_setup(cell, pos, sigma, q, omega, tol):
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    gmax = math.sqrt(2.0) * float(sigma.max())
    if omega is None:
        # balance O(n_G) structure factors against O(neighbours) real space
        V = volume(cell)
        omega = max(gmax, 0.9 * (V / 1.0e4) ** (1.0 / 6.0) * 2.0)
    omega = max(float(omega), gmax)
    return cell, pos, sigma, q, omega, realspace_cut(omega, tol * 1e-1), recip_cut(omega, tol)


def ewald_matvec(cell, pos, sigma, q, k_e=1.0, omega=None, tol=1e-13, rows=None):
    """y = A_elec q (no hardness) for large cells; ``rows`` selects output rows."""
    cell, pos, sigma, q, omega, r_cut, g_cut = _ewald_setup(cell, pos, sigma, q, omega, tol)
    n = len(pos)
    if rows is None:
        y = np.zeros(n)
        rc = _clib().oracle_ewald_matvec(n, _dp(cell), _dp(pos), _dp(sigma), _dp(q), omega, r_cut, g_cut,
                                         0, None, _dp(y))
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        y = np.zeros(len(rows))
        rc = _clib().oracle_ewald_matvec(n, _dp(cell), _dp(pos), _dp(sigma), _dp(q), omega, r_cut, g_cut,
                                         len(rows), rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(y))
    if rc != 0:
        raise RuntimeError(f"oracle_ewald_matvec failed ({rc})")
    return k_e * y


def ewald_potential_gradient(cell, pos, sigma, x, rows, k_e=1.0, omega=None, tol=1e-13):
    """g[o] = d/dR_i sum_j A_ij x_j at atom i = rows[o] (positions of the other atoms and x
    fixed), shape (len(rows), 3): the position derivative of a row of the Ewald sum, term by
    term (SI "Ewald Summation"); the self and G = 0 width terms do not depend on positions."""
    cell, pos, sigma, x, omega, r_cut, g_cut = _ewald_setup(cell, pos, sigma, x, omega, tol)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    g = np.zeros(3 * len(rows))
    rc = _clib().oracle_ewald_potential_grad(len(pos), _dp(cell), _dp(pos), _dp(sigma), _dp(x), omega, r_cut,
                                             g_cut, len(rows), rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                             _dp(g))
    if rc != 0:
        raise RuntimeError(f"oracle_ewald_potential_grad failed ({rc})")
    return k_e * g.reshape(-1, 3)


def electrostatic_forces_ewald(cell, pos, sigma, q, rows, lam=None, k_e=1.0, omega=None, tol=1e-13):
    """The electrostatic terms of the force trick, SI eq. (4g_force_trick), at atoms ``rows``
    of a cell too large for the dense matrix:

        F_k = -d/dR_k [(q/2 + lam)^T A q] = -(q_k + lam_k) grad phi_q(k) - q_k grad phi_lam(k)

    (A symmetric: the R_k dependence sits in row and column k), with grad phi_x(k) from
    ewald_potential_gradient.  lam = None leaves the lam terms out."""
    rows = np.asarray(rows)
    q = np.asarray(q, np.float64)
    gq = ewald_potential_gradient(cell, pos, sigma, q, rows, k_e, omega, tol)
    F = -q[rows, None] * gq
    if lam is not None:
        lam = np.asarray(lam, np.float64)
        gl = ewald_potential_gradient(cell, pos, sigma, lam, rows, k_e, omega, tol)
        F -= lam[rows, None] * gq + q[rows, None] * gl
    return F


def projected_residual(y_elec, J, chi, q):
    """r = A q + chi with A = E + diag J, projected onto 1^T r = 0; also mu = mean(A q + chi)."""
    r = y_elec + J * q + chi
    mu = float(np.mean(r))
    return r - mu, mu


def certified_bound(Pr, J) -> float:
    """||q - q*||_2 <= ||P(Aq + chi)||_2 / J_min (A - diag J is PSD on 1^perp)."""
    return float(np.linalg.norm(Pr) / np.min(J))


# --------------------------------------------------------------------------- forces (force trick)

def electrostatic_forces_fd(cell, pos, sigma, q, lam=None, k_e=1.0, h=1e-4, atoms=None, omega=None):
    """The electrostatic terms of the force trick, SI eq. (4g_force_trick), by central
    differences of the dense Coulomb matrix:

        F_k = -d/dR_k [ 1/2 q^T A(R) q + lam^T A(R) q ] = -dE_elec/dR_k|_q - lam^T (dA/dR_k) q

    with A the Gaussian-charge Coulomb matrix (the hardness diagonal does not depend on
    the positions).  lam = None leaves the second term out.  ``atoms`` selects the atoms
    whose force is returned (default: all), shape (len(atoms), 3).  The Ewald width is held
    fixed over the displacements (any width gives the same matrix).
    """
    pos = np.asarray(pos, np.float64)
    q = np.asarray(q, np.float64)
    lam = np.zeros_like(q) if lam is None else np.asarray(lam, np.float64)
    sigma = np.asarray(sigma, np.float64)
    if omega is None:
        omega = default_omega(cell, sigma)
    wvec = 0.5 * q + lam  # 1/2 q^T A q + lam^T A q = (q/2 + lam)^T A q for symmetric A
    atoms = list(range(len(pos))) if atoms is None else list(atoms)
    F = np.zeros((len(atoms), 3))
    for a, k in enumerate(atoms):
        for c in range(3):
            e = []
            for sgn in (1.0, -1.0):
                p = pos.copy()
                p[k, c] += sgn * h
                A = coulomb_matrix(cell, p, sigma, k_e=k_e, omega=omega)
                e.append(float(wvec @ (A @ q)))
            F[a, c] = -(e[0] - e[1]) / (2.0 * h)
    return F


def strained(cell, pos, eps):
    """Cell rows and positions under the homogeneous deformation r -> (1 + eps) r."""
    F = np.eye(3) + np.asarray(eps, np.float64)
    return np.asarray(cell, np.float64) @ F.T, np.asarray(pos, np.float64) @ F.T


def electrostatic_strain_derivative_fd(cell, pos, sigma, q, lam=None, k_e=1.0, h=1e-5, omega=None):
    """D[a, b] = d/d eps_ab [(q/2 + lam)^T A q] at fixed charges, A the Gaussian-charge Coulomb
    matrix of the deformed cell and positions (r -> (1 + eps) r), by central differences: the
    electrostatic part of the strain derivative in the force trick (SI eq. 4g_force_trick,
    applied to the cell instead of an atom).  The stress of the form is D / V."""
    q = np.asarray(q, np.float64)
    lam = np.zeros_like(q) if lam is None else np.asarray(lam, np.float64)
    sigma = np.asarray(sigma, np.float64)
    if omega is None:
        omega = default_omega(cell, sigma)
    wvec = 0.5 * q + lam
    D = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            e = []
            for sgn in (1.0, -1.0):
                eps = np.zeros((3, 3))
                eps[a, b] = sgn * h
                c2, p2 = strained(cell, pos, eps)
                A = coulomb_matrix(c2, p2, sigma, k_e=k_e, omega=omega)
                e.append(float(wvec @ (A @ q)))
            D[a, b] = (e[0] - e[1]) / (2.0 * h)
    return D


def electrostatic_strain_derivative_ewald(cell, pos, sigma, q, lam=None, k_e=1.0, omega=None, tol=1e-13):
    """The same strain derivative for cells too large for the dense matrix, term by term from
    the Ewald split (oracle_ewald_strain_derivative): D = d/d eps [(q/2 + lam)^T A q]."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    wvec = 0.5 * q + (0.0 if lam is None else np.asarray(lam, np.float64))
    cell, pos, sigma, q, omega, r_cut, g_cut = _ewald_setup(cell, pos, sigma, q, omega, tol)
    wvec = np.ascontiguousarray(wvec, dtype=np.float64)
    D = np.zeros(9)
    rc = _clib().oracle_ewald_strain_derivative(len(pos), _dp(cell), _dp(pos), _dp(sigma), _dp(wvec), _dp(q),
                                                omega, r_cut, g_cut, _dp(D))
    if rc != 0:
        raise RuntimeError(f"oracle_ewald_strain_derivative failed ({rc})")
    return k_e * D.reshape(3, 3)


# --------------------------------------------------------------------------- electrostatic embedding

def element_potentials(A_elec, species, q, n_species):
    """Element-resolved electrostatic potentials at every atomic site (the ee4G embedding
    of Sec. 2.2 and Fig. 1c): Gamma[i, z] = sum_{j of element z} E_ij q_j, with E the
    Gaussian-charge Coulomb matrix; summed over z they give E q."""
    species = np.asarray(species)
    G = np.zeros((len(q), n_species))
    for z in range(n_species):
        m = species == z
        G[:, z] = A_elec[:, m] @ np.asarray(q, np.float64)[m]
    return G
