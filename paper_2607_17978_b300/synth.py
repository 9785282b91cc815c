"""Seeded synthetic QEq inputs shaped like the paper's periodic workloads.

This module only draws inputs: periodic cells, atom positions, species labels
and per-atom electronegativity / hardness / Gaussian-width values.  It holds
none of the charge-equilibration arithmetic, so both the CUDA path and the CPU
oracle can take their inputs from here without sharing any method code.

Every draw goes through ``rng_for(cfg_id, struct_id)``, a numpy Generator on
``SeedSequence([20260, cfg_id, struct_id])``.

Workloads (cf. the paper's water benchmarks of Sec. 3 and the 4G charge
equilibration of Sec. 2.4 / SI "Fourth-Generation HDNNPs and Charge
Equilibration"; the water data are not available, so rock-salt and random
ionic cells stand in for them):

* ``rocksalt``: n1 x n2 x n3 conventional rock-salt cells (4 A + 4 B atoms
  each, B displaced by a/2 along x), Gaussian jitter, optional random
  vacancies and an optional random upper-triangular shear.
* ``random_ionic``: random orthorhombic or triclinic cells at a fixed number
  density, random sequential placement with a minimum distance, 2-4 species.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_ROOT = 20260

# Coulomb constant e^2/(4 pi eps0) in eV*Angstrom/e^2 (CODATA).
COULOMB_K_EV_A = 14.3996454784


def rng_for(cfg_id: int, struct_id: int = 0) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([SEED_ROOT, int(cfg_id), int(struct_id)]))


@dataclasses.dataclass
class Structure:
    """One periodic cell with per-atom QEq parameters.

    cell    (3,3) float64, rows are the lattice vectors a1, a2, a3 [Angstrom]
    pos     (N,3) float64 Cartesian positions [Angstrom] (not necessarily wrapped)
    species (N,)  int32 in [0, n_species)
    chi     (N,)  float64 electronegativity [eV/e]
    J       (N,)  float64 hardness [eV/e^2], > 0
    sigma_s (n_species,) float64 Gaussian width per species [Angstrom], > 0
    q_tot   total charge [e]
    """

    cell: np.ndarray
    pos: np.ndarray
    species: np.ndarray
    chi: np.ndarray
    J: np.ndarray
    sigma_s: np.ndarray
    q_tot: float = 0.0

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_species(self) -> int:
        return int(self.sigma_s.shape[0])

    @property
    def sigma(self) -> np.ndarray:
        return self.sigma_s[self.species]

    def copy(self) -> "Structure":
        return Structure(self.cell.copy(), self.pos.copy(), self.species.copy(), self.chi.copy(),
                         self.J.copy(), self.sigma_s.copy(), float(self.q_tot))


# --------------------------------------------------------------------------- cells

_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
_B_SHIFT = np.array([0.5, 0.0, 0.0])


def rocksalt_sites(n1: int, n2: int, n3: int):
    """Fractional sites (in units of the supercell) and species of a rock-salt supercell."""
    idx = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1).reshape(-1, 3)
    a_sites = (idx[:, None, :] + _FCC[None, :, :]).reshape(-1, 3)
    b_sites = (idx[:, None, :] + (_FCC + _B_SHIFT)[None, :, :]).reshape(-1, 3)
    frac = np.concatenate([a_sites, b_sites], 0) / np.array([n1, n2, n3], dtype=np.float64)
    species = np.concatenate([np.zeros(len(a_sites), np.int32), np.ones(len(b_sites), np.int32)])
    return frac, species


def sheared_cell(lengths, tilt_deg, rng):
    """Upper-triangular cell (rows a1, a2, a3) with random xy/xz/yz tilts of up to ``tilt_deg``."""
    L1, L2, L3 = lengths
    h = np.diag([L1, L2, L3]).astype(np.float64)
    if tilt_deg > 0:
        th = np.deg2rad(rng.uniform(-tilt_deg, tilt_deg, size=3))
        h[0, 1] = L2 * math.tan(th[0])
        h[0, 2] = L3 * math.tan(th[1])
        h[1, 2] = L3 * math.tan(th[2])
    return h


def rocksalt(n_cells, a: float, jitter: float, rng: np.random.Generator, *,
             vacancy_frac: float = 0.0, shear_deg: float = 0.0,
             chi_mean=(-2.0, 2.0), chi_std=0.3, J_s=(2.0, 1.5), sigma_s=(1.0, 1.8),
             q_tot: float = 0.0) -> Structure:
    if np.isscalar(n_cells):
        n_cells = (int(n_cells),) * 3
    n1, n2, n3 = n_cells
    frac, species = rocksalt_sites(n1, n2, n3)
    cell = sheared_cell((n1 * a, n2 * a, n3 * a), shear_deg, rng)
    if vacancy_frac > 0:
        n_rm = int(math.floor(vacancy_frac * len(frac)))
        keep = np.sort(rng.permutation(len(frac))[n_rm:])
        frac, species = frac[keep], species[keep]
    pos = frac @ cell
    if jitter > 0:
        pos = pos + rng.normal(0.0, jitter, size=pos.shape)
    chi = rng.normal(np.asarray(chi_mean)[species], chi_std)
    J = np.asarray(J_s, dtype=np.float64)[species]
    return Structure(cell, pos, species.astype(np.int32), chi, J, np.asarray(sigma_s, np.float64), float(q_tot))


def _place_with_min_distance(n: int, cell: np.ndarray, min_dist: float, rng: np.random.Generator) -> np.ndarray:
    """Uniform random fractional positions, redrawing one atom of every pair closer than
    min_dist (periodic images included) until none is left."""
    from scipy.spatial import cKDTree
    u = rng.random((n, 3))
    V = abs(np.linalg.det(cell))
    wd = np.array([V / np.linalg.norm(np.cross(cell[(d + 1) % 3], cell[(d + 2) % 3])) for d in range(3)])
    delta = min_dist / wd                      # fractional distance to a face that matters
    shifts = np.stack(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij"), -1).reshape(-1, 3)
    shifts = shifts[np.any(shifts != 0, axis=1)]
    for _ in range(1000):
        # the cell plus the periodic images of atoms near the faces they are shifted across
        ids, pts = [np.arange(n)], [u]
        for sh in shifts:
            m = np.ones(n, bool)
            for d in range(3):
                if sh[d] == 1:
                    m &= u[:, d] < delta[d]
                elif sh[d] == -1:
                    m &= u[:, d] > 1.0 - delta[d]
            if m.any():
                ids.append(np.nonzero(m)[0])
                pts.append(u[m] + sh)
        ids = np.concatenate(ids)
        X = np.concatenate(pts) @ cell
        pairs = cKDTree(X).query_pairs(min_dist, output_type="ndarray")
        if len(pairs):
            pairs = pairs[(pairs[:, 0] < n) | (pairs[:, 1] < n)]
        if not len(pairs):
            return u
        idx = np.unique(np.maximum(ids[pairs[:, 0]], ids[pairs[:, 1]]))
        u[idx] = rng.random((len(idx), 3))
    raise RuntimeError("random placement with minimum distance failed")


def random_ionic(n_atoms: int, rng: np.random.Generator, *, density: float = 0.045,
                 min_dist: float = 1.5, triclinic: bool = False, max_tilt_deg: float = 20.0,
                 n_species: int = 2, chi_std_atom: float = 0.3) -> Structure:
    """Random cell at ``density`` atoms/A^3, atoms at least ``min_dist`` apart."""
    V = n_atoms / density
    ratios = rng.uniform(0.75, 1.33, size=3)
    ratios = ratios / np.prod(ratios) ** (1.0 / 3.0)
    lengths = ratios * V ** (1.0 / 3.0)
    cell = sheared_cell(lengths, max_tilt_deg if triclinic else 0.0, rng)
    frac = _place_with_min_distance(n_atoms, cell, min_dist, rng)
    species = rng.integers(0, n_species, size=n_atoms).astype(np.int32)
    chi_s = rng.normal(0.0, 1.5, size=n_species)
    J_s = rng.uniform(1.0, 3.0, size=n_species)
    sigma_s = rng.uniform(0.8, 2.0, size=n_species)
    chi = chi_s[species] + rng.normal(0.0, chi_std_atom, size=n_atoms)
    q_tot = float(rng.integers(-1, 2))
    return Structure(cell, frac @ cell, species, chi, J_s[species].copy(), sigma_s, q_tot)


# --------------------------------------------------------------------------- workloads

ROCKSALT_A = 5.64


def workload(cfg_id: int, struct_id: int = 0, *, scale: int | None = None) -> Structure:
    """The synthetic cell of workload ``cfg_id`` (1, 2, 3 or 5); ``scale`` overrides n per edge."""
    rng = rng_for(cfg_id, struct_id)
    if cfg_id == 1:
        return rocksalt(scale or 3, ROCKSALT_A, 0.1, rng)
    if cfg_id == 2:
        return rocksalt(scale or 12, ROCKSALT_A, 0.15, rng)
    if cfg_id == 3:
        return rocksalt(scale or 24, ROCKSALT_A, 0.15, rng, vacancy_frac=0.05, shear_deg=10.0)
    if cfg_id == 5:
        return rocksalt(scale or 50, ROCKSALT_A, 0.2, rng, vacancy_frac=0.02)
    raise ValueError(f"workload {cfg_id} is not a single cell")


def batch_workload(n_struct: int = 512, cfg_id: int = 4, n_min: int = 64, n_max: int = 4096,
                   first: int = 0) -> list:
    """Uneven training-set batch: atom counts log-uniform in [n_min, n_max]."""
    out = []
    for s in range(first, first + n_struct):
        rng = rng_for(cfg_id, s)
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        out.append(random_ionic(n, rng, triclinic=bool(rng.random() < 0.5),
                                n_species=int(rng.integers(2, 5))))
    return out


def training_structures(n_struct: int, cfg_id: int = 6, first: int = 0, n_min: int = 64,
                        n_max: int = 4096) -> list:
    """Rock-salt-recipe training cells of n1 x n2 x n3 conventional cells (jitter 0.2, 2% vacancies)."""
    out = []
    for s in range(first, first + n_struct):
        rng = rng_for(cfg_id, s)
        target = math.exp(rng.uniform(math.log(n_min), math.log(n_max))) / 8.0
        n1 = max(1, int(round(target ** (1 / 3) * rng.uniform(0.8, 1.25))))
        n2 = max(1, int(round(math.sqrt(target / n1) * rng.uniform(0.8, 1.25))))
        n3 = max(1, int(round(target / (n1 * n2))))
        out.append(rocksalt((n1, n2, n3), ROCKSALT_A, 0.2, rng, vacancy_frac=0.02))
    return out
