"""The seeded synthetic inputs follow the stated recipes: atom counts of the five workloads, vacancy
fractions, shear, species tables, the batch's size range, density, species counts, total charges and
minimum atom distance (brute force over periodic images), and seeding (the same draw twice)."""
import itertools
import math

import numpy as np

from paper_2607_17978_b300 import synth


def test_single_cell_workloads():
    counts = {1: 216, 2: 13824, 3: 105063, 5: 980000}
    for w, n in counts.items():
        st = synth.workload(w)
        assert st.n == n and st.n_species == 2 and st.q_tot == 0.0
        assert np.array_equal(st.sigma_s, [1.0, 1.8]) and set(np.unique(st.J)) == {2.0, 1.5}
        A = st.chi[st.species == 0].mean()
        B = st.chi[st.species == 1].mean()
        assert abs(A + 2.0) < 0.1 and abs(B - 2.0) < 0.1
    full = {3: 24 ** 3 * 8, 5: 50 ** 3 * 8}
    assert counts[3] == full[3] - math.floor(0.05 * full[3]) and counts[5] == full[5] - math.floor(0.02 * full[5])
    h = synth.workload(3).cell                            # sheared: tilts of at most 10 degrees
    assert np.allclose(np.tril(h, -1), 0) and np.count_nonzero(np.triu(h, 1)) == 3
    L = np.diag(h)
    tilts = np.degrees(np.arctan(np.array([h[0, 1] / L[1], h[0, 2] / L[2], h[1, 2] / L[2]])))
    assert np.all(np.abs(tilts) <= 10.0)
    assert np.allclose(synth.workload(2).cell, np.eye(3) * 12 * synth.ROCKSALT_A)


def test_seeding_is_reproducible():
    a, b = synth.workload(3), synth.workload(3)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.chi, b.chi) and np.array_equal(a.species, b.species)
    c = synth.workload(3, struct_id=1)
    assert not np.array_equal(a.pos[:100], c.pos[:100])


def _min_image_distance(st):
    shifts = np.array(list(itertools.product([-1, 0, 1], repeat=3))) @ st.cell
    d = st.pos[None, :, None, :] - st.pos[:, None, None, :] + shifts[None, None, :, :]
    r = np.linalg.norm(d, axis=-1)
    r[np.arange(st.n), np.arange(st.n), 13] = np.inf       # the atom itself (zero shift)
    return r.min()


def test_batch_recipe():
    batch = synth.batch_workload()
    assert len(batch) == 512 and sum(s.n for s in batch) == 519537
    for s in batch:
        assert 64 <= s.n <= 4096 and 2 <= s.n_species <= 4 and s.q_tot in (-1.0, 0.0, 1.0)
        assert abs(s.n / abs(np.linalg.det(s.cell)) - 0.045) < 1e-9
        assert np.all((s.sigma_s >= 0.8) & (s.sigma_s <= 2.0)) and np.all((s.J >= 1.0) & (s.J <= 3.0))
    small = [s for s in batch if s.n <= 300][:8]
    assert small
    for s in small:
        assert _min_image_distance(s) >= 1.5
