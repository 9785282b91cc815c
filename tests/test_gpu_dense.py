"""GPU parity of the 4G charge-training path (qeq_dense_*, Sec. "4G-HDNNP Charge Training")
against the FP64 CPU oracle, through the C ABI.

Tolerances: the GPU assembles E by its own Ewald split truncated at ewald_tol = 1e-12 and
inverts in FP64, so E, A'^{-1}, the charges and the gradients agree with the oracle to
~1e-10 relative (rounding of O(n) sums and of the inverse's conditioning); the tests use
1e-9 relative to the largest entry of each compared quantity.
"""
import numpy as np
import pytest

from oracle import qeq_oracle as O
from paper_2607_17978_b300 import synth

KE = synth.COULOMB_K_EV_A
TOL = 1e-9
pytestmark = pytest.mark.gpu


def _dense(structs, **kw):
    from paper_2607_17978_b300 import build, qeq
    build.build()
    return qeq.dense_for_structures(structs, **kw)


def _batch():
    """Training-like batch: rock-salt cells of 64-512 atoms (unsheared, jittered, vacancies),
    a sheared cell, ragged tiles (n not a multiple of 32), random ionic cells with 2-4 species
    and charged totals, and a single atom."""
    out = synth.training_structures(4, cfg_id=62, n_min=64, n_max=512)
    out.append(synth.rocksalt(2, 5.64, 0.15, synth.rng_for(63, 0), vacancy_frac=0.05, shear_deg=10.0))
    for s in range(3):
        out.append(synth.batch_workload(1, cfg_id=64, n_min=40, n_max=300, first=s)[0])
    out.append(synth.Structure(np.eye(3) * 9.0, np.array([[1.0, 2.0, 3.0]]), np.array([0], np.int32),
                               np.array([-0.4]), np.array([1.7]), np.array([1.2]), 1.0))
    return out


def _rel(a, b):
    """Largest difference relative to the largest reference entry; a reference that is zero in
    exact arithmetic (a one-atom structure's charge gradient) is compared absolutely at 1e-15."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-6))


@pytest.fixture(scope="module")
def batch_and_oracle():
    structs = _batch()
    refs = [O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=KE) for st in structs]
    return structs, refs


def test_dense_assembly_matches_the_oracle_matrix(batch_and_oracle):
    from paper_2607_17978_b300 import qeq
    structs, refs = batch_and_oracle
    d = _dense(structs)
    pos, spc, *_ = qeq.pack(structs)
    d.assemble(pos, spc)
    for i, (st, A) in enumerate(zip(structs, refs)):
        E = d.matrix(i, 0).cpu().numpy()
        err = _rel(E, A)
        print(f"E of structure {i} ({st.n} atoms, {st.n_species} species): rel max {err:.2e}, "
              f"omega {d.query(i)['omega']:.3f} A, {d.query(i)['n_g']} G vectors")
        assert err < TOL, (i, err)
        assert np.array_equal(E, E.T) or np.abs(E - E.T).max() < 1e-14 * np.abs(E).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_dense_charges_gradients_and_inverse(batch_and_oracle, precision):
    """Charges, multipliers and the backward pass against the oracle at 1e-9 in both modes (the
    mixed mode's FP32 inverse is refined in FP64); the cached inverse itself at 1e-9 (FP64) or
    at FP32 accuracy (1e-4 relative to its largest entry, mixed)."""
    from paper_2607_17978_b300 import qeq
    structs, refs = batch_and_oracle
    d = _dense(structs, precision=precision)
    pos, spc, chi, J, qt = qeq.pack(structs)
    d.assemble(pos, spc)
    rng = np.random.default_rng(7)
    J2 = J * rng.uniform(0.8, 1.25, size=len(J))  # "learned" hardness: re-invert
    for Juse in (J, J2):
        d.invert(Juse)
        q, mu = d.charges(chi, qt)
        q, mu = q.cpu().numpy(), mu.cpu().numpy()
        gq = rng.normal(size=len(q))
        gchi, gJ = [x.cpu().numpy() for x in d.backward(q, gq)]
        off = np.concatenate([[0], np.cumsum([s.n for s in structs])])
        for i, (st, A) in enumerate(zip(structs, refs)):
            sl = slice(off[i], off[i + 1])
            Kinv = O.bordered_inverse(A, Juse[sl])
            qr, mur = O.charges_from_inverse(Kinv, st.chi, st.q_tot)
            gcr, gJr = O.charges_backward(Kinv, qr, gq[sl])
            assert _rel(q[sl], qr) < TOL, (i, _rel(q[sl], qr))
            assert abs(mu[i] - mur) < TOL * max(1.0, abs(mur))
            assert abs(q[sl].sum() - st.q_tot) < 1e-10
            assert _rel(gchi[sl], gcr) < TOL, (i, _rel(gchi[sl], gcr))
            assert _rel(gJ[sl], gJr) < TOL, (i, _rel(gJ[sl], gJr))
            K = d.matrix(i, 1).cpu().numpy()
            assert _rel(K, Kinv) < (TOL if precision == "fp64" else 1e-4), (i, _rel(K, Kinv))


def test_dense_matches_the_iterative_solver_and_is_repeatable():
    """The cached-inverse charges equal the plane-wave PCG solve of the same cell (to the
    PCG's 1e-5 e), and repeated calls are bitwise equal (fixed summation orders)."""
    from paper_2607_17978_b300 import qeq
    st = synth.workload(1)
    d = _dense([st])
    pos, spc, chi, J, qt = qeq.pack([st])
    d.assemble(pos, spc)
    d.invert(J)
    q1 = d.charges(chi, qt)[0].cpu().numpy()
    d.assemble(pos, spc)
    d.invert(J)
    q2 = d.charges(chi, qt)[0].cpu().numpy()
    assert np.array_equal(q1, q2)
    plan = qeq.plan_for_structures([st], ewald_tol=1e-7, r_cut=9.0)
    qp = plan.solve(pos, spc, chi, J, qt).q.cpu().numpy()
    assert np.abs(q1 - qp).max() < 1e-5


def test_dense_errors_are_reported():
    from paper_2607_17978_b300 import qeq
    st = synth.workload(1)
    d = _dense([st])
    pos, spc, chi, J, qt = qeq.pack([st])
    with pytest.raises(qeq.QEqError) as e:
        d.invert(J)  # not assembled yet
    assert e.value.status == qeq.QEQ_ERR_INVALID
    sb = spc.copy()
    sb[2] = 9
    with pytest.raises(qeq.QEqError) as e:
        d.assemble(pos, sb)
    assert e.value.status == qeq.QEQ_ERR_INVALID
    d.assemble(pos, spc)
    Jb = J.copy()
    Jb[:] = -50.0  # E + diag J indefinite
    with pytest.raises(qeq.QEqError) as e:
        d.invert(Jb)
    assert e.value.status == qeq.QEQ_ERR_NOT_PD
    d.invert(J)  # recovers
    q = d.charges(chi, qt)[0].cpu().numpy()
    assert abs(q.sum()) < 1e-10
    big = synth.rocksalt(6, 5.64, 0.1, synth.rng_for(1, 3))  # 1728 atoms > QEQ_DENSE_MAX_ATOMS
    with pytest.raises(qeq.QEqError) as e:
        _dense([big])
    assert e.value.status == qeq.QEQ_ERR_CAPACITY
