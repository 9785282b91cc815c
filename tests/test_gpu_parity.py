"""GPU parity of the CUDA path against the FP64 CPU oracle (through the C ABI).

Tolerances: charges within 1e-5 e max-abs and energies within 1e-6 relative of
the dense oracle; matvec relative RMS within the plan's ewald_tol.
"""
import math

import numpy as np
import pytest

from oracle import qeq_oracle as O
from paper_2607_17978_b300 import synth

KE = synth.COULOMB_K_EV_A
pytestmark = pytest.mark.gpu


def _plan(structs, **kw):
    from paper_2607_17978_b300 import build, qeq
    build.build()
    return qeq.plan_for_structures(structs, **kw)


def _oracle(st):
    A = O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=KE)
    q, mu = O.solve_bordered(A, st.J, st.chi, st.q_tot)
    E, Ee = O.energies(A, st.J, st.chi, q)
    return A, q, mu, E, Ee


@pytest.fixture(scope="module")
def cfg1():
    st = synth.workload(1)
    return st, _oracle(st)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_matvec_parity_config1(cfg1, precision):
    from paper_2607_17978_b300 import qeq
    st, (A, q, *_r) = cfg1
    tol = 1e-7
    plan = _plan([st], precision=precision, ewald_tol=tol, r_cut=9.0)
    pos, spc, chi, J, _ = qeq.pack([st])
    rng = np.random.default_rng(0)
    for x in (rng.normal(size=st.n), q):
        y = plan.matvec(pos, spc, x, J=J).cpu().numpy()
        ref = A @ x + st.J * x
        err = np.sqrt(np.mean((y - ref) ** 2)) / np.sqrt(np.mean(ref ** 2))
        # FP32 mesh arithmetic: single-precision rounding of potentials much larger than (A q)_i
        assert err < (tol if precision == "fp64" else 5e-6), err
    y64 = plan.matvec(pos, spc, q, J=J, fp64=True).cpu().numpy()
    ref = A @ q + st.J * q
    assert np.sqrt(np.mean((y64 - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)) < tol


def test_double_float_checks_in_a_mixed_solve():
    """A mixed-precision solve whose final checks run on double-float FFT passes (forced) gives
    the charges of the dense oracle to 1e-5 e and the same charges as with FP64 checks to the
    certification's resolution (both certify max|P r| below the same threshold)."""
    from paper_2607_17978_b300 import qeq
    st = synth.rocksalt(5, 5.64, 0.15, synth.rng_for(73, 0), vacancy_frac=0.05, shear_deg=10.0)
    A = O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=synth.COULOMB_K_EV_A)
    q_ref, _ = O.solve_bordered(A, st.J, st.chi, st.q_tot)
    pos, spc, chi, J, qt = qeq.pack([st])
    qs = {}
    for check in ("dd", "fp64"):
        plan = _plan([st], precision="mixed", ewald_tol=1e-7, r_cut=9.0, check=check, preconditioner="fourier")
        res = plan.solve(pos, spc, chi, J, qt)
        qs[check] = res.q.cpu().numpy()
        assert res.info[0]["status"] == 0
        assert np.abs(qs[check] - q_ref).max() < 1e-5, (check, np.abs(qs[check] - q_ref).max())
        plan.close()
    assert np.abs(qs["dd"] - qs["fp64"]).max() < 2e-6


def test_double_float_check_matvec_equals_fp64():
    """The FP64-accurate matvec of a mixed-precision plan (final checks, energies) with its FFT
    passes in double-float arithmetic (forced here; by default on meshes of 2^21 points or more
    with at most two species) equals the FP64 plan's matvec on the same mesh to ~1e-13 of the
    potentials' size (FP64 rounding is ~1e-16, double-float ~2^-44 per operation): a rock-salt
    cell, a sheared cell with vacancies, and a batch with 2-4 species (the general reciprocal
    multiply)."""
    from paper_2607_17978_b300 import qeq
    cases = [[synth.workload(1)],
             [synth.rocksalt(5, 5.64, 0.15, synth.rng_for(71, 0), vacancy_frac=0.05, shear_deg=10.0)],
             synth.batch_workload(3, cfg_id=72, n_min=100, n_max=600)]
    for structs in cases:
        p_mix = _plan(structs, precision="mixed", ewald_tol=1e-6, r_cut=8.0, check="dd")
        p_64 = _plan(structs, precision="fp64", ewald_tol=1e-6, r_cut=8.0)
        assert [p_mix.query(i)["mesh"] for i in range(len(structs))] == \
            [p_64.query(i)["mesh"] for i in range(len(structs))]
        pos, spc, chi, J, _ = qeq.pack(structs)
        x = np.random.default_rng(5).normal(size=len(spc))
        y_dd = p_mix.matvec(pos, spc, x, J=J, fp64=True).cpu().numpy()
        y_64 = p_64.matvec(pos, spc, x, J=J).cpu().numpy()
        scale = np.sqrt(np.mean(y_64 ** 2))
        err = np.abs(y_dd - y_64).max() / scale
        print(f"{len(structs)} structure(s), {len(spc)} atoms: max |y_dd - y_fp64| / rms = {err:.2e}")
        assert err < 1e-11, err
        p_mix.close()
        p_64.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_parity_config1(cfg1, precision):
    from paper_2607_17978_b300 import qeq
    st, (A, q, mu, E, Ee) = cfg1
    plan = _plan([st], precision=precision, ewald_tol=1e-7, r_cut=9.0)
    pos, spc, chi, J, qt = qeq.pack([st])
    res = plan.solve(pos, spc, chi, J, qt)
    qg = res.q.cpu().numpy()
    assert np.abs(qg - q).max() < 1e-5
    assert abs(qg.sum() - st.q_tot) < 1e-10
    assert abs(res.mu.cpu().numpy()[0] - mu) < 1e-5 * max(1.0, abs(mu))
    Eg, Eeg = plan.energy(pos, spc, chi, J, res.q)
    assert abs(Eg.item() - E) < 1e-6 * abs(E)
    assert abs(Eeg.item() - Ee) < 1e-6 * abs(Ee)
    assert res.info[0]["status"] == 0 and res.info[0]["iterations"] > 0


def _small_structs():
    rng = synth.rng_for(40, 0)
    out = [synth.rocksalt(3, 5.64, 0.15, rng, vacancy_frac=0.05, shear_deg=10.0)]      # triclinic, vacancies
    out.append(synth.rocksalt((2, 3, 2), 5.64, 0.2, synth.rng_for(40, 1)))              # ragged mesh bins
    for s in range(3):
        out.append(synth.batch_workload(1, cfg_id=41, n_min=64, n_max=600, first=s)[0])
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_solve_parity_uneven_structures(precision):
    from paper_2607_17978_b300 import qeq
    structs = _small_structs()
    plan = _plan(structs, precision=precision)
    pos, spc, chi, J, qt = qeq.pack(structs)
    res = plan.solve(pos, spc, chi, J, qt)
    qg = res.q.cpu().numpy()
    off = np.concatenate([[0], np.cumsum([s.n for s in structs])])
    for i, st in enumerate(structs):
        _, q, mu, E, _ = _oracle(st)
        assert np.abs(qg[off[i]:off[i + 1]] - q).max() < 1e-5, (i, plan.query(i))
        assert abs(qg[off[i]:off[i + 1]].sum() - st.q_tot) < 1e-9
    # batched == one structure at a time
    for i, st in enumerate(structs[:3]):
        p1 = _plan([st], precision=precision)
        a, b, c, d, e = qeq.pack([st])
        r1 = p1.solve(a, b, c, d, e).q.cpu().numpy()
        assert np.abs(r1 - qg[off[i]:off[i + 1]]).max() < 2e-6


def test_reduced_config2_dense():
    from paper_2607_17978_b300 import qeq
    st = synth.rocksalt(5, 5.64, 0.15, synth.rng_for(2, 7))
    _, q, mu, E, _ = _oracle(st)
    for precision in ("fp64", "mixed"):
        plan = _plan([st], precision=precision, r_cut=8.0)
        pos, spc, chi, J, qt = qeq.pack([st])
        res = plan.solve(pos, spc, chi, J, qt)
        assert np.abs(res.q.cpu().numpy() - q).max() < 1e-5


def test_edge_cases_single_atom_two_atoms_and_charged():
    from paper_2607_17978_b300 import qeq
    one = synth.Structure(np.eye(3) * 9.0, np.array([[1.0, 2.0, 3.0]]), np.array([0], np.int32),
                          np.array([-0.4]), np.array([1.7]), np.array([1.2]), 1.0)
    two = synth.Structure(np.diag([8.0, 9.0, 10.0]), np.array([[0.5, 0.5, 0.5], [3.0, 4.0, 5.5]]),
                          np.array([0, 1], np.int32), np.array([-1.1, 0.8]), np.array([2.0, 1.5]),
                          np.array([1.0, 1.8]), 0.4)
    for st in (one, two):
        _, q, mu, *_ = _oracle(st)
        plan = _plan([st])
        res = plan.solve(*qeq.pack([st]))
        assert np.abs(res.q.cpu().numpy() - q).max() < 1e-6
        assert abs(res.mu.cpu().numpy()[0] - mu) < 1e-5


def test_user_warm_start_and_repeatability(cfg1):
    from paper_2607_17978_b300 import qeq
    st, (A, q, *_r) = cfg1
    plan = _plan([st], ewald_tol=1e-7, r_cut=9.0)
    pos, spc, chi, J, qt = qeq.pack([st])
    r1 = plan.solve(pos, spc, chi, J, qt)
    r2 = plan.solve(pos, spc, chi, J, qt)
    # no floating-point atomics and fixed reduction orders: repeated solves are bitwise equal
    assert np.array_equal(r1.q.cpu().numpy(), r2.q.cpu().numpy())
    assert r1.info[0]["iterations"] == r2.info[0]["iterations"]
    r3 = plan.solve(pos, spc, chi, J, qt, q0=r1.q)
    assert r3.info[0]["iterations"] <= 4
    assert np.abs(r3.q.cpu().numpy() - q).max() < 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_preconditioned_solves_are_bitwise_repeatable(precision):
    """The Fourier preconditioner's coarse spread adds integers (fixed-point contributions, 32-bit
    tile sums, 64-bit mesh sums), whose order does not matter, so repeated preconditioned solves
    (and batches of them) give identical charges and iteration counts."""
    from paper_2607_17978_b300 import qeq
    structs = [synth.rocksalt(6, 5.64, 0.2, synth.rng_for(5, 6), vacancy_frac=0.02)]
    structs += synth.batch_workload(4, n_min=64, n_max=800)
    plan = _plan(structs, precision=precision, preconditioner="fourier")
    args = qeq.pack(structs)
    r1 = plan.solve(*args)
    r2 = plan.solve(*args)
    assert np.array_equal(r1.q.cpu().numpy(), r2.q.cpu().numpy())
    assert [i["iterations"] for i in r1.info] == [i["iterations"] for i in r2.info]


@pytest.mark.parametrize("precision,pre", [("fp64", "jacobi"), ("fp64", "fourier"), ("mixed", "jacobi"),
                                           ("mixed", "fourier")])
def test_tight_charge_tolerances_converge_or_report(cfg1, precision, pre):
    """charge_tol down to 1e-9 e: the constraint holds whatever the status; FP64 plans converge
    to the oracle charges within the mesh operator's own error (ewald_tol 1e-7: ~3e-8 e); mixed
    plans either do the same or report QEQ_ERR_NOCONV, never a converged status with charges
    that have left the constraint plane."""
    from paper_2607_17978_b300 import qeq
    st, (A, q_ref, *_r) = cfg1
    pos, spc, chi, J, qt = qeq.pack([st])
    for ct in (1e-7, 1e-8, 1e-9):
        plan = _plan([st], precision=precision, preconditioner=pre, ewald_tol=1e-7, r_cut=9.0, charge_tol=ct)
        res = plan.solve(pos, spc, chi, J, qt, raise_on_noconv=False)
        q = res.q.cpu().numpy()
        info = res.info[0]
        assert abs(q.sum() - st.q_tot) < 1e-9, (ct, q.sum())
        if precision == "fp64":
            assert info["status"] == 0, (ct, info)
        if info["status"] == 0:
            assert np.abs(q - q_ref).max() < 2e-7 + 10 * ct, (ct, np.abs(q - q_ref).max(), info)
            # the reported l2 residual is the projected one, not lost to cancellation
            assert info["residual_l2"] > 0.0
        else:
            assert info["status"] == qeq.QEQ_ERR_NOCONV, info
        plan.close()


@pytest.mark.parametrize("precision,pre", [("fp64", "jacobi"), ("fp64", "fourier"), ("mixed", "jacobi"),
                                           ("mixed", "fourier")])
def test_two_rhs_solver_matches_the_oracle(precision, pre):
    """The two-RHS formulation (plain PCG on A t = 1 and A s = -chi, q = s + mu' t) on an
    uneven batch with charged cells: charges within 1e-5 e of the dense oracle, the constraint
    exact, mu from the combined charges, the same charges as the projected solver."""
    from paper_2607_17978_b300 import qeq
    structs = _small_structs()
    plan = _plan(structs, precision=precision, preconditioner=pre, solver="two_rhs")
    args = qeq.pack(structs)
    res = plan.solve(*args)
    qg = res.q.cpu().numpy()
    mug = res.mu.cpu().numpy()
    off = np.concatenate([[0], np.cumsum([s.n for s in structs])])
    for i, st in enumerate(structs):
        _, q, mu, *_r = _oracle(st)
        sl = slice(off[i], off[i + 1])
        assert np.abs(qg[sl] - q).max() < 1e-5, (i, np.abs(qg[sl] - q).max(), res.info[i])
        assert abs(qg[sl].sum() - st.q_tot) < 1e-9
        assert abs(mug[i] - mu) < 1e-4 * max(1.0, abs(mu))
        assert res.info[i]["status"] == 0 and res.info[i]["iterations"] > 0
    qp = _plan(structs, precision=precision, preconditioner=pre).solve(*args).q.cpu().numpy()
    assert np.abs(qg - qp).max() < 2e-5
    with pytest.raises(qeq.QEqError) as e:
        plan.solve(*args, q0=qp)  # the two-RHS solver starts cold
    assert e.value.status == qeq.QEQ_ERR_INVALID


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sqnm_solver_matches_the_oracle(precision):
    """The stabilised quasi-Newton minimiser (QEQ_FLAG_SQNM) on an uneven batch with charged
    cells: charges within 1e-5 e of the dense oracle, the constraint exact, the same charges as
    the CG; repeated solves bitwise equal (fixed-order sums, deterministic subspace algebra)."""
    from paper_2607_17978_b300 import qeq
    structs = _small_structs()
    plan = _plan(structs, precision=precision, solver="sqnm")
    args = qeq.pack(structs)
    res = plan.solve(*args)
    qg = res.q.cpu().numpy()
    mug = res.mu.cpu().numpy()
    off = np.concatenate([[0], np.cumsum([s.n for s in structs])])
    for i, st in enumerate(structs):
        _, q, mu, *_r = _oracle(st)
        sl = slice(off[i], off[i + 1])
        print(f"SQNM {precision} structure {i} ({st.n} atoms): {res.info[i]['iterations']} steps, "
              f"max|dq| {np.abs(qg[sl] - q).max():.2e}")
        assert np.abs(qg[sl] - q).max() < 1e-5, (i, np.abs(qg[sl] - q).max(), res.info[i])
        assert abs(qg[sl].sum() - st.q_tot) < 1e-9
        assert abs(mug[i] - mu) < 1e-4 * max(1.0, abs(mu))
        assert res.info[i]["status"] == 0 and res.info[i]["iterations"] > 0
    res2 = plan.solve(*args)
    assert np.array_equal(qg, res2.q.cpu().numpy())
    qp = _plan(structs, precision=precision).solve(*args).q.cpu().numpy()
    assert np.abs(qg - qp).max() < 2e-5


def test_translation_invariance_within_mesh_error(cfg1):
    from paper_2607_17978_b300 import qeq
    st, (A, q, *_r) = cfg1
    t = st.copy()
    t.pos = t.pos + np.array([0.37, -1.21, 2.93])
    plan = _plan([t], ewald_tol=1e-7, r_cut=9.0)
    res = plan.solve(*qeq.pack([t]))
    assert np.abs(res.q.cpu().numpy() - q).max() < 1e-5


def test_invalid_inputs_are_reported():
    from paper_2607_17978_b300 import qeq
    st = synth.workload(1)
    plan = _plan([st])
    pos, spc, chi, J, qt = qeq.pack([st])
    Jb = J.copy()
    Jb[5] = -1.0
    with pytest.raises(qeq.QEqError) as e:
        plan.solve(pos, spc, chi, Jb, qt)
    assert e.value.status == qeq.QEQ_ERR_NOT_PD
    sb = spc.copy()
    sb[3] = 7
    with pytest.raises(qeq.QEqError) as e:
        plan.solve(pos, sb, chi, J, qt)
    assert e.value.status == qeq.QEQ_ERR_INVALID
    pb = pos.copy()
    pb[2, 1] = np.nan
    with pytest.raises(qeq.QEqError) as e:
        plan.solve(pb, spc, chi, J, qt)
    assert e.value.status == qeq.QEQ_ERR_INVALID
    # the plan still works afterwards
    res = plan.solve(pos, spc, chi, J, qt)
    assert res.info[0]["status"] == 0


def test_iteration_cap_reports_noconv():
    from paper_2607_17978_b300 import qeq
    st = synth.workload(1)
    plan = _plan([st], max_iter=2)
    res = plan.solve(*qeq.pack([st]), raise_on_noconv=False)
    assert res.info[0]["status"] == qeq.QEQ_ERR_NOCONV


def test_config4_batch_subset_against_dense_oracle():
    """Uneven training-set batch (config-4 recipe, sizes capped for the dense oracle), one batched solve."""
    from paper_2607_17978_b300 import qeq
    structs = synth.batch_workload(20, n_min=64, n_max=1024)
    for precision in ("mixed", "fp64"):
        plan = _plan(structs, precision=precision)
        pos, spc, chi, J, qt = qeq.pack(structs)
        res = plan.solve(pos, spc, chi, J, qt)
        qg = res.q.cpu().numpy()
        mu = res.mu.cpu().numpy()
        off = np.concatenate([[0], np.cumsum([s.n for s in structs])])
        for i, st in enumerate(structs):
            _, q, mu_ref, _, _ = _oracle(st)
            assert np.abs(qg[off[i]:off[i + 1]] - q).max() < 1e-5, (precision, i)
            assert abs(qg[off[i]:off[i + 1]].sum() - st.q_tot) < 1e-9
            assert abs(mu[i] - mu_ref) < 1e-4
            assert res.info[i]["status"] == 0
        plan.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fourier_preconditioner_same_charges_fewer_iterations(precision):
    from paper_2607_17978_b300 import qeq
    st = synth.rocksalt(6, 5.64, 0.2, synth.rng_for(5, 6), vacancy_frac=0.02)
    _, q, mu, E, _ = _oracle(st)
    args = qeq.pack([st])
    pj = _plan([st], precision=precision)
    pf = _plan([st], precision=precision, preconditioner="fourier")
    rj = pj.solve(*args)
    rf = pf.solve(*args)
    assert np.abs(rf.q.cpu().numpy() - q).max() < 1e-5
    assert abs(rf.mu.cpu().numpy()[0] - mu) < 1e-5
    assert rf.info[0]["iterations"] < 0.6 * rj.info[0]["iterations"], (rf.info, rj.info)
    # batches and warm starts go through the same preconditioned iteration
    structs = synth.batch_workload(6, n_min=64, n_max=800) + [st]
    pb = _plan(structs, precision=precision, preconditioner="fourier")
    rb = pb.solve(*qeq.pack(structs))
    qb = rb.q.cpu().numpy()
    off = np.concatenate([[0], np.cumsum([s.n for s in structs])])
    for i, s in enumerate(structs):
        _, qi, *_ = _oracle(s)
        assert np.abs(qb[off[i]:off[i + 1]] - qi).max() < 1e-5, i
    r2 = pf.solve(*args, q0=rf.q)
    assert r2.info[0]["iterations"] <= 4


def test_mixed_final_check_bounds_the_fp64_residual():
    """After an FP64 check, the mixed path certifies the final charges from the FP64
    residual of that check plus the FP32 product of the later change, with an error
    bound. The true FP64 residual must still meet the check's threshold, and the
    charges must agree with the plain FP64 solve."""
    import torch
    from paper_2607_17978_b300 import qeq
    st = synth.workload(2)
    args = qeq.pack([st])
    pm = _plan([st], precision="mixed", preconditioner="fourier", ewald_tol=1e-6, r_cut=8.0)
    pd = _plan([st], precision="fp64", ewald_tol=1e-6, r_cut=8.0)
    rm = pm.solve(*args)
    rd = pd.solve(*args)
    assert rm.info[0]["restarts"] >= 1  # the change-based check was the one that accepted
    q = rm.q
    y = pd.matvec(torch.tensor(st.pos, device=q.device), torch.tensor(st.species, device=q.device), q,
                  J=torch.tensor(st.J, device=q.device), fp64=True).cpu().numpy()
    r = -st.chi - y
    pinf = np.abs(r - r.mean()).max()
    assert pinf <= 0.5 * 1e-5 * st.J.min(), pinf
    assert np.abs(q.cpu().numpy() - rd.q.cpu().numpy()).max() < 1e-5


def test_bounded_wait_that_runs_out_returns_timeout_and_the_gpu_keeps_working():
    """QEQ_FLAG_TEST_STALL makes the first tile of every x FFT pass announce 16 more bytes on
    its copy barrier than its bulk copies deliver: that wait runs out after its bound (0.5 s
    of the GPU's global timer), the kernel flags it and returns, the PCG stops, and the solve
    reports QEQ_ERR_TIMEOUT.  No fault: the copies themselves complete, and a new plan on the
    same GPU solves correctly afterwards."""
    from paper_2607_17978_b300 import qeq
    st = synth.workload(1)
    args = qeq.pack([st])
    bad = _plan([st], ewald_tol=1e-7, r_cut=9.0, test_stall=True)
    with pytest.raises(qeq.QEqError) as e:
        bad.solve(*args)
    assert e.value.status == qeq.QEQ_ERR_TIMEOUT
    bad.close()
    good = _plan([st], ewald_tol=1e-7, r_cut=9.0)
    res = good.solve(*args)
    A = O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=KE)
    q_ref, _ = O.solve_bordered(A, st.J, st.chi, st.q_tot)
    assert res.info[0]["status"] == 0
    assert np.abs(res.q.cpu().numpy() - q_ref).max() < 1e-5
    good.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_device_paced_solve_graph_equals_host_loop(precision):
    """The solve graph (WHILE over rounds, WHILE over 4-iteration blocks, IF between the
    change-based and the FP64 final check, conditions set on the device) runs the same
    kernels in the same order as the host-paced loop: identical charges, iteration and
    restart counts, for a batch of uneven structures."""
    from paper_2607_17978_b300 import qeq
    structs = synth.batch_workload(5, n_min=64, n_max=700) + [synth.rocksalt(5, 5.64, 0.2, synth.rng_for(5, 9))]
    if precision == "mixed":  # a cell whose mixed solve restarts, so both check branches run
        structs = [synth.workload(2)] + structs[:2]
    args = qeq.pack(structs)
    pg = _plan(structs, precision=precision, preconditioner="fourier", ewald_tol=1e-6, r_cut=8.0)
    ph = _plan(structs, precision=precision, preconditioner="fourier", ewald_tol=1e-6, r_cut=8.0, graph=False)
    rg = pg.solve(*args)
    rh = ph.solve(*args)
    assert np.array_equal(rg.q.cpu().numpy(), rh.q.cpu().numpy())
    for a, b in zip(rg.info, rh.info):
        assert (a["iterations"], a["restarts"], a["status"]) == (b["iterations"], b["restarts"], b["status"])
    assert any(i["restarts"] >= 1 for i in rg.info) or precision == "fp64"
    # a second solve on the same instantiated graph
    rg2 = pg.solve(*args)
    assert np.array_equal(rg.q.cpu().numpy(), rg2.q.cpu().numpy())
