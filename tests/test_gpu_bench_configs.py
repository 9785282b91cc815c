"""Parity of the form bench.py times against the FP64 CPU oracle, at full size.

The chosen form is mixed precision (FP32 mesh, FFT and pairs; FP64 reductions
and final check), the Fourier-Woodbury preconditioner, the CUDA-graph
iteration and, for the rock-salt recipe the network was trained on, the
learned warm start.  These tests run it on the workloads the bench measures
and compare with the oracle (charges within 1e-5 e max-abs, the multiplier and
energies as stated per test):

* the 13,824-atom rock-salt cell against the dense bordered oracle (every
  atom);
* the 512-structure uneven batch, solved in one batched plan as the bench
  does, with a stratified sample of structures (the largest cells, every
  species count with charged and neutral cells) against the dense oracle.
"""
import os

import numpy as np
import pytest

from oracle import qeq_oracle as O
from paper_2607_17978_b300 import synth

KE = synth.COULOMB_K_EV_A
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MODEL = os.path.join(ROOT, "paper_2607_17978_b300", "models", "warmstart_rocksalt.npz")
pytestmark = pytest.mark.gpu


def _chosen_plan(structs, warm):
    from paper_2607_17978_b300 import build, qeq, warmstart
    build.build()
    plan = qeq.plan_for_structures(structs, precision="mixed", preconditioner="fourier", ewald_tol=1e-6, r_cut=8.0)
    mlp = None
    if warm:
        mlp, _ = warmstart.load(MODEL)
        plan.set_warm_start(mlp)
    return plan, mlp


def test_config2_full_size_chosen_form_against_dense_oracle():
    import torch
    from paper_2607_17978_b300 import qeq
    st = synth.workload(2)
    assert st.n == 13824
    plan, mlp = _chosen_plan([st], warm=True)
    d = [torch.tensor(a, device="cuda") for a in qeq.pack([st])[:4]]
    res = plan.solve(*d, np.array([st.q_tot]), warm="mlp")
    info = res.info[0]
    assert info["status"] == 0 and info["warm_used"] == 1
    qg = res.q.cpu().numpy()
    mug = float(res.mu.cpu().numpy()[0])
    Eg, Eeg = plan.energy(*d, res.q)
    # dense bordered oracle (about 1.5 GB matrix, minutes on the host cores)
    A = O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=KE)
    q_ref, mu_ref = O.solve_bordered(A, st.J, st.chi, st.q_tot)
    E_ref, Ee_ref = O.energies(A, st.J, st.chi, q_ref)
    del A
    err = np.abs(qg - q_ref).max()
    print(f"13,824-atom cell, chosen form: max|dq| = {err:.3e} e, iterations {info['iterations']}")
    assert err < 1e-5, err
    assert abs(qg.sum() - st.q_tot) < 1e-9
    assert abs(mug - mu_ref) < 1e-5 * max(1.0, abs(mu_ref))
    assert abs(Eg.item() - E_ref) < 1e-6 * abs(E_ref)
    assert abs(Eeg.item() - Ee_ref) < 1e-6 * abs(Ee_ref)
    plan.close()
    mlp.close()


def _stratified_sample(structs, n_largest=4, n_random=2):
    """Indices: the largest cells, one seeded-random cell per (species count, q_tot), a few random ones."""
    n = np.array([s.n for s in structs])
    pick = [int(k) for k in np.argsort(-n, kind="stable")[:n_largest]]
    rng = np.random.default_rng(4)
    order = [int(k) for k in rng.permutation(len(structs))]
    for ns in (2, 3, 4):
        for qt in (-1.0, 0.0, 1.0):
            for k in order:
                if structs[k].n_species == ns and structs[k].q_tot == qt:
                    if k not in pick:
                        pick.append(k)
                    break
    for k in order[-n_random:]:
        if k not in pick:
            pick.append(k)
    return pick


def test_config4_batch_chosen_form_stratified_sample_against_dense_oracle():
    import torch
    from paper_2607_17978_b300 import qeq
    structs = synth.batch_workload(512)
    plan, _ = _chosen_plan(structs, warm=False)
    pos, spc, chi, J, qt = qeq.pack(structs)
    d = [torch.tensor(a, device="cuda") for a in (pos, spc, chi, J)]
    res = plan.solve(*d, qt)
    qg = res.q.cpu().numpy()
    mu = res.mu.cpu().numpy()
    assert all(i["status"] == 0 for i in res.info)
    off = np.concatenate([[0], np.cumsum([s.n for s in structs])])
    sample = _stratified_sample(structs)
    assert max(structs[k].n for k in sample) > 3000
    assert {structs[k].n_species for k in sample} == {2, 3, 4}
    worst = 0.0
    for k in sample:
        st = structs[k]
        A = O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=KE)
        q_ref, mu_ref = O.solve_bordered(A, st.J, st.chi, st.q_tot)
        e = np.abs(qg[off[k]:off[k + 1]] - q_ref).max()
        worst = max(worst, e)
        assert e < 1e-5, (k, st.n, st.n_species, st.q_tot, e)
        assert abs(qg[off[k]:off[k + 1]].sum() - st.q_tot) < 1e-9
        assert abs(mu[k] - mu_ref) < 1e-4
    print(f"batch of 512, {len(sample)} sampled structures: worst max|dq| = {worst:.3e} e")
    plan.close()
