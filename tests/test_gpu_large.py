"""Full-size cells where the dense oracle is infeasible: sampled-row parity.

For the 105,062-atom triclinic cell with vacancies and the 980,000-atom cell,
the form bench.py times (mixed precision, Fourier preconditioner, CUDA graph;
learned warm start on the 980,000-atom rock-salt cell) and the plain FP64 GPU
PCG are both checked:
  * the GPU FP64 matvec agrees with the oracle's FP64 Ewald matvec on sampled
    rows within the plan's ewald_tol (relative to the RMS of the sampled rows);
  * the chosen form's charges agree with the FP64 solve within 1e-5 e max-abs;
  * the oracle's residual of the chosen form's charges, (A q + chi)_i - mu on
    the sampled rows, is within the stopping tolerance plus the matvec error
    (and so is the FP64 solve's).
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


@pytest.mark.parametrize("cfg,n_rows,omega,warm", [(3, 300, 8.0, False), (5, 64, 11.0, True)])
def test_large_cell_sampled_rows(cfg, n_rows, omega, warm):
    import torch
    from paper_2607_17978_b300 import build, qeq, warmstart
    build.build()
    st = synth.workload(cfg)
    pos, spc, chi, J, qt = qeq.pack([st])
    dev = torch.device("cuda")
    d = [torch.tensor(a, device=dev) for a in (pos, spc, chi, J)]
    tol = 1e-6
    p64 = qeq.plan_for_structures([st], precision="fp64", ewald_tol=tol, r_cut=8.0)
    r64 = p64.solve(*d, qt)
    pmx = qeq.plan_for_structures([st], precision="mixed", preconditioner="fourier", ewald_tol=tol, r_cut=8.0)
    mlp = None
    if warm:
        mlp, _ = warmstart.load(MODEL)
        pmx.set_warm_start(mlp)
    rmx = pmx.solve(*d, qt, warm="mlp" if warm else None)
    q64 = r64.q.cpu().numpy()
    qmx = rmx.q.cpu().numpy()
    assert r64.info[0]["status"] == 0 and rmx.info[0]["status"] == 0
    if warm:
        assert rmx.info[0]["warm_used"] == 1
    assert np.abs(qmx - q64).max() < 1e-5
    assert abs(q64.sum() - st.q_tot) < 1e-8 and abs(qmx.sum() - st.q_tot) < 1e-8
    rows = np.sort(np.random.default_rng(cfg).choice(st.n, n_rows, replace=False))
    y_or = O.ewald_matvec(st.cell, st.pos, st.sigma, q64, k_e=KE, omega=omega, rows=rows)
    y_gpu = p64.matvec(d[0], d[1], r64.q, J=None, fp64=True).cpu().numpy()[rows]
    # accuracy relative to the QEq operator output (E + J) q, which sets the charge error
    full = y_or + st.J[rows] * q64[rows]
    rel = np.sqrt(np.mean((y_gpu - y_or) ** 2)) / np.sqrt(np.mean(full ** 2))
    assert rel < tol, rel
    jmin = st.J.min()
    bound = 0.5 * 1e-5 * jmin + 5 * tol * np.sqrt(np.mean(full ** 2))
    mu64 = r64.mu.cpu().numpy()[0]
    res64 = y_or + st.J[rows] * q64[rows] + st.chi[rows] - mu64
    assert np.abs(res64).max() < bound, (np.abs(res64).max(), bound)
    # the oracle's residual of the chosen form's charges on the same rows
    y_mx = O.ewald_matvec(st.cell, st.pos, st.sigma, qmx, k_e=KE, omega=omega, rows=rows)
    mumx = rmx.mu.cpu().numpy()[0]
    resmx = y_mx + st.J[rows] * qmx[rows] + st.chi[rows] - mumx
    print(f"workload {cfg}: chosen form max|res| on {n_rows} oracle rows = {np.abs(resmx).max():.3e} eV/e "
          f"(bound {bound:.3e}); max|q_chosen - q_fp64| = {np.abs(qmx - q64).max():.3e} e; "
          f"iterations {rmx.info[0]['iterations']} (FP64 Jacobi {r64.info[0]['iterations']})")
    assert np.abs(resmx).max() < bound, (np.abs(resmx).max(), bound)
    p64.close()
    pmx.close()
    if mlp is not None:
        mlp.close()
