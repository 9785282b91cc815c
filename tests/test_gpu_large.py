"""Full-size cells where the dense oracle is infeasible: sampled-row parity.

For the 105,062-atom triclinic cell with vacancies and the 980,000-atom cell:
  * the GPU FP64 matvec agrees with the oracle's FP64 Ewald matvec on sampled
    rows within the plan's ewald_tol (relative to the RMS of the sampled rows);
  * the mixed-precision and FP64 GPU solves agree within 1e-5 e max-abs;
  * the oracle's residual of the GPU charges, (A q + chi)_i - mu on sampled
    rows, is within the stopping tolerance plus the matvec error.
"""
import numpy as np
import pytest

from oracle import qeq_oracle as O
from paper_2607_17978_b300 import synth

KE = synth.COULOMB_K_EV_A
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg,n_rows,omega", [(3, 300, 8.0), (5, 64, 11.0)])
def test_large_cell_sampled_rows(cfg, n_rows, omega):
    import torch
    from paper_2607_17978_b300 import build, qeq
    build.build()
    st = synth.workload(cfg)
    pos, spc, chi, J, qt = qeq.pack([st])
    dev = torch.device("cuda")
    d = [torch.tensor(a, device=dev) for a in (pos, spc, chi, J)]
    tol = 1e-6
    p64 = qeq.plan_for_structures([st], precision="fp64", ewald_tol=tol, r_cut=8.0)
    r64 = p64.solve(*d, qt)
    pmx = qeq.plan_for_structures([st], precision="mixed", ewald_tol=tol, r_cut=8.0)
    rmx = pmx.solve(*d, qt)
    q64 = r64.q.cpu().numpy()
    qmx = rmx.q.cpu().numpy()
    assert r64.info[0]["status"] == 0 and rmx.info[0]["status"] == 0
    assert np.abs(qmx - q64).max() < 1e-5
    assert abs(q64.sum() - st.q_tot) < 1e-8
    rows = np.sort(np.random.default_rng(cfg).choice(st.n, n_rows, replace=False))
    y_or = O.ewald_matvec(st.cell, st.pos, st.sigma, q64, k_e=KE, omega=omega, rows=rows)
    y_gpu = p64.matvec(d[0], d[1], r64.q, J=None, fp64=True).cpu().numpy()[rows]
    # accuracy relative to the QEq operator output (E + J) q, which sets the charge error
    full = y_or + st.J[rows] * q64[rows]
    rel = np.sqrt(np.mean((y_gpu - y_or) ** 2)) / np.sqrt(np.mean(full ** 2))
    assert rel < tol, rel
    mu = r64.mu.cpu().numpy()[0]
    res = y_or + st.J[rows] * q64[rows] + st.chi[rows] - mu
    jmin = st.J.min()
    bound = 0.5 * 1e-5 * jmin + 5 * tol * np.sqrt(np.mean(full ** 2))
    assert np.abs(res).max() < bound, (np.abs(res).max(), bound)
    p64.close()
    pmx.close()
