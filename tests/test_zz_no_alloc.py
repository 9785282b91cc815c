"""The allocation-free matvec entry point (qeq_matvec_static) against qeq_matvec and the oracle.

qeq_matvec_static serves callers that cannot call cudaMalloc: its scratch is a
file-scope device array, so the library allocates nothing during the call.
This file is collected last on purpose; it must pass on its own in a fresh
process and after the rest of the suite (the shared scratch array keeps the
previous call's contents, so two calls in a row are checked).
"""
import numpy as np
import pytest

from oracle import qeq_oracle as O
from paper_2607_17978_b300 import synth

pytestmark = pytest.mark.gpu


def _cases():
    yield synth.workload(1)                                                   # 2 species, real-space pairs
    yield synth.batch_workload(1, cfg_id=43, n_min=200, n_max=400, first=2)[0]  # triclinic, 2-4 species


@pytest.mark.parametrize("case", [0, 1])
def test_static_matvec_matches_plan_matvec_twice(case):
    import torch
    from paper_2607_17978_b300 import build, qeq
    build.build()
    st = list(_cases())[case]
    pos, spc, chi, J, _ = qeq.pack([st])
    dev = torch.device("cuda")
    d_pos = torch.tensor(pos, device=dev)
    d_spc = torch.tensor(spc, device=dev)
    d_J = torch.tensor(J, device=dev)
    tol = 1e-6
    plan = qeq.plan_for_structures([st], ewald_tol=tol, r_cut=8.0)
    # the oracle's dense (E + diag J) of this cell: an independent check of the shared kernels
    A = O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=synth.COULOMB_K_EV_A) + np.diag(st.J)
    rng = np.random.default_rng(case)
    xs = [rng.normal(size=st.n), rng.normal(size=st.n) * 0.3 + 0.1]
    for x in xs:                                   # two calls in a row share the scratch array
        d_x = torch.tensor(x, device=dev)
        y_ref = plan.matvec(d_pos, d_spc, d_x, J=d_J, fp64=True)
        y = qeq.matvec_static(st.cell, st.sigma_s, d_pos, d_spc, d_x, d_J, ewald_tol=tol, r_cut=8.0)
        torch.cuda.synchronize()
        yr, yc = y_ref.cpu().numpy(), y.cpu().numpy()
        rel = np.sqrt(np.mean((yc - yr) ** 2)) / np.sqrt(np.mean(yr ** 2))
        assert rel < tol, rel
        yo = A @ x
        rel_o = np.sqrt(np.mean((yc - yo) ** 2)) / np.sqrt(np.mean(yo ** 2))
        assert rel_o < tol, rel_o
    plan.close()


def test_static_matvec_rejects_oversized_input():
    import torch
    from paper_2607_17978_b300 import qeq
    n = 4097
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    pos = torch.zeros(n, 3, dtype=torch.float64, device="cuda")
    spc = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(qeq.QEqError) as e:
        qeq.matvec_static(np.eye(3) * 40.0, [1.0], pos, spc, x)
    assert e.value.status == qeq.QEQ_ERR_CAPACITY
