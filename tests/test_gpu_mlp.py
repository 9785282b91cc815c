"""GPU warm start: descriptors, the BF16 tensor-core network (tcgen05, inference and training)
and its training against the CPU oracle, and what the trained network gains over the cold
start."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from oracle import qeq_oracle as O
from paper_2607_17978_b300 import synth

pytestmark = pytest.mark.gpu
KE = synth.COULOMB_K_EV_A


def _structs():
    return [synth.rocksalt(2, 5.64, 0.2, synth.rng_for(50, 0), vacancy_frac=0.05, shear_deg=10.0),
            synth.batch_workload(1, cfg_id=51, n_min=150, n_max=300, first=1)[0]]


def test_features_match_oracle():
    import torch
    from paper_2607_17978_b300 import build, qeq
    build.build()
    structs = _structs()
    plan = qeq.plan_for_structures(structs)
    pos, spc, chi, J, qt = qeq.pack(structs)
    f = plan.features(pos, spc, chi, J).cpu().numpy()
    off = np.concatenate([[0], np.cumsum([s.n for s in structs])])
    for i, st in enumerate(structs):
        ref = M.features(st.cell, st.pos, st.species, st.chi, st.J, st.sigma_s)
        got = f[off[i]:off[i + 1]]
        assert np.abs(got - ref).max() < 2e-5 * max(1.0, np.abs(ref).max())


def _random_net(n_species, seed, feat, species):
    rng = np.random.default_rng(seed)
    params = M.xavier(n_species, rng)
    for s in range(n_species):
        params[s, M.P_B1:M.P_W2] = rng.normal(size=M.NH) * 0.2
        params[s, M.P_B2:M.P_W3] = rng.normal(size=M.NH) * 0.2
        params[s, M.P_B3] = 0.1
    scale = M.scale_from_features(feat, species, n_species)
    return params, scale


def _bf16_net(params, scale, feat):
    """CPU inputs as the GPU sees them: BF16 weights (biases FP32) and BF16 scaled features."""
    pr = params.copy()
    for s in range(len(pr)):
        pr[s, M.P_W1:M.P_B1] = M.bf16_round(pr[s, M.P_W1:M.P_B1])
        pr[s, M.P_W2:M.P_B2] = M.bf16_round(pr[s, M.P_W2:M.P_B2])
    return pr


def test_forward_and_gradient_match_oracle():
    import torch
    from paper_2607_17978_b300 import qeq
    rng = np.random.default_rng(3)
    n, S = 300, 2
    feat = rng.normal(size=(n, M.NF)) * 2 + 1
    feat[:, 27:] = 0
    sp = rng.integers(0, S, n)
    tgt = rng.normal(size=n) * 0.5
    params, scale = _random_net(S, 4, feat, sp)
    mlp = qeq.Mlp(S, max_batch=1024)
    mlp.set_params(params.astype(np.float32), scale.astype(np.float32))
    dev = torch.device("cuda")
    f_t = torch.tensor(feat, dtype=torch.float32, device=dev)
    s_t = torch.tensor(sp, dtype=torch.int32, device=dev)
    t_t = torch.tensor(tgt, dtype=torch.float32, device=dev)
    y = mlp.forward(f_t, s_t).cpu().numpy()
    # CPU oracle on the GPU's BF16-rounded weights and inputs
    p32 = params.astype(np.float32).astype(np.float64)
    pr = _bf16_net(p32, scale, feat)
    # scaled inputs rounded to BF16: fold the rounding into features with identity scaling
    Xs = np.zeros_like(feat)
    for s in range(S):
        m = sp == s
        Xs[m] = M.bf16_round((feat[m].astype(np.float32) - scale[s, 0].astype(np.float32)) * scale[s, 1].astype(np.float32))
    ident = np.zeros_like(scale)
    ident[:, 1] = 1.0
    y_ref, _ = M.forward(Xs, sp, pr, ident)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 2e-2
    loss, g = mlp.train_step(f_t, s_t, t_t, apply=False, want_grad=True)
    L_ref, g_ref = M.loss_and_grad(Xs, sp, tgt, pr, ident)
    g = g.cpu().numpy().reshape(S, -1)
    assert abs(loss - L_ref) < 2e-2 * L_ref
    for s in range(S):
        rel = np.linalg.norm(g[s] - g_ref[s]) / np.linalg.norm(g_ref[s])
        assert rel < 1e-2, (s, rel)
    # one Adam step equals the CPU update applied to the GPU's gradient
    before = mlp.get_state()["params"].reshape(S, -1).astype(np.float64)
    mlp.train_step(f_t, s_t, t_t, lr=1e-3, apply=True, want_grad=False)
    after = mlp.get_state()["params"].reshape(S, -1).astype(np.float64)
    exp, _, _ = M.adam_step(before, g.astype(np.float64), 0 * before, 0 * before, 1, 1e-3)
    assert np.abs(after - exp).max() < 1e-6
    mlp.close()


def test_adam_over_several_steps_matches_oracle():
    """Four Adam steps (bias corrections 1 - beta^t for t = 1..4, moments carried between steps)
    equal the oracle's updates applied to the gradients the GPU reports for each step; a fifth
    step from a restored state (set_adam_state) continues the same sequence."""
    import torch
    from paper_2607_17978_b300 import qeq
    rng = np.random.default_rng(11)
    n, S = 400, 2
    feat = rng.normal(size=(n, M.NF)) * 2 + 1
    feat[:, 27:] = 0
    sp = rng.integers(0, S, n)
    tgt = rng.normal(size=n) * 0.5
    params, scale = _random_net(S, 12, feat, sp)
    mlp = qeq.Mlp(S, max_batch=1024)
    mlp.set_params(params.astype(np.float32), scale.astype(np.float32))
    dev = torch.device("cuda")
    f_t = torch.tensor(feat, dtype=torch.float32, device=dev)
    s_t = torch.tensor(sp, dtype=torch.int32, device=dev)
    t_t = torch.tensor(tgt, dtype=torch.float32, device=dev)
    p = params.astype(np.float32).astype(np.float64).reshape(-1)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for step in range(1, 5):
        _, g = mlp.train_step(f_t, s_t, t_t, lr=2e-3, apply=True, want_grad=True)
        g = g.cpu().numpy().astype(np.float64)
        # the GPU holds beta1, beta2 as FP32 constants (1 - 0.999f is 4.7e-5 above 1e-3)
        p, m, v = M.adam_step(p, g, m, v, step, 2e-3, b1=float(np.float32(0.9)), b2=float(np.float32(0.999)))
        st = mlp.get_state()
        assert st["step"] == step
        assert np.abs(st["params"] - p).max() < 2e-6, (step, np.abs(st["params"] - p).max())
        assert np.abs(st["adam_m"] - m).max() < 1e-6 * max(1.0, np.abs(m).max())
        assert np.abs(st["adam_v"] - v).max() < 1e-6 * max(1e-6, np.abs(v).max())
    # restore the state into a fresh network and take step 5 in both
    st = mlp.get_state()
    mlp2 = qeq.Mlp(S, max_batch=1024)
    mlp2.set_params(st["params"].reshape(S, -1), st["scale"].reshape(S, 2, -1))
    mlp2.set_adam_state(st["adam_m"], st["adam_v"], st["step"])
    _, g1 = mlp.train_step(f_t, s_t, t_t, lr=2e-3, apply=True, want_grad=True)
    _, g2 = mlp2.train_step(f_t, s_t, t_t, lr=2e-3, apply=True, want_grad=True)
    assert torch.equal(g1, g2)
    assert np.array_equal(mlp.get_state()["params"], mlp2.get_state()["params"])
    mlp.close()
    mlp2.close()


@pytest.mark.parametrize("n,S", [(300, 2), (128, 1), (1000, 4), (5, 3)])
def test_tensor_core_forward_matches_bf16_emulation(n, S):
    """The inference network on tcgen05 (BF16 operands in shared memory, FP32 accumulators in
    tensor memory) against the same arithmetic emulated on the CPU: BF16 weights, scaled
    inputs and first-layer activations, everything else FP64.  Only accumulation order and the
    rare BF16 rounding of an activation that sits on a rounding boundary differ, so 99 % of the
    atoms agree to 1e-4 of the output scale and all to 5e-3.  Tiles of 128 atoms: ragged tails,
    a single full tile, a tile with every species, and fewer atoms than a warp."""
    import torch
    from paper_2607_17978_b300 import build, qeq
    build.build()
    rng = np.random.default_rng(100 + n + S)
    feat = rng.normal(size=(n, M.NF)) * 2 + 1
    feat[:, 27:] = 0
    sp = rng.integers(0, S, n)
    params, scale = _random_net(S, 7 + S, feat, sp)
    p32 = params.astype(np.float32)
    s32 = scale.astype(np.float32)
    mlp = qeq.Mlp(S, max_batch=max(n, 128))
    mlp.set_params(p32, s32)
    dev = torch.device("cuda")
    y = mlp.forward(torch.tensor(feat, dtype=torch.float32, device=dev),
                    torch.tensor(sp, dtype=torch.int32, device=dev)).cpu().numpy().astype(np.float64)
    mlp.close()
    ref = np.zeros(n)
    for s in range(S):
        idx = np.nonzero(sp == s)[0]
        if len(idx) == 0:
            continue
        W1, b1, W2, b2, W3, b3 = M.unpack(p32[s].astype(np.float64))
        X = M.bf16_round((feat[idx].astype(np.float32) - s32[s, 0]) * s32[s, 1]).astype(np.float64)
        h1 = M.bf16_round(np.tanh(X @ M.bf16_round(W1).T + b1))
        h2 = np.tanh(h1 @ M.bf16_round(W2).T + b2)
        ref[idx] = h2 @ W3 + b3
    err = np.abs(y - ref) / max(np.abs(ref).max(), 1e-3)
    assert np.all(np.isfinite(y))
    assert np.quantile(err, 0.99) < 1e-4, np.quantile(err, 0.99)
    assert err.max() < 5e-3, err.max()


def test_warm_start_gain_and_fallback():
    import torch
    from paper_2607_17978_b300 import qeq, warmstart
    train_structs = synth.training_structures(240, cfg_id=6, n_min=64, n_max=600)
    feat, spc, tgt, it_cold_train = warmstart.solve_targets(train_structs)
    mlp = qeq.Mlp(2, max_batch=4096)
    mlp.set_params(warmstart.xavier_params(2, 0), warmstart.fit_scale(feat, spc, 2))
    losses = warmstart.train(mlp, feat, spc, tgt, epochs=40, batch=2048, lr=3e-3)
    assert losses[-1] < 0.2 * losses[0]
    held = synth.training_structures(6, cfg_id=6, first=100000, n_min=200, n_max=600)
    plan = qeq.plan_for_structures(held)
    pos, sp, chi, J, qt = qeq.pack(held)
    cold = plan.solve(pos, sp, chi, J, qt)
    plan.set_warm_start(mlp)
    warm = plan.solve(pos, sp, chi, J, qt, warm="mlp")
    ic = np.array([i["iterations"] for i in cold.info])
    iw = np.array([i["iterations"] for i in warm.info])
    assert all(i["warm_used"] == 1 for i in warm.info)
    assert iw.mean() < ic.mean(), (iw, ic)
    qc, qw = cold.q.cpu().numpy(), warm.q.cpu().numpy()
    assert np.abs(qc - qw).max() < 1e-5
    st = held[0]
    A = O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=KE)
    q_ref, _ = O.solve_bordered(A, st.J, st.chi, st.q_tot)
    assert np.abs(qw[:st.n] - q_ref).max() < 1e-5
    # a network that predicts nonsense per atom (a constant offset would be removed by the
    # projection): the solve falls back to the cold start and still converges
    bad = mlp.get_state()
    p = bad["params"].reshape(2, -1).copy()
    w3 = qeq.MLP_NHIDDEN * qeq.MLP_NFEAT + qeq.MLP_NHIDDEN + qeq.MLP_NHIDDEN * qeq.MLP_NHIDDEN + qeq.MLP_NHIDDEN
    p[:, w3:w3 + qeq.MLP_NHIDDEN] *= 1e4
    mlp.set_params(p, bad["scale"])
    fb = plan.solve(pos, sp, chi, J, qt, warm="mlp")
    assert all(i["warm_used"] == 0 and i["status"] == 0 for i in fb.info)
    assert np.abs(fb.q.cpu().numpy() - qc).max() < 1e-5
    plan.close()
    mlp.close()


def test_warm_start_acceptance_is_per_structure():
    """A batch with a structure from the training recipe and one far outside it: hardnesses 25
    times larger (every training cell has the same J, so the network cannot follow J; the
    optimal charges shrink about 25-fold while the prediction stays near the training charges)
    and the electronegativities of the two sublattices swapped.  The first keeps its network
    start, the second restarts from the uniform start, and both reach the oracle's charges."""
    import os
    import torch
    from paper_2607_17978_b300 import qeq, warmstart
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    mlp, _ = warmstart.load(os.path.join(root, "paper_2607_17978_b300", "models", "warmstart_rocksalt.npz"))
    good = synth.rocksalt(4, 5.64, 0.2, synth.rng_for(5, 11), vacancy_frac=0.02)
    bad = synth.rocksalt(4, 5.64, 0.2, synth.rng_for(5, 12), vacancy_frac=0.02)
    bad.chi = -bad.chi
    bad.J = bad.J * 25.0
    structs = [good, bad]
    plan = qeq.plan_for_structures(structs, precision="mixed", preconditioner="fourier")
    plan.set_warm_start(mlp)
    pos, sp, chi, J, qt = qeq.pack(structs)
    d = [torch.tensor(a, device="cuda") for a in (pos, sp, chi, J)]
    res = plan.solve(*d, qt, warm="mlp")
    assert [i["warm_used"] for i in res.info] == [1, 0], res.info
    assert all(i["status"] == 0 for i in res.info)
    qg = res.q.cpu().numpy()
    off = [0, good.n, good.n + bad.n]
    for k, st in enumerate(structs):
        A = O.coulomb_matrix(st.cell, st.pos, st.sigma, k_e=KE)
        q_ref, _ = O.solve_bordered(A, st.J, st.chi, st.q_tot)
        assert np.abs(qg[off[k]:off[k + 1]] - q_ref).max() < 1e-5, k
    # the kept structure's solve is the one it gets alone
    p1 = qeq.plan_for_structures([good], precision="mixed", preconditioner="fourier")
    p1.set_warm_start(mlp)
    r1 = p1.solve(*[torch.tensor(a, device="cuda") for a in qeq.pack([good])[:4]], np.array([good.q_tot]), warm="mlp")
    assert r1.info[0]["warm_used"] == 1
    assert np.abs(r1.q.cpu().numpy() - qg[:good.n]).max() < 2e-6
    plan.close()
    p1.close()
    mlp.close()
