"""Pins of the warm-start oracle (descriptors and network) on the CPU."""
import math

import numpy as np

from oracle import mlp_oracle as M
from paper_2607_17978_b300 import synth


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    n, S = 40, 2
    F = rng.normal(size=(n, M.NF))
    sp = rng.integers(0, S, n)
    t = rng.normal(size=n)
    params = M.xavier(S, rng)
    for s in range(S):
        params[s, M.P_B1:M.P_W2] = rng.normal(size=M.NH) * 0.1
        params[s, M.P_B3] = 0.3
    scale = M.scale_from_features(F, sp, S)
    L, g = M.loss_and_grad(F, sp, t, params, scale)
    for s in range(S):
        for k in [M.P_W1 + 5, M.P_W1 + 700, M.P_B1 + 3, M.P_W2 + 17, M.P_W2 + 4000, M.P_B2 + 60, M.P_W3 + 9,
                  M.P_B3]:
            h = 1e-6
            p1, p2 = params.copy(), params.copy()
            p1[s, k] += h
            p2[s, k] -= h
            fd = (M.loss_and_grad(F, sp, t, p1, scale)[0] - M.loss_and_grad(F, sp, t, p2, scale)[0]) / (2 * h)
            assert abs(fd - g[s, k]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (s, k, fd, g[s, k])
    assert np.all(g[:, M.P_B3 + 1:] == 0)


def test_dimer_descriptors_closed_form():
    L = 40.0
    r = 2.3
    cell = np.eye(3) * L
    pos = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    chi = np.array([-1.2, 0.7])
    F = M.features(cell, pos, np.array([0, 1]), chi, np.array([2.0, 1.5]), np.array([1.0, 1.8]))
    g = np.exp(-2.0 * (r - (0.5 + 0.5 * np.arange(12))) ** 2) * 0.5 * (math.cos(math.pi * r / 6.0) + 1)
    assert np.allclose(F[0, :12], g, atol=1e-14) and np.allclose(F[1, :12], g, atol=1e-14)
    assert np.allclose(F[0, 12:24], chi[1] * g, atol=1e-14)
    assert np.allclose(F[1, 12:24], chi[0] * g, atol=1e-14)
    assert np.allclose(F[:, 24:27], [[-1.2, 2.0, 1.0], [0.7, 1.5, 1.8]])
    assert np.all(F[:, 27:] == 0)


def test_descriptor_cutoff_and_images():
    # one atom in a 5 A cubic cell: its own images at 5 A contribute, those at >= 6 A do not
    cell = np.eye(3) * 5.0
    F = M.features(cell, np.array([[0.3, 0.2, 0.1]]), np.array([0]), np.array([1.5]), np.array([2.0]),
                   np.array([1.0]))
    g = 6 * np.exp(-2.0 * (5.0 - (0.5 + 0.5 * np.arange(12))) ** 2) * 0.5 * (math.cos(math.pi * 5.0 / 6.0) + 1)
    assert np.allclose(F[0, :12], g, atol=1e-13)
    assert np.allclose(F[0, 12:24], 1.5 * g, atol=1e-13)


def test_descriptors_translation_and_permutation_invariant():
    st = synth.rocksalt(1, 5.64, 0.2, synth.rng_for(95, 0))
    F = M.features(st.cell, st.pos, st.species, st.chi, st.J, st.sigma_s)
    F2 = M.features(st.cell, st.pos + np.array([3.3, -1.1, 0.4]), st.species, st.chi, st.J, st.sigma_s)
    assert np.abs(F - F2).max() < 1e-12
    perm = np.random.default_rng(1).permutation(st.n)
    F3 = M.features(st.cell, st.pos[perm], st.species[perm], st.chi[perm], st.J[perm], st.sigma_s)
    assert np.abs(F3 - F[perm]).max() < 1e-12


def test_adam_first_step_is_sign_times_lr():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = M.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 1e-3)
    assert np.allclose(p, -1e-3 * np.sign(g), rtol=1e-4)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -3.14159])
    r = M.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7
    assert abs(r[3] + 3.14159) < 2 ** -6


def test_adam_matches_the_library_optimiser_over_several_steps():
    """Adam's bias-corrected update (Kingma & Ba 2015) against torch.optim.Adam in FP64, ten steps of
    random gradients with non-default betas: a slip in a bias correction or in where eps enters fails."""
    import torch
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=50)
    b1, b2, eps, lr = 0.85, 0.99, 1e-6, 3e-2
    w = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([w], lr=lr, betas=(b1, b2), eps=eps)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for step in range(1, 11):
        g = rng.normal(size=50) * (0.1 if step % 3 else 5.0)
        p, m, v = M.adam_step(p, g, m, v, step, lr, b1, b2, eps)
        w.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        assert np.abs(p - w.detach().numpy()).max() < 1e-13 * max(1.0, np.abs(p).max()), step


def test_bf16_rounding_matches_the_library_conversion():
    """Round to nearest even into bfloat16 against torch's conversion: random magnitudes over many
    binades, exact ties with an even and an odd kept bit, the largest finite values and subnormals."""
    import torch
    rng = np.random.default_rng(4)
    x = (rng.normal(size=20000) * np.exp2(rng.integers(-30, 30, size=20000))).astype(np.float32)
    hi = rng.integers(0, 1 << 16, size=4000, dtype=np.uint32) << np.uint32(16)
    ties = (hi | np.uint32(0x8000)).view(np.float32)            # exactly halfway between two bf16 values
    ties = ties[np.isfinite(ties) & (np.abs(ties) < 3e38)]
    edge = np.array([3.38e38, -3.38e38, 1e-39, -1e-39, 1e-45, 0.0, -0.0], np.float32)
    for arr in (x, ties, edge):
        expect = torch.from_numpy(arr.copy()).to(torch.bfloat16).to(torch.float64).numpy()
        got = M.bf16_round(arr)
        assert np.array_equal(got.view(np.uint64), expect.view(np.uint64))

