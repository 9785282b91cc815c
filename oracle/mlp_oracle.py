"""FP64 CPU oracle of the warm-start descriptors and network.

TEST INFRASTRUCTURE (same rules as qeq_oracle): shares no code with the CUDA
path.  Definitions follow the paper:
  * radial functions of Sec. 2.2 eq. (g2), G_mu = sum_j exp(-eta (r_ij - R_mu)^2) f_c(r_ij),
    with the cosine cutoff of SI "Cutoff Functions", f_c = (cos(pi r / r_c) + 1) / 2;
  * a second set weighted by chi_j: the element-embracing prefactor of SI
    "Element-Embracing ACSFs" with H_ij = chi_j;
  * feature scaling (G - mean) / (max - min) of SI "Feature Scaling";
  * per-species feed-forward networks z = W a + b, a = tanh(z), linear output
    (SI "Feed-Forward Neural Networks", "Activation Functions");
  * Xavier initialisation U(-a, a), a = sqrt(6 / (n_in + n_out)) (SI "Xavier");
  * the MSE loss L = 1/(2n) sum (y - t)^2 and Adam (SI "Loss Functions", "Adam").
Parameter block per species (length NPARAM, float): W1[64][32], b1[64],
W2[64][64], b2[64], W3[64], b3, zero padding.
"""
from __future__ import annotations

import math

import numpy as np

NF, NH, NPARAM = 32, 64, 6400
RC, ETA = 6.0, 2.0
R_MU = 0.5 + 0.5 * np.arange(12)
P_W1 = 0
P_B1 = P_W1 + NH * NF
P_W2 = P_B1 + NH
P_B2 = P_W2 + NH * NH
P_W3 = P_B2 + NH
P_B3 = P_W3 + NH


def cutoff(r):
    r = np.asarray(r, float)
    return np.where(r < RC, 0.5 * (np.cos(np.pi * r / RC) + 1.0), 0.0)


def features(cell, pos, species, chi, J, sigma_s):
    """Descriptors of every atom by brute force over all periodic images within RC."""
    cell = np.asarray(cell, float)
    pos = np.asarray(pos, float)
    n = len(pos)
    V = abs(np.linalg.det(cell))
    wd = np.array([V / np.linalg.norm(np.cross(cell[(d + 1) % 3], cell[(d + 2) % 3])) for d in range(3)])
    nm = [int(math.ceil(RC / wd[d])) + 1 for d in range(3)]
    shifts = np.stack(np.meshgrid(*[np.arange(-m, m + 1) for m in nm], indexing="ij"), -1).reshape(-1, 3)
    hinv = np.linalg.inv(cell)
    u = pos @ hinv
    u -= np.floor(u)
    F = np.zeros((n, NF))
    for i in range(n):
        d = (u - u[i])[None, :, :] + shifts[:, None, :]      # images x atoms x 3 (fractional)
        r = np.linalg.norm(d @ cell, axis=-1)
        zero = np.all(shifts == 0, axis=1)
        r[zero, i] = np.inf                                   # exclude the atom itself
        m = r < RC
        rr = r[m]
        cj = np.broadcast_to(np.asarray(chi, float)[None, :], r.shape)[m]
        g = np.exp(-ETA * (rr[:, None] - R_MU[None, :]) ** 2) * cutoff(rr)[:, None]
        F[i, :12] = g.sum(0)
        F[i, 12:24] = (cj[:, None] * g).sum(0)
    F[:, 24] = chi
    F[:, 25] = J
    F[:, 26] = np.asarray(sigma_s, float)[np.asarray(species)]
    return F


def unpack(p):
    return (p[P_W1:P_B1].reshape(NH, NF), p[P_B1:P_W2], p[P_W2:P_B2].reshape(NH, NH), p[P_B2:P_W3],
            p[P_W3:P_B3], p[P_B3])


def scale_from_features(F, species, n_species):
    """Per-species mean and 1/(max - min) (1 where the feature is constant)."""
    out = np.zeros((n_species, 2, NF))
    for s in range(n_species):
        X = F[species == s]
        if len(X) == 0:
            out[s, 1] = 1.0
            continue
        mn, mx = X.min(0), X.max(0)
        rng = mx - mn
        out[s, 0] = X.mean(0)
        out[s, 1] = np.where(rng > 1e-12, 1.0 / np.where(rng > 1e-12, rng, 1.0), 1.0)
    return out


def xavier(n_species, rng):
    params = np.zeros((n_species, NPARAM))
    for s in range(n_species):
        a1 = math.sqrt(6.0 / (NF + NH))
        a2 = math.sqrt(6.0 / (NH + NH))
        a3 = math.sqrt(6.0 / (NH + 1))
        params[s, P_W1:P_B1] = rng.uniform(-a1, a1, NH * NF)
        params[s, P_W2:P_B2] = rng.uniform(-a2, a2, NH * NH)
        params[s, P_W3:P_B3] = rng.uniform(-a3, a3, NH)
    return params


def forward(F, species, params, scale):
    """Network output per atom and the per-atom activations for backward."""
    n = len(F)
    y = np.zeros(n)
    cache = {}
    for s in range(len(params)):
        idx = np.nonzero(species == s)[0]
        if len(idx) == 0:
            continue
        W1, b1, W2, b2, W3, b3 = unpack(params[s])
        X = (F[idx] - scale[s, 0]) * scale[s, 1]
        h1 = np.tanh(X @ W1.T + b1)
        h2 = np.tanh(h1 @ W2.T + b2)
        y[idx] = h2 @ W3 + b3
        cache[s] = (idx, X, h1, h2)
    return y, cache


def loss_and_grad(F, species, target, params, scale):
    """L = 1/(2n) sum (y - t)^2 and dL/dparams (same layout as params)."""
    n = len(F)
    y, cache = forward(F, species, params, scale)
    e = y - target
    L = 0.5 * float(e @ e) / n
    grad = np.zeros_like(params)
    for s, (idx, X, h1, h2) in cache.items():
        W1, b1, W2, b2, W3, b3 = unpack(params[s])
        dy = e[idx] / n
        g = grad[s]
        g[P_W3:P_B3] = h2.T @ dy
        g[P_B3] = dy.sum()
        dz2 = np.outer(dy, W3) * (1 - h2 ** 2)
        g[P_W2:P_B2] = (dz2.T @ h1).reshape(-1)
        g[P_B2:P_W3] = dz2.sum(0)
        dz1 = (dz2 @ W2) * (1 - h1 ** 2)
        g[P_W1:P_B1] = (dz1.T @ X).reshape(-1)
        g[P_B1:P_W2] = dz1.sum(0)
    return L, grad


def adam_step(params, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new params, m, v."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(x):
    """Round to bfloat16 (round to nearest even) and back to float64."""
    a = np.asarray(x, np.float32).copy()
    b = a.view(np.uint32)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.view(np.float32).astype(np.float64)
