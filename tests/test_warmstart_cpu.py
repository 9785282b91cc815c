"""Host logic of the warm-start training (paper_2607_17978_b300/warmstart.py) against the oracle on CPU:
the per-species feature scaling of SI "Feature Scaling" (mean and 1/(max - min), 1 for a constant feature
and for a species absent from the data)."""
import numpy as np
import torch

from oracle import mlp_oracle as M
from paper_2607_17978_b300 import warmstart


def test_feature_scaling_matches_the_oracle():
    rng = np.random.default_rng(7)
    n, S = 500, 3
    F = rng.normal(size=(n, M.NF)) * rng.uniform(0.1, 10.0, size=M.NF)
    F[:, 5] = 2.5                                       # a constant feature
    F[:, M.NF - 4:] = 0.0                                # padding columns
    sp = rng.integers(0, S - 1, n)                       # species S - 1 absent
    got = warmstart.fit_scale(torch.from_numpy(F).float(), torch.from_numpy(sp), S)
    ref = M.scale_from_features(F.astype(np.float32).astype(np.float64), sp, S)
    assert got.shape == ref.shape == (S, 2, M.NF)
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-6)
    assert np.all(got[:, 1, 5] == 1.0) and np.all(got[S - 1] == np.stack([np.zeros(M.NF), np.ones(M.NF)]))
