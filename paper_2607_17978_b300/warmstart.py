"""Training driver of the learned warm start (host side; the arithmetic runs in libqeq).

Targets are QEq solutions the solver itself produces for generated rock-salt-
recipe cells; descriptors come from qeq_features; the network is trained with
qeq_mlp_train_step (BF16 tensor-core forward/backward, Adam on FP32 master
weights).  Checkpoints (parameters, scaling, Adam state, step, metadata) are one
.npz file, so a run can be resumed.

    python -m paper_2607_17978_b300.warmstart --n-struct 20000 --epochs 30 --out model.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import qeq, synth

NF = qeq.MLP_NFEAT
NH = qeq.MLP_NHIDDEN
NP = qeq.MLP_NPARAM


def xavier_params(n_species: int, seed: int) -> np.ndarray:
    """Xavier initialisation U(-a, a), a = sqrt(6 / (n_in + n_out)) (SI "Xavier"), zero biases."""
    rng = np.random.default_rng(seed)
    p = np.zeros((n_species, NP), np.float32)
    off_b1 = NH * NF
    off_w2 = off_b1 + NH
    off_b2 = off_w2 + NH * NH
    off_w3 = off_b2 + NH
    for s in range(n_species):
        a1, a2, a3 = math.sqrt(6 / (NF + NH)), math.sqrt(6 / (2 * NH)), math.sqrt(6 / (NH + 1))
        p[s, :off_b1] = rng.uniform(-a1, a1, NH * NF)
        p[s, off_w2:off_b2] = rng.uniform(-a2, a2, NH * NH)
        p[s, off_w3:off_w3 + NH] = rng.uniform(-a3, a3, NH)
    return p


def solve_targets(structs, batch: int = 512, precision: str = "mixed", device="cuda", **plan_kw):
    """Charges, descriptors and species of every atom of ``structs`` (torch CUDA tensors)."""
    import torch
    feats, species, targets, iters = [], [], [], []
    for b0 in range(0, len(structs), batch):
        chunk = structs[b0:b0 + batch]
        plan = qeq.plan_for_structures(chunk, precision=precision, device=device, **plan_kw)
        pos, spc, chi, J, qt = qeq.pack(chunk)
        d = [torch.tensor(a, device=device) for a in (pos, spc, chi, J)]
        res = plan.solve(*d, qt)
        feats.append(plan.features(*d))
        species.append(d[1])
        targets.append(res.q.float())
        iters += [i["iterations"] for i in res.info]
        plan.close()
    return torch.cat(feats), torch.cat(species), torch.cat(targets), iters


def fit_scale(feat, species, n_species: int) -> np.ndarray:
    """(n_species, 2, 32): per-species mean and 1/(max - min) (SI "Feature Scaling"); 1 for constant features."""
    import torch
    out = np.zeros((n_species, 2, NF), np.float32)
    for s in range(n_species):
        m = species == s
        if int(m.sum()) == 0:
            out[s, 1] = 1.0
            continue
        X = feat[m].double()
        rng = (X.max(0).values - X.min(0).values)
        inv = torch.where(rng > 1e-9, 1.0 / torch.clamp(rng, min=1e-9), torch.ones_like(rng))
        out[s, 0] = X.mean(0).cpu().numpy()
        out[s, 1] = inv.cpu().numpy()
    return out


def train(mlp, feat, species, target, epochs: int = 20, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
          log=None):
    """Mini-batch training; returns the mean loss of every epoch."""
    import torch
    n = feat.shape[0]
    g = torch.Generator(device=feat.device)
    g.manual_seed(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g, device=feat.device)
        tot, cnt = 0.0, 0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            f = feat[idx].contiguous()
            s = species[idx].contiguous()
            t = target[idx].contiguous()
            loss, _ = mlp.train_step(f, s, t, lr=lr)
            tot += loss * len(idx)
            cnt += len(idx)
        losses.append(tot / cnt)
        if log:
            log(f"epoch {ep} loss {losses[-1]:.3e}")
    return losses


def save(path: str, mlp, meta: dict) -> None:
    st = mlp.get_state()
    np.savez(path, params=st["params"], scale=st["scale"], adam_m=st["adam_m"], adam_v=st["adam_v"],
             step=np.int64(st["step"]), n_species=np.int64(mlp.n_species), meta=json.dumps(meta))


def load(path: str, device="cuda", max_batch: int = 65536):
    z = np.load(path, allow_pickle=False)
    mlp = qeq.Mlp(int(z["n_species"]), max_batch=max_batch, device=device)
    mlp.set_params(z["params"], z["scale"])
    mlp.set_adam_state(z["adam_m"], z["adam_v"], int(z["step"]))
    return mlp, json.loads(str(z["meta"]))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--n-struct", type=int, default=20000)
    ap.add_argument("--n-min", type=int, default=64)
    ap.add_argument("--n-max", type=int, default=4096)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--resume", default=None)
    ap.add_argument("--out", required=True)
    args = ap.parse_args(argv)
    from . import build
    build.build()
    t0 = time.time()
    structs = synth.training_structures(args.n_struct, n_min=args.n_min, n_max=args.n_max)
    t1 = time.time()
    feat, species, target, iters = solve_targets(structs, ewald_tol=1e-6, r_cut=8.0)
    t2 = time.time()
    print(f"{len(structs)} structures, {feat.shape[0]} atoms: generated in {t1 - t0:.1f} s, solved in {t2 - t1:.1f} s "
          f"(mean {np.mean(iters):.1f} PCG iterations)", flush=True)
    if args.resume:
        mlp, meta = load(args.resume, max_batch=args.batch)
    else:
        mlp = qeq.Mlp(2, max_batch=args.batch)
        mlp.set_params(xavier_params(2, args.seed), fit_scale(feat, species, 2))
        meta = {}
    losses = train(mlp, feat, species, target, epochs=args.epochs, batch=args.batch, lr=args.lr, seed=args.seed,
                   log=lambda m: print(m, flush=True))
    meta.update({"n_struct": args.n_struct, "atoms": int(feat.shape[0]), "epochs": args.epochs, "lr": args.lr,
                 "batch": args.batch, "final_loss": losses[-1], "recipe": "rocksalt n1 x n2 x n3, jitter 0.2 A, "
                 "2% vacancies, chi_A~N(-2,.3) chi_B~N(2,.3), J 2/1.5, sigma 1.0/1.8", "train_seconds": time.time() - t2})
    save(args.out, mlp, meta)
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    sys.exit(main())
