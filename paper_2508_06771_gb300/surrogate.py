"""Training and evaluation of the rate-coefficient surrogate on data the particle
method generates.

Every network computation (features from the cell moments, subsampled
features, forward, backward, Adam, in-loop inference) runs in the CUDA library;
this module only orchestrates: it steps a collision context, collects feature
and target tensors, shuffles mini-batches and computes the dataset's feature
statistics (PyTorch bookkeeping on the device).

Targets are the exact per-cell rates k_c = sum sigma_c |v| / N of the whole
cell.  Inputs are the cell's features either from all its particles or from a
random subsample of `per_cell` particles: the surrogate learns to predict the
well-resolved rate from a poorly sampled distribution, which is the situation
of a simulation with few particles per cell (the paper notes that resolving the
tail can take tens of thousands of particles per cell, Sec. 1).
"""
from __future__ import annotations

import numpy as np

from . import ltpc


def collect(col, net, dt, step0, nsteps, every=4, per_cells=(100, 300, 1000), salt0=0):
    """Step `col` and collect (X_raw, T_exact) every `every` steps; X from subsamples of each size in
    `per_cells` (0 = the whole cell).  The network's normalisation must be the identity here."""
    import torch
    Xs, Ts = [], []
    step = step0
    for k in range(nsteps // every):
        col.run(dt, step, every)
        step += every
        _, T = net.features(col, normalize=False)
        for i, pc in enumerate(per_cells):
            if pc == 0:
                X, _ = net.features(col, normalize=False)
            else:
                X, _ = net.subsample_features(col, pc, salt0 + 1000 * k + i)
            Xs.append(X.clone())
            Ts.append(T.clone())
    return torch.cat(Xs), torch.cat(Ts), step


def identity_norm(net):
    net.set_norm(np.zeros(66, np.float32), np.ones(66, np.float32), np.ones(2, np.float32))


def fit_norm(net, X_raw, T_raw):
    """Feature means/stds and target scales of a dataset; installs them and returns normalised tensors."""
    mean = X_raw.mean(0)
    std = X_raw.std(0).clamp_min(1e-3)
    tscale = T_raw.abs().mean(0).clamp_min(1e-30)
    net.set_norm(mean.cpu().numpy(), std.cpu().numpy(), tscale.cpu().numpy())
    return (X_raw - mean) / std, T_raw / tscale


def train(net, Xn, Tn, epochs=20, batch=4096, lr=1e-3, seed=0):
    """Adam on shuffled mini-batches; returns the mean loss of each epoch."""
    import torch
    g = torch.Generator(device=Xn.device).manual_seed(seed)
    n = Xn.shape[0]
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g, device=Xn.device)
        tot, nb = 0.0, 0
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            loss = net.train_step(Xn[idx].contiguous(), Tn[idx].contiguous(), lr)
            tot += float(loss.item()) if (nb % 50 == 0) else 0.0
            nb += 1
        hist.append(tot / max(1, (nb + 49) // 50))
    return hist


def predict(net, Xn):
    """Rates in physical units for normalised features."""
    import torch
    ys = []
    for b0 in range(0, Xn.shape[0], net.batch_max):
        ys.append(net.forward(Xn[b0:b0 + net.batch_max].contiguous()))
    Y = torch.cat(ys)
    t = torch.as_tensor(net.norm[2], device=Y.device)
    return Y * t


def relative_errors(pred, truth, mask=None):
    """Median and mean |pred - truth| / truth over the rows where `mask` holds."""
    import torch
    e = (pred - truth).abs() / truth.abs().clamp_min(1e-30)
    if mask is not None:
        e = e[mask]
    return float(e.median()), float(e.mean())
