"""Training set and training driver of the row-size predictor.

The targets come from the method itself: for each training matrix the
library's exact symbolic phase gives every row's nnz(C_i), and the features
come from smash_row_features. Rows with no products are left out (their size
is known to be zero). Training runs on the device (smash_mlp_train).
"""
from __future__ import annotations

import multiprocessing as mp
import time

import numpy as np


def _gen(seed):
    from .rmat import training_matrix
    return training_matrix(seed)


def training_matrices(seeds, workers: int = 0):
    """R-MAT training matrices (scale 12 + seed mod 5, edge factor 16), generated
    in a spawn-started process pool (safe after CUDA initialisation)."""
    seeds = list(seeds)
    if workers <= 1 or len(seeds) < 4:
        return [_gen(s) for s in seeds]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        return pool.map(_gen, seeds, chunksize=1)


def training_set(handle, mats, device="cuda"):
    """(features [n,6] float32, targets [n] float32) on the device for C = M*M:
    the library's smash_training_rows per matrix, concatenated."""
    import torch
    from . import smash
    feats, targets = [], []
    for M in mats:
        dM = smash.to_device(M, device, dtype=np.float32)
        f, t = handle.training_rows(dM, dM)
        feats.append(f)
        targets.append(t)
    return torch.cat(feats), torch.cat(targets)


def train(handle, mats, epochs: int = 8, batch: int = 4096, lr: float = 2e-3, seed: int = 1):
    """Train a fresh model on C = M*M for the given matrices. Returns
    (model, final loss, seconds of device training, number of samples)."""
    import torch
    from . import smash
    feats, targets = training_set(handle, mats)
    model = smash.Model(handle, seed=seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = handle.mlp_train(model, feats, targets, epochs=epochs, batch=batch, lr=lr, seed=seed)
    torch.cuda.synchronize()
    return model, loss, time.perf_counter() - t0, int(feats.shape[0])
