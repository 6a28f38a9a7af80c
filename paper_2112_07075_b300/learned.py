"""Learned form driver: record training examples with the method, train the MLP
with liblh's own kernels, and measure the learned initial guess.

Training data are the method's own mass-solve solutions: a context in recording
mode stores one (features, target) example per element at every mass solve that
has three earlier solutions (see lh_learn_attach in include/lh.h).
"""
from __future__ import annotations

import numpy as np

from . import lh


def record_examples(vertex_sets, n, steps, order=3, q1=6, cfl=0.5, t_end=1.0):
    """Run `steps` CFL steps of 3D Taylor-Green on each vertex set in recording mode.

    Returns (X, T, rows): DEVICE tensors [cap][586] and [cap][192] and the rows filled.
    """
    import torch
    ne = n ** 3
    cap = len(vertex_sets) * ne * 2 * steps
    X = torch.zeros((cap, lh.MLP_IN), dtype=torch.float32, device="cuda")
    T = torch.zeros((cap, lh.MLP_OUT), dtype=torch.float32, device="cuda")
    rows = 0
    for V in vertex_sets:
        ctx = lh.Context(3, n, V, order, q1, cfl=cfl)
        lh.learn_attach(ctx, None, 1, X[rows:], T[rows:])
        x, v, e = ctx.init_state()
        info = ctx.new_step_info(0.0, t_end)
        for _ in range(steps):
            ctx.rk2avg_step(x, v, e, 0.0, info)
        torch.cuda.synchronize()
        rows += lh.learn_stats(ctx)["rows"]
        ctx.close()
    return X, T, rows


def train(net, X, T, epochs=10, batch=4096, lr=1e-3, seed=0):
    """Adam on shuffled minibatches (host-side shuffling, device-side kernels). Returns the loss history."""
    import torch
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        for i in range(0, n - batch + 1 if n >= batch else 1, batch):
            idx = perm[i:i + batch]
            net.train_step(X.index_select(0, idx).contiguous(), T.index_select(0, idx).contiguous(), lr)
        hist.append(float(net.loss.item()))
    return hist
