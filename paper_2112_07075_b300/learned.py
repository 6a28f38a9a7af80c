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


# The learned workload: 3D Taylor-Green, Q3/Q2, q1 = 6, 48^3 hexes, interior nodes
# jittered by +-0.1h; training seeds 1-8, held-out seeds 9 and 10.
LEARNED_N, LEARNED_ORDER, LEARNED_Q1, LEARNED_JITTER = 48, 3, 6, 0.1
TRAIN_SEEDS, HELD_OUT_SEEDS = tuple(range(1, 9)), (9, 10)


def record_configured(steps_total=2000, stride=32, precision="fp32_ir", seeds=TRAIN_SEEDS):
    """Training data of the learned workload: `steps_total` CFL steps from t = 0 shared
    equally by the training seeds (2000 steps from 8 seeds: 250 per seed) on the full
    48^3 mesh, keeping a rotating 1/stride of the elements of every mass solve.

    Returns (X, T, rows) as DEVICE tensors. precision: the mass-solve precision of the
    recording runs (the solutions agree with the FP64 ones to the CG tolerance).
    """
    import torch
    from . import inputs
    n = LEARNED_N
    ne = n ** 3
    steps = steps_total // len(seeds)
    per_solve = (ne + stride - 1) // stride
    cap = len(seeds) * 2 * steps * per_solve
    X = torch.zeros((cap, lh.MLP_IN), dtype=torch.float32, device="cuda")
    T = torch.zeros((cap, lh.MLP_OUT), dtype=torch.float32, device="cuda")
    rows = 0
    for seed in seeds:
        V = inputs.box_vertices(3, n, jitter=LEARNED_JITTER, seed=seed)
        ctx = lh.Context(3, n, V, LEARNED_ORDER, LEARNED_Q1, precision=precision)
        lh.learn_attach(ctx, None, 1, X[rows:], T[rows:])
        lh.learn_set_record_stride(ctx, stride)
        x, v, e = ctx.init_state()
        info = ctx.new_step_info(0.0, 1.0)
        for _ in range(steps):
            ctx.rk2avg_step(x, v, e, 0.0, info)
        torch.cuda.synchronize()
        if ctx.sync_status() != 0:
            raise RuntimeError("recording run failed: " + ctx.lib.lh_last_error(ctx.h).decode())
        rows += lh.learn_stats(ctx)["rows"]
        ctx.close()
    return X, T, rows


def train_configured(out_path, steps_total=2000, stride=32, schedule=((10, 1e-3), (6, 2e-4)), seed=7):
    """Record the configured training budget, train the MLP with liblh's kernels
    (Adam, batches of 8192; schedule = (epochs, learning rate) phases) and save its
    FP32 master weights (npz with the loss history and the recipe)."""
    import time
    t0 = time.perf_counter()
    X, T, rows = record_configured(steps_total, stride)
    t1 = time.perf_counter()
    net = lh.MLP(seed=seed, max_rows=LEARNED_N ** 3)
    hist = []
    for k, (ep, lr) in enumerate(schedule):
        hist += train(net, X[:rows], T[:rows], epochs=ep, batch=8192, lr=lr, seed=k)
    epochs = "+".join(f"{ep} at lr {lr:g}" for ep, lr in schedule)
    t2 = time.perf_counter()
    np.savez(out_path, params=net.get_params(), loss=np.array(hist), rows=rows,
             recipe=np.array(f"3D Taylor-Green {LEARNED_N}^3 Q{LEARNED_ORDER} q{LEARNED_Q1} jitter "
                             f"{LEARNED_JITTER}h, seeds {TRAIN_SEEDS}, {steps_total} CFL steps in total "
                             f"({steps_total // len(TRAIN_SEEDS)} per seed), every {stride}th element of "
                             f"each solve (rotating), epochs of Adam (batch 8192): {epochs}, "
                             f"MLP seed {seed}"),
             record_s=t1 - t0, train_s=t2 - t1)
    net.close()
    return rows, hist, t1 - t0, t2 - t1


def load_weights(path, max_rows=LEARNED_N ** 3):
    """An MLP with the weights saved by train_configured."""
    w = np.load(path)
    net = lh.MLP(seed=0, max_rows=max_rows)
    net.set_params(w["params"])
    return net


def evaluate(path, steps, precision="fp32_ir", seed=HELD_OUT_SEEDS[0], learned=True):
    """CFL steps from t = 0 of the learned workload on a held-out seed with the weights
    at `path` (learned=False: the plain previous-solve guess). Returns the step record."""
    import torch
    from . import inputs
    net = load_weights(path) if learned else None
    c = lh.Context(3, LEARNED_N, inputs.box_vertices(3, LEARNED_N, jitter=LEARNED_JITTER, seed=seed),
                   LEARNED_ORDER, LEARNED_Q1, precision=precision)
    if net is not None:
        lh.learn_attach(c, net, 2)
    x, v, e = c.init_state()
    info = c.new_step_info(0.0, 1.0)
    for _ in range(steps):
        c.rk2avg_step(x, v, e, 0.0, info)
    torch.cuda.synchronize()
    si = c.read_step_info(info)
    c.close()
    if net is not None:
        net.close()
    return si


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train the learned-form MLP on the configured budget, or "
                                             "evaluate trained weights on a held-out seed")
    ap.add_argument("--out", help="train: write the weights here")
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--stride", type=int, default=32)
    ap.add_argument("--eval", help="evaluate these weights instead of training")
    ap.add_argument("--eval-steps", type=int, default=6)
    ap.add_argument("--precision", default="fp32_ir", choices=["fp64", "fp32_ir", "bf16tc_ir"])
    a = ap.parse_args()
    if a.eval:
        si = evaluate(a.eval, a.eval_steps, a.precision)
        print(json.dumps({"steps": si.steps, "t": si.t, "status": si.status, "cg_iters_last": list(si.cg_iters)}))
    else:
        rows, hist, rs, ts = train_configured(a.out, a.steps, a.stride)
        print(json.dumps({"rows": rows, "loss": hist, "record_s": rs, "train_s": ts}))
