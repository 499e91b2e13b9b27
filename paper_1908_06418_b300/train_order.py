"""Trains the branching-order network on the GPU with the library's own
forward, backward and Adam kernels (mcs_order_train).

    python -m paper_1908_06418_b300.train_order --data tests/golden/order_train.npz \\
        --out paper_1908_06418_b300/data/order_mlp_bvg.npy

The data file holds branching decisions logged by a sequential McSplit on
seeded bounded-valence training pairs (n <= 30): columns pair, v, u (original
vertex ids) and y (1 when the search below (v, u) reached the optimum).  This
script only marshals it: pairs are rebuilt from their seeds with ``synth``,
uploaded as a device batch, and every arithmetic step runs in CUDA kernels.
Positives are up-weighted by negatives / positives.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "data", "order_mlp_bvg.npy")


def load_model(path: str = DEFAULT_MODEL) -> np.ndarray:
    return np.load(path).astype(np.float32)


def init_params(seed: int) -> np.ndarray:
    """He-style initialisation; inputs 36..47 of W1 are padding and stay 0."""
    r = np.random.default_rng(seed)
    d_in, d_pad, h = 36, 48, 128
    W1 = r.normal(0, np.sqrt(2.0 / d_in), (d_pad, h))
    W1[d_in:] = 0.0
    W2 = r.normal(0, np.sqrt(2.0 / h), (h, h))
    w3 = r.normal(0, np.sqrt(1.0 / h), h)
    return np.concatenate([W1.ravel(), np.zeros(h), W2.ravel(), np.zeros(h), w3, [0.0]]).astype(np.float32)


def main():
    import synth
    from . import Solver, DeviceBatch
    ap = argparse.ArgumentParser()
    ap.add_argument("--data", required=True)
    ap.add_argument("--out", default=DEFAULT_MODEL)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--holdout", type=float, default=0.05, help="fraction of pairs held out")
    ap.add_argument("--family", default="bvg", choices=["bvg", "planted"],
                    help="training pairs: synth.config4_train_pair or synth.planted_bvg_pair "
                         "(n 16..30, config id 46)")
    a = ap.parse_args()

    d = np.load(a.data)
    pair, v, u, y = d["pair"], d["v"], d["u"], d["y"].astype(np.float32)
    ids = np.unique(pair)
    rng = np.random.default_rng(a.seed)
    hold = set(rng.choice(ids, max(1, int(a.holdout * len(ids))), replace=False).tolist())
    t0 = time.time()
    if a.family == "bvg":
        pairs = [synth.config4_train_pair(int(i)) for i in ids]
    else:
        pairs = [synth.planted_bvg_pair(int(i), 16, 30, cid=46) for i in ids]
    pos = {int(i): k for k, i in enumerate(ids)}
    rows = np.stack([np.array([pos[int(p)] for p in pair], np.int32), v, u], axis=1).astype(np.int32)
    is_hold = np.array([int(p) in hold for p in pair])
    npos, nneg = float(y[~is_hold].sum()), float((1 - y[~is_hold]).sum())
    w = np.where(y > 0, nneg / max(npos, 1.0), 1.0).astype(np.float32)
    print(f"{len(ids)} pairs, {len(y)} rows ({int(y.sum())} positive), built in {time.time() - t0:.1f} s",
          flush=True)

    with Solver(0) as s:
        batch = DeviceBatch(pairs)
        s.set_order_model(init_params(a.seed))
        tr = ~is_hold
        t1 = time.time()
        losses = s.order_train(batch, rows[tr], y[tr], w[tr], steps=a.steps, batch_size=a.batch,
                               lr=a.lr, seed=a.seed)
        train_s = time.time() - t1
        ev_tr = s.order_eval(batch, rows=rows[tr], y=y[tr], w=w[tr], loss_grad=True, scores=True)
        ev_ho = s.order_eval(batch, rows=rows[is_hold], y=y[is_hold], w=w[is_hold], loss_grad=True,
                             scores=True)
        theta = s.get_order_model()

    def acc(scores, yy):
        return float(np.mean((scores > 0) == (yy > 0)))

    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    np.save(a.out, theta)
    meta = dict(data=os.path.basename(a.data), pairs=int(len(ids)), rows=int(len(y)),
                steps=a.steps, batch=a.batch, lr=a.lr, seed=a.seed, train_seconds=round(train_s, 2),
                loss_first=float(losses[:50].mean()), loss_last=float(losses[-50:].mean()),
                train_loss=ev_tr["loss"], holdout_loss=ev_ho["loss"],
                train_acc=acc(ev_tr["scores"], y[tr]), holdout_acc=acc(ev_ho["scores"], y[is_hold]))
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
