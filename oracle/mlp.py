"""fp64 reference of the branching-order network (TEST INFRASTRUCTURE ONLY).

The library's CUDA kernels score candidate pairs (v, u) with a small MLP to
choose the order in which McSplit tries candidates; this module is the plain
numpy definition those kernels are checked against.  The order never changes
the optimum (every candidate is still tried), only how soon a good incumbent
appears.

Vertex features (18 per vertex), for a graph with adjacency a (n x n):
    deg(x)  = number of y != x with a[x,y] (undirected) or a[x,y] + a[y,x]
              (directed; an arc in each direction counts twice)
    N(x)    = { y != x : a[x,y] or a[y,x] }
    f0 = deg(x) / 16
    f1 = min(label(x), 63) / 8      (0 when unlabelled)
    f2+b = #{ y in N(x) : min(deg(y), 15) == b } / 4,   b = 0..15
Pair input x(v, u) = [f_G(v), f_H(u)] (36 values), zero-padded to 48.
Network: z1 = x W1 + b1, h1 = relu(z1) (128); z2 = h1 W2 + b2, h2 = relu(z2)
(128); s = h2 . w3 + b3 (a logit).  Loss per row: w * (softplus(s) - y s)
(binary cross-entropy with logits), averaged over the rows.

Parameter vector layout (float32/float64, 22,913 values):
    W1 [48][128] (row = input), b1 [128], W2 [128][128] (row = input),
    b2 [128], w3 [128], b3 [1]
"""
from __future__ import annotations

import numpy as np

D_IN, D_PAD, H = 36, 48, 128
N_PARAMS = D_PAD * H + H + H * H + H + H + 1


def vertex_features(adj: np.ndarray, labels=None, directed: bool = False) -> np.ndarray:
    a = (np.asarray(adj) != 0).astype(np.int64)
    n = a.shape[0]
    off = a.copy()
    np.fill_diagonal(off, 0)
    deg = off.sum(1) + (off.sum(0) if directed else 0)
    nb = (off | off.T) if directed else off
    f = np.zeros((n, 18), np.float64)
    f[:, 0] = deg / 16.0
    if labels is not None:
        f[:, 1] = np.minimum(np.asarray(labels, np.int64), 63) / 8.0
    dbin = np.minimum(deg, 15)
    for x in range(n):
        for y in np.nonzero(nb[x])[0]:
            f[x, 2 + dbin[y]] += 0.25
    return f


def unpack(theta: np.ndarray):
    t = np.asarray(theta, np.float64)
    i = 0
    W1 = t[i:i + D_PAD * H].reshape(D_PAD, H); i += D_PAD * H
    b1 = t[i:i + H]; i += H
    W2 = t[i:i + H * H].reshape(H, H); i += H * H
    b2 = t[i:i + H]; i += H
    w3 = t[i:i + H]; i += H
    b3 = t[i]
    return W1, b1, W2, b2, w3, b3


def pair_inputs(fG: np.ndarray, fH: np.ndarray, v: np.ndarray, u: np.ndarray) -> np.ndarray:
    x = np.zeros((len(v), D_PAD), np.float64)
    x[:, :18] = fG[v]
    x[:, 18:36] = fH[u]
    return x


def forward(theta, x, round_h1_fp16: bool = False):
    """Returns (s, cache).  round_h1_fp16 mirrors a device that feeds layer 2
    with h1 rounded to fp16."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    z1 = x @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    if round_h1_fp16:
        h1 = h1.astype(np.float16).astype(np.float64)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    s = h2 @ w3 + b3
    return s, (x, z1, h1, z2, h2)


def loss_and_grad(theta, x, y, w=None, round_h1_fp16: bool = False):
    """Mean weighted BCE-with-logits loss and its gradient w.r.t. theta."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    y = np.asarray(y, np.float64)
    w = np.ones_like(y) if w is None else np.asarray(w, np.float64)
    B = len(y)
    s, (x, z1, h1, z2, h2) = forward(theta, x, round_h1_fp16)
    loss = float(np.sum(w * (np.logaddexp(0.0, s) - y * s)) / B)
    ds = w * (1.0 / (1.0 + np.exp(-s)) - y) / B
    g_w3 = h2.T @ ds
    g_b3 = ds.sum()
    dz2 = np.outer(ds, w3) * (z2 > 0)
    g_W2 = h1.T @ dz2
    g_b2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * (z1 > 0)
    g_W1 = x.T @ dz1
    g_b1 = dz1.sum(0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g


def init_params(seed: int = 0) -> np.ndarray:
    """He-style initialisation (the library's training starts from the same)."""
    r = np.random.default_rng(seed)
    W1 = r.normal(0, np.sqrt(2.0 / D_IN), (D_PAD, H))
    W1[D_IN:] = 0.0
    W2 = r.normal(0, np.sqrt(2.0 / H), (H, H))
    w3 = r.normal(0, np.sqrt(1.0 / H), H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, [0.0]])
