"""Training and evaluation of the learned prolongation.

The network (``mm.Net``) adds a drift to the polar prolongation of Sec. 3.2
("Uncoarsening").  It is trained on pairs the method itself produces: for
every level l of a hierarchy, the converged layout of the coarse level l+1
is the input and the converged layout of level l (after its own sweeps) is
the target.  Everything here drives the C-ABI: the layouts, the forward and
backward passes and the Adam steps all run in the library's kernels.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import mm


def level_pairs(h: mm.Hierarchy, params: mm.Params = None):
    """Coarse-to-converged training pairs of one hierarchy (a plain layout
    records every level's final layout)."""
    p = params if params is not None else mm.default_params()
    xs = mm.layout_levels(h, p)
    ex = [mm.level_export(h, l) for l in range(len(xs))]
    pairs = []
    for l in range(len(xs) - 1):
        fine, coarse = ex[l], ex[l + 1]
        pairs.append(dict(
            fine=dict(row_ptr=fine["row_ptr"], col=fine["col"], map=fine["map"]),
            coarse=dict(row_ptr=coarse["row_ptr"], col=coarse["col"], c=coarse["c"]),
            x_coarse=xs[l + 1].contiguous(), x_target=xs[l].contiguous(), level=l,
            seed=int(p.seed), n=int(fine["row_ptr"].numel() - 1)))
    return pairs


def _sample(pair):
    return mm.Net.sample(pair["fine"], pair["coarse"], pair["x_coarse"], pair["seed"],
                         pair["level"], pair["x_target"])


def train(net: mm.Net, pairs, steps: int, lr: float = 3e-3, seed: int = 0,
          min_lr_frac: float = 0.05):
    """Adam over `steps` samples drawn (seeded) with probability proportional
    to sqrt(n), cosine learning-rate decay; returns the per-step losses."""
    rng = np.random.default_rng(seed)
    w = np.sqrt(np.array([p["n"] for p in pairs], dtype=np.float64))
    w /= w.sum()
    smps = [_sample(p) for p in pairs]
    losses = []
    for t in range(steps):
        i = int(rng.choice(len(pairs), p=w))
        frac = min_lr_frac + (1 - min_lr_frac) * 0.5 * (1 + math.cos(math.pi * t / steps))
        losses.append(net.train_step(smps[i][0], lr * frac))
    return losses


def zero_net() -> mm.Net:
    """A network whose drift is identically 0: the plain polar prolongation."""
    return mm.Net(np.zeros(mm.MM_NET_PARAMS, dtype=np.float32))


def pair_loss(net: mm.Net, pair) -> float:
    """Mean |x_v - x*_v|^2 / c(p) of the network's prolongation of one pair."""
    smp, keep = _sample(pair)
    return net.forward(smp)[1]


def init_params(seed: int) -> np.ndarray:
    """Seeded He-normal weights of the three message-passing layers, a small
    head (drift near 0 at the start) and zero biases, in the flat layout of
    mm_net_create: W0 [16x64], b0, W1 [128x64], b1, W2 [128x64], b2,
    Wo [64x4], bo."""
    rng = np.random.default_rng(seed)
    parts = []
    for rows, cols, scale in [(16, 64, math.sqrt(2 / 16)), (128, 64, math.sqrt(2 / 128)),
                              (128, 64, math.sqrt(2 / 128)), (64, 4, 0.1 / 8.0)]:
        parts.append(rng.standard_normal(rows * cols) * scale)
        parts.append(np.zeros(cols))
    out = np.concatenate(parts).astype(np.float32)
    assert out.size == mm.MM_NET_PARAMS
    return out
