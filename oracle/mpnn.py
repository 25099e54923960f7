"""FP64 oracle of the learned prolongation -- TEST INFRASTRUCTURE ONLY.

The paper (Sec. 3.2, "Uncoarsening") places a fine vertex v of the coarse
vertex v' at a random polar offset r_v around v' (angle uniform in
[0, 2 pi), radius uniform in [0, sqrt(c(v')))).  The learned prolongation
keeps that placement and adds a drift o_v predicted by a small
message-passing network from the coarse layout and the local structure:

    x_v = x'_p + r_v + o_v,      p = M(v).

Inputs per fine vertex (all rotation/translation/scale invariant except the
four basis vectors, which rotate and scale with the layout):
    a_v = mean over fine neighbours w with M(w) != p of (x'_{M(w)} - x'_p)
    b_v = mean over coarse neighbours q of p of (x'_q - x'_p)
    r_v = the polar offset of the paper's prolongation (Philox draws)
    g_v = x'_p - m, m = mean of the coarse layout (unweighted): the layout
        grows by a few percent about its centre while a level refines, and
        o = beta_3 g expresses that growth (beta_3 = factor - 1)
    scalars f (8): |g|/S with S the RMS distance of the coarse vertices from
        m, ln c(p), ln(1 + deg v), fraction of v's neighbours outside its
        cluster, |a|/R, |b|/R, cos(a, b), (a . r)/(|a| R), R = sqrt(c(p)).
Network (3 message-passing layers, hidden 64, mean aggregation over the
fine graph):
    H0 = f;  H_l = ReLU([H_{l-1} | A H_{l-1}] W_l + b_l),  l = 1..3
    beta = H_3 W_o + b_o  (4 coefficients)
    o_v = beta_0 a_v + beta_1 b_v + beta_2 r_v + beta_3 g_v
so o is equivariant by construction.  Loss: mean over v of
|o_v - t_v|^2 / c(p) with target t_v = x*_v - x'_p - r_v (x* = the level's
converged layout).

The method fixes BF16 operands with FP32 accumulation for the dense layers.
With ``quant=bf16_round`` the forward and backward passes round to BF16 at
exactly the points where those operands are formed -- the features, both
halves of every [H | A H], every W_l, every ReLU output H_l, and, in the
backward pass, dZ_l (for both [H | A H]^T dZ_l and dZ_l W_l^T) and W_l --
and stay FP64 elsewhere.
Without it (the default) everything is FP64.

Pins (tests/test_oracle_mpnn.py): analytic gradients against central finite
differences; equivariance of o under rotation and translation of the coarse
layout; the mean aggregation and its transpose against a dense adjacency;
bf16_round against an independent library conversion, including ties and
the extremes of the range.
"""
from __future__ import annotations

import math

import numpy as np

import oracle

F_IN = 8
HIDDEN = 64
N_OUT = 4
LAYERS = 3


def bf16_round(x):
    """Nearest BF16 value of every FP32-rounded element (ties to even), as an
    FP64 array.  BF16 keeps the sign, the 8 exponent bits and the top 7
    mantissa bits of an IEEE binary32 value: add half of the dropped 16-bit
    field (minus one, plus the kept low bit, for ties to even) and clear it."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _ident(x):
    return x


def layer_shapes():
    """(rows, cols) of W_1..W_3 and W_o."""
    return [(2 * F_IN, HIDDEN), (2 * HIDDEN, HIDDEN), (2 * HIDDEN, HIDDEN), (HIDDEN, N_OUT)]


def init_params(seed: int):
    """He-scaled normal weights, zero biases (seeded; passed to both sides)."""
    rng = np.random.default_rng(seed)
    P = {}
    for i, (r, c) in enumerate(layer_shapes()):
        scale = math.sqrt(2.0 / r) if i < LAYERS else 0.1 / math.sqrt(r)
        P[f"W{i}"] = rng.standard_normal((r, c)) * scale
        P[f"b{i}"] = np.zeros(c)
    return P


def polar_offsets(n_fine, mp, cc, seed, level):
    """r_v of the paper's prolongation (the oracle's own Philox draws)."""
    xc = np.zeros((len(cc), 2))
    return oracle.prolong(mp, xc, cc, seed, level)


def mean_agg(rp, col, H):
    """(A H)_v = mean over the CSR neighbours of v (0 for isolated v)."""
    n = len(rp) - 1
    deg = np.diff(rp)
    src = np.repeat(np.arange(n), deg)
    out = np.zeros((n,) + H.shape[1:])
    np.add.at(out, src, H[col])
    return out / np.maximum(deg, 1)[:, None]


def mean_agg_T(rp, col, G):
    """(A^T G)_w = sum over v with w in N(v) of G_v / deg(v)."""
    n = len(rp) - 1
    deg = np.diff(rp)
    src = np.repeat(np.arange(n), deg)
    out = np.zeros((n,) + G.shape[1:])
    np.add.at(out, col, G[src] / np.maximum(deg, 1)[src, None])
    return out


def features(rp, col, mp, xc, crp, ccol, cc, r):
    """Scalar features f [n, 8] and basis vectors a, b, r, g [n, 2] each."""
    n = len(rp) - 1
    deg = np.diff(rp)
    src = np.repeat(np.arange(n), deg)
    p = mp
    outside = mp[col] != mp[src]
    a = np.zeros((n, 2))
    cnt = np.zeros(n)
    np.add.at(a, src[outside], xc[mp[col[outside]]] - xc[p[src[outside]]])
    np.add.at(cnt, src[outside], 1)
    a = a / np.maximum(cnt, 1)[:, None]
    nc = len(crp) - 1
    cdeg = np.diff(crp)
    csrc = np.repeat(np.arange(nc), cdeg)
    bc = np.zeros((nc, 2))
    np.add.at(bc, csrc, xc[ccol] - xc[csrc])
    bc = bc / np.maximum(cdeg, 1)[:, None]
    b = bc[p]
    R = np.sqrt(cc[p])
    na = np.linalg.norm(a, axis=1)
    nb = np.linalg.norm(b, axis=1)
    m = xc.mean(axis=0)
    S = math.sqrt(((xc - m) ** 2).sum(1).mean())
    g = xc[p] - m
    f = np.zeros((n, F_IN))
    f[:, 0] = np.linalg.norm(g, axis=1) / max(S, 1e-30)
    f[:, 1] = np.log(cc[p])
    f[:, 2] = np.log1p(deg)
    f[:, 3] = cnt / np.maximum(deg, 1)
    f[:, 4] = na / R
    f[:, 5] = nb / R
    f[:, 6] = (a * b).sum(1) / (na * nb + 1e-12)
    f[:, 7] = (a * r).sum(1) / (na * R + 1e-12)
    return f, a, b, r, g


def forward(P, rp, col, f, a, b, r, g, quant=None):
    """Returns (o [n,2], cache for backward)."""
    q = quant or _ident
    H = q(f)
    cache = []
    for l in range(LAYERS):
        Hc = np.concatenate([H, q(mean_agg(rp, col, H))], axis=1)
        Z = Hc @ q(P[f"W{l}"]) + P[f"b{l}"]
        cache.append((Hc, Z))
        H = q(np.maximum(Z, 0.0))
    beta = H @ P[f"W{LAYERS}"] + P[f"b{LAYERS}"]
    o = beta[:, 0:1] * a + beta[:, 1:2] * b + beta[:, 2:3] * r + beta[:, 3:4] * g
    return o, dict(layers=cache, H=H, beta=beta)


def loss(o, t, cp):
    """mean_v |o_v - t_v|^2 / c(p)."""
    d = o - t
    return float(((d * d).sum(1) / cp).mean())


def backward(P, rp, col, cache, a, b, r, g, o, t, cp, quant=None):
    """Analytic gradients of the loss with respect to every W_l and b_l."""
    q = quant or _ident
    n = len(o)
    do = 2.0 * (o - t) / (n * cp)[:, None]
    dbeta = np.stack([(do * a).sum(1), (do * b).sum(1), (do * r).sum(1), (do * g).sum(1)],
                     axis=1)
    G = {}
    H = cache["H"]
    G[f"W{LAYERS}"] = H.T @ dbeta
    G[f"b{LAYERS}"] = dbeta.sum(0)
    dH = dbeta @ P[f"W{LAYERS}"].T
    for l in range(LAYERS - 1, -1, -1):
        Hc, Z = cache["layers"][l]
        dZ = dH * (Z > 0)
        # the weight gradient of a dense layer is a BF16 x BF16 product with
        # FP32 accumulation on the device: dZ is rounded as for dZ W^T below
        G[f"W{l}"] = Hc.T @ q(dZ)
        G[f"b{l}"] = dZ.sum(0)
        dHc = q(dZ) @ q(P[f"W{l}"]).T
        d = Hc.shape[1] // 2
        dH = dHc[:, :d] + mean_agg_T(rp, col, dHc[:, d:])
    return G


def adam_step(P, G, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) of every parameter, in place."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        m = state.setdefault("m" + k, np.zeros_like(P[k]))
        v = state.setdefault("v" + k, np.zeros_like(P[k]))
        m[:] = beta1 * m + (1 - beta1) * G[k]
        v[:] = beta2 * v + (1 - beta2) * G[k] * G[k]
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P
