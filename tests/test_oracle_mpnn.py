"""Pins of the FP64 oracle of the learned prolongation.

* analytic gradients against central finite differences of the loss;
* the predicted drift rotates and translates with the coarse layout;
* the mean aggregation and its transpose against a dense adjacency matrix.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mpnn
from paper_1506_04383_gb300 import graphs


def _sample(n_pts=300, seed=3):
    rp, col, pts, _ = graphs.rgg(n_pts, 7.0, seed, tune=False)
    n = len(rp) - 1
    c = np.ones(n)
    lab = oracle.sclap(rp, col, c, 3.0, 10, seed, 0)
    mp, cc, crp, ccol, _ = oracle.contract(rp, col, c, lab)
    rng = np.random.default_rng(seed)
    xc = rng.random((len(cc), 2)) * 20.0
    r = mpnn.polar_offsets(n, mp, cc, 1506, 0)
    t = rng.normal(0.0, 0.5, (n, 2))
    return rp, col, mp, xc, crp, ccol, cc, r, t


def test_aggregation_against_dense_adjacency():
    rp, col, *_ = _sample(120)
    n = len(rp) - 1
    A = np.zeros((n, n))
    src = np.repeat(np.arange(n), np.diff(rp))
    A[src, col] = 1.0
    A = A / np.maximum(A.sum(1, keepdims=True), 1)
    H = np.random.default_rng(0).random((n, 5))
    np.testing.assert_allclose(mpnn.mean_agg(rp, col, H), A @ H, atol=1e-12)
    np.testing.assert_allclose(mpnn.mean_agg_T(rp, col, H), A.T @ H, atol=1e-12)


def test_gradients_match_finite_differences():
    rp, col, mp, xc, crp, ccol, cc, r, t = _sample()
    f, a, b, r, g = mpnn.features(rp, col, mp, xc, crp, ccol, cc, r)
    P = mpnn.init_params(7)
    # move the biases off zero so ReLU kinks are not hit exactly
    rng = np.random.default_rng(1)
    for k in P:
        if k.startswith("b"):
            P[k] = rng.normal(0, 0.05, P[k].shape)
    cp = cc[mp]
    o, cache = mpnn.forward(P, rp, col, f, a, b, r, g)
    G = mpnn.backward(P, rp, col, cache, a, b, r, g, o, t, cp)
    h = 1e-6
    for k in ["W0", "b0", "W1", "W2", "b2", "W3", "b3"]:
        flat = P[k].reshape(-1)
        idx = rng.choice(len(flat), size=min(6, len(flat)), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = mpnn.loss(mpnn.forward(P, rp, col, f, a, b, r, g)[0], t, cp)
            flat[i] = old - h
            lm = mpnn.loss(mpnn.forward(P, rp, col, f, a, b, r, g)[0], t, cp)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = G[k].reshape(-1)[i]
            assert an == pytest.approx(fd, rel=1e-4, abs=1e-9), (k, i)


def test_drift_is_equivariant():
    rp, col, mp, xc, crp, ccol, cc, r, t = _sample()
    P = mpnn.init_params(9)
    f, a, b, r0, g = mpnn.features(rp, col, mp, xc, crp, ccol, cc, r)
    o, _ = mpnn.forward(P, rp, col, f, a, b, r0, g)
    ang = 0.9
    Rm = np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
    xc2 = xc @ Rm.T + np.array([5.0, -3.0])
    f2, a2, b2, r2, g2 = mpnn.features(rp, col, mp, xc2, crp, ccol, cc, r @ Rm.T)
    o2, _ = mpnn.forward(P, rp, col, f2, a2, b2, r2, g2)
    np.testing.assert_allclose(f2, f, atol=1e-9)
    np.testing.assert_allclose(o2, o @ Rm.T, atol=1e-9)
    # the centre direction g rotates with the layout and ignores translation
    np.testing.assert_allclose(g2, g @ Rm.T, atol=1e-9)


def test_centre_basis_expresses_a_uniform_growth():
    # a target that is the coarse layout scaled by s about its mean is
    # reproduced exactly by beta = (0, 0, 0, s - 1) -- a head with zero
    # weights and that bias -- so the loss is 0 there
    rp, col, mp, xc, crp, ccol, cc, r, _ = _sample()
    f, a, b, r, g = mpnn.features(rp, col, mp, xc, crp, ccol, cc, r)
    m = xc.mean(0)
    s = 1.07
    t_abs = m + s * (xc[mp] - m) + r
    t = t_abs - xc[mp] - r
    P = mpnn.init_params(3)
    P["W3"][:] = 0.0
    P["b3"][:] = [0.0, 0.0, 0.0, s - 1.0]
    o, _ = mpnn.forward(P, rp, col, f, a, b, r, g)
    assert mpnn.loss(o, t, cc[mp]) < 1e-20


def test_adam_matches_closed_form_first_step():
    # the first Adam step moves every parameter by -lr * sign(g) (bias
    # corrected moments equal g and g^2)
    P = {"W0": np.array([[1.0, -2.0]]), "b0": np.array([0.5])}
    G = {"W0": np.array([[0.3, -0.7]]), "b0": np.array([-2.0])}
    P2 = mpnn.adam_step({k: v.copy() for k, v in P.items()}, G, {}, lr=0.01)
    np.testing.assert_allclose(P2["W0"], P["W0"] - 0.01 * np.sign(G["W0"]), atol=1e-7)
    np.testing.assert_allclose(P2["b0"], P["b0"] - 0.01 * np.sign(G["b0"]), atol=1e-7)


def test_bf16_round_against_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-30, 30, 4000),
                        [0.0, -0.0, 1.0, 3.4e38, -3.4e38, 1e-40, 1.00390625, 1.01171875,
                         1.0 + 2.0 ** -8 + 2.0 ** -20]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = mpnn.bf16_round(x)
    np.testing.assert_array_equal(got, want)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert mpnn.bf16_round(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert mpnn.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6


def test_quantised_gradients_match_finite_differences_of_quantised_loss():
    # with BF16 operands the loss is piecewise smooth in the non-quantised
    # parameters (biases and the head); its gradient there is still exact
    rp, col, mp, xc, crp, ccol, cc, r, t = _sample()
    f, a, b, r, g = mpnn.features(rp, col, mp, xc, crp, ccol, cc, r)
    P = mpnn.init_params(7)
    cp = cc[mp]
    q = mpnn.bf16_round
    o, cache = mpnn.forward(P, rp, col, f, a, b, r, g, quant=q)
    G = mpnn.backward(P, rp, col, cache, a, b, r, g, o, t, cp, quant=q)
    h = 1e-7
    for k, i in [("W3", 5), ("W3", 100), ("W3", 131), ("b3", 0), ("b3", 3)]:
        flat = P[k].reshape(-1)
        old = flat[i]
        flat[i] = old + h
        lp = mpnn.loss(mpnn.forward(P, rp, col, f, a, b, r, g, quant=q)[0], t, cp)
        flat[i] = old - h
        lm = mpnn.loss(mpnn.forward(P, rp, col, f, a, b, r, g, quant=q)[0], t, cp)
        flat[i] = old
        assert G[k].reshape(-1)[i] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)
