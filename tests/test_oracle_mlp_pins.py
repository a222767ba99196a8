"""Pins of the FP64 reference of the learned near-singular correction.

The network is the library's own addition (the paper has none), so the
pins are mathematical facts: the gradient against central finite
differences of the loss, closed forms of special networks, the GELU
identities, and the invariances the pair features are built to have.
"""
import math

import numpy as np

from oracle import mlp_oracle as M
import oracle as O


def _rand_params(rng, scale=0.3):
    return rng.standard_normal(M.N_PARAMS) * scale


def _rand_batch(rng, n=7):
    feat = rng.standard_normal((n, 12))
    q = rng.random((n, 16))
    return feat, q / q.sum(1, keepdims=True), rng.standard_normal(n) * 0.1


def test_param_count_matches_architecture():
    assert M.N_PARAMS == 12 * 64 + 64 + 64 * 64 + 64 + 16 * 64 + 16 == 6032


def test_gelu_identities():
    z = np.linspace(-6, 6, 25)
    assert np.allclose(M.gelu(z) - M.gelu(-z), z, atol=1e-15)          # z Phi(z) - (-z) Phi(-z) = z
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert abs(M.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15  # Phi(1)
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(M.gelu_d(z), fd, atol=1e-8)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    P = _rand_params(rng)
    feat, q, c = _rand_batch(rng)
    loss, g = M.loss_and_grad(P, feat, q, c)
    assert abs(loss - np.mean((M.forward(P, feat, q) - c) ** 2)) < 1e-14
    idx = np.concatenate([rng.choice(M.N_PARAMS, 60, replace=False),
                          [0, 767, 768, 831, 832, 4927, 4928, 4991, 4992, 6015, 6016, 6031]])
    h = 1e-6
    for i in idx:
        e = np.zeros(M.N_PARAMS)
        e[i] = h
        fd = (M.loss_and_grad(P + e, feat, q, c)[0] - M.loss_and_grad(P - e, feat, q, c)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_bias_only_network_closed_form():
    """W3 = 0: dw = b3 for every pair, prediction sum_k b3_k qhat_k; with
    b3 constant the prediction is that constant (qhat sums to 1) and the
    loss and the b3 gradient have closed forms."""
    rng = np.random.default_rng(2)
    P = _rand_params(rng)
    P[4992:6016] = 0.0
    P[6016:] = 0.25
    feat, q, c = _rand_batch(rng, n=5)
    assert np.allclose(M.forward(P, feat, q), 0.25, atol=1e-15)
    loss, g = M.loss_and_grad(P, feat, q, c)
    e = 0.25 - c
    assert abs(loss - np.mean(e * e)) < 1e-15
    assert np.allclose(g[6016:], (2.0 / 5) * (e[:, None] * q).sum(0), atol=1e-15)
    assert np.all(g[:832] == 0) and np.all(g[832:4992] == 0)   # no signal reaches layers 1-2 through W3 = 0


def test_bf16_rounding():
    # spacing near 1 is 2^-7 (8 significant bits); 1 + 2^-8 and 1 + 3 2^-8 are ties
    x = np.array([1.0, 1.00390625, 1.001953125, 3.0e-3, -2.5, 1.01171875], np.float32)
    r = M.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 and r[5] == 1.015625   # ties to the even neighbour
    assert abs(r[3] - 3.0e-3) <= 2 ** -8 * 3.0e-3 and r[4] == -2.5      # unit roundoff 2^-8
    assert np.all(M.bf16_round(r) == r)


def _tet(rng, c, s):
    return c + s * rng.standard_normal((4, 3))


def test_pair_features_invariances():
    rng = np.random.default_rng(3)
    t = _tet(rng, np.zeros(3), 1.0)
    s = _tet(rng, np.array([2.5, 0.3, -0.4]), 0.8)
    f0, q0, Q0 = M.pair_features(t, s)
    assert abs(q0.sum() - 1.0) < 1e-15
    # similarity: rotation, translation, scale k -> same features and qhat, Q * k^5
    R, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    k = 0.37
    f1, q1, Q1 = M.pair_features(k * t @ R.T + 1.5, k * s @ R.T + 1.5)
    assert np.allclose(f1, f0, atol=1e-12) and np.allclose(q1, q0, atol=1e-14)
    assert abs(Q1 / Q0 - k ** 5) < 1e-12 * k ** 5
    # vertex order of the inputs does not matter
    f2, q2, Q2 = M.pair_features(t[[2, 0, 3, 1]], s[[3, 1, 0, 2]])
    assert np.allclose(f2, f0, atol=1e-13) and np.allclose(q2, q0, atol=1e-15) and abs(Q2 - Q0) < 1e-15 * Q0
    # features are affine coordinates: mapping them back gives the source vertices
    ct = t.mean(0)
    tv = t[np.argsort(((t - s.mean(0)) ** 2).sum(1))]
    A = np.stack([tv[1] - tv[0], tv[2] - tv[0], tv[3] - tv[0]], axis=1)
    back = (A @ f0.reshape(4, 3).T).T + ct
    assert np.allclose(np.sort(back, axis=0), np.sort(s, axis=0), atol=1e-12)


def test_pair_features_product_rule_matches_oracle_quadrature():
    """Q is the product rule of the pair: oracle element rules, summed."""
    rng = np.random.default_rng(4)
    t = _tet(rng, np.zeros(3), 1.0)
    s = _tet(rng, np.array([0.4, 2.9, 0.1]), 1.1)
    _, _, Q = M.pair_features(t, s)
    tp, tw = O.tet_quad(t[None])
    sp, sw = O.tet_quad(s[None])
    ref = sum(tw[i] * sw[j] / (4 * math.pi * np.linalg.norm(tp[i] - sp[j])) for i in range(4) for j in range(4))
    assert abs(Q - ref) <= 1e-14 * ref
    tri = s[:3]
    _, qh, Q = M.pair_features(t, tri)
    sp, sw = O.tri_quad(tri[None])
    ref = sum(tw[i] * sw[j] / (4 * math.pi * np.linalg.norm(tp[i] - sp[j])) for i in range(4) for j in range(3))
    assert abs(Q - ref) <= 1e-14 * ref and np.all(qh.reshape(4, 4)[:, 3] == 0)
