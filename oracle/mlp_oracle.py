"""FP64 CPU reference of the learned near-singular correction.

Test infrastructure only: the product path never imports this module.
It restates, from their definitions, what the library's training and
inference kernels compute, so that the tests can check the GPU gradients
and features against it:

  features  source vertices in the affine frame of the target, centred at
            the target centroid; both vertex orders canonical (ascending
            distance to the other element's centroid).  A triangle target's
            third frame axis is its unit normal times sqrt(2 * area), on
            the side of the source.  A triangle source fills 9 of the 12
            slots (the rest 0).
  qhat      product-rule terms q_ij = W_i W_j / (4 pi r_ij) of the pair in
            the canonical orders, over their sum Q; i target point, j
            source point, 4 x 4 slots (unused slots 0).  Quadrature point k
            carries the largest barycentric weight at vertex k (tet rule
            (a, b, b, b), triangle rule (2/3, 1/6, 1/6)).
  network   x(12) -> GELU(W1 x + b1)(64) -> GELU(W2 . + b2)(64) -> W3 . + b3
            (16) = dw;  prediction chat_pred = sum_k dw_k qhat_k
  loss      mean over pairs of (chat_pred - chat)^2
  GELU      z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 (exact form)

Parameter vector: W1[64][12] b1[64] W2[64][64] b2[64] W3[16][64] b3[16].
Nothing here is pinned to the paper (the network is this library's own
addition); the pins are the mathematics: finite differences of the loss,
closed forms of special networks, invariances of the features.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_H, N_OUT = 12, 64, 16
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_OUT, N_H)),
          ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)          # 6032

_erf = np.vectorize(math.erf)


def unpack(params):
    params = np.asarray(params, np.float64)
    assert params.shape == (N_PARAMS,)
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = params[o:o + k].reshape(shp)
        o += k
    return out


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_d(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, feat, qhat):
    """Prediction for every pair: feat [n,12], qhat [n,16] -> [n]."""
    P = unpack(params)
    x = np.asarray(feat, np.float64)
    z1 = x @ P["W1"].T + P["b1"]
    h1 = gelu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(z2)
    y = h2 @ P["W3"].T + P["b3"]
    return np.einsum("nk,nk->n", y, np.asarray(qhat, np.float64))


def loss_and_grad(params, feat, qhat, chat):
    """Mean squared error of the prediction and its gradient (chain rule
    through the three layers, written out layer by layer)."""
    P = unpack(params)
    x = np.asarray(feat, np.float64)
    q = np.asarray(qhat, np.float64)
    n = x.shape[0]
    z1 = x @ P["W1"].T + P["b1"]
    h1 = gelu(z1)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = gelu(z2)
    y = h2 @ P["W3"].T + P["b3"]
    e = np.einsum("nk,nk->n", y, q) - np.asarray(chat, np.float64)
    loss = float(np.mean(e * e))
    dy = (2.0 / n) * e[:, None] * q                 # d loss / d y
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dz2 = (dy @ P["W3"]) * gelu_d(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * gelu_d(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return loss, np.concatenate([g[name].ravel() for name, _ in SHAPES])


def bf16_round(a):
    """Round FP32-representable values to the nearest BF16 (ties to even),
    the weights the kernels compute with."""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# --------------------------------------------------------------- features
_TA = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
_TB = (5.0 - math.sqrt(5.0)) / 20.0


def _quad_points(v):
    nv = len(v)
    out = []
    for q in range(nv):
        if nv == 4:
            w = [_TA if i == q else _TB for i in range(4)]
        else:
            w = [2.0 / 3.0 if i == q else 1.0 / 6.0 for i in range(3)]
        out.append(sum(w[i] * v[i] for i in range(nv)))
    return out


def _size(v):
    v = np.asarray(v, np.float64)
    n = np.cross(v[1] - v[0], v[2] - v[0])
    if len(v) == 3:
        return 0.5 * np.linalg.norm(n)
    return abs(np.dot(n, v[3] - v[0])) / 6.0


def pair_features(tgt, src):
    """(feat [12], qhat [16], Q) of one pair from its vertex coordinates."""
    tgt = np.asarray(tgt, np.float64)
    src = np.asarray(src, np.float64)
    ct, cs = tgt.mean(0), src.mean(0)
    tv = tgt[np.argsort(((tgt - cs) ** 2).sum(1), kind="stable")]
    sv = src[np.argsort(((src - ct) ** 2).sum(1), kind="stable")]
    a0, a1 = tv[1] - tv[0], tv[2] - tv[0]
    if len(tv) == 4:
        a2 = tv[3] - tv[0]
    else:
        nrm = np.cross(a0, a1)
        a2 = nrm / np.linalg.norm(nrm) * math.sqrt(np.linalg.norm(nrm))
        if np.dot(a2, cs - ct) < 0:
            a2 = -a2
    A = np.stack([a0, a1, a2], axis=1)
    feat = np.zeros(12)
    for k in range(len(sv)):
        feat[3 * k:3 * k + 3] = np.linalg.solve(A, sv[k] - ct)
    xq, yq = _quad_points(tv), _quad_points(sv)
    wt, ws = _size(tv) / len(tv), _size(sv) / len(sv)
    q = np.zeros(16)
    for i in range(len(tv)):
        for j in range(len(sv)):
            q[4 * i + j] = wt * ws / (4.0 * math.pi * np.linalg.norm(xq[i] - yq[j]))
    Q = q.sum()
    return feat, q / Q, Q
