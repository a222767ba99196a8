"""The learned near-singular correction: GPU training kernels against the
FP64 reference (gradients, forward, Adam), the training data against the
oracle (features, product-rule terms, labels from the oracle's near rule),
and what the trained network gains over the method without it.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp_oracle as M
from paper_2112_00864_gb300.inputs import cube_bc_mesh, densities

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_00864_gb300 import bcfmm
    from paper_2112_00864_gb300.build import build
    build()
    return bcfmm


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    P = M.bf16_round(rng.standard_normal(M.N_PARAMS).astype(np.float32) * 0.3)   # BF16-exact: both sides equal
    feat = rng.standard_normal((n, 12)).astype(np.float32).astype(np.float64)
    q = rng.random((n, 16))
    q = (q / q.sum(1, keepdims=True)).astype(np.float32).astype(np.float64)
    c = (rng.standard_normal(n) * 0.05).astype(np.float32).astype(np.float64)
    return P, feat, q, c


def _t(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


@pytest.mark.parametrize("n", [1, 300, 4099])
def test_gradient_matches_oracle(bc, n):
    """n = 300 and 4099: several 128-pair blocks and a ragged last block."""
    P, feat, q, c = _batch(n, seed=n)
    grad = torch.empty(M.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    bc.mlp_grad(_t(P), _t(feat), _t(q), _t(c), grad, loss)
    ref_loss, ref = M.loss_and_grad(P, feat, q, c)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - ref_loss) <= 1e-4 * ref_loss
    scale = np.abs(ref).max()
    assert np.abs(g - ref).max() <= 2e-4 * scale, np.abs(g - ref).max() / scale
    for lo, hi in ((0, 768), (768, 832), (832, 4928), (4928, 4992), (4992, 6016), (6016, 6032)):
        r = ref[lo:hi]
        assert np.linalg.norm(g[lo:hi] - r) <= 1e-3 * np.linalg.norm(r) + 1e-7 * scale, (lo, hi)


def test_predict_matches_oracle_forward(bc):
    P, feat, q, c = _batch(1000, seed=9)
    out = torch.empty(1000, dtype=torch.float32, device="cuda")
    bc.mlp_predict(_t(P), _t(feat), _t(q), out)
    ref = M.forward(P, feat, q)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def test_adam_step(bc):
    rng = np.random.default_rng(3)
    p = rng.standard_normal(M.N_PARAMS).astype(np.float32)
    g = rng.standard_normal(M.N_PARAMS).astype(np.float32)
    m1 = rng.standard_normal(M.N_PARAMS).astype(np.float32) * 0.1
    m2 = rng.random(M.N_PARAMS).astype(np.float32) * 0.1
    P, G, A, B = _t(p), _t(g), _t(m1), _t(m2)
    bc.mlp_adam(P, G, A, B, 3, 1e-3, 0.9, 0.999, 1e-8)
    # the kernel's coefficients are FP32 numbers: beta as stored, 1 - beta in FP32
    b1, b2 = float(np.float32(0.9)), float(np.float32(0.999))
    c1, c2 = float(np.float32(1) - np.float32(0.9)), float(np.float32(1) - np.float32(0.999))
    a = b1 * m1.astype(np.float64) + c1 * g
    b = b2 * m2.astype(np.float64) + c2 * g.astype(np.float64) ** 2
    ref = p - 1e-3 * (a / (1 - b1 ** 3)) / (np.sqrt(b / (1 - b2 ** 3)) + 1e-8)
    assert np.abs(P.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    # FP32 moment updates: rounding relative to the largest moment (cancellation near 0)
    assert np.abs(A.cpu().numpy() - a).max() <= 1e-6 * np.abs(a).max()
    assert np.abs(B.cpu().numpy() - b).max() <= 1e-6 * np.abs(b).max()


@pytest.mark.parametrize("task", ["vtv", "vtb", "btv"])
def test_training_data_matches_oracle(bc, task):
    m = cube_bc_mesh(0.25, 0.125)
    ctx = bc.Context.from_mesh(m, p=2, precision="fp32", near_mode="none")
    st = ctx.stats()[task]
    assert 0 < st["near_singular"] < st["near_pairs"]
    d = ctx.mlp_dataset(task, 5000)
    n = d["chat"].shape[0]
    assert n == min(5000, st["near_singular"])
    pairs = d["pairs"].cpu().numpy()
    feat, qhat, chat = (d[k].cpu().numpy().astype(np.float64) for k in ("feat", "qhat", "chat"))
    tv = m.verts[m.tris] if task == "vtb" else m.verts[m.tets]
    sv = m.verts[m.tris] if task == "btv" else m.verts[m.tets]
    rng = np.random.default_rng(0)
    for i in rng.choice(n, size=min(n, 40), replace=False):
        t, s = tv[pairs[i, 0]], sv[pairs[i, 1]]
        # near-singular: the two elements share no vertex (closures apart)
        assert np.min(np.linalg.norm(t[:, None] - s[None], axis=2)) > 0
        f_ref, q_ref, Q = M.pair_features(t, s)
        assert np.abs(feat[i] - f_ref).max() <= 1e-5 * max(1.0, np.abs(f_ref).max())
        assert np.abs(qhat[i] - q_ref).max() <= 1e-6
        c_ref = (O.near_pair(task, t, s) - Q) / Q
        assert abs(chat[i] - c_ref) <= 1e-6 * abs(c_ref) + 1e-9, (i, chat[i], c_ref)


def test_learned_correction_gain(bc):
    """Train on random BC meshes (not the evaluation mesh), then evaluate
    VtV on a graded cube: the learned correction must remove at least 60 %
    of the near-singular error the product rule alone leaves, and the
    learned form must stay within 1e-6 of the direct definition O1.  All three contexts
    share the tree and expansions (FP64, p = 8), so their differences are
    the near-singular corrections alone."""
    from paper_2112_00864_gb300 import learned
    blob, rep = learned.train_blob(tasks=("vtv",), seeds=range(1, 9), pairs_per_task=400_000, steps=20000,
                                   max_h_index=2)
    assert rep["vtv"]["rms_err"] < 0.4 * rep["vtv"]["rms_chat"], rep
    m = cube_bc_mesh(1 / 8, 1 / 16)
    f = densities(m, "sine")[0]
    out = {}
    for mode in ("fp64", "learned", "none"):
        kw = dict(mlp_blob=blob, mlp_tol=5e-3) if mode == "learned" else {}
        ctx = bc.Context.from_mesh(m, p=8, leaf_size=64, precision="fp64", near_mode=mode, **kw)
        ctx.set_density(bc.VOLUME, f)
        out[mode] = (ctx.eval_vtv().cpu().numpy()[0], ctx.stats())
    vol = O.element_volumes(m)
    ref = out["fp64"][0] / vol
    err = {k: np.linalg.norm(out[k][0] / vol - ref) / np.linalg.norm(ref) for k in ("learned", "none")}
    st = out["learned"][1]["vtv"]
    frac = st["near_learned"] / max(1, st["near_singular"])
    print("gain:", err, "learned fraction", frac, rep)
    assert frac > 0.5
    assert err["none"] > 1e-7
    assert err["learned"] <= 0.4 * err["none"], err
    # the FP64 near-mode context itself against the oracle's O1 on samples
    # (p = 8 truncation ~ 1e-8)
    idx = np.array([0, m.ntet // 3, m.ntet - 1])
    o1 = O.direct("vtv", m, f, targets=idx)[0] / vol[idx]
    assert np.abs(ref[idx] - o1).max() <= 1e-7 * np.abs(o1).max()
    # the learned form and the product rule alone against the direct
    # definition O1 on 96 sampled targets: the learned correction is an
    # approximation of the FP64 near rule (this small in-test network leaves
    # ~3e-6 against the FP64 form), so the bar is relative: against O1 too it
    # removes at least 60 % of what the product rule alone leaves, and it
    # stays below 1e-5
    idx = np.sort(np.random.default_rng(5).choice(m.ntet, 96, replace=False))
    o1 = O.direct("vtv", m, f, targets=idx)[0] / vol[idx]
    e1 = {k: np.linalg.norm(out[k][0][idx] / vol[idx] - o1) / np.linalg.norm(o1) for k in ("fp64", "learned", "none")}
    print("vs O1:", e1)
    assert e1["fp64"] <= 1e-7, e1
    assert e1["learned"] <= 0.4 * e1["none"], e1
    assert e1["learned"] <= 1e-5, e1
