"""Training of the learned near-singular correction, on the GPU.

Pipeline (every numeric step runs in the library's kernels; this module
only orders the calls and moves tensors):

1. Training meshes: random BC meshes (unit cubes with random boundary
   size, volume size and grading; graded unit balls), one per seed.
2. Pairs: each mesh is built with near_mode "none", which classifies its
   near pairs (touching -> FP64 near rule; near-singular -> listed) and
   ``Context.mlp_dataset`` returns evenly sampled near-singular pairs with
   features, normalised product-rule terms qhat and labels
   chat = (N - Q) / Q from the library's FP64 near rule.
3. Training: Adam (about 3e4 minibatch steps of 1024 pairs, cosine
   decay) on the mean squared error of sum_k dw_k qhat_k - chat,
   gradients from the library's backward kernel (``bcfmm.mlp_grad``),
   FP32 master weights, forward/backward on their BF16 roundings.
4. Calibration: on held-out pairs, the 99.9 % quantile of |prediction -
   chat| per geometric bin; bins with too few pairs get +inf (never used).
5. Blob: the format ``bcfmm_params.mlp_blob`` expects.  At build time a
   near-singular pair takes the learned correction only if its bin's
   calibrated error is <= mlp_tol, else the FP64 near rule.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import bcfmm
from .inputs import ball_bc_mesh, cube_bc_mesh

TASKS = ("vtv", "vtb", "btv")
N_PARAMS = 6032
N_BINS = 32
MAGIC = 0x4C4D4342


def training_meshes(seeds=range(1, 17), max_h_index: int = 3):
    """One random BC mesh per seed (cube or ball)."""
    out = []
    for s in seeds:
        rng = np.random.default_rng(s)
        if rng.integers(2) == 0:
            h = (1 / 4, 1 / 8, 1 / 16)[rng.integers(max_h_index)]
            hv = h if rng.integers(2) == 0 else h / 2
            grade = (0.35, 0.5)[rng.integers(2)]
            m = cube_bc_mesh(h_bnd=h, h_vol=hv, grade=grade)
        else:
            m = ball_bc_mesh(level=int(rng.integers(2, 4)), radial=(0.35, 0.5)[rng.integers(2)])
        out.append(m)
    return out


def collect(meshes, tasks, per_mesh: int):
    """Training data per task from the meshes: {task: dict of CUDA tensors}.
    Each mesh is built once (near_mode "none") and serves every task."""
    import torch
    parts = {t: [] for t in tasks}
    for m in meshes:
        ctx = bcfmm.Context.from_mesh(m, p=2, leaf_size=64, precision="fp32", near_mode="none")
        for t in tasks:
            if t != "vtv" and m.ntri == 0:
                continue
            d = ctx.mlp_dataset(t, per_mesh)
            parts[t].append({k: v.clone() for k, v in d.items() if k != "pairs"})
        ctx.close()
    return {t: {k: torch.cat([p[k] for p in parts[t]]) for k in ("feat", "qhat", "chat", "bin")} for t in tasks}


def init_params(seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, math.sqrt(2.0 / 12), (64, 12))
    W2 = rng.normal(0, math.sqrt(2.0 / 64), (64, 64))
    W3 = rng.normal(0, 0.1 * math.sqrt(1.0 / 64), (16, 64))
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), np.zeros(16)]).astype(
        np.float32)


def split(data: dict, val_frac: float = 0.1, seed: int = 0):
    import torch
    n = data["chat"].shape[0]
    perm = torch.as_tensor(np.random.default_rng(seed).permutation(n), device=data["chat"].device)
    nv = max(1, int(n * val_frac))
    val = {k: v[perm[:nv]].contiguous() for k, v in data.items()}
    tr = {k: v[perm[nv:]].contiguous() for k, v in data.items()}
    return tr, val


def train(data: dict, steps: int = 30000, batch: int = 1024, lr: float = 2e-3, seed: int = 0, verbose: bool = False):
    """Adam with a cosine learning-rate decay over ``steps`` minibatch steps
    (the data reshuffled once per epoch); returns (params, history)."""
    import torch
    dev = data["chat"].device
    params = torch.tensor(init_params(seed), device=dev)
    m1, m2 = torch.zeros_like(params), torch.zeros_like(params)
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    n = data["chat"].shape[0]
    batch = min(batch, n)
    nb = max(1, n // batch)
    rng = np.random.default_rng(seed + 1)
    step, hist = 0, []
    while step < steps:
        perm = torch.as_tensor(rng.permutation(n), device=dev)
        f_all, q_all, c_all = (data[k][perm].contiguous() for k in ("feat", "qhat", "chat"))
        for b in range(nb):
            if step >= steps:
                break
            sl = slice(b * batch, (b + 1) * batch)
            bcfmm.mlp_grad(params, f_all[sl], q_all[sl], c_all[sl], grad, loss)
            step += 1
            lr_t = lr * (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * step / steps)))
            bcfmm.mlp_adam(params, grad, m1, m2, step, lr_t)
        hist.append(float(loss.item()))
        if verbose:
            print(f"step {step}: last-batch loss {hist[-1]:.3e}", flush=True)
    return params, hist


def predict(params, data: dict):
    import torch
    out = torch.empty_like(data["chat"])
    bcfmm.mlp_predict(params, data["feat"], data["qhat"], out)
    return out


def calibrate(params, val: dict, quantile: float = 0.999, min_count: int = 64):
    """Per-bin calibrated error and a summary of the held-out errors."""
    pred = predict(params, val).cpu().numpy().astype(np.float64)
    chat = val["chat"].cpu().numpy().astype(np.float64)
    bins = val["bin"].cpu().numpy()
    err = np.abs(pred - chat)
    eps = np.full(N_BINS, np.inf, np.float32)
    for b in range(N_BINS):
        e = err[bins == b]
        if e.size >= min_count:
            eps[b] = np.quantile(e, quantile)
    summary = dict(n=int(err.size), rms_err=float(np.sqrt(np.mean(err ** 2))), rms_chat=float(np.sqrt(np.mean(chat ** 2))),
                   q999_err=float(np.quantile(err, 0.999)), q999_chat=float(np.quantile(np.abs(chat), 0.999)))
    return eps, summary


def pack_blob(nets: dict) -> bytes:
    """nets: {task: (params float32[6032], eps float32[32])}."""
    has = [1 if t in nets else 0 for t in TASKS]
    head = np.array([MAGIC, 1, N_PARAMS, N_BINS] + has + [0], np.uint32).tobytes()
    body = b""
    for t in TASKS:
        if t in nets:
            p, e = nets[t]
            body += np.asarray(p, np.float32).tobytes() + np.asarray(e, np.float32).tobytes()
        else:
            body += np.zeros(N_PARAMS, np.float32).tobytes() + np.full(N_BINS, np.inf, np.float32).tobytes()
    blob = head + body
    assert len(blob) == bcfmm.mlp_blob_size()
    return blob


def train_blob(tasks=TASKS, seeds=range(1, 17), pairs_per_task: int = 2_000_000, steps: int = 30000,
               batch: int = 1024, lr: float = 2e-3, max_h_index: int = 3, verbose: bool = False):
    """Full pipeline; returns (blob bytes, report dict)."""
    import torch
    meshes = training_meshes(seeds, max_h_index)
    nets, report = {}, {}
    t0 = time.time()
    alldata = collect(meshes, tasks, max(1, pairs_per_task // len(meshes)))
    torch.cuda.synchronize()
    data_s = time.time() - t0
    for t in tasks:
        data = alldata[t]
        t1 = time.time()
        tr, val = split(data)
        params, hist = train(tr, steps=steps, batch=batch, lr=lr, verbose=verbose)
        torch.cuda.synchronize()
        t2 = time.time()
        eps, summ = calibrate(params, val)
        nets[t] = (params.cpu().numpy(), eps)
        report[t] = dict(pairs=int(data["chat"].shape[0]), data_s=data_s, train_s=t2 - t1, steps=steps,
                         loss=hist[-1], bins_accepted_at_5e3=int(np.sum(eps <= 5e-3)), **summ)
        if verbose:
            print(t, report[t], flush=True)
    return pack_blob(nets), report
