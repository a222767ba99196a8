"""Autotuner: pick the fastest evaluation configuration that meets an
accuracy target on the caller's own meshes and densities.

Search space (all of it is cheap to try because ``Context.build_like``
copies the near pairs and their FP64 corrections instead of recomputing
them): leaf size, the box-neighbour parameter eta0 (Eq. def:neighbors: the
near-field / interaction-list trade-off), the level-order schedule
q_l = min(p, q0 + L - l) of Sec. 4.3, and the M2L form: FP32 Taylor form on
CUDA cores, or the tensor-core BF16 hi+lo split (orders <= 6 on the tensor
cores) with its work-unit size ("tile" of the M2L launch: interaction
entries per CTA).  Each candidate is timed with CUDA events as the graph
launch a user makes (``Context.eval_graph``) and its error is measured on
sampled target elements against the library's FP64 direct evaluation of
the discrete operator (``Context.direct_sample``), as the relative L2
error of cell averages.  The winner is the fastest candidate whose error
is at most ``safety * tol`` for every task (the sample stands for meshes
and targets the tuner did not see; the margin covers that).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

from . import bcfmm

DEFAULT_SPACE = dict(leaf_size=(64, 128), eta0=(0.5, 0.6, 0.7), q0=(4, 5, 6, 7), p=7,
                     tc_space=dict(eta0=(0.5,), q0=(4, 5), tc_unit=(0, 32)))


@dataclass
class Trial:
    params: dict
    ms: float = float("nan")
    err: dict = field(default_factory=dict)
    ok: bool = False
    note: str = ""


def candidates(space: dict | None = None):
    """FP32 Taylor-form candidates over leaf x eta0 x q0, then the
    tensor-core ones over leaf x the (smaller) tc_space."""
    space = dict(DEFAULT_SPACE, **(space or {}))
    p = int(space["p"])
    out = []
    for ls, eta0, q0 in itertools.product(space["leaf_size"], space["eta0"], space["q0"]):
        out.append(dict(leaf_size=int(ls), eta0=float(eta0), q0=int(q0), p=p, precision="fp32"))
    tcs = space.get("tc_space") or {}
    for ls, eta0, q0, u in itertools.product(space["leaf_size"], tcs.get("eta0", ()), tcs.get("q0", ()),
                                             tcs.get("tc_unit", (0,))):
        out.append(dict(leaf_size=int(ls), eta0=float(eta0), q0=int(q0), p=p, precision="bf16x2", tc_unit=int(u)))
    return out


def _cell_sizes(ctx, task: str) -> np.ndarray:
    if task == "vtb":
        v = ctx.element_vertices(bcfmm.BOUNDARY)
        return 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1)
    v = ctx.element_vertices(bcfmm.VOLUME)
    return np.abs(np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])) / 6.0


def _time_graph(ctx, tasks, outs, reps: int) -> float:
    import torch
    st = torch.cuda.current_stream()
    outs = ctx.eval_graph(tasks, outs)                  # capture
    for _ in range(2):
        ctx.eval_graph(tasks, outs)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
    ms = []
    for r in range(reps):
        ev[2 * r].record(st)
        ctx.eval_graph(tasks, outs)
        ev[2 * r + 1].record(st)
    torch.cuda.synchronize()
    for r in range(reps):
        ms.append(ev[2 * r].elapsed_time(ev[2 * r + 1]))
    return float(np.median(ms))


def autotune(base: "bcfmm.Context", dens_volume, dens_boundary=None, tasks=("vtv", "vtb"), tol: float = 1e-6,
             space: dict | None = None, nsample: int = 64, reps: int = 5, seed: int = 0, safety: float = 0.5,
             verbose: bool = False, timer=None):
    """Returns (best params dict, list of Trial).  ``base`` is any context on
    the meshes (its near pairs are reused); densities as for set_density.
    ``timer(ctx, tasks, reps) -> ms`` replaces the CUDA-event timing of the
    graph launches (default) when given."""
    timer = timer or (lambda c, t, r: _time_graph(c, t, None, r))
    rng = np.random.default_rng(seed)
    base.set_density(bcfmm.VOLUME, dens_volume)
    if dens_boundary is not None:
        base.set_density(bcfmm.BOUNDARY, dens_boundary)
    refs = {}
    for t in tasks:
        n = base.ntri if t == "vtb" else base.ntet
        idx = np.sort(rng.choice(n, size=min(nsample, n), replace=False))
        size = _cell_sizes(base, t)[idx]
        refs[t] = (idx, base.direct_sample(t, idx) / size, size)
    trials = []
    for cand in candidates(space):
        tr = Trial(params=cand)
        try:
            ctx = base.build_like(**cand)
            ctx.set_density(bcfmm.VOLUME, dens_volume)
            if dens_boundary is not None:
                ctx.set_density(bcfmm.BOUNDARY, dens_boundary)
            tr.ms = timer(ctx, tasks, reps)
            outs = ctx.eval_graph(tasks)
            for t in tasks:
                idx, ref, size = refs[t]
                u = outs[t].cpu().numpy()[:, idx] / size
                tr.err[t] = float(np.linalg.norm(u - ref) / np.linalg.norm(ref))
            tr.ok = all(e <= safety * tol for e in tr.err.values())
            ctx.close()
        except bcfmm.BcfmmError as ex:
            tr.note = str(ex)
        if verbose:
            print(f"autotune {cand} ms={tr.ms:.3f} err={tr.err} ok={tr.ok} {tr.note}", flush=True)
        trials.append(tr)
    good = [t for t in trials if t.ok]
    if not good:
        raise RuntimeError(f"autotune: no configuration reaches {safety:g} * tol = {safety * tol:g}")
    best = min(good, key=lambda t: t.ms)
    return dict(best.params), trials
