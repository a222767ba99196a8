"""Batched evaluation of independent meshes and the CUDA-graph entry point.

A batch is the paper's computation for every mesh on its own (no
interaction between meshes), run as one forest so that each stage is one
launch over all meshes.  Per mesh, the batch must reproduce the CPU FMM
oracle O2 (same p, leaf size and eta0) and the single-mesh contexts; the
graph entry point must reproduce the per-task entry points.
Norms are taken over cell averages u_t / |t|.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_00864_gb300.inputs import batch_meshes, densities

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


@pytest.fixture(scope="module")
def small_batch():
    """Ragged batch of cubes and balls at h in {1/4, 1/8}, 2 bump densities each."""
    meshes = batch_meshes(n=5, seed=3, hs=(1 / 4, 1 / 8))
    F, G = [], []
    for i, m in enumerate(meshes):
        f, g = densities(m, "bumps", ndens=2, seed=100 + i)
        F.append(f)
        G.append(g)
    return meshes, F, G


def rel(a, b, size):
    a, b = np.asarray(a) / size, np.asarray(b) / size
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max()


def _sizes(m, task):
    return O.element_areas(m) if task == "vtb" else O.element_volumes(m)


def _batch_ctx(bc, meshes, F, G, **kw):
    ctx = bc.Context.from_meshes(meshes, **kw)
    ctx.set_density(bc.VOLUME, np.concatenate(F, axis=1))
    ctx.set_density(bc.BOUNDARY, np.concatenate(G, axis=1))
    return ctx


def test_batch_forest_shape(bc, small_batch):
    meshes, F, G = small_batch
    ctx = _batch_ctx(bc, meshes, F, G, p=4, leaf_size=32, precision="fp64")
    st = ctx.stats()
    assert st["nmesh"] == len(meshes)
    assert st["ntet"] == sum(m.ntet for m in meshes) and st["ntri"] == sum(m.ntri for m in meshes)
    # every mesh has its own root
    assert st["boxes_per_level"][0] == len(meshes)
    kinds = {m.name.split("_")[0] for m in meshes}
    assert kinds == {"cube", "ball"}, kinds


@pytest.mark.parametrize("task", ["vtv", "vtb", "btv"])
def test_batch_fp64_matches_oracle_per_mesh(bc, small_batch, task):
    meshes, F, G = small_batch
    ctx = _batch_ctx(bc, meshes, F, G, p=4, leaf_size=32, precision="fp64")
    u = ctx.eval(task).cpu().numpy()
    parts = ctx.split(u, task)
    for m, f, g, um in zip(meshes, F, G, parts):
        dens = g if task == "btv" else f
        ref = O.fmm(task, m, dens, p=4, leaf_size=32)
        for d in range(dens.shape[0]):
            r2, rm = rel(um[d], ref[d], _sizes(m, task))
            assert r2 <= 1e-10 and rm <= 1e-10, (m.name, d, r2, rm)


@pytest.mark.parametrize("task", ["vtv", "vtb", "btv"])
def test_batch_equals_single_mesh_contexts(bc, small_batch, task):
    """Same kernels, same per-mesh lists: only the tensor-core tiles and
    work units mix meshes, which changes the FP32 summation order of the
    interaction phase, so the batch agrees with one context per mesh to
    FP32 rounding (2^-24 ~ 6e-8 per operation, amplified where the bump
    densities cancel), well inside the 1e-6 parity bar."""
    meshes, F, G = small_batch
    kw = dict(p=6, leaf_size=64, precision="bf16x3")
    ctx = _batch_ctx(bc, meshes, F, G, **kw)
    parts = ctx.split(ctx.eval(task).cpu().numpy(), task)
    for m, f, g, um in zip(meshes, F, G, parts):
        one = bc.Context.from_mesh(m, **kw)
        one.set_density(bc.VOLUME, f)
        one.set_density(bc.BOUNDARY, g)
        u1 = one.eval(task).cpu().numpy()
        r2, rm = rel(um, u1, _sizes(m, task))
        assert r2 <= 5e-7 and rm <= 1e-6, (m.name, r2, rm)


def test_graph_matches_eval(bc, small_batch):
    meshes, F, G = small_batch
    ctx = _batch_ctx(bc, meshes, F, G, p=6, leaf_size=64, precision="bf16x2")
    ref = {t: ctx.eval(t).cpu().numpy() for t in ("vtv", "vtb", "btv")}
    size_b = np.concatenate([_sizes(m, "vtb") for m in meshes])

    def check(outs, ref):
        # VtV and BtV run the same launches as the per-task calls; VtB takes
        # VtV's local expansions, whose tensor-core tiles sum in another
        # FP32 order than VtB's own, so it agrees to FP32 rounding
        for t in ("vtv", "btv"):
            if t in ref:
                np.testing.assert_array_equal(outs[t].cpu().numpy(), ref[t])
        r2, rm = rel(outs["vtb"].cpu().numpy(), ref["vtb"], size_b)
        assert r2 <= 5e-7 and rm <= 1e-6, (r2, rm)

    outs = None
    for _ in range(2):                              # capture, then replay
        outs = ctx.eval_graph(("vtv", "vtb", "btv"), outs)
        torch.cuda.synchronize()
        check(outs, ref)
    # new density values, same sizes: the replayed graph reads them
    F2 = [np.flip(f, axis=0).copy() * 0.5 for f in F]
    ctx.set_density(bc.VOLUME, np.concatenate(F2, axis=1))
    ref2 = {t: ctx.eval(t).cpu().numpy() for t in ("vtv", "vtb")}
    outs = ctx.eval_graph(("vtv", "vtb", "btv"), outs)
    torch.cuda.synchronize()
    check(outs, ref2)
    assert ctx.stats()["device_error"] == 0


def test_graph_rejects_misuse(bc, small_batch):
    meshes, F, G = small_batch
    ctx = bc.Context.from_meshes(meshes[:2], p=4, precision="fp32")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(bc.BcfmmError) as e:
        ctx.eval_graph(("vtv",), {"vtv": out})      # no density yet
    assert e.value.code == -6
    import ctypes
    rc = ctx._lib.bcfmm_eval_graph(ctx._ctx, 0, None, None, None)
    assert rc == -1
    rc = ctx._lib.bcfmm_eval_graph(ctx._ctx, 8, None, None, None)
    assert rc == -1
    ctx.set_density(bc.VOLUME, np.concatenate([np.ones((1, m.ntet)) for m in meshes[:2]], axis=1))
    rc = ctx._lib.bcfmm_eval_graph(ctx._ctx, 1, None, None, None)   # null output
    assert rc == -1
    del ctypes
