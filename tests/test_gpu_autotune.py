"""The FP64 GPU direct evaluation, context rebuilds that reuse near pairs,
and the autotuner built on both.

The direct evaluation is the discrete operator summed pair by pair, the
same quantity as the oracle's O1, so the two agree to FP64 rounding.  The
autotuner's pick is then checked against O1 itself.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_00864_gb300.inputs import batch_meshes, cube_bc_mesh, densities

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
def c1():
    m = cube_bc_mesh(0.25, 0.125)
    f, g = densities(m, "sine")
    return m, f, g


@pytest.mark.parametrize("task", ["vtv", "vtb", "btv"])
def test_direct_sample_matches_oracle_direct(bc, c1, task):
    m, f, g = c1
    dens = np.concatenate([g, 0.5 * g]) if task == "btv" else np.concatenate([f, -f])
    ctx = bc.Context.from_mesh(m, p=2, precision="fp32")
    ctx.set_density(bc.BOUNDARY if task == "btv" else bc.VOLUME, dens)
    n = m.ntri if task == "vtb" else m.ntet
    idx = np.array([0, 1, n // 3, n // 2, n - 1], np.int64)
    u = ctx.direct_sample(task, idx)
    ref = O.direct(task, m, dens, targets=idx)
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max(), np.abs(u - ref).max()


def test_build_like_equals_fresh_build(bc, c1):
    m, f, g = c1
    base = bc.Context.from_mesh(m, p=4, leaf_size=64, precision="fp64")
    like = base.build_like(p=6, leaf_size=32)
    fresh = bc.Context.from_mesh(m, p=6, leaf_size=32, precision="fp64")
    for c in (like, fresh):
        c.set_density(bc.VOLUME, f)
        c.set_density(bc.BOUNDARY, g)
    for t in ("vtv", "vtb", "btv"):
        np.testing.assert_array_equal(like.eval(t).cpu().numpy(), fresh.eval(t).cpu().numpy())
    st = like.stats()
    assert st["p"] == 6 and st["leaf_size"] == 32
    with pytest.raises(bc.BcfmmError):
        base.build_like(eta_ns=0.5)


def test_autotune_pick_meets_tolerance(bc):
    from paper_2112_00864_gb300.autotune import autotune
    meshes = batch_meshes(n=4, seed=5, hs=(1 / 4, 1 / 8))
    F = np.concatenate([densities(m, "bumps", ndens=2, seed=i)[0] for i, m in enumerate(meshes)], axis=1)
    base = bc.Context.from_meshes(meshes, p=4, precision="fp32")
    tol = 1e-6
    space = dict(leaf_size=(32, 128), eta0=(0.5, 0.7), q0=(3, 6), tc_space=dict(eta0=(0.5,), q0=(4,), tc_unit=(0, 16)))
    best, trials = autotune(base, F, tasks=("vtv", "vtb"), tol=tol, space=space, nsample=48, reps=3)
    # per leaf size: FP32 Taylor form over eta0 x q0 (2 x 2), tensor cores 1 x 1 x 2 units
    assert len(trials) == 2 * (2 * 2 + 2)
    chosen = [t for t in trials if t.params == best][0]
    assert chosen.ok and chosen.ms == min(t.ms for t in trials if t.ok)
    # the pick against the oracle's O1 on sampled targets of every mesh
    ctx = base.build_like(**best)
    ctx.set_density(bc.VOLUME, F)
    outs = ctx.eval_graph(("vtv", "vtb"))
    for t in ("vtv", "vtb"):
        parts = ctx.split(outs[t].cpu().numpy(), t)
        dparts = ctx.split(F, bc.VOLUME)
        errs = []
        for m, u, f in zip(meshes, parts, dparts):
            n = m.ntri if t == "vtb" else m.ntet
            idx = np.unique(np.linspace(0, n - 1, 24).astype(np.int64))
            size = O.element_areas(m)[idx] if t == "vtb" else O.element_volumes(m)[idx]
            ref = O.direct(t, m, f, targets=idx) / size
            errs.append(np.linalg.norm(u[:, idx] / size - ref) / np.linalg.norm(ref))
        assert max(errs) <= tol, (t, errs)


def test_direct_sample_in_a_batch_sees_own_mesh_only(bc):
    meshes = batch_meshes(n=3, seed=2, hs=(1 / 4, 1 / 8))
    F = [densities(m, "bumps", ndens=1, seed=i)[0] for i, m in enumerate(meshes)]
    ctx = bc.Context.from_meshes(meshes, p=2, precision="fp32")
    ctx.set_density(bc.VOLUME, np.concatenate(F, axis=1))
    for t in ("vtv", "vtb"):
        off = ctx.tri_off if t == "vtb" else ctx.tet_off
        for mi, (m, f) in enumerate(zip(meshes, F)):
            n = m.ntri if t == "vtb" else m.ntet
            loc = np.array([0, n // 2, n - 1], np.int64)
            u = ctx.direct_sample(t, loc + off[mi])
            ref = O.direct(t, m, f, targets=loc)
            assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max(), (t, mi)
