"""GPU parity of the C-ABI library against the FP64 CPU oracle.

Plain FP64 path vs O2 (same tree parameters): rel L2 <= 1e-10.
Chosen FP32 path vs O2 at the same p (precision error only) and vs O1
(truncation + precision) at an order that resolves 1e-6: rel L2 <= 1e-6.
Box neighbours use the paper's eta0 = 0.5 (Sec. 5) unless stated.
Norms are taken over cell averages u_t / |t|.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_00864_gb300.inputs import ball_bc_mesh, cube_bc_mesh, densities

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


def rel(a, b, size):
    a, b = np.asarray(a) / size, np.asarray(b) / size
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module")
def c1():
    m = cube_bc_mesh(0.25, 0.125)
    f, g = densities(m, "sine")
    return m, f, g


def _sizes(m, task):
    return O.element_areas(m) if task == "vtb" else O.element_volumes(m)


@pytest.mark.parametrize("task", ["vtv", "vtb", "btv"])
def test_fp64_matches_oracle_fmm(bc, c1, task):
    m, f, g = c1
    dens = g if task == "btv" else f
    ctx = bc.Context.from_mesh(m, p=4, leaf_size=64, precision="fp64")
    ctx.set_density(bc.BOUNDARY if task == "btv" else bc.VOLUME, dens)
    u = ctx.eval(task).cpu().numpy()
    ref = O.fmm(task, m, dens, p=4, leaf_size=64)
    r2, rm = rel(u, ref, _sizes(m, task))
    assert r2 <= 1e-10 and rm <= 1e-10, (r2, rm)


@pytest.mark.parametrize("task", ["vtv", "vtb", "btv"])
def test_fp32_matches_oracle(bc, c1, task):
    m, f, g = c1
    dens = g if task == "btv" else f
    kind = bc.BOUNDARY if task == "btv" else bc.VOLUME
    ctx = bc.Context.from_mesh(m, p=8, leaf_size=64, precision="fp32")
    ctx.set_density(kind, dens)
    u = ctx.eval(task).cpu().numpy()
    direct = O.direct(task, m, dens)
    r2, rm = rel(u, direct, _sizes(m, task))
    assert r2 <= 1e-6, (r2, rm)
    ref = O.fmm(task, m, dens, p=8, leaf_size=64)
    r2, rm = rel(u, ref, _sizes(m, task))
    assert r2 <= 1e-6, (r2, rm)


@pytest.mark.parametrize("prec,task", [("bf16x2", "vtv"), ("bf16x2", "vtb"),
                                       ("bf16x3", "vtv"), ("bf16x3", "vtb"), ("bf16x3", "btv")])
def test_tensor_core_m2l_matches_oracle(bc, c1, prec, task):
    """tcgen05 M2L (BF16 split, FP32 accumulation, compensated window sums)
    against O2 at the same p (precision error only) and O1.  The hi+lo split
    (16 significant bits per operand) holds 1e-6 for volume sources; surface
    sources (BtV) need the hi+mid+lo split."""
    m, f, g = c1
    dens = g if task == "btv" else f
    kind = bc.BOUNDARY if task == "btv" else bc.VOLUME
    ctx = bc.Context.from_mesh(m, p=6, leaf_size=64, precision=prec)
    ctx.set_density(kind, dens)
    u = ctx.eval(task).cpu().numpy()
    assert ctx.stats()["device_error"] == 0
    ref = O.fmm(task, m, dens, p=6, leaf_size=64)
    r2, rm = rel(u, ref, _sizes(m, task))
    assert r2 <= 1e-6, (r2, rm)
    r2, rm = rel(u, O.direct(task, m, dens), _sizes(m, task))
    assert r2 <= 1e-6, (r2, rm)


@pytest.mark.parametrize("p,prec", [(2, "bf16x2"), (3, "bf16x2"), (4, "bf16x2"), (5, "bf16x2"), (7, "bf16x2"),
                                    (2, "bf16x3"), (4, "bf16x3"), (5, "bf16x3")])
def test_tensor_core_m2l_every_order(bc, c1, p, prec):
    """Every padded width of the tensor-core M2L (16, 32, 48, 64, 96, 128
    columns for p = 2..7) against the FP64 path at the same p: the
    difference is the split-precision error alone.  Surface sources (BtV)
    need the 3-term split, as at p = 6; the 2-term split is checked on the
    volume-source tasks."""
    m, f, g = c1
    legs = ((("vtv", f, bc.VOLUME), ("vtb", f, bc.VOLUME)) if prec == "bf16x2" else
            (("vtv", f, bc.VOLUME), ("btv", g, bc.BOUNDARY)))
    for task, dens, kind in legs:
        u = {}
        for pr in (prec, "fp64"):
            ctx = bc.Context.from_mesh(m, p=p, leaf_size=32, precision=pr)
            ctx.set_density(kind, dens)
            u[pr] = ctx.eval(task).cpu().numpy()
            assert ctx.stats()["device_error"] == 0
        r2, rm = rel(u[prec], u["fp64"], _sizes(m, task))
        assert r2 <= 1e-6, (task, p, prec, r2, rm)


def test_multiple_densities_and_device_io(bc, c1):
    m, f, g = c1
    rng = np.random.default_rng(7)
    F = np.concatenate([f, rng.standard_normal((2, m.ntet))])          # 3 densities, padded to 4
    ctx = bc.Context.from_mesh(m, p=4, precision="fp64")
    ctx.set_density(bc.VOLUME, torch.tensor(F, device="cuda"))
    out = torch.zeros((3, m.ntet), dtype=torch.float64, device="cuda")
    ctx.eval_vtv(out)
    host = np.zeros((3, m.ntet))
    ctx.eval_vtv(host)
    assert np.array_equal(out.cpu().numpy(), host)
    for d in range(3):
        one = bc.Context.from_mesh(m, p=4, precision="fp64")
        one.set_density(bc.VOLUME, F[d])
        assert np.abs(one.eval_vtv().cpu().numpy()[0] - host[d]).max() <= 1e-13 * np.abs(host[d]).max()


def test_state_errors(bc, c1):
    m, f, g = c1
    ctx = bc.Context.from_mesh(m, p=2)
    with pytest.raises(bc.BcfmmError) as e:
        ctx.eval_vtv()
    assert e.value.code == -6
    with pytest.raises(bc.BcfmmError):
        ctx.set_density(bc.VOLUME, np.full((1, m.ntet), np.nan))
    with pytest.raises(bc.BcfmmError):
        ctx.set_density(bc.VOLUME, np.ones((17, m.ntet)))


def test_degenerate_meshes(bc):
    # one tet, no triangles: every pair is near (self pair only)
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    t = np.array([[0, 1, 2, 3]], np.int32)
    from paper_2112_00864_gb300.inputs import Mesh
    m = Mesh(v, t, np.zeros((0, 3), np.int32))
    ctx = bc.Context(v, t, None, p=4)
    ctx.set_density(bc.VOLUME, np.array([[2.0]]))
    u = ctx.eval_vtv().cpu().numpy()
    ref = O.direct("vtv", m, np.array([[2.0]]))
    assert abs(u[0, 0] / ref[0, 0] - 1) < 1e-12
    with pytest.raises(bc.BcfmmError):
        ctx.set_density(bc.BOUNDARY, np.ones((1, 1)))
    with pytest.raises(bc.BcfmmError):
        ctx.eval_btv()
    # tiny leaves: many levels, ragged last leaves
    m = cube_bc_mesh(0.5, 0.25)
    f, g = densities(m, "random", seed=3)
    ctx = bc.Context.from_mesh(m, p=3, leaf_size=5, precision="fp64")
    ctx.set_density(bc.VOLUME, f)
    u = ctx.eval_vtv().cpu().numpy()
    ref = O.fmm("vtv", m, f, p=3, leaf_size=5)
    r2, rm = rel(u, ref, O.element_volumes(m))
    assert r2 <= 1e-10, r2


def test_ball_full_size_sampled(bc):
    """Config-2 workload (unit ball, 5120 boundary triangles, ~1.9e5 tets)
    in the benchmark's launch configuration (the chosen form: BF16x2
    tensor-core M2L, the paper's order schedule q0 = 4 capped at p = 7,
    eta0 = 0.5; VtV + VtB through one CUDA graph) against O1 on 512
    sampled target elements per task: rel L2 <= 5e-7."""
    import bench
    m = ball_bc_mesh(4, radial=0.35)
    f = np.ones((1, m.ntet))
    ctx = bc.Context.from_mesh(m, **bench.CHOSEN)
    ctx.set_density(bc.VOLUME, torch.tensor(f, device="cuda"))
    outs = ctx.eval_graph(("vtv", "vtb"))
    assert ctx.stats()["device_error"] == 0
    rng = np.random.default_rng(11)
    for task, nel, size in (("vtv", m.ntet, O.element_volumes(m)), ("vtb", m.ntri, O.element_areas(m))):
        u = outs[task].cpu().numpy()[0]
        idx = np.sort(rng.choice(nel, 512, replace=False))
        ref = O.direct(task, m, f, targets=idx)[0]
        r2, rm = rel(u[idx], ref, size[idx])
        assert r2 <= 5e-7, (task, r2, rm)
