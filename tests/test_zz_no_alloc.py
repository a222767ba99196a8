"""bcfmm_eval_noalloc: the no-allocation evaluation entry point.

It serves callers that must not call the CUDA allocator during an
evaluation (a host framework that owns and budgets all device memory, or a
latency-critical loop where cudaMalloc/cudaFree could synchronise the
device).  Its interaction phase (tensor cores or the Taylor form) keeps its
partial sums in the library's fixed static device array instead of context
scratch.  Its
results must match the ordinary entry points on the same context, for two
calls in a row (the shared array keeps the previous call's contents).
This file is collected last on purpose.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("prec", ["bf16x2", "fp32"])
def test_eval_noalloc_matches_eval(bc, prec):
    from paper_2112_00864_gb300.inputs import cube_bc_mesh, densities
    m = cube_bc_mesh(0.25, 0.125)
    f, g = densities(m, "sine")
    ctx = bc.Context.from_mesh(m, p=6, leaf_size=64, precision=prec)
    f_dev = torch.tensor(f, device="cuda")
    g_dev = torch.tensor(g, device="cuda")
    ctx.set_density(bc.VOLUME, f_dev)
    ctx.set_density(bc.BOUNDARY, g_dev)
    for task, dens, n in (("vtv", f_dev, m.ntet), ("vtb", f_dev, m.ntri), ("btv", g_dev, m.ntet)):
        ref = ctx.eval(task)[0].cpu().numpy()
        for _ in range(2):
            out = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            ctx.eval_noalloc(task, dens[0].contiguous(), out)
            torch.cuda.synchronize()
            u = out.cpu().numpy()
            assert np.all(np.isfinite(u))
            err = np.linalg.norm(u - ref) / np.linalg.norm(ref)
            assert err <= 1e-12, (task, err)
    assert ctx.stats()["device_error"] == 0


def test_eval_noalloc_rejects_misuse(bc):
    from paper_2112_00864_gb300.inputs import cube_bc_mesh
    m = cube_bc_mesh(0.5, 0.25)
    f = torch.ones(m.ntet, dtype=torch.float64, device="cuda")
    out = torch.empty(m.ntet, dtype=torch.float64, device="cuda")
    plain = bc.Context.from_mesh(m, p=4, precision="fp64")
    plain.set_density(bc.VOLUME, f[None])
    with pytest.raises(bc.BcfmmError) as e:
        plain.eval_noalloc("vtv", f, out)
    assert e.value.code == -1
    tc = bc.Context.from_mesh(m, p=4, precision="bf16x2")
    with pytest.raises(bc.BcfmmError) as e:
        tc.eval_noalloc("vtv", f, out)         # no set_density yet
    assert e.value.code == -6


def test_eval_noalloc_expired_wait_shows_in_stats(bc):
    """The entry point does not synchronise, so an expired bounded wait of
    the tensor-core M2L is reported through the context's device error word
    (bcfmm_stats), and the next evaluation with host output returns
    BCFMM_ERR_TIMEOUT and clears it.  The expiry is made on purpose by the
    library's test hook (a bounded wait on a barrier that nothing
    completes); nothing faults or hangs."""
    from paper_2112_00864_gb300.inputs import cube_bc_mesh, densities
    m = cube_bc_mesh(0.5, 0.25)
    f = densities(m, "sine")[0]
    ctx = bc.Context.from_mesh(m, p=4, precision="bf16x2")
    f_dev = torch.tensor(f, device="cuda")
    ctx.set_density(bc.VOLUME, f_dev)
    ref = ctx.eval_vtv().cpu().numpy()[0]
    assert ctx._lib.bcfmm_debug_expire_wait(ctx._ctx, 1000) == 0
    out = torch.empty(m.ntet, dtype=torch.float64, device="cuda")
    ctx.eval_noalloc("vtv", f_dev[0].contiguous(), out)
    torch.cuda.synchronize()
    assert ctx.stats()["device_error"] == 1
    host = np.zeros((1, m.ntet))
    with pytest.raises(bc.BcfmmError) as e:
        ctx.eval_vtv(host)
    assert e.value.code == -5
    assert ctx.stats()["device_error"] == 0
    ctx.eval_noalloc("vtv", f_dev[0].contiguous(), out)
    u = out.cpu().numpy()
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= 1e-12
