"""Failure paths tested without faulting the GPU: an expired bounded device
wait reports BCFMM_ERR_TIMEOUT to the host and the context stays usable,
and near-singular pairs whose calibrated error is over the tolerance (or
that have no network) are routed to the FP64 near rule."""
import numpy as np
import pytest

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


def test_expired_wait_reports_timeout_and_context_recovers(bc):
    m = cube_bc_mesh(0.5, 0.25)
    f = densities(m, "sine")[0]
    ctx = bc.Context.from_mesh(m, p=4, precision="bf16x2")
    ctx.set_density(bc.VOLUME, f)
    ref = ctx.eval_vtv().cpu().numpy()
    assert ctx._lib.bcfmm_debug_expire_wait(ctx._ctx, 1000) == 0       # a wait that nothing completes
    host = np.zeros((1, m.ntet))
    with pytest.raises(bc.BcfmmError) as e:
        ctx.eval_vtv(host)
    assert e.value.code == -5                                          # BCFMM_ERR_TIMEOUT
    ctx.eval_vtv(host)                                                 # the error word was cleared
    np.testing.assert_array_equal(host, ref)
    assert ctx.stats()["device_error"] == 0
    assert ctx._lib.bcfmm_debug_expire_wait(ctx._ctx, 0) == -1


def test_learned_fallback_routing(bc):
    from paper_2112_00864_gb300 import learned
    m = cube_bc_mesh(0.25, 0.125)
    f = densities(m, "sine")[0]
    ref = bc.Context.from_mesh(m, p=4, precision="fp64")
    ref.set_density(bc.VOLUME, f)
    u_ref = {t: ref.eval(t).cpu().numpy() for t in ("vtv", "vtb")}
    P = learned.init_params(0)
    cases = ((np.full(32, np.inf), 5e-3, "none"),       # no bin calibrated: everything falls back
             (np.full(32, 1e-3), 1e-4, "none"),         # every bin over the tolerance
             (np.full(32, 1e-3), 5e-3, "all"))          # every bin accepted
    for eps, tol, expect in cases:
        blob = learned.pack_blob({"vtv": (P, eps.astype(np.float32))})
        ctx = bc.Context.from_mesh(m, p=4, precision="fp64", near_mode="learned", mlp_blob=blob, mlp_tol=tol)
        ctx.set_density(bc.VOLUME, f)
        st = ctx.stats()
        assert 0 < st["vtv"]["near_singular"] < st["vtv"]["near_pairs"]
        # VtB has no network in this blob: all of its near pairs stay on the FP64 rule
        assert st["vtb"]["near_learned"] == 0 and st["vtb"]["near_fp64"] == st["vtb"]["near_pairs"]
        np.testing.assert_array_equal(ctx.eval("vtb").cpu().numpy(), u_ref["vtb"])
        if expect == "none":
            assert st["vtv"]["near_learned"] == 0 and st["vtv"]["near_fp64"] == st["vtv"]["near_pairs"]
            np.testing.assert_array_equal(ctx.eval("vtv").cpu().numpy(), u_ref["vtv"])
        else:
            assert st["vtv"]["near_learned"] == st["vtv"]["near_singular"]
            assert st["vtv"]["near_fp64"] == st["vtv"]["near_pairs"] - st["vtv"]["near_singular"]
