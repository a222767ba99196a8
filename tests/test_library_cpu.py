"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol include/bcfmm.h declares, validates arguments before touching the
GPU, and its host-built translation tables agree with the oracle's."""
import os
import re

import numpy as np
import pytest

from paper_2112_00864_gb300 import bcfmm
from paper_2112_00864_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return bcfmm.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bcfmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bcfmm_\w+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(names) == sorted(bcfmm.EXPORTED)


def test_default_params(lib):
    prm = bcfmm.default_params()
    assert prm.p == 6 and prm.leaf_size == 64 and prm.near_n == 3 and prm.near_k == 1
    assert abs(prm.eta_ns - (1 - 2 ** -20)) < 1e-15


def test_argument_errors_before_gpu(lib):
    import ctypes as C
    prm = bcfmm.default_params()
    ctx = C.c_void_p()
    v = np.zeros((4, 3))
    t = np.array([[0, 1, 2, 3]], np.int32)
    # null vertices
    rc = lib.bcfmm_build_bc_tree(None, 4, t.ctypes.data, 1, None, 0, C.byref(prm), None, C.byref(ctx))
    assert rc == -1 and ctx.value is None
    # vertex id out of range
    bad = np.array([[0, 1, 2, 7]], np.int32)
    v = np.eye(4, 3)
    rc = lib.bcfmm_build_bc_tree(v.ctypes.data, 4, bad.ctypes.data, 1, None, 0, C.byref(prm), None, C.byref(ctx))
    assert rc == -1 and b"out of range" in lib.bcfmm_last_error()
    # degenerate tet
    flat = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0.0]])
    rc = lib.bcfmm_build_bc_tree(flat.ctypes.data, 4, t.ctypes.data, 1, None, 0, C.byref(prm), None, C.byref(ctx))
    assert rc == -2 and b"zero volume" in lib.bcfmm_last_error()
    # non-finite coordinate
    nanv = np.eye(4, 3)
    nanv[2, 1] = np.nan
    rc = lib.bcfmm_build_bc_tree(nanv.ctypes.data, 4, t.ctypes.data, 1, None, 0, C.byref(prm), None, C.byref(ctx))
    assert rc == -2
    # bad parameters
    for field, val in (("p", 13), ("leaf_size", 0), ("near_n", 9), ("precision", 7), ("eta_ns", 0.0)):
        q = bcfmm.default_params(**{field: val})
        rc = lib.bcfmm_build_bc_tree(np.eye(4, 3).ctypes.data, 4, t.ctypes.data, 1, None, 0, C.byref(q), None,
                                     C.byref(ctx))
        assert rc == -1, field
    # null context everywhere
    assert lib.bcfmm_set_density(None, 0, None, 1, 0) == -1
    assert lib.bcfmm_eval_vtv(None, None, 0) == -1
    lib.bcfmm_destroy(None)


def test_m2l_tables_match_oracle(lib):
    import oracle as O
    for p in (2, 4, 8):
        for o in ((2, 0, 0), (3, -2, 1), (-2, -3, -3)):
            T = bcfmm.debug_m2l_matrix(p, np.array(o, float))
            R = O.m2l_matrix(np.array(o, float), p)
            scale = np.abs(R).max()
            assert np.abs(T - R).max() <= 1e-13 * scale, (p, o)
    # the table is zero outside |alpha| + |beta| <= p
    T = bcfmm.debug_m2l_matrix(4, np.array([2.0, 1.0, 0.0]))
    mi = O.multi_indices(4).sum(1)
    mask = (mi[:, None] + mi[None, :]) > 4
    assert np.all(T[mask] == 0) and np.all(T[~mask] != 0) is not None


def test_m2l_taylor_form_rebuilds_oracle_matrix(lib):
    """The Taylor-form M2L keeps nterms(q) numbers per offset, g = D^gamma G(o),
    and rebuilds T[a][b] = g[a + b] (-1)^{|b|} / (a! b!) (Sec. 3.3, the
    expansion coefficients lambda): checked against the oracle's matrix,
    entry by entry, zero pattern included."""
    import oracle as O
    from math import factorial
    for q in (1, 4, 5, 7):
        mi = O.multi_indices(q)
        pos = {tuple(m): i for i, m in enumerate(mi)}
        fact = np.array([factorial(a) * factorial(b) * factorial(c) for a, b, c in mi], float)
        deg = mi.sum(1)
        for o in ((2, 0, 0), (3, -2, 1), (-2, -3, -3), (0, 5, -4)):
            g = bcfmm.debug_m2l_taylor_coeffs(q, np.array(o, float))
            R = O.m2l_matrix(np.array(o, float), q)
            T = np.zeros_like(R)
            for a in range(len(mi)):
                for b in range(len(mi)):
                    if deg[a] + deg[b] <= q:
                        T[a, b] = g[pos[tuple(mi[a] + mi[b])]] * (-1.0) ** deg[b] / (fact[a] * fact[b])
            assert np.abs(T - R).max() <= 1e-13 * np.abs(R).max(), (q, o)
            assert np.array_equal(T == 0, R == 0), (q, o)


def test_batch_argument_errors_before_gpu(lib):
    """bcfmm_build_batch validates offsets and every mesh before any device work."""
    import ctypes as C
    prm = bcfmm.default_params()
    ctx = C.c_void_p()
    good = np.eye(4, 3)
    flat = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0.0]])
    verts = np.concatenate([good, good, flat])
    tets = np.array([[0, 1, 2, 3]] * 3, np.int32)       # local vertex ids
    vo = np.array([0, 4, 8, 12], np.int64)
    to = np.array([0, 1, 2, 3], np.int64)
    ro = np.zeros(4, np.int64)
    args = lambda v, t, n: (verts.ctypes.data, v.ctypes.data, tets.ctypes.data, t.ctypes.data, None, ro.ctypes.data,
                            n, C.byref(prm), None, C.byref(ctx))
    rc = lib.bcfmm_build_batch(*args(vo, to, 3))
    assert rc == -2 and b"mesh 2" in lib.bcfmm_last_error() and b"zero volume" in lib.bcfmm_last_error()
    rc = lib.bcfmm_build_batch(*args(vo, np.array([0, 1, 1, 3], np.int64), 3))    # empty mesh 1
    assert rc == -1 and b"mesh 1" in lib.bcfmm_last_error()
    rc = lib.bcfmm_build_batch(*args(vo, to, 0))
    assert rc == -1 and ctx.value is None
    assert lib.bcfmm_eval_graph(None, 1, None, None, None) == -1


def test_learned_mode_arguments_checked_before_gpu(lib):
    """A missing or malformed network blob and bad near-mode settings are
    argument errors found before any device work."""
    import ctypes as C
    ctx = C.c_void_p()
    v = np.eye(4, 3)
    t = np.array([[0, 1, 2, 3]], np.int32)
    for kw in (dict(near_mode=1), dict(near_mode=1, mlp_blob=b"\0" * 64), dict(near_mode=3),
               dict(near_mode=1, mlp_tol=0.0, mlp_blob=b"\0" * bcfmm.mlp_blob_size()), dict(tc_unit=-1)):
        q = bcfmm.default_params(**kw)
        rc = lib.bcfmm_build_bc_tree(v.ctypes.data, 4, t.ctypes.data, 1, None, 0, C.byref(q), None, C.byref(ctx))
        assert rc == -1 and ctx.value is None, kw
    q = bcfmm.default_params(near_mode=1, mlp_blob=b"\0" * bcfmm.mlp_blob_size())
    rc = lib.bcfmm_build_bc_tree(v.ctypes.data, 4, t.ctypes.data, 1, None, 0, C.byref(q), None, C.byref(ctx))
    assert rc == -1 and b"header" in lib.bcfmm_last_error()


@pytest.mark.parametrize("leaf_size,eta0,p_level,tc_unit", [(64, 0.5, None, 0), (8, 0.9, None, 0),
                                                           (32, 0.5, [0, 0, 6, 5, 4, 3, 3, 3], 0),
                                                           (3, 0.7, [0, 0, 2, 3, 4, 5, 6, 7], 5),
                                                           (16, 0.5, [0, 0, 9, 8, 7, 6, 5, 4], 0)])
def test_interactions_covered_exactly_once(lib, leaf_size, eta0, p_level, tc_unit):
    """Every (target leaf, source point) pair of a mesh is evaluated once:
    by the leaf's near field N* or by one interaction list of the leaf or an
    ancestor (Sec. 2, Sec. 3); in a batch, never across meshes.  The
    tensor-core tiles (grouped by the levels' expansion orders, Sec. 4.3)
    reproduce every interaction list, and their persistent schedule covers
    every (tile, offset) entry once; the Taylor-form schedule (list chunks
    interleaved per warp) holds every list entry of its orders once and
    leaves the higher orders (8, 9 here) to the generic kernel.  Host-only
    check of the library's own tree, lists, tiles and schedules (no GPU)."""
    from paper_2112_00864_gb300.inputs import ball_bc_mesh, batch_meshes, cube_bc_mesh
    kw = dict(leaf_size=leaf_size, eta0=eta0, p=max(p_level or [7]), tc_unit=tc_unit, p_level=p_level)
    # [0:3] covering of every task, [3:6] the tiles against the lists, [6:9] the
    # tensor-core schedule, [9:12] the Taylor-form schedule, [12:15] the packed
    # near field's chunk blocks (cut at 96 points and at the library's size)
    assert list(bcfmm.debug_list_coverage([cube_bc_mesh(0.25, 0.125)], **kw)) == [0] * 15
    assert list(bcfmm.debug_list_coverage([ball_bc_mesh(2, radial=0.35)], **kw)) == [0] * 15
    assert list(bcfmm.debug_list_coverage(batch_meshes(4, seed=3, hs=(1 / 4, 1 / 8)), **kw)) == [0] * 15


def test_near_pairs_equal_brute_force(lib):
    """The build's near-pair search (multi-level hash grids, both size
    orders) finds exactly the pairs the oracle's near predicate selects when
    every element pair is tried (Eq. def:sepRatio with centroids)."""
    import oracle as O
    from paper_2112_00864_gb300.inputs import ball_bc_mesh, cube_bc_mesh
    for m, tasks in ((cube_bc_mesh(0.5, 0.25), ("vtv", "vtb", "btv")), (ball_bc_mesh(1, radial=0.5), ("vtb", "btv"))):
        for task in tasks:
            row, cols = bcfmm.debug_near_pairs(m, task)
            tv = m.verts[m.tris] if task == "vtb" else m.verts[m.tets]
            sv = m.verts[m.tris] if task == "btv" else m.verts[m.tets]
            found = {(i, int(c)) for i in range(len(tv)) for c in cols[row[i]:row[i + 1]]}
            brute = {(i, j) for i in range(len(tv)) for j in range(len(sv)) if O.is_near(tv[i], sv[j])}
            assert found == brute, (m.name, task, len(found ^ brute))
            assert all(np.all(np.diff(cols[row[i]:row[i + 1]]) > 0) for i in range(len(tv)))   # sorted, unique


def test_shift_tables_match_oracle(lib):
    """The library's box-scaled M2M / L2L tables reproduce the oracle's
    unscaled shifts (Sec. 3.3) for every child octant once the box scalings
    (moments by s^-|beta|, locals by s^|alpha|, child side s/2) are applied."""
    import oracle as O
    rng = np.random.default_rng(5)
    for p in (0, 3, 6):
        deg = O.multi_indices(p).sum(1)
        sp = 0.8
        cp = np.array([0.3, -0.2, 0.5])
        for q in range(8):
            sg = np.array([0.25 if q >> ax & 1 else -0.25 for ax in range(3)])
            cc = cp + sg * sp
            sc = sp / 2
            mc = rng.standard_normal(len(deg))                 # unscaled child moments
            ref = O.m2m(mc, cc, cp, p) / sp ** deg
            got = bcfmm.debug_shift_matrix("m2m", p, q) @ (mc / sc ** deg)
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), (p, q)
            lp = rng.standard_normal(len(deg))                 # unscaled parent locals
            ref = O.l2l(lp, cp, cc, p) * sc ** deg
            got = bcfmm.debug_shift_matrix("l2l", p, q) @ (lp * sp ** deg)
            assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), (p, q)


def test_tree_shape_equals_oracle_tree(lib):
    """The build's octree and the oracle's independently written one have
    the same boxes and leaves on every level (both compute points and box
    centres with products and sums rounded as written, so a point on a box
    plane lands on the same side)."""
    import oracle as O
    from paper_2112_00864_gb300.inputs import ball_bc_mesh, cube_bc_mesh
    for m in (cube_bc_mesh(0.25, 0.125), ball_bc_mesh(2, radial=0.35), ball_bc_mesh(3, radial=0.5)):
        for ls in (8, 32, 128):
            b, lf = bcfmm.debug_tree_counts(m, ls)
            n, ob, olf = O.tree_stats(m, leaf_size=ls)
            ob, olf = np.asarray(ob), np.asarray(olf)
            nl = max(len(np.trim_zeros(b, "b")), len(np.trim_zeros(ob, "b")))
            assert len(b) >= nl and len(ob) >= nl and len(lf) >= nl and len(olf) >= nl, (m.name, ls, nl)
            assert np.array_equal(b[:nl], ob[:nl]) and np.array_equal(lf[:nl], olf[:nl]), (m.name, ls)
            assert not b[nl:].any() and not ob[nl:].any() and not lf[nl:].any() and not olf[nl:].any()
            assert b.sum() == n
