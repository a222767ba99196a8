"""The synthetic input recipe: the meshes every configuration runs on.

Checks of geometry that do not depend on the method: positive orientation
and tiling (volumes sum to the domain's), boundary triangles that cover the
domain's surface with outward normals, the boundary triangle counts the
configurations state, and the ragged batch's size range.
"""
import numpy as np

from paper_2112_00864_gb300.inputs import (ball_bc_mesh, batch_meshes, cube_bc_mesh, densities,
                                           gaussian_bumps)


def _signed_volumes(m):
    v = m.tet_vertices()
    return np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0]) / 6


def _tri_normals(m):
    v = m.tri_vertices()
    return 0.5 * np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])


def test_cube_meshes_tile_the_unit_cube():
    for h_bnd, h_vol, nt_expect, nf_expect in ((0.25, 0.125, 3072, 192), (1 / 8, 1 / 8, 3072, 768),
                                                (1 / 16, 1 / 16, 21888, 3072)):
        m = cube_bc_mesh(h_bnd, h_vol)
        vol = _signed_volumes(m)
        assert np.all(vol > 0), "tets positively oriented"
        assert abs(vol.sum() - 1.0) < 1e-12
        assert m.ntet == nt_expect and m.ntri == nf_expect      # 6 faces x 2 / h^2 boundary triangles
        n = _tri_normals(m)
        assert abs(np.linalg.norm(n, axis=1).sum() - 6.0) < 1e-12
        c = m.tri_centroids()
        # outward: the normal points away from the cube centre
        assert np.all(np.einsum("ij,ij->i", n, c - 0.5) > 0)
        # divergence theorem: sum over the boundary of (x . n) / 3 = volume
        assert abs(np.einsum("ij,ij->i", c, n).sum() / 3 - 1.0) < 1e-12


def test_ball_mesh_fills_the_icosphere_polyhedron():
    m = ball_bc_mesh(3, radial=0.35)
    vol = _signed_volumes(m)
    assert np.all(vol > 0)
    n = _tri_normals(m)
    c = m.tri_centroids()
    assert m.ntri == 20 * 4 ** 3
    assert np.all(np.einsum("ij,ij->i", n, c) > 0)
    poly = np.einsum("ij,ij->i", c, n).sum() / 3        # volume enclosed by the boundary
    assert abs(vol.sum() - poly) < 1e-13 * poly
    assert np.allclose(np.linalg.norm(m.tri_vertices().reshape(-1, 3), axis=1), 1.0, atol=1e-14)
    assert m.ntri == 1280 and 2e4 < m.ntet < 1e5
    m4 = ball_bc_mesh(4, radial=0.35)
    assert m4.ntri == 5120 and 1.5e5 < m4.ntet < 2.5e5       # "~2e5 tets" of the ball configuration


def test_batch_sizes_and_densities():
    meshes = batch_meshes(64, seed=0)
    sizes = np.array([m.ntet for m in meshes])
    assert len(meshes) == 64 and sizes.min() >= 1e3 and sizes.max() <= 2e5
    kinds = {m.name.split("_")[0] for m in meshes}
    hs = {m.info["h_req"] for m in meshes}
    assert kinds == {"cube", "ball"} and hs == {1 / 8, 1 / 16, 1 / 32}
    assert batch_meshes(3, seed=4)[1].ntet == batch_meshes(3, seed=4)[1].ntet     # seeded
    f, g = densities(meshes[0], "bumps", ndens=4, seed=7)
    assert f.shape == (4, meshes[0].ntet) and g.shape == (4, meshes[0].ntri)
    assert np.all(np.isfinite(f)) and not np.allclose(f[0], f[1])


def test_gaussian_bumps_definition():
    rng = np.random.default_rng(1)
    x = np.array([[0.5, 0.5, 0.5], [0.0, 0.0, 0.0], [0.9, 0.1, 0.4]])
    f = gaussian_bumps(x, rng, np.zeros(3), np.ones(3), lambda c: True, nb=1)
    rng = np.random.default_rng(1)
    c = rng.uniform(np.zeros(3), np.ones(3), size=3)
    w = rng.uniform(0.1, 0.3)
    a = rng.normal()
    assert np.allclose(f, a * np.exp(-((x - c) ** 2).sum(1) / w ** 2), rtol=1e-15)
