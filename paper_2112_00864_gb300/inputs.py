"""Seeded synthetic boundary-concentrated (BC) meshes and densities.

This module only generates inputs: vertex coordinates, tetrahedra, boundary
triangles and P0 density coefficients.  It holds none of the method's
arithmetic (no quadrature, no kernel evaluation, no expansions), so both the
CUDA path and the CPU oracle can be fed from it.

Meshes follow the workloads of the paper's numerical section (Sec. 5): a BC
tetrahedral volume mesh whose element size grows with the distance to the
boundary (Sec. 2), plus a conforming, quasi-uniform triangle mesh of the
boundary surface (Sec. 1.2).

* ``cube_bc_mesh``: unit cube [0,1]^3.  Octree cells of size
  ``max(h_vol, grade * dist(cell, boundary))``, each hexahedron split into the
  six Kuhn tetrahedra sharing its main diagonal.  Boundary: every face an
  ``n x n`` grid of squares, each split into two triangles (n = 1/h_bnd).
* ``ball_bc_mesh``: unit ball.  Boundary: the icosphere obtained by ``level``
  midpoint subdivisions of the icosahedron.  Volume: spherical shells of
  triangular prisms over icosphere triangles, three tetrahedra per prism; the
  icosphere level drops by one inward where the BC size rule allows it.  At a
  level change the fine shell's inner vertices sit on the flat coarse
  triangles (hanging nodes, no gaps).  The core is a fan of tetrahedra from
  the origin.
* ``batch_meshes``: ragged batch of cube and ball meshes.
* densities: the P0 test functions used by the workloads.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    """A tetrahedral volume mesh with a triangulated boundary surface.

    verts: [nv, 3] float64; tets: [nt, 4] int32 (positively oriented);
    tris: [nf, 3] int32 (outward normal by the right-hand rule).
    """
    verts: np.ndarray
    tets: np.ndarray
    tris: np.ndarray
    name: str = ""
    info: dict = field(default_factory=dict)

    @property
    def ntet(self) -> int:
        return int(self.tets.shape[0])

    @property
    def ntri(self) -> int:
        return int(self.tris.shape[0])

    def tet_vertices(self) -> np.ndarray:
        return self.verts[self.tets]          # [nt, 4, 3]

    def tri_vertices(self) -> np.ndarray:
        return self.verts[self.tris]          # [nf, 3, 3]

    def tet_centroids(self) -> np.ndarray:
        return self.tet_vertices().mean(axis=1)

    def tri_centroids(self) -> np.ndarray:
        return self.tri_vertices().mean(axis=1)


# --------------------------------------------------------------------------
# cube
# --------------------------------------------------------------------------
_KUHN_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def _orient_tets(verts: np.ndarray, tets: np.ndarray) -> np.ndarray:
    p = verts[tets]
    d = np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])
    tets = tets.copy()
    neg = d < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


def cube_bc_mesh(h_bnd: float = 0.25, h_vol: float = 0.125, grade: float = 0.5,
                 max_level: int = 12) -> Mesh:
    """BC tet mesh of [0,1]^3 (octree cells + Kuhn split) and its boundary.

    A cell of size s at octree level l is split while
    s > max(h_vol, grade * d), d = distance from the cell to the cube surface.
    """
    nb = int(round(1.0 / h_bnd))
    assert abs(nb * h_bnd - 1.0) < 1e-12, "1/h_bnd must be an integer"
    lv = np.zeros(1, np.int64)
    ijk = np.zeros((1, 3), np.int64)
    leaves_l, leaves_ijk = [], []
    for level in range(max_level + 1):
        if ijk.shape[0] == 0:
            break
        s = 2.0 ** (-level)
        lo = ijk * s
        hi = lo + s
        d = np.minimum(lo, 1.0 - hi).min(axis=1)
        target = np.maximum(h_vol, grade * d)
        split = (s > target * (1 + 1e-12)) & (level < max_level)
        leaves_l.append(np.full(int((~split).sum()), level))
        leaves_ijk.append(ijk[~split])
        par = ijk[split]
        kids = (2 * par[:, None, :] + np.array([[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1]
                                                 for c in range(8)])[None]).reshape(-1, 3)
        ijk = kids
    L = np.concatenate(leaves_l)
    C = np.concatenate(leaves_ijk)
    fine = int(max(L.max(), math.ceil(math.log2(nb))))
    scale = 2 ** (fine - L)                       # cell size in finest units
    base = C * scale[:, None]
    corners = []
    for perm in _KUHN_PERMS:
        e = np.eye(3, dtype=np.int64)
        v0 = np.zeros(3, np.int64)
        v1 = e[perm[0]]
        v2 = v1 + e[perm[1]]
        v3 = np.ones(3, np.int64)
        corners.append(np.stack([v0, v1, v2, v3]))
    corners = np.stack(corners)                   # [6, 4, 3]
    tv = base[:, None, None, :] + corners[None] * scale[:, None, None, None]   # [nc, 6, 4, 3]
    tv = tv.reshape(-1, 3)
    # boundary triangles on the same integer grid
    tri_pts = []
    g = 2 ** fine // nb
    for axis in range(3):
        for side in (0, 1):
            a1, a2 = [a for a in range(3) if a != axis]
            for i in range(nb):
                for j in range(nb):
                    def P(di, dj):
                        p = np.zeros(3, np.int64)
                        p[axis] = side * 2 ** fine
                        p[a1] = (i + di) * g
                        p[a2] = (j + dj) * g
                        return p
                    q00, q10, q11, q01 = P(0, 0), P(1, 0), P(1, 1), P(0, 1)
                    tri_pts.append(np.stack([q00, q10, q11]))
                    tri_pts.append(np.stack([q00, q11, q01]))
    tri_pts = np.stack(tri_pts).reshape(-1, 3)
    allp = np.concatenate([tv, tri_pts])
    uniq, inv = np.unique(allp, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    verts = uniq.astype(np.float64) / float(2 ** fine)
    tets = inv[: tv.shape[0]].reshape(-1, 4).astype(np.int32)
    tris = inv[tv.shape[0]:].reshape(-1, 3).astype(np.int32)
    tets = _orient_tets(verts, tets).astype(np.int32)
    # outward triangle normals
    tp = verts[tris]
    n = np.cross(tp[:, 1] - tp[:, 0], tp[:, 2] - tp[:, 0])
    out = tp.mean(axis=1) - 0.5
    flip = np.einsum("ij,ij->i", n, out) < 0
    tris = tris.copy()
    tris[flip, 1], tris[flip, 2] = tris[flip, 2].copy(), tris[flip, 1].copy()
    return Mesh(verts, tets, tris.astype(np.int32), name=f"cube_h{nb}",
                info={"h_bnd": h_bnd, "h_vol": h_vol, "grade": grade, "cells": int(L.size)})


# --------------------------------------------------------------------------
# ball
# --------------------------------------------------------------------------
def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], np.int64)
    return v, f


def _icosphere_levels(level: int):
    """Icosphere hierarchy.  Returns per level (unit vertices, faces,
    parent pair of every vertex: (a, a) for vertices inherited from the
    coarser level, (a, b) for the midpoint of coarse edge a-b)."""
    v, f = _icosahedron()
    out = [(v.copy(), f.copy(), np.stack([np.arange(len(v))] * 2, axis=1))]
    for _ in range(level):
        nv = len(v)
        edges = np.sort(np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]]), axis=1)
        ue, inv = np.unique(edges, axis=0, return_inverse=True)
        inv = inv.reshape(3, -1)
        mid = v[ue[:, 0]] + v[ue[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        m01, m12, m20 = nv + inv[0], nv + inv[1], nv + inv[2]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate([np.stack([a, m01, m20], 1), np.stack([b, m12, m01], 1),
                            np.stack([c, m20, m12], 1), np.stack([m01, m12, m20], 1)])
        parent = np.concatenate([np.stack([np.arange(nv)] * 2, 1), ue])
        v = np.concatenate([v, mid])
        out.append((v.copy(), f.copy(), parent))
    return out


def ball_bc_mesh(level: int = 4, radial: float = 0.5, grade: float = 0.5,
                 core_radius: float = 0.12) -> Mesh:
    """BC tet mesh of the unit ball bounded by the level-``level`` icosphere.

    Shell thickness = radial * (tangential edge length of the current
    icosphere level at that radius).  The level drops by one inward once
    2 * edge(level) <= max(h, grade * depth), h = surface edge length.
    """
    levels = _icosphere_levels(level)
    mean_edge = []
    for (v, f, _) in levels:
        e = np.linalg.norm(v[f[:, 0]] - v[f[:, 1]], axis=1)
        mean_edge.append(float(e.mean()))
    h = mean_edge[level]
    verts = []
    vcount = 0
    tets = []

    def add_verts(p):
        nonlocal vcount
        verts.append(p)
        idx = np.arange(vcount, vcount + len(p))
        vcount += len(p)
        return idx

    # surfaces are stored as (positions of the level's vertices, level)
    lv = level
    r = 1.0
    v_unit, faces, _ = levels[lv]
    outer_idx = add_verts(v_unit * r)
    bnd_idx = outer_idx
    while True:
        edge = mean_edge[lv] * r
        depth = 1.0 - r
        target = max(h, grade * depth)
        if lv > 0 and 2.0 * edge <= target:
            # coarsen: the fine shell below has its inner face on the flat
            # coarse triangles.  Build that shell now.
            t = radial * edge
            r_in = r - t
            v_c, f_c, _ = levels[lv - 1]
            _, _, parent = levels[lv]
            inner_pos = 0.5 * (v_c[parent[:, 0]] + v_c[parent[:, 1]]) * r_in
            inner_idx = add_verts(inner_pos)
            tets.append(_prism_tets(faces, outer_idx, inner_idx))
            # the coarse level continues from the coarse vertices at r_in
            lv -= 1
            v_unit, faces, _ = levels[lv]
            outer_idx = inner_idx[: len(v_unit)]
            r = r_in
            continue
        t = radial * edge
        r_in = r - t
        if r_in < core_radius:
            break
        inner_idx = add_verts(v_unit * r_in)
        tets.append(_prism_tets(faces, outer_idx, inner_idx))
        outer_idx = inner_idx
        r = r_in
    # core: fan from the origin to the current surface
    o = add_verts(np.zeros((1, 3)))
    core = np.concatenate([outer_idx[faces], np.full((len(faces), 1), o[0])], axis=1)
    tets.append(core)
    V = np.concatenate(verts)
    T = np.concatenate(tets).astype(np.int64)
    T = _orient_tets(V, T)
    tris = bnd_idx[levels[level][1]].astype(np.int64)
    tp = V[tris]
    n = np.cross(tp[:, 1] - tp[:, 0], tp[:, 2] - tp[:, 0])
    flip = np.einsum("ij,ij->i", n, tp.mean(axis=1)) < 0
    tris[flip, 1], tris[flip, 2] = tris[flip, 2].copy(), tris[flip, 1].copy()
    return Mesh(V, T.astype(np.int32), tris.astype(np.int32), name=f"ball_l{level}",
                info={"level": level, "radial": radial, "grade": grade, "h": h})


def _prism_tets(faces: np.ndarray, outer_idx: np.ndarray, inner_idx: np.ndarray) -> np.ndarray:
    """Split each prism (outer triangle over inner triangle) into three tets.
    Quad faces are cut from the lowest-numbered outer vertex to the next
    inner vertex, a rule neighbours share, so the split is conforming."""
    f = np.sort(faces, axis=1)                   # icosphere vertex ids, ascending
    a, b, c = f[:, 0], f[:, 1], f[:, 2]
    A, B, C = outer_idx[a], outer_idx[b], outer_idx[c]
    A2, B2, C2 = inner_idx[a], inner_idx[b], inner_idx[c]
    t1 = np.stack([A, B, C, C2], 1)
    t2 = np.stack([A, B, B2, C2], 1)
    t3 = np.stack([A, A2, B2, C2], 1)
    return np.concatenate([t1, t2, t3])


# --------------------------------------------------------------------------
# batches and densities
# --------------------------------------------------------------------------
def batch_meshes(n: int = 64, seed: int = 0, hs=(1 / 8, 1 / 16, 1 / 32)):
    """Ragged batch: kind in {cube, ball} and h in ``hs``, uniformly drawn."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        kind = "cube" if rng.integers(2) == 0 else "ball"
        h = float(hs[rng.integers(len(hs))])
        if kind == "cube":
            m = cube_bc_mesh(h_bnd=h, h_vol=h)
        else:
            lev = max(1, int(round(np.log2(1.0 / h))) - 1)      # 1/8 -> 2, 1/16 -> 3, 1/32 -> 4
            m = ball_bc_mesh(level=lev)
        m.info["h_req"] = h
        out.append(m)
    return out


def f_sine(x: np.ndarray) -> np.ndarray:
    """1 + sin(pi x) sin(pi y) sin(pi z)."""
    return 1.0 + np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 2])


def f_gauss(x: np.ndarray, c=(0.5, 0.5, 0.5), a: float = 0.05) -> np.ndarray:
    """exp(-|x-c|^2 / a)."""
    d = x - np.asarray(c)[None]
    return np.exp(-np.einsum("ij,ij->i", d, d) / a)


def g_cos(x: np.ndarray) -> np.ndarray:
    """cos(2 pi x) cos(2 pi y) cos(2 pi z)."""
    return np.cos(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1]) * np.cos(2 * np.pi * x[:, 2])


def gaussian_bumps(x: np.ndarray, rng: np.random.Generator, lo, hi, inside, nb: int = 8) -> np.ndarray:
    """Sum of ``nb`` Gaussian bumps: centres uniform in the box [lo,hi]
    (rejected if ``inside(c)`` is false), widths U[0.1,0.3], amplitudes N(0,1)."""
    f = np.zeros(x.shape[0])
    k = 0
    while k < nb:
        c = rng.uniform(lo, hi, size=3)
        if not inside(c):
            continue
        w = rng.uniform(0.1, 0.3)
        a = rng.normal()
        d = x - c[None]
        f += a * np.exp(-np.einsum("ij,ij->i", d, d) / w ** 2)
        k += 1
    return f


def densities(mesh: Mesh, kind: str, ndens: int = 1, seed: int = 0):
    """P0 coefficients at element centroids: (f [ndens, ntet], g [ndens, ntri])."""
    xc, xt = mesh.tet_centroids(), mesh.tri_centroids()
    if kind == "sine":
        f, g = f_sine(xc), f_sine(xt)
        return np.tile(f, (ndens, 1)), np.tile(g, (ndens, 1))
    if kind == "one":
        return np.ones((ndens, mesh.ntet)), np.ones((ndens, mesh.ntri))
    if kind == "gauss":
        return np.tile(f_gauss(xc), (ndens, 1)), np.tile(g_cos(xt), (ndens, 1))
    if kind == "bumps":
        rng = np.random.default_rng(seed)
        lo, hi = mesh.verts.min(axis=0), mesh.verts.max(axis=0)
        if mesh.name.startswith("ball"):
            inside = lambda c: float(np.dot(c, c)) < 1.0
        else:
            inside = lambda c: True
        F = np.stack([gaussian_bumps(xc, rng, lo, hi, inside) for _ in range(ndens)])
        G = np.stack([gaussian_bumps(xt, rng, lo, hi, inside) for _ in range(ndens)])
        return F, G
    if kind == "random":
        rng = np.random.default_rng(seed)
        return rng.standard_normal((ndens, mesh.ntet)), rng.standard_normal((ndens, mesh.ntri))
    raise ValueError(kind)
