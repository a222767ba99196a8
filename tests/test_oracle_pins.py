"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test ties one oracle function to a closed form, a textbook identity,
brute-force quadrature written here independently, or an invariant of the
method (Sec. 3.3 expansions, Eq. est:remain:G), so that a dropped term, a
sign or index error or a transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2112_00864_gb300.inputs import _KUHN_PERMS, ball_bc_mesh, cube_bc_mesh, densities


def kuhn_cube(lo=(0.0, 0.0, 0.0), s=1.0):
    e = np.eye(3)
    out = []
    for perm in _KUHN_PERMS:
        v1 = e[perm[0]]
        v2 = v1 + e[perm[1]]
        out.append(np.asarray(lo) + s * np.stack([np.zeros(3), v1, v2, np.ones(3)]))
    return out


def cuboid_potential(p, lo, hi):
    """Textbook closed form of int_box dy/|p-y| (corner sum of
    uv ln(w+r) - w^2/2 atan(uv/(wr)) over cyclic (u,v,w))."""
    def F(x, y, z):
        r = math.sqrt(x * x + y * y + z * z)
        def t(u, v, w):
            a = u * v * math.log(w + r) if (w + r) > 0 else 0.0
            b = 0.5 * w * w * math.atan(u * v / (w * r)) if w != 0 else 0.0
            return a - b
        return t(x, y, z) + t(y, z, x) + t(z, x, y)
    s = 0.0
    for i, xx in enumerate([hi[0] - p[0], lo[0] - p[0]]):
        for j, yy in enumerate([hi[1] - p[1], lo[1] - p[1]]):
            for k, zz in enumerate([hi[2] - p[2], lo[2] - p[2]]):
                s += (-1) ** (i + j + k) * F(xx, yy, zz)
    return s


def brute_tri(x, tri, n=120):
    """Collapsed tensor Gauss on the triangle (written here, independent)."""
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1), 0.5 * w
    u, v = np.meshgrid(g, g, indexing="ij")
    W = np.outer(w, w) * (1 - u)
    P = tri[0] + u[..., None] * (tri[1] - tri[0]) + ((1 - u) * v)[..., None] * (tri[2] - tri[0])
    area2 = np.linalg.norm(np.cross(tri[1] - tri[0], tri[2] - tri[0]))
    return float((W * area2 / np.linalg.norm(P - x, axis=-1)).sum())


# ---------------------------------------------------------------- quadrature
def test_element_rules_exact_for_degree_two():
    rng = np.random.default_rng(1)
    for _ in range(5):
        v = rng.standard_normal((4, 3))
        pts, w = O.tet_quad(v[None])
        vol = abs(np.linalg.det(v[1:] - v[0])) / 6
        S = v.sum(0)
        exact2 = vol / 20 * (v.T @ v + np.outer(S, S))      # int x x^T over a tet
        assert np.allclose(w.sum(), vol, rtol=1e-14)
        assert np.allclose((w[:, None] * pts).sum(0), vol * v.mean(0), rtol=1e-13)
        assert np.allclose(np.einsum("q,qi,qj->ij", w, pts, pts), exact2, rtol=1e-12, atol=1e-14)
        t = rng.standard_normal((3, 3))
        pts, w = O.tri_quad(t[None])
        ar = 0.5 * np.linalg.norm(np.cross(t[1] - t[0], t[2] - t[0]))
        S = t.sum(0)
        exact2 = ar / 12 * (t.T @ t + np.outer(S, S))       # int x x^T over a triangle
        assert np.allclose(w.sum(), ar, rtol=1e-14)
        assert np.allclose(np.einsum("q,qi,qj->ij", w, pts, pts), exact2, rtol=1e-12, atol=1e-14)
        # interior rule: no point on an edge
        bary = np.linalg.lstsq(np.vstack([t.T, np.ones(3)]), np.vstack([pts.T, np.ones(3)]), rcond=None)[0]
        assert bary.min() > 0.1


# ---------------------------------------------------------- closed forms
def test_triangle_potential_vs_brute_force():
    rng = np.random.default_rng(2)
    tri = rng.standard_normal((3, 3))
    for _ in range(6):
        x = 2.5 * rng.standard_normal(3)
        assert abs(O.tri_potential(x, tri) - brute_tri(x, tri)) < 1e-11
    c = tri.mean(0)
    x = c + 2.0 * (tri[0] - c)                     # in the plane, outside
    assert abs(O.tri_potential(x, tri) - brute_tri(x, tri, 300)) < 1e-10


def test_triangle_potential_at_vertex_equilateral():
    # at a vertex of an equilateral triangle of side a: (a sqrt3 / 2) ln 3
    a = 0.7
    tri = np.array([[0, 0, 0], [a, 0, 0], [a / 2, a * math.sqrt(3) / 2, 0.0]])
    assert abs(O.tri_potential(tri[0], tri) - a * math.sqrt(3) / 2 * math.log(3)) < 1e-14
    # at the centroid: 3 isosceles pieces with apex angle 120 deg, height a/(2 sqrt3)
    h = a / (2 * math.sqrt(3))
    exact = 3 * 2 * h * math.asinh(math.tan(math.pi / 3))
    assert abs(O.tri_potential(tri.mean(0), tri) - exact) < 1e-14


def test_tet_potential_vs_cuboid_closed_form():
    tets = kuhn_cube((0.2, -0.1, 0.3), 0.5)
    lo, hi = np.array([0.2, -0.1, 0.3]), np.array([0.7, 0.4, 0.8])
    for x in [(0.3, 0.0, 0.5), (0.45, 0.15, 0.55), (1.2, -0.6, 0.4), (0.2, 0.1, 0.5), (0.7, 0.4, 0.8)]:
        x = np.array(x)
        s = sum(O.tet_potential(x, t) for t in tets)
        assert abs(s - cuboid_potential(x, lo, hi)) < 1e-13 * max(1, abs(s))


def test_tet_potential_is_poisson_inside():
    # inside the tet, psi + 2 pi/3 |x|^2 is harmonic: discrete Laplacian of psi = -4 pi
    rng = np.random.default_rng(3)
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]) + 0.01 * rng.standard_normal((4, 3))
    x = v.mean(0)
    h = 1e-3
    lap = sum(O.tet_potential(x + h * e, v) + O.tet_potential(x - h * e, v) for e in np.eye(3))
    lap = (lap - 6 * O.tet_potential(x, v)) / h ** 2
    assert abs(lap + 4 * math.pi) < 1e-4


# ------------------------------------------------------------- near rule
def test_cube_self_energy():
    """int_C int_C dx dy/|x-y| for the unit cube, from the 36 Kuhn-tet pairs
    (near rule and adaptive), against the cuboid closed form integrated by
    tensor Gauss-Legendre here."""
    g, w = np.polynomial.legendre.leggauss(24)
    g, w = 0.5 * (g + 1), 0.5 * w
    ref = 0.0
    for i in range(24):
        for j in range(24):
            for k in range(24):
                ref += w[i] * w[j] * w[k] * cuboid_potential((g[i], g[j], g[k]), (0, 0, 0), (1, 1, 1))
    assert abs(ref - 1.8823126) < 2e-6            # mean inverse distance in the unit cube
    tets = kuhn_cube()
    rule = sum(O.near_pair("vtv", t, s) for t in tets for s in tets) * 4 * math.pi
    assert abs(rule / ref - 1) < 5e-5
    ad = sum(O.adaptive_pair("vtv", t, s, tol=1e-11, maxdepth=4) for t in tets for s in tets) * 4 * math.pi
    assert abs(ad / ref - 1) < 2e-6


def test_near_rule_vs_adaptive_and_far_limit():
    m = cube_bc_mesh(0.25, 0.125)
    T = m.verts[m.tets]
    c = T.mean(1)
    t0 = 100
    order = np.argsort(np.linalg.norm(c - c[t0], axis=1))
    for s in order[:30:6]:
        ref = O.adaptive_pair("vtv", T[t0], T[s], tol=1e-13, maxdepth=5)
        assert abs(O.near_pair("vtv", T[t0], T[s]) / ref - 1) < 3e-5
    # well separated pair: the smooth integrand is integrated to rounding
    s = order[-1]
    ref = O.adaptive_pair("vtv", T[t0], T[s], tol=1e-15, maxdepth=2)
    assert abs(O.near_pair("vtv", T[t0], T[s], n=5, k=1) / ref - 1) < 1e-10
    # BtV near rule against brute force of the triangle potential integrated over the tet
    tri = m.verts[m.tris][0]
    tet = T[np.argmin(np.linalg.norm(c - tri.mean(0), axis=1))]
    a = O.near_pair("btv", tet, tri, n=5, k=2)
    b = O.adaptive_pair("btv", tet, tri, tol=1e-13, maxdepth=5)
    assert abs(a / b - 1) < 1e-5


def test_is_near_threshold():
    t = kuhn_cube()[0]
    assert O.is_near(t, t)
    far = t + 10.0
    assert not O.is_near(t, far)
    # touching pairs (shared vertex) are always near
    for s in kuhn_cube((1.0, 1.0, 1.0)):
        assert O.is_near(t, s)


# -------------------------------------------------- expansions (Sec. 3.3)
def test_taylor_coefficients_vs_sympy_and_fd():
    sp = pytest.importorskip("sympy")
    X, Y, Z = sp.symbols("x y z")
    phi = 1 / sp.sqrt(X * X + Y * Y + Z * Z)
    r = np.array([0.3, -0.7, 1.1])
    b = O.taylor_b(r, 5)
    mi = O.multi_indices(5)
    for q, (a1, a2, a3) in enumerate(mi):
        expr = phi
        if a1:
            expr = sp.diff(expr, X, int(a1))
        if a2:
            expr = sp.diff(expr, Y, int(a2))
        if a3:
            expr = sp.diff(expr, Z, int(a3))
        d = float(expr.subs({X: r[0], Y: r[1], Z: r[2]}).evalf(30))
        fact = math.factorial(a1) * math.factorial(a2) * math.factorial(a3)
        assert abs(b[q] - (-1) ** (a1 + a2 + a3) * d / fact) < 1e-12 * max(1.0, abs(d / fact))
    # high orders: the Taylor series of 1/|r - h| with these coefficients
    bh = O.taylor_b(r, 16)
    mi = O.multi_indices(16)
    h = 0.05 * np.array([1.0, 2.0, -1.5])
    series = sum(bh[q] * np.prod(h ** mi[q]) for q in range(len(mi)))
    assert abs(series - 1 / np.linalg.norm(r - h)) < 1e-15


def test_m2m_l2l_polynomial_identities():
    rng = np.random.default_rng(4)
    p = 6
    pts = rng.uniform(-0.5, 0.5, (50, 3))
    w = rng.standard_normal(50)
    cc = np.array([0.1, -0.2, 0.05])
    cp = np.array([0.35, 0.05, -0.2])
    mc = O.p2m(pts, w, cc, p)
    assert np.allclose(O.m2m(mc, cc, cp, p), O.p2m(pts, w, cp, p), rtol=1e-12, atol=1e-13)
    loc = rng.standard_normal(O.nterms(p))
    lc = O.l2l(loc, cp, cc, p)
    for x in rng.uniform(-1, 1, (5, 3)):
        assert abs(O.l2p(lc, cc, p, x) - O.l2p(loc, cp, p, x)) < 1e-11


def test_single_source_m2l_remainder_bound():
    """P2M -> M2L -> L2P of one source equals G up to the Taylor remainder
    C/|r| (|h|/|r|)^(p+1) (Eq. est:remain:G), which falls geometrically."""
    x = np.array([0.11, -0.07, 0.05])
    y = np.array([2.0, 0.13, -0.09])
    ct, cs = np.zeros(3), np.array([2.0, 0.0, 0.0])
    r = ct - cs
    h = (x - ct) - (y - cs)
    ratio = np.linalg.norm(h) / np.linalg.norm(r)
    G = 1 / (4 * math.pi * np.linalg.norm(x - y))
    errs = []
    for p in range(1, 12):
        m = O.p2m(y[None], np.ones(1), cs, p)
        loc = O.m2l_matrix(r, p) @ m
        errs.append(abs(O.l2p(loc, ct, p, x) - G))
        assert errs[-1] <= 2.0 / (4 * math.pi * np.linalg.norm(r)) * ratio ** (p + 1) / (1 - ratio)
    assert errs[-1] < 1e-12 and errs[-1] < errs[2] * 1e-6


# --------------------------------------------------------- whole operator
def test_fmm_converges_to_direct_geometrically():
    m = cube_bc_mesh(0.25, 0.25)
    f, g = densities(m, "sine")
    u1 = O.direct("vtv", m, f)
    e = []
    for p in (2, 4, 6, 8):
        u2 = O.fmm("vtv", m, f, p=p, leaf_size=16)
        e.append(np.linalg.norm(u2 - u1) / np.linalg.norm(u1))
    assert e[0] > 5 * e[1] > 25 * e[2] > 125 * e[3]
    assert e[3] < 1e-6
    u1 = O.direct("btv", m, g)
    u2 = O.fmm("btv", m, g, p=10, leaf_size=16)
    assert np.linalg.norm(u2 - u1) / np.linalg.norm(u1) < 2e-6


def test_fmm_vtb_converges_to_direct_geometrically():
    """O2's triangle-target branch (VtB: tet sources, triangle targets,
    Algorithm 2) against O1: the truncation error falls geometrically in p
    (Eq. est:remain:G), so a slip in the triangle-target lists or the
    evaluation at triangle points fails here, on the CPU."""
    m = cube_bc_mesh(0.25, 0.25)
    f, g = densities(m, "sine")
    u1 = O.direct("vtb", m, f)
    e = []
    for p in (2, 4, 6, 8):
        u2 = O.fmm("vtb", m, f, p=p, leaf_size=16)
        e.append(np.linalg.norm(u2 - u1) / np.linalg.norm(u1))
    assert e[0] > 5 * e[1] > 25 * e[2] > 125 * e[3], e
    assert e[3] < 1e-6, e


def test_fmm_level_orders():
    """Level-dependent expansion orders (Sec. 4.3, Eq. def:q0; Sec. 5 uses
    q_l = 4 + L - l).  A schedule whose every entry equals p reproduces the
    uniform-order O2 bit for bit; with the paper's schedule the error
    against O1 falls geometrically as q0 grows; and raising only the
    coarse levels' orders changes the result by less than the error of the
    finest level's order (the coarse levels carry the larger orders)."""
    m = cube_bc_mesh(0.25, 0.25)
    f, g = densities(m, "sine")
    u1 = O.direct("vtv", m, f)
    _, st = O.fmm("vtv", m, f, p=4, leaf_size=16, return_stats=True)
    L = st["maxlevel"]
    a = O.fmm("vtv", m, f, p=6, leaf_size=16)
    b = O.fmm("vtv", m, f, p=6, leaf_size=16, p_level=[6] * 20)
    assert np.array_equal(a, b)
    e = []
    for q0 in (1, 2, 3, 4):
        q = O.paper_orders(q0, L)
        u2 = O.fmm("vtv", m, f, p=max(q), leaf_size=16, p_level=q)
        e.append(np.linalg.norm(u2 - u1) / np.linalg.norm(u1))
    assert e[0] > 4 * e[1] > 16 * e[2] > 64 * e[3], e
    # the finest level at order 2 carries most of the error: raising every
    # other level to order 8 removes only part of it
    q = [8] * 20
    q[L] = 2
    u3 = O.fmm("vtv", m, f, p=8, leaf_size=16, p_level=q)
    u4 = O.fmm("vtv", m, f, p=8, leaf_size=16, p_level=[2] * 20)
    e3 = np.linalg.norm(u3 - u1) / np.linalg.norm(u1)
    e4 = np.linalg.norm(u4 - u1) / np.linalg.norm(u1)
    assert e3 < e4, (e3, e4)


def test_galerkin_symmetry_and_transpose():
    m = cube_bc_mesh(0.25, 0.25)
    rng = np.random.default_rng(5)
    f1, f2 = rng.standard_normal((2, m.ntet))
    u1 = O.direct("vtv", m, f1)[0]
    a, b = f2 @ u1, f1 @ O.direct("vtv", m, f2)[0]
    scale = np.linalg.norm(f2) * np.linalg.norm(u1)
    assert abs(a - b) / scale < 1e-6                       # exact for far pairs; near rule accuracy
    g = rng.standard_normal(m.ntri)
    ub = O.direct("vtb", m, f1)[0]
    a, b = g @ ub, f1 @ O.direct("btv", m, g)[0]
    assert abs(a - b) / (np.linalg.norm(g) * np.linalg.norm(ub)) < 2e-5    # two different near rules


def test_cube_total_and_ball_closed_form():
    # f = 1: sum_t u_t -> int int G over the cube = 1.8823126/(4 pi)
    m = cube_bc_mesh(0.25, 0.25)
    u = O.direct("vtv", m, np.ones(m.ntet))[0]
    assert abs(u.sum() * 4 * math.pi / 1.8823126 - 1) < 2e-3
    # unit ball, f = 1: u = (3 - r^2)/6 inside, 1/3 on the sphere (O(h^2) on the polyhedron)
    b = ball_bc_mesh(2, radial=0.5)
    vol = O.element_volumes(b)
    tgt = np.arange(0, b.ntet, 97)
    u = O.direct("vtv", b, np.ones(b.ntet), targets=tgt)[0] / vol[tgt]
    pts, w = O.tet_quad(b.verts[b.tets[tgt]])
    exact = (w * (3 - (pts ** 2).sum(1)) / 6).reshape(-1, 4).sum(1) / vol[tgt]
    assert np.abs(u - exact).max() < 0.02
    area = O.element_areas(b)
    ub = O.direct("vtb", b, np.ones(b.ntet), targets=np.arange(0, b.ntri, 7))[0] / area[::7]
    assert np.abs(ub - 1 / 3).max() < 0.02
    # single layer of g = 1 on the sphere equals 1 inside (to O(h^2))
    ui = O.direct("btv", b, np.ones(b.ntri), targets=tgt)[0] / vol[tgt]
    assert np.abs(ui - 1).max() < 0.03


# --- double layer (Algorithm 3, K~[gamma_0 u]) and the Green representation (Sec. 5)
def test_solid_angle_closed_form():
    """int_T n.(x-y)/|x-y|^3 ds_y (the double-layer potential of a flat
    triangle with unit density) is the signed solid angle: over a closed
    outward-oriented polyhedral surface it adds up to -4 pi inside and 0
    outside (Gauss), far away it tends to |T| n.(x-c)/|x-c|^3, and it is
    positive on the side the right-hand-rule normal points to; against
    brute-force quadrature on a near point."""
    m = ball_bc_mesh(1, radial=0.35)
    tri = m.verts[m.tris]
    for x in ([0.1, -0.2, 0.05], [0.0, 0.0, 0.0], [0.5, 0.4, -0.3]):
        s = sum(O.tri_solid_angle(np.array(x), t) for t in tri)
        assert abs(s / (4 * np.pi) + 1.0) < 1e-12, (x, s)
    for x in ([1.7, 0.3, -0.2], [0.0, -3.0, 0.1]):
        assert abs(sum(O.tri_solid_angle(np.array(x), t) for t in tri)) < 1e-12
    t = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    c = t.mean(0)
    for x in ([0.3, 0.2, 50.0], [-20.0, 5.0, -30.0]):
        x = np.array(x)
        ref = 0.5 * (x - c)[2] / np.linalg.norm(x - c) ** 3
        assert abs(O.tri_solid_angle(x, t) - ref) < 1e-3 * abs(ref)
    assert O.tri_solid_angle(np.array([0.2, 0.2, 0.1]), t) > 0 > O.tri_solid_angle(np.array([0.2, 0.2, -0.1]), t)
    # brute force: tensor Gauss rule on the collapsed square
    x = np.array([0.25, 0.3, 0.4])
    gx, gw = np.polynomial.legendre.leggauss(80)
    gx, gw = 0.5 * (gx + 1), 0.5 * gw
    U, Vv = np.meshgrid(gx, gx, indexing="ij")
    W = np.outer(gw, gw) * (1 - U)
    y = np.stack([U, (1 - U) * Vv, 0 * U], -1)
    d = x - y
    bf = np.sum(W * d[..., 2] / np.linalg.norm(d, axis=-1) ** 3)
    assert abs(O.tri_solid_angle(x, t) - bf) < 1e-9 * abs(bf)


def test_double_layer_of_constant_density():
    """K~[1] = -1 inside the domain (the Green representation of u = 1),
    so the discrete double-layer operator maps g = 1 to -|t| on every target
    tet: exactly when every pair takes the near rule (closed-form solid
    angle, any outer rule integrates the constant sum exactly), and to
    product-rule accuracy with the default near/far split."""
    m = ball_bc_mesh(1, radial=0.35)
    tg = np.arange(0, m.ntet, 7)
    vol = O.element_volumes(m)[tg]
    u = O.direct("btv_dl", m, np.ones((1, m.ntri)), targets=tg, eta_ns=0.0)[0] / vol
    assert np.abs(u + 1.0).max() < 1e-12
    u = O.direct("btv_dl", m, np.ones((1, m.ntri)), targets=tg)[0] / vol
    assert np.abs(u + 1.0).max() < 3e-3


def test_fmm_double_layer_converges_to_direct_geometrically():
    """O2's double-layer leg (moments <gamma_1 (y-c)^beta, g>, near field
    with dG/dn_y, Algorithm 3) against O1: geometric decay in p."""
    m = cube_bc_mesh(0.25, 0.25)
    f, g = densities(m, "sine")
    u1 = O.direct("btv_dl", m, g)
    e = []
    for p in (2, 4, 6, 8):
        u2 = O.fmm("btv_dl", m, g, p=p, leaf_size=16)
        e.append(np.linalg.norm(u2 - u1) / np.linalg.norm(u1))
    assert e[0] > 4 * e[1] > 16 * e[2] > 64 * e[3], e
    assert e[3] < 2e-6, e


_B4 = np.array([[(5 + 3 * 5 ** 0.5) / 20] + [(5 - 5 ** 0.5) / 20] * 3,
                [(5 - 5 ** 0.5) / 20, (5 + 3 * 5 ** 0.5) / 20] + [(5 - 5 ** 0.5) / 20] * 2,
                [(5 - 5 ** 0.5) / 20] * 2 + [(5 + 3 * 5 ** 0.5) / 20, (5 - 5 ** 0.5) / 20],
                [(5 - 5 ** 0.5) / 20] * 3 + [(5 + 3 * 5 ** 0.5) / 20]])
_B3 = np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]])


def _p0_boundary_data(m, u, du):
    """P0 Dirichlet and Neumann data: triangle averages of u and du/dn (3-point rule)."""
    tri = m.verts[m.tris]
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    n /= np.linalg.norm(n, axis=1)[:, None]
    qp = np.einsum("qk,tkd->tqd", _B3, tri)
    return u(qp).mean(1), du(qp, n[:, None, :]).mean(1)


def _cell_avg(m, u, tg):
    return u(np.einsum("qk,tkd->tqd", _B4, m.verts[m.tets[tg]])).mean(1)


def test_green_representation_laplace():
    """Sec. 5's BtV test: u_L = 1/|x - (3,0,0)| is harmonic in the ball, so
    V~[gamma_1 u_L] - K~[gamma_0 u_L] = u_L inside (Eq. green:ie:vol with
    f = 0).  With P0 boundary data the cell averages converge at least at
    the paper's O(h): the error falls by >= 1.8x per halving of h."""
    x0 = np.array([3.0, 0.0, 0.0])
    uL = lambda x: 1.0 / np.linalg.norm(x - x0, axis=-1)
    duL = lambda x, n: -np.sum((x - x0) * n, -1) / np.linalg.norm(x - x0, axis=-1) ** 3
    err = []
    for lev in (1, 2, 3):
        m = ball_bc_mesh(lev, radial=0.35)
        g, q = _p0_boundary_data(m, uL, duL)
        tg = np.sort(np.random.default_rng(0).choice(m.ntet, min(300, m.ntet), replace=False))
        vol = O.element_volumes(m)[tg]
        num = (O.direct("btv", m, q[None], targets=tg)[0] - O.direct("btv_dl", m, g[None], targets=tg)[0]) / vol
        ref = _cell_avg(m, uL, tg)
        err.append(np.linalg.norm(num - ref) / np.linalg.norm(ref))
    assert err[0] > 1.8 * err[1] > 1.8 ** 2 * err[2], err
    assert err[2] < 1e-3, err


def test_green_representation_poisson():
    """Sec. 5's VtV test: u_P = exp(-r^2) solves -Lap u_P = f = (6 - 4 r^2)
    exp(-r^2), so V~[gamma_1 u_P] - K~[gamma_0 u_P] + N~f = u_P inside
    (Eq. green:ie:vol), on the ball and on the cube; O(h) or better."""
    uP = lambda x: np.exp(-np.sum(x * x, -1))
    fP = lambda x: (6 - 4 * np.sum(x * x, -1)) * np.exp(-np.sum(x * x, -1))
    duP = lambda x, n: -2 * np.sum(x * n, -1) * uP(x)
    for mk in (lambda l: ball_bc_mesh(l + 1, radial=0.35), lambda l: cube_bc_mesh(0.5 / 2 ** l, 0.25 / 2 ** l)):
        err = []
        for lev in (0, 1, 2):
            m = mk(lev)
            g, q = _p0_boundary_data(m, uP, duP)
            f = _cell_avg(m, fP, np.arange(m.ntet))
            tg = np.sort(np.random.default_rng(1).choice(m.ntet, min(200, m.ntet), replace=False))
            vol = O.element_volumes(m)[tg]
            num = (O.direct("btv", m, q[None], targets=tg)[0] - O.direct("btv_dl", m, g[None], targets=tg)[0]
                   + O.direct("vtv", m, f[None], targets=tg)[0]) / vol
            ref = _cell_avg(m, uP, tg)
            err.append(np.linalg.norm(num - ref) / np.linalg.norm(ref))
        assert err[0] > 1.8 * err[1] > 1.8 ** 2 * err[2], err


def _cube_frame():
    """Sec. 5's functions on the cube meshes of [0,1]^3 through x' = 2(x - 1/2)."""
    c = np.array([0.5, 0.5, 0.5])
    xp = lambda x: 2.0 * (x - c)
    x0 = np.array([3.0, 0.0, 0.0])
    uL = lambda x: 1.0 / np.linalg.norm(xp(x) - x0, axis=-1)
    duL = lambda x, n: -2.0 * np.sum((xp(x) - x0) * n, -1) / np.linalg.norm(xp(x) - x0, axis=-1) ** 3
    uP = lambda x: np.exp(-np.sum(xp(x) ** 2, -1))
    fP = lambda x: 4.0 * (6.0 - 4.0 * np.sum(xp(x) ** 2, -1)) * uP(x)
    duP = lambda x, n: -4.0 * np.sum(xp(x) * n, -1) * uP(x)
    return uL, duL, uP, fP, duP


def _boundary_tets(m):
    """Tets with a face on the cube's surface (the set B_L of Sec. 2)."""
    tv = m.verts[m.tets]
    onb = (np.abs(tv) < 1e-12) | (np.abs(tv - 1.0) < 1e-12)
    return np.where((onb.sum(1) >= 3).any(1))[0]


def test_green_laplace_boundary_tets_need_the_wider_near_rule():
    """Sec. 5's BtV test on the cube's boundary tets.  With only the
    touching element pairs on the near rule, the 4 x 3-point product rule on
    the next ring of triangles keeps a relative error that a self-similar
    mesh does not shrink: here the error still halves from h = 1/16 to 1/32
    (4.4e-4 to 2.2e-4 on these 120 targets), and the library's runs at 1/64
    and 1/128 stay near 1.9e-4.  With eta_ns = 0.5 (that ring on the near rule
    too) it falls faster than O(h) over the same meshes (8.1e-4, 3.7e-4,
    1.3e-4) and ends 0.57x below the default at 1/32.  The floor is the
    product rule's, not the FMM's, the P0 data's or the near rule order's
    (6 instead of 3 Gauss points changes the error in the third digit)."""
    uL, duL, _, _, _ = _cube_frame()
    err = {O.ETA_NS: [], 0.5: []}
    for inv_h in (8, 16, 32):
        m = cube_bc_mesh(1 / inv_h, 1 / inv_h)
        g, q = _p0_boundary_data(m, uL, duL)
        tg = np.sort(np.random.default_rng(0).choice(_boundary_tets(m), 120, replace=False))
        vol = O.element_volumes(m)[tg]
        ref = _cell_avg(m, uL, tg)
        for en in err:
            num = (O.direct("btv", m, q[None], targets=tg, eta_ns=en)[0]
                   - O.direct("btv_dl", m, g[None], targets=tg, eta_ns=en)[0]) / vol
            err[en].append(np.linalg.norm(num - ref) / np.linalg.norm(ref))
    wide, default = err[0.5], err[O.ETA_NS]
    assert wide[0] > 1.8 * wide[1] > 1.8 ** 2 * wide[2], wide
    # the wider rule converges faster and ends well below the default
    assert default[1] / default[2] < 0.8 * wide[1] / wide[2], (default, wide)
    assert wide[2] < 0.7 * default[2], (default, wide)


def test_green_poisson_floor_is_the_coarse_interior():
    """Sec. 5's VtV + BtV test on the cube at h = 1/32: the P0 cell averages
    of f on the BC mesh's coarse interior cells (a cell is split while larger
    than half its distance to the surface) fix an error in N~f at every
    target, the boundary tets included.  Grading the interior twice as
    finely lowers it at the same h: the floor lies in the interior cells,
    which Sec. 5 treats with the degree schedule p_l = L - l."""
    _, _, uP, fP, duP = _cube_frame()
    err = {}
    for grade in (0.5, 0.25):
        m = cube_bc_mesh(1 / 32, 1 / 32, grade=grade)
        g, q = _p0_boundary_data(m, uP, duP)
        f = _cell_avg(m, fP, np.arange(m.ntet))
        tg = np.sort(np.random.default_rng(0).choice(_boundary_tets(m), 120, replace=False))
        vol = O.element_volumes(m)[tg]
        num = (O.direct("btv", m, q[None], targets=tg)[0] - O.direct("btv_dl", m, g[None], targets=tg)[0]
               + O.direct("vtv", m, f[None], targets=tg)[0]) / vol
        ref = _cell_avg(m, uP, tg)
        err[grade] = np.linalg.norm(num - ref) / np.linalg.norm(ref)
    assert err[0.25] < 0.6 * err[0.5], err
