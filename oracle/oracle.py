"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Arithmetic lives in ``bcfmm_oracle.c`` (closed-form element potentials,
element quadrature, the near rule, O1) and ``bcfmm_oracle_fmm.c`` (O2).  Gauss-
Legendre nodes for the near rule come from ``numpy.polynomial.legendre``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "bcfmm_oracle.c"), os.path.join(_HERE, "bcfmm_oracle_fmm.c")]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
_lock = threading.Lock()

# btv_dl: the double-layer part K~[gamma_0 u] of BtV (Algorithm 3, Eq.
# green:ie:vol), tet targets, triangle sources with their right-hand-rule
# normals; the BtV of Algorithm 3 is btv(gamma_1 u) - btv_dl(gamma_0 u)
TASKS = {"vtv": 0, "vtb": 1, "btv": 2, "btv_dl": 3}

# defaults of the discrete operator (shared by convention with the library)
ETA_NS = 1.0 - 2.0 ** -20      # near iff eta > ETA_NS: every touching pair (eta >= 1) is near
NEAR_N = 3                      # Gauss-Legendre nodes per collapsed direction
NEAR_K = 1                      # uniform refinements of the target element
ETA0 = 0.5                      # box neighbours: eta = sqrt3/|o| > ETA0 (Sec. 5 value; 0.9: the 27 touching boxes)


def build_lib(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into oracle/_build."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        # -ffp-contract=off: every product and sum rounds as written, so the
        # quadrature points (and the octree built on them) do not depend on
        # whether the host compiler fuses multiply-adds (it does on aarch64)
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-ffp-contract=off", "-o", tmp] + _SRC + ["-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build_lib()
            L = C.CDLL(_LIB_PATH)
            d, i, i64, p = C.c_double, C.c_int, C.c_int64, C.c_void_p
            L.orc_tri_potential.restype = d
            L.orc_tri_potential.argtypes = [p, p]
            L.orc_tet_potential.restype = d
            L.orc_tet_potential.argtypes = [p, p]
            L.orc_tri_solid_angle.restype = d
            L.orc_tri_solid_angle.argtypes = [p, p]
            L.orc_near_pair.restype = d
            L.orc_near_pair.argtypes = [i, p, p, p, p, i, i]
            L.orc_adaptive_pair.restype = d
            L.orc_adaptive_pair.argtypes = [i, p, p, p, p, i, d, i]
            L.orc_is_near.restype = i
            L.orc_is_near.argtypes = [p, i, p, i, d]
            L.orc_tet_quad.argtypes = [p, i64, p, p]
            L.orc_tri_quad.argtypes = [p, i64, p, p]
            L.orc_direct.argtypes = [i, p, i64, p, i64, p, i, p, i64, d, p, p, i, i, p, i]
            L.orc_fmm.restype = i
            L.orc_fmm.argtypes = [i, p, i64, p, i64, p, i, i, i, d, d, p, p, i, i, p, i64, p, p, i, p, p]
            L.orc_taylor_b.argtypes = [p, i, p]
            L.orc_m2l_matrix.argtypes = [p, i, p]
            L.orc_p2m.argtypes = [p, p, i64, p, i, p]
            L.orc_m2m.argtypes = [p, p, p, i, p]
            L.orc_l2l.argtypes = [p, p, p, i, p]
            L.orc_l2p.restype = d
            L.orc_l2p.argtypes = [p, p, i, p]
            L.orc_tree_stats.restype = i
            L.orc_tree_stats.argtypes = [p, i64, p, i64, i, p, p]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def gauss_legendre01(n: int):
    """Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return _f64(0.5 * (x + 1.0)), _f64(0.5 * w)


def nterms(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


def multi_indices(p: int) -> np.ndarray:
    """Multi-indices of total degree <= p, by degree then lexicographic (descending)."""
    out = []
    for d in range(p + 1):
        for a in range(d, -1, -1):
            for b in range(d - a, -1, -1):
                out.append((a, b, d - a - b))
    return np.array(out, dtype=np.int64)


# --- element-level functions ------------------------------------------------
def tri_potential(x, tri) -> float:
    """int_T ds_y / |x - y| (closed form)."""
    return lib().orc_tri_potential(_ptr(_f64(x)), _ptr(_f64(tri)))


def tri_solid_angle(x, tri) -> float:
    """int_T n.(x - y)/|x - y|^3 ds_y: the signed solid angle (closed form),
    positive on the side of the right-hand-rule normal."""
    return lib().orc_tri_solid_angle(_ptr(_f64(x)), _ptr(_f64(tri)))


def tet_potential(x, tet) -> float:
    """int_tau dy / |x - y| (closed form via the faces)."""
    return lib().orc_tet_potential(_ptr(_f64(x)), _ptr(_f64(tet)))


def tet_quad(tets):
    tets = _f64(tets).reshape(-1, 4, 3)
    pts = np.zeros((tets.shape[0] * 4, 3))
    w = np.zeros(tets.shape[0] * 4)
    lib().orc_tet_quad(_ptr(tets), tets.shape[0], _ptr(pts), _ptr(w))
    return pts, w


def tri_quad(tris):
    tris = _f64(tris).reshape(-1, 3, 3)
    pts = np.zeros((tris.shape[0] * 3, 3))
    w = np.zeros(tris.shape[0] * 3)
    lib().orc_tri_quad(_ptr(tris), tris.shape[0], _ptr(pts), _ptr(w))
    return pts, w


def near_pair(task: str, tgt, src, n: int = NEAR_N, k: int = NEAR_K) -> float:
    """The near rule N_ts = int_t int_s G (inner closed form, outer fixed rule)."""
    gx, gw = gauss_legendre01(n)
    return lib().orc_near_pair(TASKS[task], _ptr(_f64(tgt)), _ptr(_f64(src)), _ptr(gx), _ptr(gw), n, k)


def adaptive_pair(task: str, tgt, src, tol: float = 1e-12, n: int = 4, maxdepth: int = 7) -> float:
    """Adaptive (pin-only) evaluation of int_t int_s G for tet targets."""
    gx, gw = gauss_legendre01(n)
    return lib().orc_adaptive_pair(TASKS[task], _ptr(_f64(tgt)), _ptr(_f64(src)), _ptr(gx), _ptr(gw),
                                   n, tol, maxdepth)


def is_near(tgt, src, eta_ns: float = ETA_NS) -> bool:
    tgt, src = _f64(tgt), _f64(src)
    return bool(lib().orc_is_near(_ptr(tgt), tgt.size // 3, _ptr(src), src.size // 3, eta_ns))


# --- whole-operator functions ---------------------------------------------
def _task_arrays(task, mesh):
    tets = _f64(mesh.verts[mesh.tets])
    tris = _f64(mesh.verts[mesh.tris])
    tgt = tris if task == "vtb" else tets
    src = tris if task in ("btv", "btv_dl") else tets
    return tets, tris, tgt, src


def direct(task: str, mesh, dens, targets=None, eta_ns: float = ETA_NS, n: int = NEAR_N,
           k: int = NEAR_K, nthreads: int = 0) -> np.ndarray:
    """O1: u[d, t] = sum_s (near ? N_ts : Q_ts) dens[d, s] for target elements t."""
    tets, tris, tgt, src = _task_arrays(task, mesh)
    dens = _f64(np.atleast_2d(dens))
    ntgt = tgt.shape[0]
    targets = np.arange(ntgt, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
    out = np.zeros((dens.shape[0], targets.size))
    gx, gw = gauss_legendre01(n)
    lib().orc_direct(TASKS[task], _ptr(tgt), ntgt, _ptr(src), src.shape[0], _ptr(dens), dens.shape[0],
                     _ptr(targets), targets.size, eta_ns, _ptr(gx), _ptr(gw), n, k, _ptr(out), nthreads)
    return out


def fmm(task: str, mesh, dens, p: int = 4, leaf_size: int = 64, targets=None, eta0: float = ETA0,
        eta_ns: float = ETA_NS,
        n: int = NEAR_N, k: int = NEAR_K, nthreads: int = 0, return_stats: bool = False, p_level=None):
    """O2: the FP64 reference FMM; returns u[d, t] (and tree statistics).

    p_level: optional expansion order per octree level (index = level,
    at most 20 entries; entries <= 0 mean p), the level-dependent orders of
    Sec. 4.3; moments are kept to order p on every level."""
    tets, tris, tgt, src = _task_arrays(task, mesh)
    dens = _f64(np.atleast_2d(dens))
    targets = (np.arange(tgt.shape[0], dtype=np.int64) if targets is None
               else np.ascontiguousarray(targets, np.int64))
    out = np.zeros((dens.shape[0], targets.size))
    raw = np.zeros_like(out)
    st = np.zeros(8, np.int64)
    gx, gw = gauss_legendre01(n)
    ql = None
    if p_level is not None:
        ql = np.zeros(20, np.int32)
        q = np.asarray(p_level, np.int32)[:20]
        ql[:len(q)] = q
    lib().orc_fmm(TASKS[task], _ptr(tets), tets.shape[0], _ptr(tris), tris.shape[0], _ptr(dens),
                  dens.shape[0], p, leaf_size, eta0, eta_ns, _ptr(gx), _ptr(gw), n, k, _ptr(targets),
                  targets.size, _ptr(out), _ptr(raw), nthreads, _ptr(st), None if ql is None else _ptr(ql))
    if return_stats:
        keys = ["nbox", "nleaf", "maxlevel", "n_m2l", "n_p2p"]
        return out, dict(zip(keys, st[:5].tolist()), raw=raw)
    return out


def paper_orders(q0: int, finest_level: int, nlevels: int = 20):
    """Level-dependent expansion orders of Sec. 4.3 (Eq. def:q0, and Sec. 5's
    q_l = 4 + L - l with q0 = 4): q_l = q0 + L - l for l <= L."""
    return [q0 + finest_level - l if l <= finest_level else q0 for l in range(nlevels)]


def tree_stats(mesh, leaf_size: int = 64):
    tets = _f64(mesh.verts[mesh.tets])
    tris = _f64(mesh.verts[mesh.tris])
    b = np.zeros(20, np.int64)
    lf = np.zeros(20, np.int64)
    n = lib().orc_tree_stats(_ptr(tets), tets.shape[0], _ptr(tris), tris.shape[0], leaf_size, _ptr(b), _ptr(lf))
    return n, b, lf


# --- expansion pieces (for pins) ------------------------------------------------
def taylor_b(r, P: int) -> np.ndarray:
    """b_k(r) = (-1)^|k| D^k(1/|r|)/k!, |k| <= P."""
    out = np.zeros(nterms(P))
    lib().orc_taylor_b(_ptr(_f64(r)), P, _ptr(out))
    return out


def m2l_matrix(r, p: int) -> np.ndarray:
    npc = nterms(p)
    T = np.zeros((npc, npc))
    lib().orc_m2l_matrix(_ptr(_f64(r)), p, _ptr(T))
    return T


def p2m(pts, w, c, p: int) -> np.ndarray:
    pts = _f64(pts).reshape(-1, 3)
    m = np.zeros(nterms(p))
    lib().orc_p2m(_ptr(pts), _ptr(_f64(w)), pts.shape[0], _ptr(_f64(c)), p, _ptr(m))
    return m


def m2m(mc, cc, cp, p: int) -> np.ndarray:
    out = np.zeros(nterms(p))
    lib().orc_m2m(_ptr(_f64(mc)), _ptr(_f64(cc)), _ptr(_f64(cp)), p, _ptr(out))
    return out


def l2l(lp, cp, cc, p: int) -> np.ndarray:
    out = np.zeros(nterms(p))
    lib().orc_l2l(_ptr(_f64(lp)), _ptr(_f64(cp)), _ptr(_f64(cc)), p, _ptr(out))
    return out


def l2p(loc, c, p: int, x) -> float:
    return lib().orc_l2p(_ptr(_f64(loc)), _ptr(_f64(c)), p, _ptr(_f64(x)))


def element_volumes(mesh) -> np.ndarray:
    p = mesh.verts[mesh.tets]
    return np.abs(np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])) / 6.0


def element_areas(mesh) -> np.ndarray:
    p = mesh.verts[mesh.tris]
    return 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1)
