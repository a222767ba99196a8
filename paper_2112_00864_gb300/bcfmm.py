"""Thin Python binding of the bcfmm C ABI (``include/bcfmm.h``).

Argument marshalling only: every step of the evaluation runs in the CUDA
library ``_build/libbcfmm.so``.  PyTorch supplies device memory and the CUDA
stream.  There is no CPU fallback: loading fails loudly when the library is
missing (build it with ``paper_2112_00864_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes as C
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbcfmm.so")

BCFMM_OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_MESH", -3: "ERR_CUDA", -4: "ERR_OOM", -5: "ERR_TIMEOUT", -6: "ERR_STATE"}
PRECISION = {"fp64": 0, "fp32": 1, "bf16x2": 2, "bf16x3": 3}
VOLUME, BOUNDARY, DIPOLE = 0, 1, 2
EXPORTED = ["bcfmm_default_params", "bcfmm_build_bc_tree", "bcfmm_set_density", "bcfmm_eval_vtv",
            "bcfmm_eval_vtb", "bcfmm_eval_btv", "bcfmm_stats", "bcfmm_last_error", "bcfmm_destroy",
            "bcfmm_debug_m2l_matrix", "bcfmm_eval_noalloc", "bcfmm_build_batch", "bcfmm_eval_graph",
            "bcfmm_build_like", "bcfmm_direct_sample", "bcfmm_mlp_blob_size", "bcfmm_mlp_dataset",
            "bcfmm_mlp_grad", "bcfmm_mlp_adam", "bcfmm_mlp_predict", "bcfmm_debug_expire_wait",
            "bcfmm_debug_list_coverage", "bcfmm_debug_near_pairs", "bcfmm_debug_shift_matrix",
            "bcfmm_debug_tree_counts", "bcfmm_debug_m2l_taylor_coeffs", "bcfmm_measure_ffma"]
NEAR_MODE = {"fp64": 0, "learned": 1, "none": 2}
TASK_BIT = {"vtv": 1, "vtb": 2, "btv": 4}


class Params(C.Structure):
    _fields_ = [("p", C.c_int32), ("leaf_size", C.c_int32), ("eta_ns", C.c_double), ("near_n", C.c_int32),
                ("near_k", C.c_int32), ("precision", C.c_int32), ("timing", C.c_int32), ("eta0", C.c_double),
                ("tc_unit", C.c_int32), ("near_mode", C.c_int32), ("mlp_tol", C.c_double), ("mlp_blob", C.c_void_p),
                ("mlp_blob_bytes", C.c_int64), ("p_level", C.c_int32 * 20), ("q0", C.c_int32),
                ("double_layer", C.c_int32)]


class BcfmmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"bcfmm CUDA library not built: {path} is missing "
                              "(run paper_2112_00864_gb300.build.build())")
        L = C.CDLL(path)
        p, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.bcfmm_default_params.argtypes = [C.POINTER(Params)]
        L.bcfmm_default_params.restype = None
        L.bcfmm_build_bc_tree.argtypes = [p, i64, p, i64, p, i64, C.POINTER(Params), p, C.POINTER(p)]
        L.bcfmm_build_bc_tree.restype = C.c_int
        L.bcfmm_set_density.argtypes = [p, i32, p, i32, i32]
        L.bcfmm_set_density.restype = C.c_int
        for f in ("bcfmm_eval_vtv", "bcfmm_eval_vtb", "bcfmm_eval_btv"):
            getattr(L, f).argtypes = [p, p, i32]
            getattr(L, f).restype = C.c_int
        L.bcfmm_stats.argtypes = [p, C.c_char_p, C.c_size_t]
        L.bcfmm_stats.restype = C.c_int
        L.bcfmm_last_error.argtypes = []
        L.bcfmm_last_error.restype = C.c_char_p
        L.bcfmm_destroy.argtypes = [p]
        L.bcfmm_destroy.restype = None
        L.bcfmm_debug_m2l_matrix.argtypes = [i32, p, p]
        L.bcfmm_debug_m2l_matrix.restype = C.c_int
        L.bcfmm_debug_m2l_taylor_coeffs.argtypes = [i32, p, p]
        L.bcfmm_debug_m2l_taylor_coeffs.restype = C.c_int
        L.bcfmm_measure_ffma.argtypes = [i32, p]
        L.bcfmm_measure_ffma.restype = C.c_int
        L.bcfmm_eval_noalloc.argtypes = [p, i32, p, p]
        L.bcfmm_eval_noalloc.restype = C.c_int
        L.bcfmm_build_batch.argtypes = [p, p, p, p, p, p, i32, C.POINTER(Params), p, C.POINTER(p)]
        L.bcfmm_build_batch.restype = C.c_int
        L.bcfmm_eval_graph.argtypes = [p, i32, p, p, p]
        L.bcfmm_eval_graph.restype = C.c_int
        L.bcfmm_build_like.argtypes = [p, C.POINTER(Params), C.POINTER(p)]
        L.bcfmm_build_like.restype = C.c_int
        L.bcfmm_direct_sample.argtypes = [p, i32, p, i64, p]
        L.bcfmm_direct_sample.restype = C.c_int
        L.bcfmm_mlp_blob_size.argtypes = []
        L.bcfmm_mlp_blob_size.restype = C.c_int64
        L.bcfmm_mlp_dataset.argtypes = [p, i32, i64, p, p, p, p, p, C.POINTER(C.c_int64)]
        L.bcfmm_mlp_dataset.restype = C.c_int
        L.bcfmm_mlp_grad.argtypes = [p, p, p, p, i64, p, p, p]
        L.bcfmm_mlp_grad.restype = C.c_int
        L.bcfmm_mlp_adam.argtypes = [p, p, p, p, i32, C.c_float, C.c_float, C.c_float, C.c_float, p]
        L.bcfmm_mlp_adam.restype = C.c_int
        L.bcfmm_mlp_predict.argtypes = [p, p, p, i64, p, p]
        L.bcfmm_mlp_predict.restype = C.c_int
        L.bcfmm_debug_expire_wait.argtypes = [p, i32]
        L.bcfmm_debug_expire_wait.restype = C.c_int
        L.bcfmm_debug_list_coverage.argtypes = [p, p, p, p, p, p, i32, C.POINTER(Params), p]
        L.bcfmm_debug_list_coverage.restype = C.c_int
        L.bcfmm_debug_near_pairs.argtypes = [p, i64, p, i64, p, i64, d, i32, i64, p, p, C.POINTER(C.c_int64)]
        L.bcfmm_debug_near_pairs.restype = C.c_int
        L.bcfmm_debug_shift_matrix.argtypes = [i32, i32, i32, p]
        L.bcfmm_debug_shift_matrix.restype = C.c_int
        L.bcfmm_debug_tree_counts.argtypes = [p, i64, p, i64, p, i64, i32, p, p, i32]
        L.bcfmm_debug_tree_counts.restype = C.c_int
        _lib = L
    return _lib


def _check(rc: int):
    if rc != BCFMM_OK:
        raise BcfmmError(rc, load().bcfmm_last_error().decode())


def _set(prm: Params, k, v):
    if k == "precision" and isinstance(v, str):
        v = PRECISION[v]
    if k == "near_mode" and isinstance(v, str):
        v = NEAR_MODE[v]
    if k == "p_level":
        # expansion order per octree level (index = level; 0 or missing: p)
        arr = (C.c_int32 * 20)()
        for i, q in enumerate(list(v or [])[:20]):
            arr[i] = int(q)
        v = arr
    if k == "mlp_blob":
        # keep the bytes alive with the Params object; the library reads
        # them during the build only
        buf = C.create_string_buffer(bytes(v), len(v))
        prm._blob = buf
        prm.mlp_blob_bytes = len(v)
        v = C.cast(buf, C.c_void_p)
    setattr(prm, k, v)


def default_params(**kw) -> Params:
    prm = Params()
    load().bcfmm_default_params(C.byref(prm))
    for k, v in kw.items():
        _set(prm, k, v)
    return prm


def nterms(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


def debug_m2l_matrix(p: int, o) -> np.ndarray:
    o = np.ascontiguousarray(o, np.float64)
    T = np.zeros((nterms(p), nterms(p)))
    _check(load().bcfmm_debug_m2l_matrix(p, o.ctypes.data, T.ctypes.data))
    return T


def measure_ffma(device: int = 0) -> float:
    """Measured FP32 FMA throughput of a CUDA device in flop/s (FMA = 2)."""
    out = C.c_double(0.0)
    _check(load().bcfmm_measure_ffma(device, C.byref(out)))
    return out.value


def debug_m2l_taylor_coeffs(q: int, o) -> np.ndarray:
    """D^gamma G(o), |gamma| <= q: the per-offset numbers of the Taylor-form M2L."""
    o = np.ascontiguousarray(o, np.float64)
    g = np.zeros(nterms(q))
    _check(load().bcfmm_debug_m2l_taylor_coeffs(q, o.ctypes.data, g.ctypes.data))
    return g


def debug_shift_matrix(kind: str, p: int, octant: int) -> np.ndarray:
    """Box-scaled M2M ("m2m") or L2L ("l2l") matrix for a child octant."""
    T = np.zeros((nterms(p), nterms(p)))
    _check(load().bcfmm_debug_shift_matrix({"m2m": 0, "l2l": 1}[kind], p, octant, T.ctypes.data))
    return T


def _ptr(x):
    """(address, is_device) of a numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data, 0
    return x.data_ptr(), int(x.is_cuda)


class Context:
    """One mesh, or a batch of independent meshes, on the current CUDA
    device, bound to ``stream`` (a torch.cuda.Stream, an int handle, or None
    for the current torch stream).

    ``Context(verts, tets, tris)`` builds one mesh; ``Context.from_meshes``
    builds a batch whose densities and outputs are the concatenation of the
    meshes' element columns (``tet_off`` / ``tri_off`` give the ranges)."""

    def __init__(self, verts, tets, tris, params: Params | None = None, stream=None, *, vert_off=None,
                 tet_off=None, tri_off=None, **kw):
        import torch
        self._lib = load()
        self.params = params if params is not None else default_params(**kw)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream if isinstance(stream, int) else stream.cuda_stream
        self._v = np.ascontiguousarray(verts, np.float64)
        self._t = np.ascontiguousarray(tets, np.int32)
        self._f = np.ascontiguousarray(tris, np.int32) if tris is not None else np.zeros((0, 3), np.int32)
        self.ntet, self.ntri = self._t.shape[0], self._f.shape[0]
        ctx = C.c_void_p()
        self.vert_off = np.array([0, self._v.shape[0]], np.int64) if vert_off is None else \
            np.ascontiguousarray(vert_off, np.int64)
        if vert_off is None:
            self.nmesh = 1
            self.tet_off = np.array([0, self.ntet], np.int64)
            self.tri_off = np.array([0, self.ntri], np.int64)
            _check(self._lib.bcfmm_build_bc_tree(self._v.ctypes.data, self._v.shape[0], self._t.ctypes.data,
                                                 self.ntet, self._f.ctypes.data, self.ntri, C.byref(self.params),
                                                 C.c_void_p(handle), C.byref(ctx)))
        else:
            vo = np.ascontiguousarray(vert_off, np.int64)
            self.tet_off = np.ascontiguousarray(tet_off, np.int64)
            self.tri_off = np.ascontiguousarray(tri_off, np.int64)
            self.nmesh = len(vo) - 1
            assert len(self.tet_off) == len(self.tri_off) == len(vo)
            _check(self._lib.bcfmm_build_batch(self._v.ctypes.data, vo.ctypes.data, self._t.ctypes.data,
                                               self.tet_off.ctypes.data, self._f.ctypes.data,
                                               self.tri_off.ctypes.data, self.nmesh, C.byref(self.params),
                                               C.c_void_p(handle), C.byref(ctx)))
        self._ctx = ctx
        self.ndens = {VOLUME: 0, BOUNDARY: 0, DIPOLE: 0}

    @classmethod
    def from_meshes(cls, meshes, **kw):
        """Batch of independent meshes (objects with verts, tets, tris)."""
        vo, to, ro = [0], [0], [0]
        for m in meshes:
            vo.append(vo[-1] + len(m.verts))
            to.append(to[-1] + len(m.tets))
            ro.append(ro[-1] + len(m.tris))
        verts = np.concatenate([np.asarray(m.verts, np.float64) for m in meshes])
        tets = np.concatenate([np.asarray(m.tets, np.int32) for m in meshes])
        tris = np.concatenate([np.asarray(m.tris, np.int32).reshape(-1, 3) for m in meshes])
        return cls(verts, tets, tris, vert_off=vo, tet_off=to, tri_off=ro, **kw)

    def build_like(self, **overrides) -> "Context":
        """New context on the same meshes with other tree / precision
        parameters (p, leaf_size, eta0, precision, tc_unit); the near pairs and
        their corrections are copied from this context, not recomputed."""
        new = object.__new__(Context)
        new._lib = self._lib
        prm = Params()
        C.pointer(prm)[0] = self.params
        for k, v in overrides.items():
            _set(prm, k, v)
        new.params = prm
        new.stream = self.stream
        new._v, new._t, new._f = self._v, self._t, self._f
        new.ntet, new.ntri, new.nmesh = self.ntet, self.ntri, self.nmesh
        new.tet_off, new.tri_off, new.vert_off = self.tet_off, self.tri_off, self.vert_off
        ctx = C.c_void_p()
        new._ctx = None
        _check(self._lib.bcfmm_build_like(self._ctx, C.byref(prm), C.byref(ctx)))
        new._ctx = ctx
        new.ndens = {VOLUME: 0, BOUNDARY: 0, DIPOLE: 0}
        return new

    def direct_sample(self, task: str, targets) -> np.ndarray:
        """FP64 direct evaluation (no expansions) of the target elements
        ``targets`` on the GPU: [ndens, len(targets)] host array."""
        t = {"vtv": 0, "vtb": 1, "btv": 2}[task]
        kind = BOUNDARY if task == "btv" else VOLUME
        tg = np.ascontiguousarray(targets, np.int64)
        out = np.zeros((self.ndens[kind], len(tg)))
        _check(self._lib.bcfmm_direct_sample(self._ctx, t, tg.ctypes.data, len(tg), out.ctypes.data))
        return out

    def mlp_dataset(self, task: str, max_pairs: int) -> dict:
        """Near-singular pairs of this context (built with near_mode
        "learned" or "none"), evenly sampled: features, qhat, chat (labels
        from the FP64 near rule), calibration bins and the (target, source)
        element indices, as CUDA tensors."""
        import torch
        t = {"vtv": 0, "vtb": 1, "btv": 2}[task]
        feat = torch.empty((max_pairs, 12), dtype=torch.float32, device="cuda")
        qhat = torch.empty((max_pairs, 16), dtype=torch.float32, device="cuda")
        chat = torch.empty((max_pairs,), dtype=torch.float32, device="cuda")
        bins = torch.empty((max_pairs,), dtype=torch.int32, device="cuda")
        pairs = torch.empty((max_pairs, 2), dtype=torch.int32, device="cuda")
        n = C.c_int64()
        _check(self._lib.bcfmm_mlp_dataset(self._ctx, t, max_pairs, C.c_void_p(feat.data_ptr()),
                                           C.c_void_p(qhat.data_ptr()), C.c_void_p(chat.data_ptr()),
                                           C.c_void_p(bins.data_ptr()), C.c_void_p(pairs.data_ptr()), C.byref(n)))
        k = n.value
        return dict(feat=feat[:k], qhat=qhat[:k], chat=chat[:k], bin=bins[:k], pairs=pairs[:k])

    @classmethod
    def from_mesh(cls, mesh, **kw):
        return cls(mesh.verts, mesh.tets, mesh.tris, **kw)

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.bcfmm_destroy(self._ctx)
            self._ctx = None

    __del__ = close

    def set_density(self, kind: int, vals):
        """vals: [ndens, nelem] float64 numpy array (host) or CUDA tensor (device)."""
        if isinstance(vals, np.ndarray):
            vals = np.ascontiguousarray(np.atleast_2d(vals), np.float64)
            nd = vals.shape[0]
        else:
            if vals.dim() == 1:
                vals = vals[None]
            vals = vals.contiguous()
            assert vals.dtype.is_floating_point and vals.element_size() == 8, "densities must be float64"
            nd = vals.shape[0]
        if not hasattr(self, "_keep"):
            self._keep = {}
        self._keep[kind] = vals
        ptr, dev = _ptr(vals)
        _check(self._lib.bcfmm_set_density(self._ctx, kind, C.c_void_p(ptr), nd, dev))
        self.ndens[kind] = nd

    def clear_dipole(self):
        """Remove the double-layer density (BtV then evaluates V~ q alone)."""
        _check(self._lib.bcfmm_set_density(self._ctx, DIPOLE, None, 0, 0))
        self.ndens[DIPOLE] = 0
        if hasattr(self, "_keep"):
            self._keep.pop(DIPOLE, None)

    def _eval(self, fn, nel: int, kind: int, out=None):
        nd = self.ndens[kind]
        if out is None:
            import torch
            out = torch.empty((nd, nel), dtype=torch.float64, device="cuda")
        ptr, dev = _ptr(out)
        _check(fn(self._ctx, C.c_void_p(ptr), dev))
        return out

    def eval_vtv(self, out=None):
        return self._eval(self._lib.bcfmm_eval_vtv, self.ntet, VOLUME, out)

    def eval_vtb(self, out=None):
        return self._eval(self._lib.bcfmm_eval_vtb, self.ntri, VOLUME, out)

    def eval_btv(self, out=None):
        return self._eval(self._lib.bcfmm_eval_btv, self.ntet, BOUNDARY, out)

    def eval(self, task: str, out=None):
        return {"vtv": self.eval_vtv, "vtb": self.eval_vtb, "btv": self.eval_btv}[task](out)

    def eval_noalloc(self, task: str, dens, out):
        """One task for one density with no allocation (device tensors)."""
        t = {"vtv": 0, "vtb": 1, "btv": 2}[task]
        assert dens.is_cuda and out.is_cuda and dens.dtype == out.dtype and dens.element_size() == 8
        _check(self._lib.bcfmm_eval_noalloc(self._ctx, t, C.c_void_p(dens.data_ptr()), C.c_void_p(out.data_ptr())))
        return out

    def eval_graph(self, tasks=("vtv", "vtb"), outs=None):
        """Evaluate ``tasks`` as one CUDA graph launch (captured on first use
        for this set of tasks and output buffers).  Returns {task: tensor}."""
        import torch
        outs = dict(outs or {})
        mask = 0
        ptrs = [None, None, None]
        for i, t in enumerate(("vtv", "vtb", "btv")):
            if t not in tasks:
                continue
            mask |= TASK_BIT[t]
            kind = BOUNDARY if t == "btv" else VOLUME
            nel = self.ntri if t == "vtb" else self.ntet
            if t not in outs:
                outs[t] = torch.empty((self.ndens[kind], nel), dtype=torch.float64, device="cuda")
            assert outs[t].is_cuda and outs[t].is_contiguous()
            ptrs[i] = C.c_void_p(outs[t].data_ptr())
        _check(self._lib.bcfmm_eval_graph(self._ctx, mask, *ptrs))
        return outs

    def element_vertices(self, kind: int) -> np.ndarray:
        """[n, 4 or 3, 3] vertex coordinates of the volume / boundary elements
        (mesh-local vertex ids of a batch resolved)."""
        el, off = (self._t, self.tet_off) if kind == VOLUME else (self._f, self.tri_off)
        shift = np.repeat(self.vert_off[:-1], np.diff(off))
        return self._v[el + shift[:, None]]

    def split(self, out, kind_or_task):
        """Per-mesh views of a batch output / density ([ndens][n] -> list)."""
        off = self.tri_off if kind_or_task in ("vtb", BOUNDARY) else self.tet_off
        return [out[..., off[m]:off[m + 1]] for m in range(self.nmesh)]

    def stats(self) -> dict:
        buf = C.create_string_buffer(1 << 16)
        _check(self._lib.bcfmm_stats(self._ctx, buf, len(buf)))
        return json.loads(buf.value.decode())


# ------------------------------------------------ learned correction kernels
def _dev(t):
    assert t.is_cuda and t.is_contiguous() and t.dtype.is_floating_point and t.element_size() == 4
    return C.c_void_p(t.data_ptr())


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s if isinstance(s, int) else s.cuda_stream)


def mlp_blob_size() -> int:
    return int(load().bcfmm_mlp_blob_size())


def mlp_grad(params, feat, qhat, chat, grad, loss, stream=None):
    """grad (6032) and loss (1) of the mean squared error over the pairs."""
    _check(load().bcfmm_mlp_grad(_dev(params), _dev(feat), _dev(qhat), _dev(chat), feat.shape[0], _dev(grad),
                                 _dev(loss), _stream_handle(stream)))


def mlp_adam(params, grad, m1, m2, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().bcfmm_mlp_adam(_dev(params), _dev(grad), _dev(m1), _dev(m2), step, lr, beta1, beta2, eps,
                                 _stream_handle(stream)))


def mlp_predict(params, feat, qhat, out, stream=None):
    _check(load().bcfmm_mlp_predict(_dev(params), _dev(feat), _dev(qhat), feat.shape[0], _dev(out),
                                    _stream_handle(stream)))


def debug_list_coverage(meshes, **kw) -> np.ndarray:
    """Host-only check of the FMM's interaction covering for one mesh or a
    batch: [0:3] per task the (target leaf, source point) pairs not covered
    exactly once, [3:6] per task the interaction entries the tensor-core
    tiles get wrong, [6:9] per task the faults of the tensor-core schedule,
    [9:12] per task the faults of the Taylor-form M2L schedule, [12:15] per
    task the faults of the packed near field's chunk blocks (see
    include/bcfmm.h)."""
    vo, to, ro = [0], [0], [0]
    for m in meshes:
        vo.append(vo[-1] + len(m.verts))
        to.append(to[-1] + len(m.tets))
        ro.append(ro[-1] + len(m.tris))
    verts = np.ascontiguousarray(np.concatenate([m.verts for m in meshes]), np.float64)
    tets = np.ascontiguousarray(np.concatenate([m.tets for m in meshes]), np.int32)
    tris = np.ascontiguousarray(np.concatenate([np.asarray(m.tris).reshape(-1, 3) for m in meshes]), np.int32)
    vo, to, ro = (np.asarray(x, np.int64) for x in (vo, to, ro))
    prm = default_params(**kw)
    out = np.zeros(15, np.int64)
    _check(load().bcfmm_debug_list_coverage(verts.ctypes.data, vo.ctypes.data, tets.ctypes.data, to.ctypes.data,
                                            tris.ctypes.data, ro.ctypes.data, len(meshes), C.byref(prm),
                                            out.ctypes.data))
    return out


def debug_near_pairs(mesh, task: str, eta_ns: float | None = None):
    """Host-only: the near pairs the build finds, (row_off, cols) CSR."""
    t = {"vtv": 0, "vtb": 1, "btv": 2}[task]
    v = np.ascontiguousarray(mesh.verts, np.float64)
    te = np.ascontiguousarray(mesh.tets, np.int32)
    tr = np.ascontiguousarray(np.asarray(mesh.tris).reshape(-1, 3), np.int32)
    nrow = (len(tr) if t == 1 else len(te)) + 1
    row = np.zeros(nrow, np.int64)
    nnz = C.c_int64()
    eta = default_params().eta_ns if eta_ns is None else eta_ns
    L = load()
    L.bcfmm_debug_near_pairs(v.ctypes.data, len(v), te.ctypes.data, len(te), tr.ctypes.data, len(tr), eta, t, 0,
                             row.ctypes.data, None, C.byref(nnz))
    cols = np.zeros(max(1, nnz.value), np.int32)
    _check(L.bcfmm_debug_near_pairs(v.ctypes.data, len(v), te.ctypes.data, len(te), tr.ctypes.data, len(tr), eta, t,
                                    len(cols), row.ctypes.data, cols.ctypes.data, C.byref(nnz)))
    return row, cols[:nnz.value]


def debug_tree_counts(mesh, leaf_size: int = 64):
    """Host-only: (boxes per level, leaves per level) of the build's octree."""
    v = np.ascontiguousarray(mesh.verts, np.float64)
    te = np.ascontiguousarray(mesh.tets, np.int32)
    tr = np.ascontiguousarray(np.asarray(mesh.tris).reshape(-1, 3), np.int32)
    b = np.zeros(24, np.int64)
    lf = np.zeros(24, np.int64)
    _check(load().bcfmm_debug_tree_counts(v.ctypes.data, len(v), te.ctypes.data, len(te), tr.ctypes.data, len(tr),
                                          leaf_size, b.ctypes.data, lf.ctypes.data, len(b)))
    return b, lf
