"""Thin ctypes binding of the C ABI in include/mlfma.h.

Argument marshalling only: every step of the product runs in the CUDA
library.  PyTorch supplies device memory and the current stream.  If the
compiled library is missing this module raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

FP64 = 0
FP32 = 1
MIXED_TF32 = 2      # FP32 product, tensor-core (TF32) interpolation
MIXED_3XTF32 = 3    # FP32 product, tensor-core (3xTF32 split) interpolation
MAX_LEVELS = 22

(X_PERM, X_LEAF_BOX, X_GRID, X_ALPHA, X_ALPHA_OFFS, X_INTERP, X_BOX_CENTERS, X_NEAR_COUNT, X_ANTERP, X_ALPHA_J,
 X_ALPHA_Y, X_SIB_ALPHA, X_SIB_OFFS, X_WIN_INTERP, X_WIN_ANTERP, X_WIN_SHAPE, X_SHIFT, X_SHIFT_XY,
 X_SHIFT_Z) = range(1, 20)

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "ETIMEOUT", 6: "ENOTSUP"}

EXPORTED = ["mlfma_default_opts", "mlfma_plan", "mlfma_num_unknowns", "mlfma_rwg_edges", "mlfma_matvec",
            "mlfma_matvec_adjoint", "mlfma_matvec_dk", "mlfma_matvec_dk_adjoint", "mlfma_matvec_x",
            "mlfma_matvec_r", "mlfma_matvec_host", "mlfma_sync", "mlfma_plan_info", "mlfma_export",
            "mlfma_profile_stages", "mlfma_export_field", "mlfma_tune", "mlfma_tune_get", "mlfma_tune_set", "mlfma_matvec_noalloc", "mlfma_cm_default_opts", "cm_ira_solve", "cm_block_solve", "cm_rayleigh_ritz",
            "cm_eig_derivatives", "cm_track_modes",
            "mlfma_set_create", "mlfma_set_matvec", "mlfma_set_info", "mlfma_set_plan", "mlfma_set_destroy",
            "mlfma_destroy", "mlfma_last_error"]
CM_ZINV_R, CM_XINV_R = 0, 1
STAGE_COUNT = 71
TUNE_FIELDS = 3 + 3 * 22


class MlfmaError(RuntimeError):
    """A C-ABI call returned a status other than MLFMA_OK: `status` is the
    code (1 EINVAL, 2 ENOMEM, 3 ECUDA, 4 ENOTCONV, 5 ETIMEOUT, 6 ENOTSUP),
    the message is mlfma_last_error()."""

    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Opts(ctypes.Structure):
    """mlfma_opts (include/mlfma.h)."""
    _fields_ = [("interp_order", ctypes.c_int), ("max_batch", ctypes.c_int), ("precisions", ctypes.c_int),
                ("host_only", ctypes.c_int), ("device", ctypes.c_int), ("eta", ctypes.c_double)]


class CmOpts(ctypes.Structure):
    """mlfma_cm_opts: options of cm_ira_solve / cm_block_solve."""
    _fields_ = [("nev", ctypes.c_int), ("ncv", ctypes.c_int), ("op", ctypes.c_int), ("prec", ctypes.c_int),
                ("tol", ctypes.c_double), ("gmres_tol", ctypes.c_double), ("gmres_restart", ctypes.c_int),
                ("max_inner", ctypes.c_int), ("max_restarts", ctypes.c_int), ("use_sai", ctypes.c_int),
                ("seed", ctypes.c_uint64)]


class CmStats(ctypes.Structure):
    """mlfma_cm_stats: counters of an eigensolve."""
    _fields_ = [("restarts", ctypes.c_int), ("inner_iterations", ctypes.c_int64), ("products", ctypes.c_int64),
                ("converged", ctypes.c_int), ("inner_converged", ctypes.c_int), ("seconds", ctypes.c_double)]


class Info(ctypes.Structure):
    """mlfma_info: tree and table sizes of a plan (mlfma_plan_info)."""
    _fields_ = [("n", ctypes.c_int64), ("levels", ctypes.c_int), ("leaf_level", ctypes.c_int),
                ("root_side", ctypes.c_double), ("root_center", ctypes.c_double * 3),
                ("near_nnz", ctypes.c_int64), ("leaf_boxes", ctypes.c_int64), ("max_leaf_unknowns", ctypes.c_int),
                ("box_count", ctypes.c_int * MAX_LEVELS), ("trunc_L", ctypes.c_int * MAX_LEVELS),
                ("samples_K", ctypes.c_int * MAX_LEVELS), ("translations", ctypes.c_int64 * MAX_LEVELS),
                ("device_bytes", ctypes.c_int64), ("setup_seconds", ctypes.c_double)]


_lib = None


def _check_device_pair(x, y=None):
    """The products read x and write y on the GPU, so both must be CUDA
    tensors on one device: a host buffer handed to the library would be
    accessed by the kernels as if it were device memory."""
    if not x.is_cuda:
        raise ValueError("x must be a CUDA tensor (use matvec_host for host arrays)")
    if y is not None and (not y.is_cuda or y.device != x.device):
        raise ValueError("y must be a CUDA tensor on x's device")


def _mesh_arrays(verts, tris):
    """float64 [nv, 3] and int32 [nt, 3] copies of the mesh (the library reads
    three values per row)."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    if v.ndim != 2 or v.shape[1] != 3 or t.ndim != 2 or t.shape[1] != 3:
        raise ValueError("verts must be [nv, 3] and tris [nt, 3]")
    return v, t


def library_path() -> str:
    """Path of the in-tree compiled library."""
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the compiled library (build it first when asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError("MLFMA CUDA library not built (%s); call __graft_entry__.build() or "
                               "paper_1412_1756_gb300._build.build()" % path)
        _build.build()
    L = ctypes.CDLL(path)
    P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.mlfma_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.mlfma_plan.argtypes = [P, I64, P, I64, ctypes.c_double, I, ctypes.c_double, ctypes.POINTER(Opts),
                             ctypes.POINTER(P)]
    L.mlfma_num_unknowns.argtypes = [P, ctypes.POINTER(I64)]
    L.mlfma_rwg_edges.argtypes = [P, P, P]
    for f in ("mlfma_matvec", "mlfma_matvec_adjoint", "mlfma_matvec_dk", "mlfma_matvec_dk_adjoint",
              "mlfma_matvec_x", "mlfma_matvec_r", "mlfma_matvec_host", "mlfma_matvec_noalloc"):
        getattr(L, f).argtypes = [P, P, I, P, I64, I, P]
    L.mlfma_sync.argtypes = [P, P]
    L.mlfma_profile_stages.argtypes = [P, P, I, P, I64, I, P, P]
    L.mlfma_tune.argtypes = [P, I64, I, I, P, P, P]
    L.mlfma_export_field.argtypes = [P, I, I, I, I64, P, I64, ctypes.POINTER(I64)]
    L.mlfma_tune_get.argtypes = [P, I64, I, I, P]
    L.mlfma_tune_set.argtypes = [P, I64, I, I, P]
    L.mlfma_cm_default_opts.argtypes = [ctypes.POINTER(CmOpts)]
    L.cm_ira_solve.argtypes = [P, ctypes.POINTER(CmOpts), P, P, ctypes.POINTER(CmStats)]
    L.cm_block_solve.argtypes = [P, ctypes.POINTER(CmOpts), P, P, ctypes.POINTER(CmStats)]
    L.cm_rayleigh_ritz.argtypes = [I64, I, P, P, P, P, P, ctypes.POINTER(I)]
    L.cm_eig_derivatives.argtypes = [P, I, P, P, I, P]
    L.cm_track_modes.argtypes = [I64, I, P, P, I, P, P, ctypes.c_double, P, P]
    L.mlfma_plan_info.argtypes = [P, ctypes.POINTER(Info)]
    L.mlfma_export.argtypes = [P, I, I, P, I64, ctypes.POINTER(I64)]
    L.mlfma_destroy.argtypes = [P]
    L.mlfma_destroy.restype = None
    L.mlfma_set_create.argtypes = [P, I64, P, I64, P, I, I, ctypes.c_double, ctypes.POINTER(Opts), I64,
                                   ctypes.POINTER(P)]
    L.mlfma_set_matvec.argtypes = [P, P, I, I, P, I64, I, P]
    L.mlfma_set_info.argtypes = [P, P, P, P, P, P]
    L.mlfma_set_plan.argtypes = [P, I, ctypes.POINTER(P)]
    L.mlfma_set_destroy.argtypes = [P]
    L.mlfma_set_destroy.restype = None
    L.mlfma_last_error.argtypes = []
    L.mlfma_last_error.restype = ctypes.c_char_p
    for f in EXPORTED:
        if f not in ("mlfma_destroy", "mlfma_set_destroy", "mlfma_last_error"):
            getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise MlfmaError(status, load().mlfma_last_error().decode())


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class MlfmaPlan:
    """A plan for y = Z x on one mesh at one wavenumber (include/mlfma.h)."""

    def __init__(self, verts, tris, k, levels, digits=3.0, interp_order=10, max_batch=64,
                 precisions=(FP32, FP64), host_only=False, device=None, eta=None, _handle=None):
        L = load()
        if _handle is not None:   # a plan owned by a MlfmaPlanSet
            self._lib, self._h, self._owned = L, _handle, False
            self.k, self.max_batch, self.host_only = float(k), int(max_batch), False
            self.interp_order = int(interp_order)
            n = ctypes.c_int64()
            _check(L.mlfma_num_unknowns(_handle, ctypes.byref(n)))
            self.n = int(n.value)
            return
        self._owned = True
        self._lib = L
        v, t = _mesh_arrays(verts, tris)
        o = Opts()
        _check(L.mlfma_default_opts(ctypes.byref(o)))
        o.interp_order = int(interp_order)
        o.max_batch = int(max_batch)
        o.precisions = sum(1 << p for p in precisions)
        o.host_only = 1 if host_only else 0
        if device is not None:
            o.device = int(device)
        elif not host_only:
            import torch
            o.device = torch.cuda.current_device()
        if eta is not None:
            o.eta = float(eta)
        h = ctypes.c_void_p()
        _check(L.mlfma_plan(_np_ptr(v), v.shape[0], _np_ptr(t), t.shape[0], float(k), int(levels),
                            float(digits), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.k = float(k)
        self.max_batch = int(max_batch)
        self.host_only = bool(host_only)
        self.interp_order = int(interp_order)
        n = ctypes.c_int64()
        _check(L.mlfma_num_unknowns(h, ctypes.byref(n)))
        self.n = int(n.value)

    # ------------------------------------------------------------ queries
    def info(self) -> dict:
        """Tree and table sizes (mlfma_plan_info) as a dict; per-level lists
        are indexed by level, 0 = root."""
        inf = Info()
        _check(self._lib.mlfma_plan_info(self._h, ctypes.byref(inf)))
        nl = inf.levels
        return {
            "n": inf.n, "levels": nl, "leaf_level": inf.leaf_level, "root_side": inf.root_side,
            "root_center": list(inf.root_center), "near_nnz": inf.near_nnz, "leaf_boxes": inf.leaf_boxes,
            "max_leaf_unknowns": inf.max_leaf_unknowns, "box_count": list(inf.box_count[:nl]),
            "trunc_L": list(inf.trunc_L[:nl]), "samples_K": list(inf.samples_K[:nl]),
            "translations": list(inf.translations[:nl]), "device_bytes": inf.device_bytes,
            "setup_seconds": inf.setup_seconds,
        }

    def rwg_edges(self):
        """(edge_v [N, 2], tri_pm [N, 2]): each unknown's edge vertices and its
        T+ / T- triangles, canonical order (mlfma_rwg_edges)."""
        ev = np.zeros((self.n, 2), np.int32)
        tp = np.zeros((self.n, 2), np.int32)
        _check(self._lib.mlfma_rwg_edges(self._h, _np_ptr(ev), _np_ptr(tp)))
        return ev, tp

    def export(self, what: int, level: int = 0) -> np.ndarray:
        """A plan table (mlfma_export, an X_* code) as a NumPy array of the
        layout include/mlfma.h gives for that code."""
        need = ctypes.c_int64()
        _check(self._lib.mlfma_export(self._h, what, level, None, 0, ctypes.byref(need)))
        buf = np.zeros(need.value, np.uint8)
        _check(self._lib.mlfma_export(self._h, what, level, _np_ptr(buf), need.value, ctypes.byref(need)))
        if what == X_PERM:
            return buf.view(np.int64)
        if what in (X_LEAF_BOX,):
            return buf.view(np.int32)
        if what == X_WIN_SHAPE:
            return buf.view(np.int32).reshape(4, 2)
        if what == X_NEAR_COUNT:
            return buf.view(np.int64)
        if what in (X_ALPHA_OFFS, X_SIB_OFFS):
            return buf.view(np.int32).reshape(-1, 3)
        if what == X_GRID:
            return buf.view(np.float64).reshape(-1, 4)
        if what in (X_ALPHA, X_ALPHA_J, X_ALPHA_Y, X_SIB_ALPHA):
            return buf.view(np.complex128)
        if what in (X_SHIFT, X_SHIFT_XY, X_SHIFT_Z):   # [octant][sample or theta row]
            return buf.view(np.complex128).reshape(8, -1)
        if what == X_BOX_CENTERS:
            return buf.view(np.float64).reshape(-1, 3)
        return buf.view(np.float64)

    # ----------------------------------------------------------- products
    @staticmethod
    def _prec_of(dtype):
        import torch
        if dtype in (torch.float32, torch.complex64):
            return FP32
        if dtype in (torch.float64, torch.complex128):
            return FP64
        raise TypeError("x must be float32/float64/complex64/complex128, got %s" % dtype)

    def _product(self, fn, x, y, stream, prec=None):
        import torch
        _check_device_pair(x)
        squeeze = x.dim() == 1
        x2 = x.reshape(self.n, -1) if squeeze else x
        if x2.dim() != 2 or x2.shape[0] != self.n:
            raise ValueError("x must be [N] or [N, B] with N = %d" % self.n)
        x2 = x2.contiguous()
        dprec = self._prec_of(x2.dtype)
        if prec in (MIXED_TF32, MIXED_3XTF32):
            if dprec != FP32:
                raise TypeError("the TF32 precisions take float32 / complex64 x")
        else:
            prec = dprec
        xc = 1 if x2.is_complex() else 0
        cdt = torch.complex128 if prec == FP64 else torch.complex64
        B = x2.shape[1]
        if y is None:
            y = torch.empty((self.n, B), dtype=cdt, device=x2.device)
        if y.dtype != cdt or not y.is_contiguous() or y.numel() != self.n * B:
            raise ValueError("y must be a contiguous %s tensor with N*B elements" % cdt)
        _check_device_pair(x2, y)
        s = torch.cuda.current_stream(x2.device).cuda_stream if stream is None else stream
        _check(fn(self._h, ctypes.c_void_p(x2.data_ptr()), xc, ctypes.c_void_p(y.data_ptr()), B, prec,
                  ctypes.c_void_p(s)))
        return y.reshape(self.n) if squeeze else y.reshape(self.n, B)

    def matvec(self, x, y=None, stream=None, prec=None):
        """y = Z x for a CUDA tensor x [N] or [N, B] (real or complex).  The
        precision follows x's dtype; prec = MIXED_TF32 or MIXED_3XTF32 (with
        float32 / complex64 x) selects tensor-core interpolation."""
        return self._product(self._lib.mlfma_matvec, x, y, stream, prec)

    def matvec_adjoint(self, x, y=None, stream=None, prec=None):
        """y = Z^H x."""
        return self._product(self._lib.mlfma_matvec_adjoint, x, y, stream, prec)

    def _dk_product(self, fn, x, y, stream):
        # value and tangent fields share the plan's field buffers: at most
        # max_batch / 2 internal real columns per call, so wider x is split
        import torch
        squeeze = x.dim() == 1
        x2 = x.reshape(self.n, -1) if squeeze else x
        per = max(1, (self.max_batch // 2) // (2 if x2.is_complex() else 1))
        if x2.dim() != 2 or x2.shape[1] <= per:
            return self._product(fn, x, y, stream)
        cdt = torch.complex64 if self._prec_of(x2.dtype) == FP32 else torch.complex128
        out = torch.empty((self.n, x2.shape[1]), dtype=cdt, device=x2.device) if y is None else y.view(self.n, -1)
        for c0 in range(0, x2.shape[1], per):
            c1 = min(x2.shape[1], c0 + per)
            out[:, c0:c1] = self._product(fn, x2[:, c0:c1], None, stream)
        return out

    def matvec_dk(self, x, y=None, stream=None):
        """y = (dZ/dk) x (include/mlfma.h: mlfma_matvec_dk)."""
        return self._dk_product(self._lib.mlfma_matvec_dk, x, y, stream)

    def matvec_dk_adjoint(self, x, y=None, stream=None):
        """y = (dZ/dk)^H x."""
        return self._dk_product(self._lib.mlfma_matvec_dk_adjoint, x, y, stream)

    def matvec_x(self, x, y=None, stream=None):
        """y = X x, X = Im Z, by the cos-kernel product (include/mlfma.h: mlfma_matvec_x)."""
        return self._product(self._lib.mlfma_matvec_x, x, y, stream)

    def matvec_r(self, x, y=None, stream=None):
        """y = R x, R = Re Z, by the sin-kernel sibling product (mlfma_matvec_r)."""
        return self._product(self._lib.mlfma_matvec_r, x, y, stream)

    def matvec_host(self, x: np.ndarray, prec: int = FP32, y: np.ndarray = None, stream=None) -> np.ndarray:
        """y = Z x for HOST arrays (copies inside the call; waits for completion)."""
        rdt = np.float64 if prec == FP64 else np.float32
        cdt = np.complex128 if prec == FP64 else np.complex64
        squeeze = x.ndim == 1
        x2 = x.reshape(self.n, -1)
        xc = 1 if np.iscomplexobj(x2) else 0
        x2 = np.ascontiguousarray(x2, dtype=cdt if xc else rdt)
        B = x2.shape[1]
        if y is None:
            y = np.empty((self.n, B), dtype=cdt)
        if y.dtype != cdt or not y.flags.c_contiguous or y.size != self.n * B:
            raise ValueError("y must be a C-contiguous %s array with N*B elements" % np.dtype(cdt))
        _check(self._lib.mlfma_matvec_host(self._h, _np_ptr(x2), xc, _np_ptr(y), B, prec,
                                           ctypes.c_void_p(stream or 0)))
        return y.reshape(self.n) if squeeze else y

    def tune(self, B, prec=FP32, complex_x=False, stream=None, cache=None):
        """Autotune the launch shapes for products of B columns; returns the
        serial stage-time sums (ms) with the built-in and the chosen shapes.
        cache: path of a JSON file of earlier choices keyed by GPU, tree
        geometry, columns and precision; a hit pins the stored shapes
        (mlfma_tune_set) without timing and returns (None, None)."""
        import torch
        key = None
        if cache is not None:
            key = tune_cache_key(torch.cuda.get_device_name(), self.info(), self.interp_order, B, prec, complex_x)
            entry = _read_tune_cache(cache).get(key)
            if isinstance(entry, list) and len(entry) == TUNE_FIELDS:
                try:
                    self.tune_set(B, entry, prec, complex_x)
                    return None, None
                except (MlfmaError, TypeError, ValueError):   # a damaged entry: tune again and replace it
                    pass
        d, t = ctypes.c_double(), ctypes.c_double()
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        _check(self._lib.mlfma_tune(self._h, int(B), 1 if complex_x else 0, int(prec), ctypes.c_void_p(s),
                                    ctypes.byref(d), ctypes.byref(t)))
        if key is not None:
            table = _read_tune_cache(cache)
            table[key] = self.tune_get(B, prec, complex_x).tolist()
            _write_tune_cache(cache, table)
        return d.value, t.value

    def export_field(self, prec, which, level, B) -> np.ndarray:
        """Field of a far level after the last product in `prec` (which 0 =
        outgoing S, 1 = incoming G): complex [boxes, 2, K, B], leaf box order."""
        need = ctypes.c_int64()
        _check(self._lib.mlfma_export_field(self._h, int(prec), int(which), int(level), int(B), None, 0,
                                            ctypes.byref(need)))
        buf = np.zeros(need.value, np.uint8)
        _check(self._lib.mlfma_export_field(self._h, int(prec), int(which), int(level), int(B), _np_ptr(buf),
                                            need.value, ctypes.byref(need)))
        cdt = np.complex64 if prec == FP32 else np.complex128
        K = self.info()["samples_K"][level]
        return buf.view(cdt).reshape(-1, 2, K, int(B))

    def tune_get(self, B, prec=FP32, complex_x=False) -> np.ndarray:
        """Launch shapes used for (B, prec) (include/mlfma.h: mlfma_tune_get)."""
        c = np.zeros(TUNE_FIELDS, np.int32)
        _check(self._lib.mlfma_tune_get(self._h, int(B), 1 if complex_x else 0, int(prec), _np_ptr(c)))
        return c

    def tune_set(self, B, choices, prec=FP32, complex_x=False):
        """Pin launch shapes for (B, prec) (mlfma_tune_set)."""
        c = np.ascontiguousarray(choices, dtype=np.int32).reshape(TUNE_FIELDS)
        _check(self._lib.mlfma_tune_set(self._h, int(B), 1 if complex_x else 0, int(prec), _np_ptr(c)))

    def profile_stages(self, x, y=None, stream=None, prec=None) -> dict:
        """Serial per-stage device times (ms) of one product (measurement aid)."""
        import torch
        ms = np.zeros(STAGE_COUNT)
        fn = lambda h, xp, xc, yp, B, prec, s: self._lib.mlfma_profile_stages(h, xp, xc, yp, B, prec, s, _np_ptr(ms))
        self._product(fn, x, y, stream, prec)
        out = {"prepare": ms[0], "near": ms[1], "radiate": ms[2], "receive": ms[69], "finalize": ms[70]}
        for l in range(22):
            if ms[3 + l]:
                out["up%d" % l] = ms[3 + l]
            if ms[25 + l]:
                out["translate%d" % l] = ms[25 + l]
            if ms[47 + l]:
                out["down%d" % l] = ms[47 + l]
        return out

    def cm_solve(self, nev=10, ncv=30, op=CM_ZINV_R, prec=FP32, tol=1e-8, gmres_tol=1e-6, gmres_restart=50,
                 max_inner=2000, max_restarts=200, use_sai=True, seed=1412175602, vectors=True):
        """Characteristic values nearest zero (and real currents) by IRA:
        returns (lambda [nev], J [N, nev] or None, stats dict)."""
        o = CmOpts()
        _check(self._lib.mlfma_cm_default_opts(ctypes.byref(o)))
        o.nev, o.ncv, o.op, o.prec = int(nev), int(ncv), int(op), int(prec)
        o.tol, o.gmres_tol = float(tol), float(gmres_tol)
        o.gmres_restart, o.max_inner, o.max_restarts = int(gmres_restart), int(max_inner), int(max_restarts)
        o.use_sai, o.seed = 1 if use_sai else 0, int(seed)
        lam = np.zeros(nev)
        J = np.zeros((self.n, nev)) if vectors else None
        st = CmStats()
        rc = self._lib.cm_ira_solve(self._h, ctypes.byref(o), _np_ptr(lam), _np_ptr(J) if vectors else None,
                                    ctypes.byref(st))
        stats = {f: getattr(st, f) for f, _ in CmStats._fields_}
        if rc != 0:
            err = MlfmaError(rc, self._lib.mlfma_last_error().decode())
            err.stats, err.values = stats, lam   # ENOTCONV: counters and the current Ritz values
            raise err
        return lam, J, stats

    def cm_block_solve(self, nev=10, block=32, prec=FP32, tol=1e-5, gmres_tol=1e-6, gmres_restart=200,
                       max_inner=2000, max_iters=50, use_sai=True, seed=1412175602, vectors=True):
        """Characteristic values nearest zero (and real currents) by block
        shift-invert subspace iteration on X^-1 R (include/mlfma.h:
        cm_block_solve): returns (lambda [nev], J [N, nev] or None, stats)."""
        o = CmOpts()
        _check(self._lib.mlfma_cm_default_opts(ctypes.byref(o)))
        o.nev, o.ncv, o.op, o.prec = int(nev), int(block), CM_XINV_R, int(prec)
        o.tol, o.gmres_tol = float(tol), float(gmres_tol)
        o.gmres_restart, o.max_inner, o.max_restarts = int(gmres_restart), int(max_inner), int(max_iters)
        o.use_sai, o.seed = 1 if use_sai else 0, int(seed)
        lam = np.zeros(nev)
        J = np.zeros((self.n, nev)) if vectors else None
        st = CmStats()
        rc = self._lib.cm_block_solve(self._h, ctypes.byref(o), _np_ptr(lam), _np_ptr(J) if vectors else None,
                                      ctypes.byref(st))
        stats = {f: getattr(st, f) for f, _ in CmStats._fields_}
        if rc != 0:
            err = MlfmaError(rc, self._lib.mlfma_last_error().decode())
            err.stats, err.values = stats, lam
            raise err
        return lam, J, stats

    def cm_derivatives(self, lam, J, prec=FP64) -> np.ndarray:
        """d lambda / dk of characteristic pairs (include/mlfma.h: cm_eig_derivatives)."""
        lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
        J = np.ascontiguousarray(J, dtype=np.float64).reshape(self.n, lam.shape[0])
        out = np.zeros(lam.shape[0])
        _check(self._lib.cm_eig_derivatives(self._h, lam.shape[0], _np_ptr(lam), _np_ptr(J), int(prec),
                                            _np_ptr(out)))
        return out

    def sync(self, stream=None):
        """Wait for the plan's work on `stream` and raise a pending device-side
        error (mlfma_sync)."""
        _check(self._lib.mlfma_sync(self._h, ctypes.c_void_p(stream or 0)))

    def close(self):
        """Release the plan (mlfma_destroy) unless it belongs to a set."""
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                self._lib.mlfma_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rayleigh_ritz(Y, RY, W):
    """Ritz pairs of T = X^-1 R on span Y in the R inner product from Y,
    R Y and W = T Y (include/mlfma.h: cm_rayleigh_ritz; host only): returns
    (mu [r] sorted by |mu|, largest first, lambda = 1 / mu; coef [p, r] with
    Ritz vectors Y coef)."""
    L = load()
    Y, RY, W = (np.ascontiguousarray(a, dtype=np.float64) for a in (Y, RY, W))
    if Y.ndim != 2 or Y.shape != RY.shape or Y.shape != W.shape:
        raise ValueError("Y, RY and W must be [n, p] arrays of one shape")
    n, p = Y.shape
    mu, coef, r = np.zeros(p), np.zeros((p, p)), ctypes.c_int(0)
    _check(L.cm_rayleigh_ritz(n, p, _np_ptr(Y), _np_ptr(RY), _np_ptr(W), _np_ptr(mu), _np_ptr(coef),
                              ctypes.byref(r)))
    return mu[:r.value], coef[:, :r.value]


def track_modes(lam_a, Ja, lam_b, Jb, cluster_tol=1e-2):
    """Pair the modes (lam_b, Jb) with the previous wavenumber's (lam_a, Ja)
    (cm_track_modes): returns (match [nb] indices into set a or -1,
    overlap [nb] cluster-pair scores)."""
    L = load()
    la = np.ascontiguousarray(lam_a, dtype=np.float64)
    lb = np.ascontiguousarray(lam_b, dtype=np.float64)
    A = np.ascontiguousarray(Ja, dtype=np.float64)
    Bm = np.ascontiguousarray(Jb, dtype=np.float64)
    if A.ndim != 2 or Bm.ndim != 2 or A.shape[0] != Bm.shape[0] or A.shape[1] != la.size or Bm.shape[1] != lb.size:
        raise ValueError("Ja [n][na], Jb [n][nb] with matching value counts")
    match = np.zeros(lb.size, np.int32)
    ov = np.zeros(lb.size)
    _check(L.cm_track_modes(A.shape[0], la.size, _np_ptr(la), _np_ptr(A), lb.size, _np_ptr(lb), _np_ptr(Bm),
                            float(cluster_tol), _np_ptr(match), _np_ptr(ov)))
    return match, ov


def tune_cache_key(gpu_name, info, interp_order, B, prec, complex_x) -> str:
    """Key of a tuned-shape entry: the GPU, the tree's geometry (boxes,
    truncation numbers and samples per level, leaf sizes, near entries), the
    interpolation order, the columns and the precision."""
    geo = "/".join("%d:%d:%d" % (b, l, k) for b, l, k in zip(info["box_count"], info["trunc_L"], info["samples_K"]))
    return "|".join([str(gpu_name), "n%d" % info["n"], geo, "leaf%d" % info["max_leaf_unknowns"],
                     "nnz%d" % info["near_nnz"], "p%d" % interp_order, "B%d" % int(B),
                     "fp64" if prec == FP64 else "fp32", "complex" if complex_x else "real"])


def _read_tune_cache(path) -> dict:
    import json
    try:
        with open(path) as f:
            t = json.load(f)
        return t if isinstance(t, dict) else {}
    except (OSError, ValueError):
        return {}


def _write_tune_cache(path, table: dict):
    import json
    tmp = "%s.tmp.%d" % (path, os.getpid())
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _autograd_function():
    import torch
    from torch.autograd.function import once_differentiable

    class MlfmaZ(torch.autograd.Function):
        """y = Z(k) x with gradients for x (through Z^H) and for the 0-d
        wavenumber tensor k (through dZ/dk): grad_k = Re sum conj(g) (dZ/dk x)
        for the upstream gradient g, PyTorch's convention for a real input of
        a complex output."""

        @staticmethod
        def forward(ctx, x, k, plan):
            if k.dim() != 0:
                raise ValueError("k must be a 0-d tensor")
            kv = float(k.detach().cpu())
            if abs(kv - plan.k) > 1e-12 * abs(plan.k):
                raise ValueError("k = %r differs from the plan's wavenumber %r" % (kv, plan.k))
            ctx.plan = plan
            ctx.save_for_backward(x)
            return plan.matvec(x)

        @staticmethod
        @once_differentiable
        def backward(ctx, g):
            (x,) = ctx.saved_tensors
            plan = ctx.plan
            gx = gk = None
            if ctx.needs_input_grad[0]:
                gx = plan.matvec_adjoint(g.contiguous())
                if not x.is_complex():
                    gx = gx.real.contiguous()
            if ctx.needs_input_grad[1]:
                dy = plan.matvec_dk(x)
                gk = (g.conj() * dy).real.sum().to(torch.float64)
            return gx, gk, None

    return MlfmaZ


_MlfmaZ = None


def efie_product(plan: MlfmaPlan, x, k):
    """Differentiable y = Z(k) x for a CUDA tensor x [N] or [N, B] and a 0-d
    tensor k equal to the plan's wavenumber (gradients for x and k)."""
    global _MlfmaZ
    if _MlfmaZ is None:
        _MlfmaZ = _autograd_function()
    return _MlfmaZ.apply(x, k, plan)


class MlfmaPlanSet:
    """One plan per wavenumber on one mesh, admitted by device memory, with
    the products of a wave in one graph (include/mlfma.h: mlfma_set_*)."""

    def __init__(self, verts, tris, ks, levels, digits=3.0, interp_order=10, max_batch=64,
                 precisions=(FP32, FP64), device=None, budget_bytes=0):
        L = load()
        self._lib = L
        v, t = _mesh_arrays(verts, tris)
        kk = np.ascontiguousarray(np.asarray(ks, dtype=np.float64).reshape(-1))
        o = Opts()
        _check(L.mlfma_default_opts(ctypes.byref(o)))
        o.interp_order, o.max_batch = int(interp_order), int(max_batch)
        o.precisions = sum(1 << p for p in precisions)
        if device is None:
            import torch
            device = torch.cuda.current_device()
        o.device = int(device)
        h = ctypes.c_void_p()
        _check(L.mlfma_set_create(_np_ptr(v), v.shape[0], _np_ptr(t), t.shape[0], _np_ptr(kk), kk.shape[0],
                                  int(levels), float(digits), ctypes.byref(o), int(budget_bytes), ctypes.byref(h)))
        self._h = h
        self.ks = kk.copy()
        self.max_batch = int(max_batch)
        p0 = ctypes.c_void_p()
        _check(L.mlfma_set_plan(h, 0, ctypes.byref(p0)))
        n = ctypes.c_int64()
        _check(L.mlfma_num_unknowns(p0, ctypes.byref(n)))
        self.n = int(n.value)

    def info(self) -> dict:
        """Waves, each wavenumber's wave, and estimated and actual device
        bytes per plan (mlfma_set_info)."""
        nk = len(self.ks)
        waves = ctypes.c_int()
        wave_of = np.zeros(nk, np.int32)
        est = np.zeros(nk, np.int64)
        dev = np.zeros(nk, np.int64)
        _check(self._lib.mlfma_set_info(self._h, None, ctypes.byref(waves), _np_ptr(wave_of), _np_ptr(est),
                                        _np_ptr(dev)))
        return {"waves": waves.value, "wave_of": wave_of.tolist(), "est_bytes": est.tolist(),
                "device_bytes": dev.tolist()}

    def plan(self, f: int) -> "MlfmaPlan":
        """The set's plan of wavenumber f (owned by the set)."""
        h = ctypes.c_void_p()
        _check(self._lib.mlfma_set_plan(self._h, int(f), ctypes.byref(h)))
        return MlfmaPlan(None, None, self.ks[f], 0, max_batch=self.max_batch, _handle=h)

    def matvec(self, x, y=None, stream=None):
        """y[f] = Z(k_f) x[f] for x [nk, N, B] (or one [N, B] block for every
        wavenumber); returns [nk, N, B] complex."""
        import torch
        _check_device_pair(x, y)
        nk = len(self.ks)
        shared = x.dim() == 2 or (x.dim() == 1)
        x3 = x.reshape(self.n, -1) if shared else x.reshape(nk, self.n, -1)
        x3 = x3.contiguous()
        prec = MlfmaPlan._prec_of(x3.dtype)
        xc = 1 if x3.is_complex() else 0
        cdt = torch.complex64 if prec == FP32 else torch.complex128
        B = x3.shape[-1]
        if y is None:
            y = torch.empty((nk, self.n, B), dtype=cdt, device=x3.device)
        if y.dtype != cdt or not y.is_contiguous() or y.numel() != nk * self.n * B:
            raise ValueError("y must be a contiguous %s tensor with nk*N*B elements" % cdt)
        s = torch.cuda.current_stream(x3.device).cuda_stream if stream is None else stream
        _check(self._lib.mlfma_set_matvec(self._h, ctypes.c_void_p(x3.data_ptr()), 1 if shared else 0, xc,
                                          ctypes.c_void_p(y.data_ptr()), B, prec, ctypes.c_void_p(s)))
        return y

    def close(self):
        """Release the set and all its plans (mlfma_set_destroy)."""
        if getattr(self, "_h", None):
            self._lib.mlfma_set_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
