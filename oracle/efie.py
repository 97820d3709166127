"""ctypes driver for the FP64 EFIE oracle (efie_oracle.c).  Test infrastructure.

Z follows Section II, Eq. (5): Z_ij = i k eta <f_i, G, f_j> with the
scalar Green's function exp(ikR)/R of Eq. (3) (no 1/(4 pi)).  The product
y = Z x is the plain definition: a dense matrix (small N) or exact rows
(large N) times x, with NumPy's matmul as the only library step.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build
from .rwg import rwg_list

ETA0 = 376.730313668  # free-space impedance, ohm

_lib = None


def load(path: str):
    """Open an oracle library compiled from efie_oracle.c at `path` and
    declare its entry points (lib() opens the package's own build)."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i = ctypes.c_int
    d = ctypes.c_double
    L.oracle_zfill.argtypes = [i, P, i, P, i, P, P, P, d, d, P, i]
    L.oracle_dzfill.argtypes = [i, P, i, P, i, P, P, P, d, d, P, i]
    L.oracle_zrows.argtypes = [i, P, i, P, i, P, P, P, d, d, i, P, P, i]
    L.oracle_dzrows.argtypes = [i, P, i, P, i, P, P, P, d, d, i, P, P, i]
    L.oracle_tri_potential.argtypes = [i, P, i, P, P, i, d, i, P]
    L.oracle_static_potential.argtypes = [P, P, P, P, P]
    L.oracle_pair_is_singular.argtypes = [i, P, i, P, i, i]
    L.oracle_rule7.argtypes = [P]
    for f in ("oracle_zfill", "oracle_dzfill", "oracle_zrows", "oracle_dzrows", "oracle_tri_potential",
              "oracle_static_potential", "oracle_pair_is_singular", "oracle_rule7",
              "oracle_num_threads"):
        getattr(L, f).restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Problem:
    """A meshed PEC surface at wavenumber k, with its RWG list."""

    def __init__(self, verts, tris, k, eta=ETA0):
        self.verts = np.ascontiguousarray(verts, dtype=np.float64)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.k = float(k)
        self.eta = float(eta)
        r = rwg_list(self.verts, self.tris)
        self.edge_v = r["edge_v"]
        self.tri = np.ascontiguousarray(r["tri"])
        self.vfree = np.ascontiguousarray(r["vfree"])
        self.length = np.ascontiguousarray(r["length"])
        self.n = self.tri.shape[0]

    def _mesh_args(self):
        return (self.verts.shape[0], _p(self.verts), self.tris.shape[0], _p(self.tris),
                self.n, _p(self.tri), _p(self.vfree), _p(self.length))

    def dense(self, nthreads: int = 0) -> np.ndarray:
        """Dense symmetric Z [N, N] complex128."""
        Z = np.zeros((self.n, self.n), dtype=np.complex128)
        rc = lib().oracle_zfill(*self._mesh_args(), self.k, self.eta, _p(Z), int(nthreads))
        if rc != 0:
            raise MemoryError("oracle_zfill failed")
        return Z

    def dense_dk(self, nthreads: int = 0) -> np.ndarray:
        """Dense symmetric dZ/dk [N, N] complex128 (Section II, Eq. (5)
        differentiated in k with the quadrature fixed)."""
        Z = np.zeros((self.n, self.n), dtype=np.complex128)
        rc = lib().oracle_dzfill(*self._mesh_args(), self.k, self.eta, _p(Z), int(nthreads))
        if rc != 0:
            raise MemoryError("oracle_dzfill failed")
        return Z

    def rows(self, rows, nthreads: int = 0) -> np.ndarray:
        """Rows Z[rows, :] of the symmetric Z, complex128 [len(rows), N]."""
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).reshape(-1))
        out = np.zeros((rows.shape[0], self.n), dtype=np.complex128)
        rc = lib().oracle_zrows(*self._mesh_args(), self.k, self.eta, rows.shape[0], _p(rows),
                                _p(out), int(nthreads))
        if rc != 0:
            raise MemoryError("oracle_zrows failed")
        return out

    def rows_dk(self, rows, nthreads: int = 0) -> np.ndarray:
        """Rows of the symmetric dZ/dk, complex128 [len(rows), N]."""
        rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).reshape(-1))
        out = np.zeros((rows.shape[0], self.n), dtype=np.complex128)
        rc = lib().oracle_dzrows(*self._mesh_args(), self.k, self.eta, rows.shape[0], _p(rows),
                                 _p(out), int(nthreads))
        if rc != 0:
            raise MemoryError("oracle_dzrows failed")
        return out

    def matvec_rows(self, x: np.ndarray, rows, nthreads: int = 0) -> np.ndarray:
        """(Z x)[rows] for x [N] or [N, B]: each row of Z computed exactly."""
        return self.rows(rows, nthreads) @ x

    def tri_potential(self, r, s: int, singular: bool):
        """Inner potentials of triangle s at point r: P0 = int g dS',
        P1 = int r' g dS' (complex [3])."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        out = np.zeros(8)
        lib().oracle_tri_potential(self.verts.shape[0], _p(self.verts), self.tris.shape[0],
                                   _p(self.tris), _p(r), int(s), self.k, int(singular), _p(out))
        return out[0] + 1j * out[1], out[2::2] + 1j * out[3::2]

    def pair_is_singular(self, t: int, s: int) -> bool:
        return bool(lib().oracle_pair_is_singular(self.verts.shape[0], _p(self.verts),
                                                  self.tris.shape[0], _p(self.tris), int(t), int(s)))


def static_potential(r, tri9):
    """Closed-form int_T dS'/R and int_T (rho' - rho)/R dS' for a flat triangle
    (rows of tri9 are its vertices), and rho, the projection of r."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    t = np.ascontiguousarray(tri9, dtype=np.float64).reshape(9)
    I0 = np.zeros(1)
    I1 = np.zeros(3)
    rho = np.zeros(3)
    lib().oracle_static_potential(_p(r), _p(t), _p(I0), _p(I1), _p(rho))
    return I0[0], I1, rho


def rule7() -> np.ndarray:
    out = np.zeros((7, 4))
    lib().oracle_rule7(_p(out))
    return out


def num_threads() -> int:
    return int(lib().oracle_num_threads())
