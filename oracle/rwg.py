"""RWG basis list, canonical order.  Test infrastructure.

An RWG function lives on an interior edge shared by exactly two triangles
(Section II: the current is expanded in RWG functions f_j).  Canonical order:
edges sorted by (smaller vertex index, larger vertex index).  T+ is the
triangle whose vertex cycle runs along the edge from the smaller to the
larger vertex index; T- is the other one.  Boundary edges (one triangle)
carry no function; an edge on three or more triangles, or one traversed the
same way by both of its triangles, is an error.
"""
from __future__ import annotations

import numpy as np


class MeshError(ValueError):
    pass


def rwg_list(verts: np.ndarray, tris: np.ndarray):
    """Return dict with ``edge_v`` [N,2] (lo, hi), ``tri`` [N,2] (T+, T-),
    ``vfree`` [N,2] (v+, v-), ``length`` [N] (float64)."""
    tris = np.asarray(tris, dtype=np.int64)
    nt = tris.shape[0]
    a = tris[:, [0, 1, 2]].reshape(-1)
    b = tris[:, [1, 2, 0]].reshape(-1)
    opp = tris[:, [2, 0, 1]].reshape(-1)          # vertex opposite directed edge a->b
    tid = np.repeat(np.arange(nt), 3)
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    fwd = a < b
    order = np.lexsort((~fwd, hi, lo))            # by lo, then hi, forward first
    lo, hi, fwd, tid, opp = lo[order], hi[order], fwd[order], tid[order], opp[order]
    key_change = np.ones(lo.shape[0], dtype=bool)
    key_change[1:] = (lo[1:] != lo[:-1]) | (hi[1:] != hi[:-1])
    starts = np.flatnonzero(key_change)
    counts = np.diff(np.append(starts, lo.shape[0]))
    if np.any(counts > 2):
        raise MeshError("non-manifold edge (three or more triangles)")
    two = starts[counts == 2]
    if np.any(fwd[two] == fwd[two + 1]):
        raise MeshError("inconsistent triangle orientation across an edge")
    tp, tm = tid[two], tid[two + 1]
    vp, vm = opp[two], opp[two + 1]
    edge_v = np.stack([lo[two], hi[two]], 1)
    length = np.linalg.norm(verts[edge_v[:, 1]] - verts[edge_v[:, 0]], axis=1)
    return {
        "edge_v": edge_v.astype(np.int32),
        "tri": np.stack([tp, tm], 1).astype(np.int32),
        "vfree": np.stack([vp, vm], 1).astype(np.int32),
        "length": length.astype(np.float64),
    }
