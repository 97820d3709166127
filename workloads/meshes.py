"""Seeded synthetic surface meshes: closed spheres and cubes, and an open plate
with strip dipoles.

Every generator returns ``(verts, tris)``: ``verts`` float64 [nv, 3] in metres,
``tris`` int32 [nt, 3] with a consistent orientation (counter-clockwise seen
from outside for closed surfaces, from +z for the plate and strips).  Nothing
here knows about basis functions, Green's functions or the fast multipole
method: these are the inputs that both the CPU oracle and the GPU library take.

The paper's own geometries (a 1.0 x 0.6 m plate, a sphere of radius 0.75
wavelengths, a UAV and a Boeing 787, Section V) come without meshes; these
stand in for them with the same kinds of surface (smooth closed, flat with
boundary edges, closed with sharp edges).
"""
from __future__ import annotations

import numpy as np

_PHI = (1.0 + 5.0 ** 0.5) / 2.0


def _icosahedron():
    v = np.array([
        [-1, _PHI, 0], [1, _PHI, 0], [-1, -_PHI, 0], [1, -_PHI, 0],
        [0, -1, _PHI], [0, 1, _PHI], [0, -1, -_PHI], [0, 1, -_PHI],
        [_PHI, 0, -1], [_PHI, 0, 1], [-_PHI, 0, -1], [-_PHI, 0, 1],
    ], dtype=np.float64)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int64)
    return v, f


def _orient_outward(verts, tris):
    """Flip triangles whose normal points towards the origin (closed,
    star-shaped surfaces centred at the origin only)."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    n = np.cross(b - a, c - a)
    inward = np.einsum("ij,ij->i", n, a + b + c) < 0
    tris = tris.copy()
    tris[inward, 1], tris[inward, 2] = tris[inward, 2].copy(), tris[inward, 1].copy()
    return tris


def icosphere(subdivisions: int, radius: float):
    """Icosahedron refined ``subdivisions`` times (each triangle split in four
    at its edge midpoints), every vertex projected onto the sphere.
    20 * 4**s triangles and 30 * 4**s edges."""
    v, f = _icosahedron()
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    f = _orient_outward(v, f)
    for _ in range(subdivisions):
        nf = f.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        uniq, inv = np.unique(e, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mid = 0.5 * (v[uniq[:, 0]] + v[uniq[:, 1]])
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        base = v.shape[0]
        v = np.concatenate([v, mid], axis=0)
        ab = base + inv[0:nf]
        bc = base + inv[nf:2 * nf]
        ca = base + inv[2 * nf:3 * nf]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate([
            np.stack([a, ab, ca], 1), np.stack([ab, b, bc], 1),
            np.stack([ca, bc, c], 1), np.stack([ab, bc, ca], 1),
        ], axis=0)
    return (v * radius).astype(np.float64), f.astype(np.int32)


def _grid_patch(origin, u, v, nu, nv, hu, hv):
    """Flat rectangle origin + i*hu*u + j*hv*v, nu x nv cells, each cell split
    along its (0,0)-(1,1) diagonal; counter-clockwise about u x v."""
    ii, jj = np.meshgrid(np.arange(nu + 1), np.arange(nv + 1), indexing="ij")
    pts = (np.asarray(origin, float)[None, :]
           + (ii.reshape(-1, 1) * hu) * np.asarray(u, float)[None, :]
           + (jj.reshape(-1, 1) * hv) * np.asarray(v, float)[None, :])
    idx = np.arange((nu + 1) * (nv + 1)).reshape(nu + 1, nv + 1)
    p00 = idx[:-1, :-1].reshape(-1)
    p10 = idx[1:, :-1].reshape(-1)
    p11 = idx[1:, 1:].reshape(-1)
    p01 = idx[:-1, 1:].reshape(-1)
    t = np.concatenate([np.stack([p00, p10, p11], 1), np.stack([p00, p11, p01], 1)], 0)
    return pts, t


def plate_with_strips(size: float = 6.0, cells: int = 60, strips: bool = True,
                      strip_len: float = 0.5, strip_w: float = 0.02,
                      strip_cells: int = 5, strip_height: float = 0.25,
                      strip_centres=(-2.25, -0.75, 0.75, 2.25)):
    """Square PEC plate in z = 0 (``cells`` x ``cells`` squares, each split by
    its (0,0)-(1,1) diagonal) plus, optionally, a 4 x 4 array of thin strips
    along x at height ``strip_height``, each meshed as ``strip_cells`` x 1 cells.
    Defaults: 7,200 plate triangles (10,680 interior edges) and 16 strips of 10
    triangles (9 interior edges each)."""
    h = size / cells
    pts, t = _grid_patch((-size / 2, -size / 2, 0.0), (1, 0, 0), (0, 1, 0), cells, cells, h, h)
    verts = [pts]
    tris = [t]
    nv = pts.shape[0]
    if strips:
        for cx in strip_centres:
            for cy in strip_centres:
                o = (cx - strip_len / 2, cy - strip_w / 2, strip_height)
                p, s = _grid_patch(o, (1, 0, 0), (0, 1, 0), strip_cells, 1,
                                   strip_len / strip_cells, strip_w)
                verts.append(p)
                tris.append(s + nv)
                nv += p.shape[0]
    return np.concatenate(verts, 0).astype(np.float64), np.concatenate(tris, 0).astype(np.int32)


def plate(lx: float, ly: float, nx: int, ny: int):
    """Rectangular plate lx x ly in z = 0 centred at the origin, nx x ny cells."""
    pts, t = _grid_patch((-lx / 2, -ly / 2, 0.0), (1, 0, 0), (0, 1, 0), nx, ny, lx / nx, ly / ny)
    return pts.astype(np.float64), t.astype(np.int32)


def cube(side: float, cells: int):
    """Closed cube centred at the origin, ``cells`` x ``cells`` squares per face,
    each split by its (0,0)-(1,1) diagonal, vertices shared along the cube's
    edges; outward orientation.  12 * cells**2 triangles, 18 * cells**2 edges."""
    n = cells
    faces = [  # (fixed axis, fixed value, u axis, v axis) with u x v outward
        (0, n, 1, 2), (0, 0, 2, 1),
        (1, n, 2, 0), (1, 0, 0, 2),
        (2, n, 0, 1), (2, 0, 1, 0),
    ]
    keys = []
    tris = []
    for ax, val, ua, va in faces:
        ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
        lat = np.zeros((n + 1, n + 1, 3), dtype=np.int64)
        lat[..., ax] = val
        lat[..., ua] = ii
        lat[..., va] = jj
        lat = lat.reshape(-1, 3)
        key = (lat[:, 0] * (n + 1) + lat[:, 1]) * (n + 1) + lat[:, 2]
        idx = np.arange((n + 1) * (n + 1)).reshape(n + 1, n + 1)
        p00 = idx[:-1, :-1].reshape(-1)
        p10 = idx[1:, :-1].reshape(-1)
        p11 = idx[1:, 1:].reshape(-1)
        p01 = idx[:-1, 1:].reshape(-1)
        t = np.concatenate([np.stack([p00, p10, p11], 1), np.stack([p00, p11, p01], 1)], 0)
        keys.append(key)
        tris.append(key[t])
    allkeys = np.concatenate(keys)
    uniq, inv = np.unique(allkeys, return_inverse=True)
    tri_keys = np.concatenate(tris, 0)
    tri_idx = np.searchsorted(uniq, tri_keys)
    k = uniq
    lat = np.stack([k // ((n + 1) * (n + 1)), (k // (n + 1)) % (n + 1), k % (n + 1)], 1)
    verts = (lat.astype(np.float64) - n / 2.0) * (side / n)
    return verts, tri_idx.astype(np.int32)


def two_triangle_pairs(separation: float, size: float = 0.05):
    """Two small separated RWG pairs (four triangles, two interior edges): a
    tiny far-interaction case.  Pair 1 sits at the origin, pair 2 at
    (separation, 0.3*separation, 0.1*separation)."""
    base = np.array([[0, 0, 0], [1, 0, 0], [0.4, 0.9, 0.1], [0.6, -0.8, -0.1]], float) * size
    t = np.array([[0, 1, 2], [1, 0, 3]], dtype=np.int32)
    off = np.array([separation, 0.3 * separation, 0.1 * separation])
    verts = np.concatenate([base, base + off], 0)
    tris = np.concatenate([t, t + 4], 0)
    return verts, tris
