"""The seeded synthetic inputs that both the oracle and the GPU path take
(workloads/): the right-hand sides are reproducible from their seed and
N(0, 1); the closed meshes (spheres, cube) are 2-manifolds of genus 0
(V - E + F = 2, every edge on exactly two triangles traversed in opposite
directions), oriented outward (positive enclosed volume, equal to the
solid's to the mesh's accuracy); the plate's triangles are finite, in range
and of positive area (its RWG count is pinned with the others in
test_oracle_matrix)."""
import math

import numpy as np
import pytest

import workloads


def test_rhs_reproducible_and_standard_normal():
    a, b = workloads.rhs(5000, 8, 3), workloads.rhs(5000, 8, 3)
    assert np.array_equal(a, b) and a.shape == (5000, 8) and a.dtype == np.float64
    assert not np.array_equal(a, workloads.rhs(5000, 8, 4))
    assert abs(a.mean()) < 0.02 and abs(a.std() - 1.0) < 0.02
    c = workloads.rhs_complex(5000, 8, 3)
    assert np.array_equal(c, workloads.rhs_complex(5000, 8, 3)) and c.dtype == np.complex128
    assert abs(c.real.std() - 1.0) < 0.02 and abs(c.imag.std() - 1.0) < 0.02


def _edges(t):
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    return e


@pytest.mark.parametrize("mesh,volume", [
    (lambda: workloads.icosphere(3, 0.5), 4 / 3 * math.pi * 0.5 ** 3),
    (lambda: workloads.icosphere(5, 2.0), 4 / 3 * math.pi * 2.0 ** 3),
    (lambda: workloads.cube(8.0, 10), 8.0 ** 3),
])
def test_closed_meshes_are_outward_genus_zero_manifolds(mesh, volume):
    v, t = mesh()
    e = _edges(t)
    directed = set(map(tuple, e))
    assert len(directed) == len(e)                                   # no edge traversed twice the same way
    assert all((b, a) in directed for a, b in directed)              # each edge once in each direction
    n_edges = len(e) // 2
    assert len(v) - n_edges + len(t) == 2                            # Euler characteristic of a sphere
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0       # divergence theorem
    assert vol > 0 and abs(vol - volume) < 0.02 * volume
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    assert area.min() > 0


def test_plate_with_strips_counts():
    v, t = workloads.plate_with_strips()
    assert np.isfinite(v).all() and t.min() >= 0 and t.max() < len(v)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    assert (0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)).min() > 0
