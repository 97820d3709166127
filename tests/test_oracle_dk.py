"""Pins of the oracle's dZ/dk, the derivative in wavenumber of the EFIE
matrix of Section II, Eq. (5), with the quadrature and the mesh fixed.

The derivative is filled by its own routine (the four terms
i eta A + i k eta A' + (i eta / k^2) Phi - (i eta / k) Phi', with
dg/dk = i exp(ikR)); it is pinned here against central differences of the
oracle's Z(k), which runs through the singularity-extraction path instead
and shares no term with it.  A dropped term, a wrong sign or a wrong power of
k each moves the result by O(1) of the tested norm."""
import numpy as np
import pytest

import workloads
from oracle import efie


def _fd(P, h):
    k = P.k
    Pp = efie.Problem(P.verts, P.tris, k + h)
    Pm = efie.Problem(P.verts, P.tris, k - h)
    return (Pp.dense() - Pm.dense()) / (2 * h)


@pytest.mark.parametrize("mesh,k", [
    (lambda: workloads.icosphere(2, 0.5), 2 * np.pi),
    (lambda: workloads.icosphere(1, 0.5), 2 * np.pi * 0.4),
    (lambda: workloads.plate(1.0, 1.0, 6, 6), 2 * np.pi * 1.3),
])
def test_dk_matches_central_differences(mesh, k):
    v, t = mesh()
    P = efie.Problem(v, t, k)
    D = P.dense_dk()
    F = _fd(P, 1e-4 * k)
    err = np.abs(D - F).max() / np.abs(F).max()
    assert err < 1e-6, err
    assert np.linalg.norm(D - F) / np.linalg.norm(F) < 1e-6


def test_dk_symmetric_and_nonzero_terms():
    v, t = workloads.icosphere(2, 0.5)
    P = efie.Problem(v, t, 2 * np.pi)
    D = P.dense_dk()
    assert np.array_equal(D, D.T)
    # both parts carry weight: the reactive part grows from both the vector
    # and the scalar potential, the resistive part is nonzero at this size
    assert np.linalg.norm(D.real) > 1e-2 * np.linalg.norm(D)
    assert np.linalg.norm(D.imag) > 1e-2 * np.linalg.norm(D)


def test_dk_reproduces_step_in_k_to_second_order():
    # Z(k + h) ~ Z(k) + h dZ/dk with error O(h^2): halving h quarters it
    v, t = workloads.icosphere(1, 0.5)
    k = 2 * np.pi
    P = efie.Problem(v, t, k)
    Z0, D = P.dense(), P.dense_dk()
    errs = []
    for h in (2e-2, 1e-2):
        Z1 = efie.Problem(v, t, k + h).dense()
        errs.append(np.linalg.norm(Z1 - Z0 - h * D))
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.5, ratio
