"""Pins of the oracle's building blocks against mathematics it does not use
itself: polynomial exactness of the seven-point rule, closed-form 1/R
potentials against brute-force Duffy quadrature, and the extracted inner
potentials of exp(ikR)/R against brute force of the full kernel."""
import math

import numpy as np
import pytest

from oracle import efie
from tests.brute import triangle_integral


def _monomial_exact(p, q):
    # int over the unit right triangle {x, y >= 0, x + y <= 1} of x^p y^q
    return math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2)


def test_rule7_weights_and_barycentrics():
    R = efie.rule7()
    assert np.allclose(R[:, :3].sum(1), 1.0, atol=1e-15)
    assert abs(R[:, 3].sum() - 1.0) < 1e-15
    assert np.all(R[:, 3] > 0)


def test_rule7_exact_to_degree_5_not_6():
    R = efie.rule7()
    x, y, w = R[:, 1], R[:, 2], R[:, 3] * 0.5  # vertices (0,0),(1,0),(0,1); area 1/2
    for deg in range(6):
        for p in range(deg + 1):
            q = deg - p
            assert abs(np.sum(w * x ** p * y ** q) - _monomial_exact(p, q)) < 1e-15
    errs = [abs(np.sum(w * x ** p * y ** (6 - p)) - _monomial_exact(p, 6 - p)) for p in range(7)]
    assert max(errs) > 1e-6


TRI = np.array([[0.0, 0.0, 0.0], [0.08, 0.01, 0.0], [0.02, 0.07, 0.0]])


def _points():
    rng = np.random.default_rng(11)
    pts = []
    c = TRI.mean(0)
    pts.append(c)                                              # centroid, on plane
    for _ in range(6):                                         # random in-plane interior
        l = rng.dirichlet([1, 1, 1])
        pts.append(l @ TRI)
    pts.append(0.5 * (TRI[0] + TRI[1]) + np.array([0, -0.03, 0]))   # in plane, outside
    pts.append(TRI[2] + np.array([0.05, 0.04, 0.0]))           # in plane, far outside
    pts.append(c + np.array([0, 0, 1e-4]))                     # just above
    pts.append(c + np.array([0, 0, 0.02]))                     # above
    pts.append(TRI[1] + np.array([0.01, 0.0, -0.003]))         # near a vertex, below
    pts.append(np.array([0.3, -0.2, 0.15]))                    # far
    # on the extension of an edge line (in plane, collinear with edge 0-1)
    pts.append(TRI[0] + 1.7 * (TRI[1] - TRI[0]))
    return pts


@pytest.mark.parametrize("idx", range(14))
def test_static_potential_matches_duffy(idx):
    r = _points()[idx]
    I0, I1, rho = efie.static_potential(r, TRI)
    f = lambda pts, R: np.concatenate([(1.0 / R)[..., None], (pts - rho) / R[..., None]], -1)
    ref = triangle_integral(r, TRI, f, n=16)
    assert abs(I0 - ref[0]) < 1e-12 * abs(ref[0])
    assert np.max(np.abs(I1 - ref[1:])) < 1e-11 * abs(ref[0])


def test_static_potential_self_known_value():
    # int over an equilateral triangle of side a, seen from its centroid:
    # 3 * int_{-pi/3}^{pi/3} (h / cos t) dt with h = a / (2 sqrt 3)
    # = sqrt(3) a * ln(2 + sqrt 3) / 1  ... derived from the polar form
    a = 0.1
    T = np.array([[0, 0, 0], [a, 0, 0], [a / 2, a * math.sqrt(3) / 2, 0]])
    c = T.mean(0)
    I0, I1, _ = efie.static_potential(c, T)
    h = a / (2 * math.sqrt(3))
    # int_T 1/R dS from an interior point = sum over edges of h_e * ln(tan(pi/4 + t/2)) |_{t-}^{t+}
    exact = 3 * h * 2 * math.log(math.tan(math.pi / 4 + math.pi / 6))
    assert abs(I0 - exact) < 1e-14 * exact
    assert np.max(np.abs(I1)) < 1e-15   # symmetric: first moment about the centroid vanishes


def _mesh_one():
    V = TRI.copy()
    T = np.array([[0, 1, 2]], dtype=np.int32)
    return V, T


@pytest.mark.parametrize("idx", [0, 1, 3, 7, 9, 10, 11])
def test_extracted_potential_matches_full_kernel(idx):
    """Inner potentials with singularity extraction against brute force of
    the full exp(ikR)/R kernel.  Im part: sin(kR)/R is smooth (only even
    powers of R), so the seven-point remainder is accurate to ~1e-9; Re part:
    (cos kR - 1)/R has a kink ~ -k^2 R / 2 at R = 0 that a degree-5 rule
    resolves to ~5e-4 of the total at this size (k h ~ 0.5).  The closed-form
    part is pinned to 1e-12 above; a mistake in it (sign, factor, dropped
    term) moves these numbers by O(1), far beyond the 1e-3 allowed here."""
    V, T = _mesh_one()
    k = 2 * math.pi
    P = efie.Problem.__new__(efie.Problem)
    P.verts, P.tris, P.k = V, T, k
    r = _points()[idx]
    P0, P1 = efie.Problem.tri_potential(P, r, 0, True)
    f = lambda pts, R: np.concatenate([(np.exp(1j * k * R) / R)[..., None],
                                       pts * (np.exp(1j * k * R) / R)[..., None]], -1)
    ref = triangle_integral(r, TRI, f, n=16)
    scale = abs(ref[0])
    assert abs(P0.imag - ref[0].imag) < 1e-8 * scale
    assert abs(P0.real - ref[0].real) < 1e-3 * scale
    scale1 = np.max(np.abs(ref[1:]))
    assert np.max(np.abs(P1.imag - ref[1:].imag)) < 1e-8 * scale1
    assert np.max(np.abs(P1.real - ref[1:].real)) < 1e-3 * scale1


def test_far_potential_plain_rule_matches_full_kernel():
    V, T = _mesh_one()
    k = 2 * math.pi
    P = efie.Problem.__new__(efie.Problem)
    P.verts, P.tris, P.k = V, T, k
    r = np.array([0.4, -0.3, 0.2])
    P0, P1 = efie.Problem.tri_potential(P, r, 0, False)
    f = lambda pts, R: np.concatenate([(np.exp(1j * k * R) / R)[..., None],
                                       pts * (np.exp(1j * k * R) / R)[..., None]], -1)
    ref = triangle_integral(r, TRI, f, n=20)
    assert abs(P0 - ref[0]) < 1e-6 * abs(ref[0])
    assert np.max(np.abs(P1 - ref[1:])) < 1e-6 * np.max(np.abs(ref[1:]))
