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


def _sphere_closed_form_dk(ka, a, nmax=6):
    """(lambda, dlambda/dk, multiplicity) of the PEC sphere's characteristic
    modes (Harrington): TE lambda = -y_n/j_n, TM lambda = -(x y_n)'/(x j_n)'.
    Differentiating through the Wronskians j_n y_n' - j_n' y_n = 1/x^2 and
    u v' - u' v = 1 (u = x j_n, v = x y_n, u'' = (n(n+1)/x^2 - 1) u):
    TE dlambda/dk = -a / (x^2 j_n^2), TM dlambda/dk = -a (1 - n(n+1)/x^2) / u'^2."""
    from scipy.special import spherical_jn, spherical_yn
    out = []
    for n in range(1, nmax + 1):
        j, y = spherical_jn(n, ka), spherical_yn(n, ka)
        out.append((-y / j, -a / (ka * ka * j * j), 2 * n + 1))
        u = j + ka * spherical_jn(n, ka, True)
        v = y + ka * spherical_yn(n, ka, True)
        out.append((-v / u, -a * (1.0 - n * (n + 1) / (ka * ka)) / (u * u), 2 * n + 1))
    return sorted(out, key=lambda t: abs(t[0]))


def _cluster_means(lam, dl, sizes):
    out, i = [], 0
    for m in sizes:
        out.append((lam[i:i + m].mean(), dl[i:i + m].mean()))
        i += m
    return np.array(out)


def test_closed_form_derivative_against_central_differences():
    a = 0.5
    for k in (2 * np.pi, 0.7 * 2 * np.pi):
        h = 1e-5 * k
        for (l0, d0, _), (lp, _, _), (lm, _, _) in zip(_sphere_closed_form_dk(k * a, a),
                                                       _sphere_closed_form_dk((k + h) * a, a),
                                                       _sphere_closed_form_dk((k - h) * a, a)):
            assert abs((lp - lm) / (2 * h) - d0) < 1e-6 * max(1.0, abs(d0))


@pytest.mark.parametrize("level,tol,method", [(2, (0.05, 0.03, 0.16), "dense"),
                                              (3, (0.015, 0.01, 0.05), "arnoldi")])
def test_sphere_dlambda_dk_against_closed_form(level, tol, method):
    """Characteristic values of the sphere r = 0.5 m at ka = pi and their
    k-derivatives by first-order perturbation of Eq. (GEP) with the oracle's
    Z and dZ/dk; cluster means of TE1 (x3), TE2 (x5), TM3 (x7) against the
    closed form, within the mesh's discretisation error (which shrinks from
    480 to 1,920 unknowns).  The two eigensolver routes must agree."""
    from oracle import cm
    a, k = 0.5, 2 * np.pi
    v, t = workloads.icosphere(level, a)
    P = efie.Problem(v, t, k)
    lam, dl = cm.cm_derivatives(P.dense(), P.dense_dk(), 15, method=method)
    ref = _sphere_closed_form_dk(k * a, a)[:3]
    got = _cluster_means(lam, dl, [m for _, _, m in ref])
    for (l_ref, d_ref, _), (l_got, d_got), tl in zip(ref, got, tol):
        assert abs(d_got - d_ref) < tl * abs(d_ref), (d_got, d_ref)
        assert np.sign(l_got) == np.sign(l_ref)


def test_dk_rows_equal_dense_rows():
    v, t = workloads.icosphere(2, 0.5)
    P = efie.Problem(v, t, 2 * np.pi)
    D = P.dense_dk()
    rows = [0, 7, 311, P.n - 1]
    assert np.array_equal(P.rows_dk(rows), D[rows])


def test_dlambda_dk_dense_and_arnoldi_agree():
    from oracle import cm
    v, t = workloads.icosphere(2, 0.5)
    P = efie.Problem(v, t, 2 * np.pi)
    Z, D = P.dense(), P.dense_dk()
    l1, d1 = cm.cm_derivatives(Z, D, 8, method="dense")
    l2, d2 = cm.cm_derivatives(Z, D, 8, method="arnoldi")
    assert np.allclose(l1, l2, rtol=1e-8)
    assert np.allclose(d1, d2, rtol=1e-6)
