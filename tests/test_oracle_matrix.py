"""Pins of the oracle's whole matrix Z (Section II, Eq. (5)) against results
fixed by mathematics and by the paper:

- RWG list: counts, canonical order, orientation (Section II, Eq. (4)).
- Re Z through the plane-wave (spectral) identity
  sin(kR)/R = (k / 4 pi) int d^2k exp(i k.(r - r')), the addition-theorem
  identity of Eq. (SinKer) with the translation summed to all orders.  It
  holds exactly for the discrete seven-point rule because sin(kR)/R has no
  singular part; it checks the prefactor i k eta, the Green's function
  normalisation and the sign and 1/k^2 of the divergence term.
- Z = Z^T, and R = -Re Z positive semidefinite.
- A far pair against an independent high-order quadrature.
- Characteristic values of a PEC sphere against Harrington's closed form
  (-y_n/j_n, TE; -(x y_n)'/(x j_n)', TM), which is itself checked against
  Table I.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg
from scipy.special import spherical_jn, spherical_yn

import workloads
from oracle import cm, efie
from oracle.rwg import MeshError, rwg_list
from tests.brute import gauss_legendre

HERE = os.path.dirname(os.path.abspath(__file__))


# ------------------------------------------------------------------ RWG ---
@pytest.mark.parametrize("mesh,n", [
    (lambda: workloads.icosphere(0, 1.0), 30),
    (lambda: workloads.icosphere(3, 1.0), 1920),
    (lambda: workloads.icosphere(5, 2.0), 30720),
    (lambda: workloads.plate_with_strips(), 10824),
    (lambda: workloads.plate_with_strips(strips=False), 10680),
    (lambda: workloads.cube(1.0, 4), 18 * 16),
])
def test_rwg_counts(mesh, n):
    v, t = mesh()
    r = rwg_list(v, t)
    assert r["tri"].shape == (n, 2)


def test_rwg_canonical_order_and_orientation():
    v, t = workloads.cube(1.0, 3)
    r = rwg_list(v, t)
    ev = r["edge_v"]
    assert np.all(ev[:, 0] < ev[:, 1])
    key = ev[:, 0].astype(np.int64) * 10 ** 6 + ev[:, 1]
    assert np.all(np.diff(key) > 0)
    for e in range(ev.shape[0]):
        lo, hi = ev[e]
        tp, tm = r["tri"][e]
        cyc_p = list(t[tp]) + [t[tp][0]]
        cyc_m = list(t[tm]) + [t[tm][0]]
        assert any(cyc_p[i] == lo and cyc_p[i + 1] == hi for i in range(3))
        assert any(cyc_m[i] == hi and cyc_m[i + 1] == lo for i in range(3))
        assert r["vfree"][e][0] in t[tp] and r["vfree"][e][0] not in (lo, hi)
        assert r["vfree"][e][1] in t[tm] and r["vfree"][e][1] not in (lo, hi)
    assert np.allclose(r["length"], np.linalg.norm(v[ev[:, 1]] - v[ev[:, 0]], axis=1))


@pytest.mark.parametrize("mesh", [lambda: workloads.icosphere(2, 0.5), lambda: workloads.cube(1.0, 3)])
def test_rwg_normal_continuity_and_divergence(mesh):
    """The defining identities of the RWG functions the oracle uses
    (f = +-l / (2 A+-) (r - v+-) on T+-, div f = +-l / A+-): across the common
    edge the normal component is 1 from both triangles (no line charge);
    along the two other edges of each triangle f is tangential (no flux
    leaves the support); and the surface divergence of the vector field,
    taken by finite differences in the triangle's plane, is the +-l / A+-
    that the scalar-potential term of Eq. (5) uses."""
    v, t = mesh()
    r = rwg_list(v, t)
    for e in range(r["tri"].shape[0]):
        lo, hi = v[r["edge_v"][e]]
        lhat = (hi - lo) / np.linalg.norm(hi - lo)
        for side, sgn in ((0, 1.0), (1, -1.0)):
            tri = r["tri"][e, side]
            vf = v[r["vfree"][e, side]]
            P = v[t[tri]]
            nrm = np.cross(P[1] - P[0], P[2] - P[0])
            A = 0.5 * np.linalg.norm(nrm)
            nhat = nrm / (2 * A)
            c = sgn * r["length"][e] / (2 * A)
            f = lambda x: c * (x - vf)
            # in-plane unit normal of the common edge in this triangle, pointing
            # from T+ into T- (away from v+ on T+, towards v- on T-)
            d = (lo - vf) if side == 0 else (vf - lo)
            mp = d - np.dot(d, lhat) * lhat
            mp /= np.linalg.norm(mp)
            for s_ in (0.2, 0.5, 0.9):
                x = lo + s_ * (hi - lo)
                assert abs(np.dot(f(x), mp) - 1.0) < 1e-12
            # the other two edges: from the free vertex to each end of the common edge
            for end in (lo, hi):
                dvec = end - vf
                nout = np.cross(dvec, nhat)
                for s_ in (0.3, 0.7):
                    assert abs(np.dot(f(vf + s_ * dvec), nout)) < 1e-12 * abs(c) * np.linalg.norm(dvec) * np.linalg.norm(nout)
            # surface divergence by central differences along two in-plane directions
            u1 = lhat
            u2 = np.cross(nhat, u1)
            x0 = P.mean(0)
            h = 1e-4 * np.sqrt(A)
            div = sum(np.dot(f(x0 + h * u) - f(x0 - h * u), u) / (2 * h) for u in (u1, u2))
            assert abs(div - sgn * r["length"][e] / A) < 1e-7 * r["length"][e] / A


def test_rwg_rejects_bad_meshes():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1]], float)
    with pytest.raises(MeshError):   # edge 0-1 on three triangles
        rwg_list(v, np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]]))
    with pytest.raises(MeshError):   # both triangles traverse 0->1
        rwg_list(v, np.array([[0, 1, 2], [0, 1, 3]]))
    r = rwg_list(v, np.array([[0, 1, 2]]))  # a lone triangle: boundary edges only
    assert r["tri"].shape[0] == 0


# ---------------------------------------------------- dense Z invariants ---
@pytest.fixture(scope="module")
def small_sphere():
    v, t = workloads.icosphere(2, 0.5)
    P = efie.Problem(v, t, 2 * math.pi)
    return P, P.dense()


def test_symmetric(small_sphere):
    _, Z = small_sphere
    assert np.max(np.abs(Z - Z.T)) == 0.0


def test_resistance_psd(small_sphere):
    """-Re Z = (k^2 eta / 4 pi) int |F_perp|^2 >= 0 holds exactly for exact
    integrals; with the seven-point rule the discrete divergence term differs
    from |k^.F|^2 by the rule's error, which shows up (~1e-9 relative) only in
    the near-null space of non-radiating currents."""
    _, Z = small_sphere
    ev = np.linalg.eigvalsh(-Z.real)
    assert ev.min() > -1e-7 * ev.max()
    assert np.sum(ev > 1e-3 * ev.max()) > 20     # a real radiating subspace


def _quad_points(P):
    R7 = efie.rule7()
    V, T = P.verts, P.tris
    tri = V[T]                                         # [nt, 3, 3]
    pts = np.einsum("qa,tad->tqd", R7[:, :3], tri)      # [nt, 7, 3]
    area = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1)
    return pts, area, R7[:, 3]


def test_re_z_spectral_identity(small_sphere):
    """Re Z_ij = -(k^2 eta / 4 pi) sum_q w_q [ conj(F_i).F_j - conj(D_i) D_j / k^2 ],
    F_j(k^) = int f_j exp(-i k k^.r), D_j(k^) = int div f_j exp(-i k k^.r),
    on a product grid exact for the band limit (L = 40 > k * diameter + 30)."""
    P, Z = small_sphere
    k, eta = P.k, P.eta
    pts, area, w7 = _quad_points(P)
    L = 40
    x, wx = np.polynomial.legendre.leggauss(L + 1)
    nphi = 2 * (L + 1)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    ct = np.repeat(x, nphi)
    st = np.sqrt(1 - ct ** 2)
    ph = np.tile(phi, L + 1)
    khat = np.stack([st * np.cos(ph), st * np.sin(ph), ct], 1)    # [Q, 3]
    wq = np.repeat(wx, nphi) * (2 * np.pi / nphi)
    n = P.n
    F = np.zeros((n, khat.shape[0], 3), complex)
    D = np.zeros((n, khat.shape[0]), complex)
    for side, sgn in ((0, 1.0), (1, -1.0)):
        t = P.tri[:, side]
        vf = P.verts[P.vfree[:, side]]
        A = area[t]
        l = P.length
        for q in range(7):
            r = pts[t, q]                                            # [n, 3]
            ph_ = np.exp(-1j * k * (r @ khat.T))                     # [n, Q]
            wA = (A * w7[q])[:, None]
            f = sgn * (l / (2 * A))[:, None] * (r - vf)              # [n, 3]
            F += (wA * ph_)[..., None] * f[:, None, :]
            D += wA * ph_ * (sgn * l / A)[:, None]
    Fw = (F * wq[None, :, None]).conj().reshape(n, -1)
    Dw = (D * wq[None, :]).conj()
    G = Fw @ F.reshape(n, -1).T - (Dw @ D.T) / k ** 2
    ReZ = -(k ** 2 * eta / (4 * np.pi)) * G
    assert np.max(np.abs(ReZ.imag)) < 1e-10 * np.max(np.abs(ReZ.real))
    err = np.max(np.abs(ReZ.real - Z.real)) / np.max(np.abs(Z.real))
    assert err < 1e-10, err


def test_far_pair_against_high_order_rule():
    """Two RWG pairs 1 m apart: the seven-point product rule against a
    15 x 15 collapsed Gauss rule on every triangle pair."""
    v, t = workloads.two_triangle_pairs(1.0)
    k = 2 * math.pi
    P = efie.Problem(v, t, k)
    assert P.n == 2
    Z = P.dense()
    xg, wg = gauss_legendre(15)
    U, Vv = np.meshgrid(xg, xg, indexing="ij")
    bary = np.stack([1 - U, U * (1 - Vv), U * Vv], -1).reshape(-1, 3)
    wb = (np.outer(wg, wg) * U).reshape(-1) * 2.0   # weights relative to area, sum 1

    def side_pts(j, side):
        tri = P.tris[P.tri[j, side]]
        X = P.verts[tri]
        A = 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
        r = bary @ X
        sgn = 1.0 if side == 0 else -1.0
        f = sgn * P.length[j] / (2 * A) * (r - P.verts[P.vfree[j, side]])
        return r, f, sgn * P.length[j] / A, A * wb

    ref = 0.0
    for si in (0, 1):
        ri, fi, di, wi = side_pts(0, si)
        for sj in (0, 1):
            rj, fj, dj, wj = side_pts(1, sj)
            R = np.linalg.norm(ri[:, None] - rj[None], axis=-1)
            g = np.exp(1j * k * R) / R
            ref += np.einsum("a,b,ab->", wi, wj, ((fi @ fj.T) - di * dj / k ** 2) * g)
    ref *= 1j * k * P.eta
    assert abs(Z[0, 1] - ref) < 1e-5 * abs(ref)


# ------------------------------------------------------------ sphere CM ---
def closed_form_sphere(ka, nmax=12):
    """(lambda, multiplicity, label) of a PEC sphere's characteristic modes."""
    out = []
    for n in range(1, nmax + 1):
        j, y = spherical_jn(n, ka), spherical_yn(n, ka)
        jd, yd = spherical_jn(n, ka, True), spherical_yn(n, ka, True)
        out.append((-y / j, 2 * n + 1, "TE%d" % n))
        out.append((-(y + ka * yd) / (j + ka * jd), 2 * n + 1, "TM%d" % n))
    return out


def nearest_zero(ka, count):
    vals = []
    for lam, mult, _ in sorted(closed_form_sphere(ka), key=lambda t: abs(t[0])):
        vals += [lam] * mult
    return np.array(vals[:count])


def test_closed_form_matches_table_cv():
    """Table I (sphere, ka = 1.5 pi, finest mesh 15,015 unknowns) against the
    closed form: a 3-fold cluster near -0.22 and a cluster near +0.286."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "sphere_table_cv.txt"))
            if l.strip() and not l.startswith("#")]
    finest = np.array([float(r[5]) for r in rows])
    cf = closed_form_sphere(1.5 * math.pi)
    tm1 = [l for l, m, s in cf if s == "TM1"][0]
    te3 = [l for l, m, s in cf if s == "TE3"][0]
    assert abs(tm1 - (-0.22221)) < 1e-4 and abs(te3 - 0.28722) < 1e-4
    assert np.all(np.abs(finest[:3] - tm1) < 0.02 * abs(tm1))
    assert np.all(np.abs(finest[3:] - te3) < 0.02 * abs(te3))
    ref = nearest_zero(1.5 * math.pi, 10)
    assert np.allclose(ref[:3], tm1) and np.allclose(ref[3:10], te3)


def test_sphere_cm_values_coarse(small_sphere):
    """480 unknowns, ka = pi: the 15 values nearest zero form the clusters
    TE1 (x3), TE2 (x5), TM3 (x7) of the closed form, each within 12 %."""
    _, Z = small_sphere
    lam = cm.cm_values(Z, 15)
    ref = nearest_zero(math.pi, 15)
    assert np.all(np.abs(lam - ref) < 0.12 * np.abs(ref)), (lam, ref)
    lam2 = cm.cm_values_arnoldi(Z, 15)
    assert np.allclose(np.sort(lam2), np.sort(lam), rtol=1e-8)


def test_symmetric_reduction_equals_qz(small_sphere):
    """cm_values_symmetric (R = L L^T, eigenvalues of L^T X^-1 L) selects
    the same values as the QZ route of cm_values on the sphere pencil."""
    _, Z = small_sphere
    lam = cm.cm_values_symmetric(-Z.real, Z.imag.copy(), 15)
    assert np.allclose(lam, cm.cm_values(Z, 15), rtol=1e-8)


def test_symmetric_reduction_random_semidefinite_pencil():
    """A random pencil with R of rank n - 3 (three infinite values) and X
    indefinite: the reduction equals the finite generalized eigenvalues
    nearest zero from a general eigensolver."""
    rng = np.random.default_rng(7)
    n = 70
    A = rng.standard_normal((n, n))
    X = A + A.T
    Bf = rng.standard_normal((n, n - 3))
    R = Bf @ Bf.T
    mu = scipy.linalg.eigvals(R, X)
    mu = mu[np.isfinite(mu)].real
    lam_ref = 1.0 / mu[np.argsort(-np.abs(mu))[:12]]
    lam_ref = lam_ref[np.argsort(np.abs(lam_ref))]
    lam = cm.cm_values_symmetric(R.copy(), X.copy(), 12, overwrite=True)
    assert np.allclose(lam, lam_ref, rtol=1e-7)


@pytest.mark.slow
def test_sphere_cm_values_converge():
    """Refining 480 -> 1,920 unknowns moves every cluster towards the closed
    form, and the finer mesh is within 3.5 %."""
    errs = []
    for sub in (2, 3):
        v, t = workloads.icosphere(sub, 0.5)
        P = efie.Problem(v, t, 2 * math.pi)
        lam = cm.cm_values_arnoldi(P.dense(), 15)
        ref = nearest_zero(math.pi, 15)
        errs.append(np.abs(lam - ref) / np.abs(ref))
    assert np.all(errs[1] < errs[0])
    assert np.all(errs[1] < 0.035), errs[1]
