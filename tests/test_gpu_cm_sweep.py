"""Characteristic modes followed over a wavenumber sweep (Section V follows
the values over frequency; the north-star's d lambda / dk for tracked
modes): on the 1,920-unknown sphere, eigenpairs from cm_ira_solve (FP64
products, 5-digit plan) at each wavenumber, slopes from cm_eig_derivatives,
modes paired from one wavenumber to the next by cm_track_modes.

Checks
- tracking keeps every cluster (TE1 x3, TE2 x5, three TM3 values) together
  over a +-4 % sweep of ka around pi;
- the tracked cluster means change as the slopes predict (trapezoidal
  integration of the slopes between sweep points, to 1e-2 relative);
- at the centre, the slopes match Richardson-extrapolated central
  differences of the tracked values (steps h and 2h, h = 1e-4 k, as in the
  workload's dk = 1e-4 k) to 1e-3 relative;
- and the sphere's closed-form slopes (derived from the Wronskians:
  -a / (x^2 j_n(x)^2) for TE, -a (1 - n(n+1)/x^2) / ((x j_n)')^2 for TM,
  x = ka) within the mesh's discretisation error (5 %; the oracle's own
  slopes on this mesh differ from the closed form by 0.9 / 0.5 / 3.4 %).
"""
import math

import numpy as np
import pytest
from scipy.special import spherical_jn

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402

NEV = 11
GROUPS = (3, 5, 3)       # TE1, TE2, three values of TM3 (whole clusters of this mesh)
A = 0.5                  # sphere radius, m


def solve(k):
    W = workloads.get("sphere-r0.5m-ico3")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, k, W.levels, 5.0, precisions=(M.FP64,))
    lam, J, st = P.cm_solve(nev=NEV, ncv=30, op=M.CM_ZINV_R, prec=M.FP64, tol=1e-10, gmres_tol=1e-9)
    assert st["converged"] == 1
    dl = P.cm_derivatives(lam, J, M.FP64)
    P.close()
    return lam, J, dl


def groups(lam):
    """Indices of the clusters, by |lambda| (the order of GROUPS)."""
    o = np.argsort(np.abs(lam))
    out, i = [], 0
    for m in GROUPS:
        out.append(sorted(o[i:i + m].tolist()))
        i += m
    return out


def closed_form(k):
    x = k * A
    te = lambda n: -A / (x * x * spherical_jn(n, x) ** 2)
    def tm(n):
        u = spherical_jn(n, x) + x * spherical_jn(n, x, derivative=True)
        return -A * (1 - n * (n + 1) / (x * x)) / u ** 2
    return np.array([te(1), te(2), tm(3)])


_c = {}


def setup_module():
    k0 = workloads.get("sphere-r0.5m-ico3").k
    ks = k0 * (1 + np.array([-0.04, -0.02, 0.0, 0.02, 0.04]))
    _c["k0"], _c["ks"] = k0, ks
    _c["sweep"] = [solve(k) for k in ks]


def test_tracking_keeps_clusters_together():
    sweep = _c["sweep"]
    for (la, Ja, _), (lb, Jb, _) in zip(sweep[:-1], sweep[1:]):
        match, ov = M.track_modes(la, Ja, lb, Jb, cluster_tol=1e-2)
        ga, gb = groups(la), groups(lb)
        for g in range(len(GROUPS)):
            src = {int(match[j]) for j in gb[g]}
            assert src <= set(ga[g]) and -1 not in src, (g, src, ga[g])
            assert min(ov[j] for j in gb[g]) > 0.9


def test_values_follow_the_slopes():
    ks, sweep = _c["ks"], _c["sweep"]
    for i in range(len(ks) - 1):
        (la, _, da), (lb, _, db) = sweep[i], sweep[i + 1]
        for ga, gb in zip(groups(la), groups(lb)):
            step = lb[gb].mean() - la[ga].mean()
            pred = 0.5 * (ks[i + 1] - ks[i]) * (da[ga].mean() + db[gb].mean())
            assert abs(step - pred) <= 1e-2 * abs(step), (i, step, pred)


def test_slopes_match_richardson_differences_and_closed_form():
    k0 = _c["k0"]
    h = 1e-4 * k0
    lam0, J0, d0 = _c["sweep"][2]
    vals = {}
    for m in (-2, -1, 1, 2):
        lam, J, _ = solve(k0 + m * h)
        match, _ = M.track_modes(lam0, J0, lam, J, cluster_tol=1e-2)
        g0, g = groups(lam0), groups(lam)
        for gi in range(len(GROUPS)):
            assert {int(match[j]) for j in g[gi]} <= set(g0[gi])
        vals[m] = np.array([lam[ix].mean() for ix in g])
    D1 = (vals[1] - vals[-1]) / (2 * h)
    D2 = (vals[2] - vals[-2]) / (4 * h)
    rich = (4 * D1 - D2) / 3
    slope = np.array([d0[ix].mean() for ix in groups(lam0)])
    err = np.abs(slope - rich) / np.abs(rich)
    assert np.all(err < 1e-3), err
    cf = closed_form(k0)
    assert np.all(np.abs(slope - cf) / np.abs(cf) < 0.05), (slope, cf)
