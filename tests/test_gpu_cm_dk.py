"""Slopes of characteristic values (cm_eig_derivatives): dlambda/dk =
J^T (X' - lambda R') J / J^T R J from the library's own eigenpairs
(cm_ira_solve) and dZ/dk products, on the 1,920-unknown sphere, against

- the dense oracle's first-order perturbation of Eq. (GEP) with its dense
  Z and dZ/dk (oracle/cm.py: cm_derivatives), and
- central differences of the library's characteristic values at
  k (1 +- 1e-4) (the same discrete operator, so the agreement is tight).

The plan has d0 = 5 (product error ~1e-5), so the values themselves match
the dense oracle's to 1e-4.

The 11 values nearest zero form whole clusters of the icosahedral mesh
(TE1 x3, TE2 x5, and 3 of the TM3 values); within a degenerate cluster
individual slopes depend on the basis the eigensolver returns, so cluster
means are compared."""
import numpy as np
import pytest

import workloads
from oracle import cm, efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402

NEV = 11
SIZES = (3, 5, 3)
_c = {}


def means(lam, dl):
    o = np.argsort(np.abs(lam))
    lam, dl = lam[o], dl[o]
    out, i = [], 0
    for m in SIZES:
        out.append((lam[i:i + m].mean(), dl[i:i + m].mean(), np.ptp(lam[i:i + m])))
        i += m
    return np.array(out)


def solve(k):
    W = workloads.get("sphere-r0.5m-ico3")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, k, W.levels, 5.0, precisions=(M.FP64,))
    lam, J, _ = P.cm_solve(nev=NEV, ncv=30, op=M.CM_ZINV_R, prec=M.FP64, tol=1e-10, gmres_tol=1e-9)
    return P, lam, J


def setup_module():
    W = workloads.get("sphere-r0.5m-ico3")
    v, t = W.mesh()
    Pr = efie.Problem(v, t, W.k)
    lo, dlo = cm.cm_derivatives(Pr.dense(), Pr.dense_dk(), NEV, method="arnoldi")
    _c["oracle"] = means(lo, dlo)
    _c["oracle_values"] = lo
    P, lam, J = solve(W.k)
    _c["lib"] = means(lam, P.cm_derivatives(lam, J, M.FP64))
    _c["lam"], _c["P"], _c["J"] = lam, P, J


def test_clusters_are_whole():
    # each compared group is one cluster, well apart from the next
    for lam, _, spread in _c["lib"]:
        assert spread < 1e-3 * abs(lam)


def test_values_match_dense_oracle():
    lo = _c["oracle_values"]
    ref = np.sort(lo[np.argsort(np.abs(lo))[:10]])
    lam = _c["lam"]
    got = np.sort(lam[np.argsort(np.abs(lam))[:10]])
    assert np.abs(got - ref).max() <= 1e-4, (got, ref)


def test_slopes_match_dense_oracle():
    lib, ora = _c["lib"], _c["oracle"]
    assert np.abs(lib[:, 0] - ora[:, 0]).max() <= 1e-4
    err = np.abs(lib[:, 1] - ora[:, 1]) / np.abs(ora[:, 1])
    assert np.all(err < 3e-3), err


def test_slopes_match_central_differences():
    W = workloads.get("sphere-r0.5m-ico3")
    h = 1e-4 * W.k
    _, lp, _ = solve(W.k + h)
    _, lm, _ = solve(W.k - h)
    fd = (means(lp, np.zeros(NEV))[:, 0] - means(lm, np.zeros(NEV))[:, 0]) / (2 * h)
    err = np.abs(_c["lib"][:, 1] - fd) / np.abs(fd)
    assert np.all(err < 1e-3), err


def test_fp32_products_give_the_same_slopes():
    """The same eigenpairs through FP32 and FP64 dZ/dk products of one
    3-digit plan (FP32 cannot carry the 5-digit expansion on this tree)."""
    lam, J = _c["lam"], _c["J"]
    W = workloads.get("sphere-r0.5m-ico3")
    v, t = W.mesh()
    P3 = M.MlfmaPlan(v, t, W.k, W.levels, W.digits)
    d32 = means(lam, P3.cm_derivatives(lam, J, M.FP32))
    d64 = means(lam, P3.cm_derivatives(lam, J, M.FP64))
    assert np.allclose(d32[:, 1], d64[:, 1], rtol=1e-4)
