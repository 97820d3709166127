"""Products on a plan whose coarsest translation level has 4-wavelength
boxes (a 30,720-unknown mesh of the r = 8 m sphere, k = 2 pi, 5 levels: level
2 holds L = 57, 6,728 samples, level 3 L = 33).  One FP64 column of the
level-2 anterpolation (Section III-B, the downward pass) stages the parent
field, the phi-anterpolated rows and the child field: 208,672 bytes of
shared memory, above 200 KB and within the 227 KB a CTA may use.  The
built-in products and the tuner must run there in both precisions and meet
exact oracle rows."""
import math

import numpy as np
import pytest

import workloads
from oracle import efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case():
    v, t = workloads.icosphere(5, 8.0)
    k = 2 * math.pi
    P = M.MlfmaPlan(v, t, k, 5, 3.0, max_batch=16, precisions=(M.FP32, M.FP64))
    info = P.info()
    assert info["trunc_L"][2] == 57 and info["samples_K"][3] == 2312
    rows = np.random.default_rng(5).choice(P.n, 8, replace=False)
    yield P, efie.Problem(v, t, k), rows
    P.close()


@pytest.mark.parametrize("prec,B", [(M.FP64, 1), (M.FP32, 16)])
def test_products_and_tuner_on_4_wavelength_boxes(case, prec, B):
    P, prob, rows = case
    dt = torch.float64 if prec == M.FP64 else torch.float32
    x = workloads.rhs(P.n, B, 3)
    xd = torch.from_numpy(x).to("cuda", dt)
    ref = prob.matvec_rows(x, rows)
    y = P.matvec(xd).cpu().numpy()
    err = rel(y[rows], ref)
    print("error against the oracle rows: %.2e" % err)
    assert err < 5e-3   # the triangles are 0.47 wavelengths across: coarser than the other meshes
    before, after = P.tune(B, prec)
    assert before > 0 and 0 < after <= before
    y2 = P.matvec(xd).cpu().numpy()
    assert rel(y2, y) < (1e-10 if prec == M.FP64 else 1e-5)
