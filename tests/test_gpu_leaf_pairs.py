"""FP32 reception with two columns per thread (tune values 4 / 5 / 6: 64 /
32 / 16 columns per CTA; the leaf disaggregation of Section III with the
field tile scaled by the quadrature weights as it is staged) and radiation
with four columns and two samples per thread (radiation tune value 5: the
leaf aggregation).  Each choice
reproduces the product of the built-in kernels to FP32 rounding (1e-5
relative) on the sphere, the plate with strips, an odd column count (no
16-byte path) and complex input, and meets exact oracle rows; FP64 refuses
the choices."""
import numpy as np
import pytest

import workloads
from oracle import efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name,B,cplx", [("sphere-r2m-ico5", 64, False), ("plate6m-strips", 16, False),
                                         ("sphere-r2m-ico5", 7, False), ("sphere-r2m-ico5", 3, True)])
def test_reception_pairs_match_builtin(name, B, cplx):
    W = workloads.get(name)
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=64, precisions=(M.FP32,))
    if cplx:
        x = workloads.rhs_complex(P.n, B, W.seed)
        xd = torch.from_numpy(x).to("cuda", torch.complex64)
    else:
        x = workloads.rhs(P.n, B, W.seed)
        xd = torch.from_numpy(x).to("cuda", torch.float32)
    y0 = P.matvec(xd).cpu().numpy()
    rows = np.random.default_rng(12).choice(P.n, 12, replace=False)
    ref = efie.Problem(v, t, W.k).matvec_rows(x, rows)
    for field, c in ((2, 4), (2, 5), (2, 6), (1, 5)):
        ch = np.zeros(M.TUNE_FIELDS, np.int32)
        ch[field] = c
        P.tune_set(B, ch, M.FP32, complex_x=cplx)
        y = P.matvec(xd).cpu().numpy()
        assert rel(y, y0) < 1e-5, (c, rel(y, y0))
        assert rel(y[rows], ref) < 1e-3, c
    P.tune_set(B, np.zeros(M.TUNE_FIELDS, np.int32), M.FP32, complex_x=cplx)
    P.close()


def test_fp64_refuses_the_pair_reception():
    W = workloads.get("sphere-r0.5m-ico3")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=4, precisions=(M.FP64,))
    for field, c in ((2, 4), (1, 5)):
        ch = np.zeros(M.TUNE_FIELDS, np.int32)
        ch[field] = c
        P.tune_set(1, ch, M.FP64)
        with pytest.raises(M.MlfmaError):
            P.matvec(torch.from_numpy(workloads.rhs(P.n, 1, 1)).to("cuda", torch.float64))
        torch.cuda.synchronize()
    P.close()
