"""FP32 translation with four columns per thread and the children four at a
time (tune values 9 / 10 / 11: 64 / 32 / 16 columns per CTA; Eq. (8) grouped
by parent, a second pass over the entries for parents with more than four
children).  Each
level pinned in turn to each choice reproduces the product of the built-in
kernels to FP32 rounding (1e-5 relative) on the sphere, the plate with
strips, a ragged column count and complex input; with every level pinned the
fields match the FP64 product's to FP32 level and the product meets exact
oracle rows; FP64 refuses the choices."""
import numpy as np
import pytest

import workloads
from oracle import efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402

ST = (9, 10, 11)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def pin(P, B, pairs, prec=M.FP32, complex_x=False):
    ch = np.zeros(M.TUNE_FIELDS, np.int32)
    for field, c in pairs:
        ch[field] = c
    P.tune_set(B, ch, prec, complex_x=complex_x)


@pytest.mark.parametrize("name,B,cplx", [("sphere-r2m-ico5", 64, False), ("plate6m-strips", 16, False),
                                         ("sphere-r2m-ico5", 7, False), ("sphere-r2m-ico5", 3, True)])
def test_each_level_matches_builtin(name, B, cplx):
    W = workloads.get(name)
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=64, precisions=(M.FP32,))
    if cplx:
        xd = torch.from_numpy(workloads.rhs_complex(P.n, B, W.seed)).to("cuda", torch.complex64)
    else:
        xd = torch.from_numpy(workloads.rhs(P.n, B, W.seed)).to("cuda", torch.float32)
    y0 = P.matvec(xd).cpu().numpy()
    for l in range(2, P.info()["leaf_level"] + 1):
        for c in ST:
            pin(P, B, [(3 + 2 * M.MAX_LEVELS + l, c)], complex_x=cplx)
            y = P.matvec(xd).cpu().numpy()
            assert rel(y, y0) < 1e-5, (l, c, rel(y, y0))
    P.tune_set(B, np.zeros(M.TUNE_FIELDS, np.int32), M.FP32, complex_x=cplx)
    P.close()


def test_all_levels_fields_oracle_rows_and_fp64_refusal():
    W = workloads.get("plate6m-strips")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=16)
    B = 16
    x = workloads.rhs(P.n, B, W.seed)
    info = P.info()
    P.matvec(torch.from_numpy(x).to("cuda", torch.float64))
    f64 = {(w, l): P.export_field(M.FP64, w, l, B) for l in range(2, info["leaf_level"] + 1) for w in (0, 1)}
    rows = np.random.default_rng(6).choice(P.n, 24, replace=False)
    ref = efie.Problem(v, t, W.k).matvec_rows(x, rows)
    for c in ST:
        pin(P, B, [(3 + 2 * M.MAX_LEVELS + l, c) for l in range(2, info["leaf_level"] + 1)])
        y = P.matvec(torch.from_numpy(x).to("cuda", torch.float32)).cpu().numpy()
        for (w, l), f in f64.items():
            e = rel(P.export_field(M.FP32, w, l, B).astype(np.complex128), f)
            assert e < 1e-5, (c, "SG"[w], l, e)
        assert rel(y[rows], ref) < 1e-3
    pin(P, 1, [(3 + 2 * M.MAX_LEVELS + 2, 9)], M.FP64)
    with pytest.raises(M.MlfmaError):
        P.matvec(torch.from_numpy(workloads.rhs(P.n, 1, 1)).to("cuda", torch.float64))
    torch.cuda.synchronize()
    P.close()
