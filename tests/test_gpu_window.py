"""FP32 windowed interpolation and anterpolation kernels (tune values 304 /
308 / 316, 4 / 8 / 16 columns per CTA; 404 / 408 with a register budget for
one more CTA per SM; down pass 504 / 508 with one CTA per parent): the stencil rows of Section III-C in
groups of four on windows of consecutive source samples, the theta windows
running over the pole reflections.  The tables are pinned on CPU
(test_plan_host.py: they rebuild the row stencils exactly); here the kernels
that read them are checked:

- each level's up and down pass pinned in turn to each choice reproduces the
  product of the built-in kernels to FP32 rounding (1e-5 relative), on the
  sphere, the plate with strips, a ragged column count and complex input;
  every level takes at least one of the choices (the tables exist wherever a
  window is at most 32 samples wide; a column count whose shared memory
  exceeds the kernel's cap at a level fails with "invalid configuration");
- with every level pinned, every far level's outgoing and incoming field
  agrees with the FP64 product's to FP32 level (1e-5), and the product meets
  exact oracle rows to the 1e-3 bound.
"""
import numpy as np
import pytest

import workloads
from oracle import efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402

WIN = (304, 308, 316, 404, 408)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def pin(P, B, pairs, prec=M.FP32, complex_x=False):
    ch = np.zeros(M.TUNE_FIELDS, np.int32)
    for field, c in pairs:
        ch[field] = c
    P.tune_set(B, ch, prec, complex_x=complex_x)


def all_levels(info, c):
    out = []
    for l in range(2, info["leaf_level"]):
        out += [(3 + l, c), (3 + M.MAX_LEVELS + l, c)]
    return out


@pytest.mark.parametrize("name,B,cplx", [("sphere-r2m-ico5", 64, False), ("plate6m-strips", 16, False),
                                         ("sphere-r2m-ico5", 7, False), ("sphere-r2m-ico5", 3, True)])
def test_each_stage_matches_builtin(name, B, cplx):
    W = workloads.get(name)
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=64, precisions=(M.FP32,))
    if cplx:
        xd = torch.from_numpy(workloads.rhs_complex(P.n, B, W.seed)).to("cuda", torch.complex64)
    else:
        xd = torch.from_numpy(workloads.rhs(P.n, B, W.seed)).to("cuda", torch.float32)
    y0 = P.matvec(xd).cpu().numpy()
    info = P.info()
    for l in range(2, info["leaf_level"]):
        for field, shapes in ((3 + l, WIN + (704, 708, 716)), (3 + M.MAX_LEVELS + l, WIN + (504, 508, 804, 808))):
            ran = []
            for c in shapes:
                pin(P, B, [(field, c)], complex_x=cplx)
                try:
                    y = P.matvec(xd).cpu().numpy()
                except M.MlfmaError as e:
                    # a shape whose shared memory exceeds the kernel's cap
                    # at this level does not apply (documented failure)
                    assert "invalid configuration" in str(e), str(e)
                    torch.cuda.synchronize()
                    continue
                ran.append(c)
                assert rel(y, y0) < 1e-5, (l, field, c, rel(y, y0))
            assert ran, (l, field)
    P.tune_set(B, np.zeros(M.TUNE_FIELDS, np.int32), M.FP32, complex_x=cplx)
    P.close()


def test_all_levels_fields_and_oracle_rows():
    W = workloads.get("plate6m-strips")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=16)
    B = 16
    x = workloads.rhs(P.n, B, W.seed)
    info = P.info()
    P.matvec(torch.from_numpy(x).to("cuda", torch.float64))
    f64 = {(w, l): P.export_field(M.FP64, w, l, B) for l in range(2, info["leaf_level"] + 1) for w in (0, 1)}
    for c in (304, 308, 404, 504, 708, 804):   # 16 columns do not fit the down kernel at this plate's level 2
        if c < 500:
            pairs = all_levels(info, c)
        elif c < 700 or c > 800:   # per-parent or z-pair down pass
            pairs = [(3 + M.MAX_LEVELS + l, c) for l in range(2, info["leaf_level"])]
        else:           # up pass with z pairs
            pairs = [(3 + l, c) for l in range(2, info["leaf_level"])]
        pin(P, B, pairs)
        y = P.matvec(torch.from_numpy(x).to("cuda", torch.float32)).cpu().numpy()
        for (w, l), ref in f64.items():
            e = rel(P.export_field(M.FP32, w, l, B).astype(np.complex128), ref)
            assert e < 1e-5, (c, "SG"[w], l, e)
        rows = np.random.default_rng(5).choice(P.n, 24, replace=False)
        ref = efie.Problem(v, t, W.k).matvec_rows(x, rows)
        assert rel(y[rows], ref) < 1e-3
    P.close()


def test_tuner_may_pick_windowed_shapes_and_fp64_refuses_them():
    """mlfma_tune times the windowed candidates with the others (the pick is
    whatever is fastest); an FP64 product pinned to one fails with an error
    instead of running another kernel."""
    W = workloads.get("sphere-r2m-ico5")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=64)
    x32 = torch.from_numpy(workloads.rhs(P.n, 64, W.seed)).to("cuda", torch.float32)
    y0 = P.matvec(x32).cpu().numpy()
    P.tune(64, M.FP32)
    assert rel(P.matvec(x32).cpu().numpy(), y0) < 1e-5
    pin(P, 1, [(3 + 2, 308)], M.FP64)
    with pytest.raises(M.MlfmaError):
        P.matvec(torch.from_numpy(workloads.rhs(P.n, 1, 1)).to("cuda", torch.float64))
    torch.cuda.synchronize()
    P.close()
