"""mlfma_tune: the tuned launch shapes change how the product is computed,
not what it computes - tuned products agree with the built-in ones to
rounding (FP32: 1e-5, FP64: 1e-12) and with the dense oracle to the product's
bound; the chosen stage-time sum never exceeds the built-in one."""
import numpy as np
import pytest

import workloads
from oracle import efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dt,prec,tol", [(torch.float32, M.FP32, 1e-5), (torch.float64, M.FP64, 1e-12)])
def test_tuned_product_matches_builtin(dt, prec, tol):
    W = workloads.get("sphere-r0.5m-ico3")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=16)
    x = workloads.rhs(P.n, 8, W.seed)
    xd = torch.from_numpy(x).to("cuda", dt)
    y0 = P.matvec(xd).cpu().numpy()
    d, tt = P.tune(8, prec)
    assert 0 < tt <= d
    y1 = P.matvec(xd).cpu().numpy()
    assert rel(y1, y0) < tol
    Z = efie.Problem(v, t, W.k).dense()
    assert rel(y1, Z @ x) < 1e-3
    xc = workloads.rhs_complex(P.n, 4, W.seed)
    cdt = torch.complex64 if prec == M.FP32 else torch.complex128
    P.tune(4, prec, complex_x=True)
    yc = P.matvec(torch.from_numpy(xc).to("cuda", cdt)).cpu().numpy()
    assert rel(yc, Z @ xc) < 1e-3


def test_tuned_full_size_rows():
    W = workloads.get("sphere-r2m-ico5")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=64, precisions=(M.FP32,))
    d, tt = P.tune(64, M.FP32)
    assert tt <= d
    x = workloads.rhs(P.n, 64, W.seed)
    y = P.matvec(torch.from_numpy(x).to("cuda", torch.float32)).cpu().numpy()
    idx = np.random.default_rng(5).choice(P.n, 8, replace=False)
    ref = efie.Problem(v, t, W.k).matvec_rows(x, idx)
    assert rel(y[idx], ref) < 1e-3


def test_tune_rejects_bad_sizes():
    W = workloads.get("sphere-r0.5m-ico2")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=8)
    with pytest.raises(M.MlfmaError):
        P.tune(9, M.FP32)


@pytest.mark.parametrize("dt,prec,tol", [(torch.float32, M.FP32, 2e-5), (torch.float64, M.FP64, 1e-12)])
def test_every_candidate_shape_computes_the_same_product(dt, prec, tol):
    """Pin each candidate of every stage in turn (mlfma_tune_set) and check
    the product against the built-in shapes: 5-level sphere (30,720
    unknowns, levels 2..4), 32 columns."""
    W = workloads.get("sphere-r2m-ico5")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=32, precisions=(prec,))
    x = torch.from_numpy(workloads.rhs(P.n, 32, W.seed)).to("cuda", dt)
    ref = P.matvec(x).cpu().numpy()
    L = 22
    cands = [(0, c) for c in (1, 2, 3)] + [(1, c) for c in (1, 2, 3, 4)] + [(2, c) for c in (1, 2, 3)]
    if prec == M.FP32:   # reception with two columns per thread, radiation with four
        cands += [(2, c) for c in (4, 5, 6)] + [(1, 5)]
    for l in (2, 3, 4):
        cands += [(3 + 2 * L + l, c) for c in range(1, 12 if prec == M.FP32 else 9)]
        if l < 4:
            cands += [(3 + l, c) for c in (1, 2, 4, 8, 16)] + [(3 + L + l, c) for c in (1, 2, 4, 8, 16, 104, 108)]
            if prec == M.FP32:   # rows in pairs; rows in groups of four on windows
                cands += [(3 + l, c) for c in (202, 204, 208, 216)] + [(3 + L + l, c) for c in (204, 208, 216)]
                cands += [(3 + l, c) for c in (304, 308, 316, 404, 408, 704, 708, 716)] + [(3 + L + l, c) for c in (304, 308, 316, 404, 408, 504, 508, 804, 808)]
    for field, c in cands:
        ch = np.zeros(M.TUNE_FIELDS, np.int32)
        ch[field] = c
        P.tune_set(32, ch, prec)
        try:
            y = P.matvec(x).cpu().numpy()
        except M.MlfmaError:
            torch.cuda.synchronize()
            continue   # a shape that does not apply to this plan
        assert rel(y, ref) < tol, (field, c, rel(y, ref))
    P.tune_set(32, np.zeros(M.TUNE_FIELDS, np.int32), prec)
    assert np.array_equal(P.matvec(x).cpu().numpy(), ref)


def test_tune_cache_reuses_shapes(tmp_path):
    """A second plan of the same tree takes its shapes from the cache file
    (no timing) and computes the same product as the tuned first plan."""
    W = workloads.get("sphere-r0.5m-ico3")
    v, t = W.mesh()
    path = str(tmp_path / "tune.json")
    P1 = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=8, precisions=(M.FP32,))
    d, tt = P1.tune(8, M.FP32, cache=path)
    assert d is not None and tt <= d
    stored = M._read_tune_cache(path)
    assert len(stored) == 1
    P2 = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=8, precisions=(M.FP32,))
    assert P2.tune(8, M.FP32, cache=path) == (None, None)
    assert np.array_equal(P2.tune_get(8, M.FP32), P1.tune_get(8, M.FP32))
    x = torch.from_numpy(workloads.rhs(P1.n, 8, W.seed)).to("cuda", torch.float32)
    assert rel(P2.matvec(x).cpu().numpy(), P1.matvec(x).cpu().numpy()) < 1e-6


def test_tune_set_rejects_undocumented_shapes():
    W = workloads.get("sphere-r0.5m-ico2")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=8)
    good = P.tune_get(4, M.FP32)
    for field, value in ((0, 4), (1, 6), (2, 7), (3 + 2, 3), (3 + 22 + 2, 100), (3 + 44 + 2, 12)):
        bad = good.copy()
        bad[field] = value
        with pytest.raises(M.MlfmaError):
            P.tune_set(4, bad, M.FP32)
    with pytest.raises(M.MlfmaError):
        P.tune_set(9, good, M.FP32)
    P.tune_set(4, good, M.FP32)
    assert np.array_equal(P.tune_get(4, M.FP32), good)


@pytest.mark.parametrize("name,B", [("sphere-r2m-ico5", 64), ("plate6m-strips", 16), ("sphere-r2m-ico5", 7)])
def test_paired_rows_variants_match_builtin(name, B):
    """The up and down passes with their interpolation / anterpolation rows
    taken in pairs (tune values 202..216: one shared-memory load feeds both
    rows of a pair) compute the same product as the one-row kernels: each
    level and stage pinned in turn to each columns-per-CTA choice, FP32
    rounding (1e-5).  A pair table wider than the kernels' tap counts leaves a
    level without the variant (the pinned product then fails, as documented);
    the variant must apply to most levels and stages."""
    W = workloads.get(name)
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=64, precisions=(M.FP32,))
    x = workloads.rhs(P.n, B, W.seed)
    xd = torch.from_numpy(x).to("cuda", torch.float32)
    y0 = P.matvec(xd).cpu().numpy()
    info = P.info()
    ran = tried = 0
    for l in range(2, info["leaf_level"]):
        for field, choices in ((3 + l, (202, 204, 208, 216)), (3 + M.MAX_LEVELS + l, (204, 208, 216))):
            for c in choices:
                if c - 200 > B:
                    continue
                ch = np.zeros(M.TUNE_FIELDS, np.int32)
                ch[field] = c
                P.tune_set(B, ch, M.FP32)
                tried += 1
                try:
                    y = P.matvec(xd).cpu().numpy()
                except M.MlfmaError:
                    torch.cuda.synchronize()
                    continue
                ran += 1
                assert rel(y, y0) < 1e-5, (l, field, c, rel(y, y0))
    assert ran >= tried // 2, (ran, tried)
    P.tune_set(B, np.zeros(M.TUNE_FIELDS, np.int32), M.FP32)
    idx = np.random.default_rng(9).choice(P.n, 8, replace=False)
    ref = efie.Problem(v, t, W.k).matvec_rows(x, idx)
    P.tune(B, M.FP32)
    assert rel(P.matvec(xd).cpu().numpy()[idx], ref) < 1e-3
