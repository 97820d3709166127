"""Tensor-core interpolation and anterpolation (Section III-C on tcgen05
TF32 tensor cores; MLFMA_MIXED_TF32 / MLFMA_MIXED_3XTF32): the product
against the FP32 CUDA-core product on the same plan, against exact oracle
rows, and stage by stage against the FP64 fields.

Tolerances
- 3xTF32 (hi/lo split of both operands) is accurate to FP32 rounding: the
  product agrees with the FP32 CUDA-core product to 2e-6 and with the FP64
  product to the FP32 path's own 1e-5, and every level's outgoing and
  incoming field agrees with FP64 to 1e-5.
- One TF32 product rounds both operands to the nearest TF32 (10 mantissa
  bits, relative error up to 2^-11 per operand): every level's fields differ
  from FP64 by 3e-4 - 6e-4 and the product by ~1e-3 (measured 1.05e-3 on the
  30,720-unknown sphere, 7.9e-4 on the plate with strips; on the 115,200-
  unknown cube the far field's cancellation magnifies it to 6e-2).  It is
  therefore not within the 1e-3 target in general; the bench reports it and
  picks its headline precision by the error on the timed inputs.
- Bilinear symmetry u^T (Z v) = v^T (Z u) holds because the down pass is the
  exact transpose of the up pass (weighted), to FP32 level for 3xTF32.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads
from oracle import efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


_c = {}


def plan(name, max_batch=64):
    if name not in _c:
        W = workloads.get(name)
        v, t = W.mesh()
        _c[name] = (W, v, t, M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=max_batch))
    return _c[name]


def gpu(x, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt)


@pytest.mark.parametrize("name", ["sphere-r2m-ico5", "plate6m-strips"])
def test_3xtf32_matches_fp32_and_oracle(name):
    W, v, t, P = plan(name)
    B = 16
    x = workloads.rhs(P.n, B, W.seed)
    y32 = P.matvec(gpu(x)).cpu().numpy()
    y3 = P.matvec(gpu(x), prec=M.MIXED_3XTF32).cpu().numpy()
    y64 = P.matvec(gpu(x, torch.float64)).cpu().numpy()
    assert rel(y3, y32) < 2e-6, rel(y3, y32)
    assert rel(y3, y64) < 1e-5, rel(y3, y64)
    rows = np.random.default_rng(3).choice(P.n, 24, replace=False)
    ref = efie.Problem(v, t, W.k).matvec_rows(x, rows)
    assert rel(y3[rows], ref) < 1e-3


@pytest.mark.parametrize("name", ["sphere-r2m-ico5", "plate6m-strips"])
def test_tf32_error_budget(name):
    """One TF32 product: ~1e-3 against FP64 (measured 1.05e-3 / 7.9e-4), and
    not the FP32 path by accident (which would give ~1e-6)."""
    W, v, t, P = plan(name)
    B = 16
    x = workloads.rhs(P.n, B, W.seed)
    y1 = P.matvec(gpu(x), prec=M.MIXED_TF32).cpu().numpy()
    y64 = P.matvec(gpu(x, torch.float64)).cpu().numpy()
    e = rel(y1, y64)
    assert 1e-4 < e < 2e-3, e
    rows = np.random.default_rng(4).choice(P.n, 24, replace=False)
    ref = efie.Problem(v, t, W.k).matvec_rows(x, rows)
    assert rel(y1[rows], ref) < 2e-3


@pytest.mark.parametrize("prec,tol", [(M.MIXED_3XTF32, 1e-5), (M.MIXED_TF32, 1e-3)])
def test_fields_stage_by_stage_against_fp64(prec, tol):
    """Every far level's outgoing field S (aggregation and up pass) and
    incoming field G (translation and down pass) of the tensor-core product
    against FP64, on the plate with strips at 16 columns."""
    W, v, t, P = plan("plate6m-strips")
    B = 16
    x = workloads.rhs(P.n, B, W.seed)
    info = P.info()
    P.matvec(gpu(x, torch.float64))
    f64 = {(w, l): P.export_field(M.FP64, w, l, B) for l in range(2, info["leaf_level"] + 1) for w in (0, 1)}
    P.matvec(gpu(x), prec=prec)
    for (w, l), ref in f64.items():
        got = P.export_field(M.FP32, w, l, B).astype(np.complex128)
        e = rel(got, ref)
        assert e < tol, ("SG"[w], l, e)


def test_ragged_columns_and_complex_input():
    W, v, t, P = plan("sphere-r2m-ico5")
    for B in (1, 3, 7, 33):
        x = workloads.rhs(P.n, B, 50 + B)
        y32 = P.matvec(gpu(x)).cpu().numpy()
        y3 = P.matvec(gpu(x), prec=M.MIXED_3XTF32).cpu().numpy()
        assert rel(y3, y32) < 2e-6, (B, rel(y3, y32))
    xc = workloads.rhs_complex(P.n, 5, 9)
    y32 = P.matvec(gpu(xc, torch.complex64)).cpu().numpy()
    y3 = P.matvec(gpu(xc, torch.complex64), prec=M.MIXED_3XTF32).cpu().numpy()
    assert rel(y3, y32) < 2e-6


def test_adjoint_and_bilinear_symmetry():
    W, v, t, P = plan("sphere-r2m-ico5")
    u = workloads.rhs(P.n, 1, 11)[:, 0]
    w = workloads.rhs(P.n, 1, 12)[:, 0]
    Zu = P.matvec(gpu(u), prec=M.MIXED_3XTF32).cpu().numpy()
    Zw = P.matvec(gpu(w), prec=M.MIXED_3XTF32).cpu().numpy()
    a, b = w @ Zu, u @ Zw
    assert abs(a - b) / (np.linalg.norm(Zu) * np.linalg.norm(w)) < 1e-5
    xc = workloads.rhs_complex(P.n, 2, 13)
    ya = P.matvec_adjoint(gpu(xc, torch.complex64), prec=M.MIXED_3XTF32).cpu().numpy()
    yr = np.conj(P.matvec(gpu(np.conj(xc), torch.complex64), prec=M.MIXED_3XTF32).cpu().numpy())
    assert rel(ya, yr) < 1e-6


def test_other_products_refuse_the_tf32_precisions():
    W, v, t, P = plan("sphere-r2m-ico5")
    x = gpu(workloads.rhs(P.n, 2, 1))
    with pytest.raises(M.MlfmaError) as e:
        P._product(P._lib.mlfma_matvec_dk, x, None, None, M.MIXED_TF32)
    assert e.value.status == 6
    with pytest.raises(TypeError):
        P.matvec(gpu(workloads.rhs(P.n, 2, 1), torch.float64), prec=M.MIXED_3XTF32)


_HOOK = r"""
import ctypes, os, sys
import numpy as np, torch
sys.path.insert(0, os.environ["REPO"])
import workloads
from paper_1412_1756_gb300 import mlfma as M
W = workloads.get("plate6m-strips")
v, t = W.mesh()
P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=16)
x = torch.from_numpy(workloads.rhs(P.n, 8, 1)).to("cuda", torch.float32)
P.matvec(x, prec=M.MIXED_3XTF32)
st = P._lib.mlfma_sync(P._h, None)
msg = P._lib.mlfma_last_error().decode()
st2 = P._lib.mlfma_sync(P._h, None)          # reported once, then clear
y = P.matvec(x).cpu()                          # the context is still usable
print("STATUS", st, st2, int(torch.isfinite(torch.view_as_real(y)).all()), "timeout" in msg or "gave up" in msg)
"""


def test_bounded_wait_reports_timeout_without_a_fault():
    """With the test hook set, the first CTA of each tensor-core launch
    withholds its first MMA arrival, so its bounded mbarrier wait runs out:
    the kernel records the failure, frees its tensor memory and returns; the
    next mlfma_sync reports MLFMA_ETIMEOUT once, and the context stays
    usable (an FP32 product afterwards is finite)."""
    env = dict(os.environ, MLFMA_TEST_WITHHOLD_ARRIVAL="1",
               REPO=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    r = subprocess.run([sys.executable, "-c", _HOOK], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("STATUS")][-1].split()
    assert line[1:] == ["5", "0", "1", "True"], r.stdout
