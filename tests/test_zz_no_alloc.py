"""mlfma_matvec_noalloc: the product for callers that cannot allocate device
memory when they need it (memory held entirely by another allocator, a
real-time loop that must not allocate).  Called through the C ABI and checked
against mlfma_matvec on the same plan and inputs, twice in a row, since every
call reuses one static scratch array that keeps the previous call's
contents.  Collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes
import math

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.fixture(scope="module")
def plan():
    W = workloads.get("sphere-r0.5m-ico3")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, max_batch=64)
    yield P
    P.close()


def _noalloc(P, x, y, B, prec, xc=0):
    lib = M.load()
    s = torch.cuda.current_stream().cuda_stream
    return lib.mlfma_matvec_noalloc(P._h, ctypes.c_void_p(x.data_ptr()), xc, ctypes.c_void_p(y.data_ptr()), B,
                                    prec, ctypes.c_void_p(s))


@pytest.mark.parametrize("prec,rdt,cdt,tol", [(M.FP32, torch.float32, torch.complex64, 1e-6),
                                              (M.FP64, torch.float64, torch.complex128, 1e-12)])
def test_noalloc_matches_matvec_twice(plan, prec, rdt, cdt, tol):
    for call, B in enumerate((3, 5)):
        x = torch.from_numpy(workloads.rhs(plan.n, B, 100 + call)).to("cuda", rdt)
        ref = plan.matvec(x)
        y = torch.full((plan.n, B), math.nan, dtype=cdt, device="cuda")
        assert _noalloc(plan, x, y, B, prec) == 0, M.load().mlfma_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(y)).all()
        assert _rel(y, ref) < tol, (call, _rel(y, ref))


def test_noalloc_complex_input(plan):
    xc = torch.from_numpy(workloads.rhs_complex(plan.n, 2, 7)).to("cuda", torch.complex64)
    ref = plan.matvec(xc)
    y = torch.empty_like(ref)
    assert _noalloc(plan, xc, y, 2, M.FP32, xc=1) == 0
    torch.cuda.synchronize()
    assert _rel(y, ref) < 1e-6


def test_noalloc_rejects_sizes_beyond_the_scratch(plan):
    # 64 FP64 columns need ~40 MB of fields: more than the 32 MiB array
    x = torch.zeros((plan.n, 64), dtype=torch.float64, device="cuda")
    y = torch.zeros((plan.n, 64), dtype=torch.complex128, device="cuda")
    assert _noalloc(plan, x, y, 64, M.FP64) == 1
    assert b"static scratch" in M.load().mlfma_last_error()
