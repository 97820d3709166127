"""GPU parity of the wavenumber derivative y = (dZ/dk) x (Eq. (5)
differentiated in k, applied through the multilevel product of Eq. (ZI))
against the FP64 oracle's dense dZ/dk, through the C ABI.

Tolerances
- levels = 2 (near field only): the stored near blocks of dZ/dk, the same
  quadrature and closed forms as the oracle in FP64: <= 1e-10.
- Central differences of the library's own product, (Z(k+h) - Z(k-h)) x / 2h
  with plans whose truncation numbers agree: the derivative pass is the exact
  derivative of the discrete multilevel operator, so FP64 agrees to the
  difference quotient's own error, <= 1e-6 (h = 2e-5 k).
- Against the dense oracle: the multilevel error of the product carries over
  to its derivative; <= 2e-3 relative (FP64 and FP32) on the 1,920-unknown
  sphere, 3e-3 on sampled rows of the full-size workloads.
- Autograd: gradients of a scalar loss through efie_product equal those of
  the same loss through a dense PyTorch model Z(k) = Z0 + (k - k0) dZ/dk
  built from the oracle, within the product's accuracy (2e-3).
"""
import numpy as np
import pytest

import workloads
from oracle import efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


_plans = {}
_mats = {}


def plan(name, levels=None, k=None, max_batch=64):
    W = workloads.get(name)
    key = (name, levels, k, max_batch)
    if key not in _plans:
        v, t = W.mesh()
        _plans[key] = M.MlfmaPlan(v, t, k or W.k, levels or W.levels, W.digits, max_batch=max_batch)
    return W, _plans[key]


def mats(name):
    if name not in _mats:
        W = workloads.get(name)
        v, t = W.mesh()
        P = efie.Problem(v, t, W.k)
        _mats[name] = (P.dense(), P.dense_dk())
    return _mats[name]


def test_near_field_only_dk_matches_dense_fp64():
    W, P = plan("sphere-r0.5m-ico2", levels=2)
    _, D = mats("sphere-r0.5m-ico2")
    x = workloads.rhs(P.n, 3, W.seed)
    y = P.matvec_dk(gpu(x, torch.float64)).cpu().numpy()
    assert rel(y, D @ x) < 1e-10


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_dk_matches_dense(dt):
    W, P = plan("sphere-r0.5m-ico3")
    _, D = mats("sphere-r0.5m-ico3")
    x = workloads.rhs(P.n, W.batch, W.seed)
    y = P.matvec_dk(gpu(x, dt)).cpu().numpy()
    err = rel(y, D @ x)
    assert err < 2e-3, err


def test_dk_is_derivative_of_the_product_fp64():
    W = workloads.get("sphere-r0.5m-ico3")
    h = 2e-5 * W.k
    _, P0 = plan(W.name)
    _, Pp = plan(W.name, k=W.k + h)
    _, Pm = plan(W.name, k=W.k - h)
    assert Pp.info()["trunc_L"] == P0.info()["trunc_L"] == Pm.info()["trunc_L"]
    x = gpu(workloads.rhs(P0.n, 4, W.seed), torch.float64)
    fd = ((Pp.matvec(x) - Pm.matvec(x)) / (2 * h)).cpu().numpy()
    y = P0.matvec_dk(x).cpu().numpy()
    err = rel(y, fd)
    assert err < 1e-6, err


def test_dk_complex_input_and_adjoint():
    W, P = plan("sphere-r0.5m-ico3")
    _, D = mats("sphere-r0.5m-ico3")
    x = workloads.rhs_complex(P.n, 3, W.seed)
    for dt in (torch.complex128, torch.complex64):
        xd = gpu(x, dt)
        y = P.matvec_dk(xd).cpu().numpy()
        assert rel(y, D @ x) < 2e-3
        ya = P.matvec_dk_adjoint(xd).cpu().numpy()
        assert rel(ya, D.conj().T @ x) < 2e-3
        yc = P.matvec_dk(xd.conj().resolve_conj()).conj().cpu().numpy()
        assert np.array_equal(ya, yc)


@pytest.mark.parametrize("B", [1, 3])
def test_dk_single_and_ragged_columns(B):
    W, P = plan("sphere-r0.5m-ico3")
    _, D = mats("sphere-r0.5m-ico3")
    x = workloads.rhs(P.n, B, W.seed + B)
    for dt in (torch.float64, torch.float32):
        y = P.matvec_dk(gpu(x, dt)).cpu().numpy()
        assert rel(y, D @ x) < 2e-3


def test_dk_column_limit_and_binding_split():
    W, P = plan("sphere-r0.5m-ico3", max_batch=8)
    _, D = mats("sphere-r0.5m-ico3")
    x = workloads.rhs(P.n, 5, W.seed)
    xd = gpu(x, torch.float64)
    with pytest.raises(M.MlfmaError) as ei:
        P._product(P._lib.mlfma_matvec_dk, xd, None, None)   # 2 x 5 columns > max_batch 8
    assert ei.value.status == 1
    y = P.matvec_dk(xd).cpu().numpy()                          # the binding splits into 4 + 1
    assert rel(y, D @ x) < 2e-3
    y1 = P.matvec_dk(xd[:, :4]).cpu().numpy()
    assert np.array_equal(y[:, :4], y1)


@pytest.mark.parametrize("name,rows", [("plate6m-strips", 12), ("sphere-r2m-ico5", 8)])
def test_dk_rows_full_size(name, rows):
    W, P = plan(name)
    v, t = W.mesh()
    B = 4
    x = workloads.rhs(P.n, B, W.seed)
    idx = np.random.default_rng(11).choice(P.n, rows, replace=False)
    ref = efie.Problem(v, t, W.k).rows_dk(idx) @ x
    y = P.matvec_dk(gpu(x, torch.float32)).cpu().numpy()[idx]
    err = rel(y, ref)
    assert err < 3e-3, err


@pytest.mark.parametrize("complex_x", [False, True])
def test_autograd_matches_dense_model(complex_x):
    name = "sphere-r0.5m-ico3"
    W, P = plan(name)
    Z0, D = mats(name)
    B = 2
    xn = workloads.rhs_complex(P.n, B, W.seed) if complex_x else workloads.rhs(P.n, B, W.seed)
    wn = np.random.default_rng(3).standard_normal((P.n, B))
    dt = torch.complex128 if complex_x else torch.float64

    x = gpu(xn, dt).requires_grad_(True)
    k = torch.tensor(W.k, dtype=torch.float64, device="cuda", requires_grad=True)
    y = M.efie_product(P, x, k)
    w = gpu(wn, torch.float64)
    loss = (w * y.real ** 2 + (1 - w) * y.imag * y.real).sum()
    loss.backward()

    xr = gpu(xn, dt).requires_grad_(True)
    kr = torch.tensor(W.k, dtype=torch.float64, device="cuda", requires_grad=True)
    Zt = gpu(Z0, torch.complex128) + (kr - W.k) * gpu(D, torch.complex128)
    yr = Zt @ (xr if complex_x else xr.to(torch.complex128))
    lr = (w * yr.real ** 2 + (1 - w) * yr.imag * yr.real).sum()
    lr.backward()

    assert rel(x.grad.cpu().numpy(), xr.grad.cpu().numpy()) < 2e-3
    assert abs(k.grad.item() - kr.grad.item()) < 2e-3 * abs(kr.grad.item())


def test_autograd_rejects_other_wavenumber():
    W, P = plan("sphere-r0.5m-ico3")
    x = gpu(workloads.rhs(P.n, 1, W.seed), torch.float64)
    with pytest.raises(ValueError):
        M.efie_product(P, x, torch.tensor(W.k * 1.01, dtype=torch.float64))
