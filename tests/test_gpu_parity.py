"""GPU parity: the CUDA product (through the C ABI) against the FP64 CPU
oracle on the same seeded meshes and vectors.

Tolerances
- levels = 2: no far work (every leaf box neighbours every other), so the
  product is the stored near field alone, the same quadrature and closed
  forms as the oracle in FP64: relative error <= 1e-10 (rounding order only).
- MLFMA against the dense oracle: relative 2-norm error <= 1e-3 (the
  accuracy target of the product; truncation with d0 = 3 digits plus local
  interpolation), for FP64 and for FP32.
- Invariants: u^T (Z v) = v^T (Z u) to 1e-10 (FP64) / 1e-5 (FP32) relative,
  which needs anterpolation to be the weighted transpose of interpolation.
"""
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


_cache = {}


def problem(name, levels=None, interp_order=10, max_batch=64):
    key = (name, levels, interp_order, max_batch)
    if key not in _cache:
        W = workloads.get(name)
        v, t = W.mesh()
        P = M.MlfmaPlan(v, t, W.k, levels or W.levels, W.digits, interp_order=interp_order, max_batch=max_batch)
        _cache[key] = (W, v, t, P)
    return _cache[key]


_dense = {}


def dense(name):
    if name not in _dense:
        W = workloads.get(name)
        v, t = W.mesh()
        _dense[name] = efie.Problem(v, t, W.k).dense()
    return _dense[name]


def gpu(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def test_near_field_only_matches_dense_fp64():
    """Two levels: the product is the near-field blocks alone."""
    W, v, t, P = problem("sphere-r0.5m-ico2", levels=2)
    Z = dense("sphere-r0.5m-ico2")
    x = workloads.rhs(P.n, 3, W.seed)
    y = P.matvec(gpu(x, torch.float64)).cpu().numpy()
    assert rel(y, Z @ x) < 1e-10


@pytest.mark.parametrize("name", ["sphere-r0.5m-ico3"])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_mlfma_matches_dense(name, dt):
    W, v, t, P = problem(name)
    Z = dense(name)
    x = workloads.rhs(P.n, W.batch, W.seed)
    y = P.matvec(gpu(x, dt)).cpu().numpy()
    err = rel(y, Z @ x)
    assert err < 1e-3, err


def test_coarse_mesh_error_is_truncation_not_arithmetic():
    """480 unknowns on the r = 0.5 m sphere: triangles (~0.15 lambda) are
    large against the 0.25 lambda leaf boxes, so RWG supports reach far out
    of their boxes and the 3-digit expansion gives ~2e-3.  FP32 and FP64 agree
    to 1e-5 (the error is the expansion's), and more digits remove it."""
    W = workloads.get("sphere-r0.5m-ico2")
    v, t = W.mesh()
    Z = dense("sphere-r0.5m-ico2")
    x = workloads.rhs(Z.shape[0], W.batch, W.seed)
    P3 = M.MlfmaPlan(v, t, W.k, W.levels, 3.0)
    P5 = M.MlfmaPlan(v, t, W.k, W.levels, 5.0)
    y64 = P3.matvec(gpu(x, torch.float64)).cpu().numpy()
    y32 = P3.matvec(gpu(x, torch.float32)).cpu().numpy()
    assert rel(y64, Z @ x) < 3e-3
    assert rel(y32, y64) < 1e-5
    assert rel(P5.matvec(gpu(x, torch.float64)).cpu().numpy(), Z @ x) < 1e-3


def test_mlfma_single_vector_and_ragged_batches():
    W, v, t, P = problem("sphere-r0.5m-ico3")
    Z = dense("sphere-r0.5m-ico3")
    for B in (1, 3, 7, 33, 64):
        x = workloads.rhs(P.n, B, W.seed + B)
        y = P.matvec(gpu(x, torch.float32)).cpu().numpy()
        assert rel(y, Z @ x) < 1e-3
        if B > 1:
            y1 = P.matvec(gpu(x[:, 1:2], torch.float32)).cpu().numpy()
            assert np.abs(y1[:, 0] - y[:, 1]).max() < 1e-5 * np.abs(y[:, 1]).max()
    with pytest.raises(M.MlfmaError):
        P.matvec(gpu(workloads.rhs(P.n, 65, 1), torch.float32))


def test_bilinear_symmetry():
    W, v, t, P = problem("sphere-r0.5m-ico3")
    u = workloads.rhs(P.n, 1, 11)[:, 0]
    w = workloads.rhs(P.n, 1, 12)[:, 0]
    for dt, tol in ((torch.float64, 1e-10), (torch.float32, 1e-5)):
        Zu = P.matvec(gpu(u, dt)).cpu().numpy()
        Zw = P.matvec(gpu(w, dt)).cpu().numpy()
        a, b = w @ Zu, u @ Zw
        scale = np.linalg.norm(Zu) * np.linalg.norm(w)
        assert abs(a - b) < tol * scale, (dt, abs(a - b) / scale)


def test_complex_input_and_adjoint():
    W, v, t, P = problem("sphere-r0.5m-ico3")
    Z = dense("sphere-r0.5m-ico3")
    xc = workloads.rhs_complex(P.n, 4, 5)
    for dt in (torch.complex128, torch.complex64):
        y = P.matvec(gpu(xc, dt)).cpu().numpy()
        assert rel(y, Z @ xc) < 1e-3
        ya = P.matvec_adjoint(gpu(xc, dt)).cpu().numpy()
        assert rel(ya, Z.conj().T @ xc) < 1e-3
        # Z^H x = conj(Z conj x) exactly (same pass, conjugated)
        yb = P.matvec(gpu(xc.conj(), dt)).cpu().numpy().conj()
        assert np.abs(ya - yb).max() <= 1e-6 * np.abs(yb).max()


def test_host_buffers_match_device():
    W, v, t, P = problem("sphere-r0.5m-ico3")
    x = workloads.rhs(P.n, 8, 3)
    for prec, dt in ((M.FP32, torch.float32), (M.FP64, torch.float64)):
        yh = P.matvec_host(x, prec)
        yd = P.matvec(gpu(x, dt)).cpu().numpy()
        assert np.array_equal(yh, yd)


@pytest.mark.parametrize("name,rows", [("plate6m-strips", 24), ("sphere-r2m-ico5", 24)])
def test_mlfma_rows_full_size(name, rows):
    """Full-size meshes: sampled rows of y = Z x computed exactly by the
    oracle, same x, same launch as the benchmark (FP32, all columns)."""
    W, v, t, P = problem(name)
    x = workloads.rhs(P.n, max(W.batch, 4), W.seed)
    y32 = P.matvec(gpu(x, torch.float32)).cpu().numpy()
    y64 = P.matvec(gpu(x, torch.float64)).cpu().numpy()
    idx = np.random.default_rng(7).choice(P.n, rows, replace=False)
    ref = efie.Problem(v, t, W.k).matvec_rows(x, idx)
    assert rel(y64[idx], ref) < 1e-3
    assert rel(y32[idx], ref) < 1e-3
    assert rel(y32, y64) < 1e-4


def test_far_pair_tiny_mesh():
    """Two RWG pairs 3 m apart land in non-neighbouring leaf boxes: the entry
    comes from the expansion alone and must match the oracle's quadrature
    to the expansion's accuracy."""
    v, t = workloads.two_triangle_pairs(3.0)
    k = 2 * math.pi
    P = M.MlfmaPlan(v, t, k, 4, 3.0)
    Z = efie.Problem(v, t, k).dense()
    for j in range(2):
        e = np.zeros(2)
        e[j] = 1.0
        y = P.matvec(gpu(e, torch.float64)).cpu().numpy()
        assert rel(y, Z[:, j]) < 1e-3


@pytest.mark.parametrize("name,B", [("sphere-r2m-ico5", 8), ("plate6m-strips", 16)])
def test_fields_per_stage_fp32_against_fp64(name, B):
    """mlfma_export_field: the outgoing and incoming fields of every far level
    after a product, FP32 against FP64 on the same columns (the per-stage
    error report of the mixed-precision path); also the product itself."""
    W, v, t, P = problem(name)
    x = workloads.rhs(P.n, B, W.seed)
    inf = P.info()
    f, y = {}, {}
    for dt, prec in ((torch.float32, M.FP32), (torch.float64, M.FP64)):
        y[prec] = P.matvec(gpu(x, dt)).cpu().numpy()
        for l in range(2, inf["leaf_level"] + 1):
            for w in (0, 1):
                f[(prec, w, l)] = P.export_field(prec, w, l, B)
    for l in range(2, inf["leaf_level"] + 1):
        for w in (0, 1):
            a, b = f[(M.FP32, w, l)].astype(np.complex128), f[(M.FP64, w, l)]
            assert a.shape == (inf["box_count"][l], 2, inf["samples_K"][l], B)
            assert np.linalg.norm(b) > 0
            assert rel(a, b) < 1e-4, (l, w, rel(a, b))
    assert rel(y[M.FP32], y[M.FP64]) < 1e-5
