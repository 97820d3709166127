"""GPU parity of the paper's kernel variants (Section IV) against the FP64
oracle's dense Z:

- R x (mlfma_matvec_r, R = Re Z) by the sin(kR)/R kernel in the form of
  Eq. (RI): near part the leaf box itself, every other pair of boxes
  translated at the level where their ancestors are siblings.  The regular
  kernel's expansion has no addition-theorem limit (Section V's point test
  reproduces it to ~1e-10), so the product meets the 1e-3 bound of the Z
  product on the 1,920-unknown sphere whose leaves are a quarter wavelength.
- X x (mlfma_matvec_x, X = Im Z) by the cos(kR)/R kernel of Eq. (XI): the
  standard tree, <= 1e-3 on a plate 4 x 4 wavelengths with wavelength
  leaves; on quarter-wavelength leaves it carries the Z product's whole
  expansion error (measured 2.4e-4, the same as Z), while the sin half is
  ~20x more accurate (1.0e-5).
- Consistency: R x + i X x reproduces mlfma_matvec where both are accurate.
"""
import numpy as np
import pytest

import workloads
from oracle import efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402

K0 = 2 * np.pi


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


_cache = {}


def case(name):
    if name not in _cache:
        if name == "sphere":
            v, t = workloads.icosphere(3, 0.5)
            levels = 3
        else:
            v, t = workloads.plate(4.0, 4.0, 24, 24)
            levels = 3
        P = M.MlfmaPlan(v, t, K0, levels, 3.0)
        Z = efie.Problem(v, t, K0).dense()
        _cache[name] = (P, Z)
    return _cache[name]


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_sin_kernel_resistance_product(dt):
    P, Z = case("sphere")
    x = workloads.rhs(P.n, 4, 1412)
    y = P.matvec_r(gpu(x, dt)).cpu().numpy()
    ref = Z.real @ x
    assert rel(y.real, ref) < 1e-3, rel(y.real, ref)
    assert np.linalg.norm(y.imag) < 1e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_cos_kernel_reactance_product_wavelength_leaves(dt):
    P, Z = case("plate")
    x = workloads.rhs(P.n, 4, 1413)
    y = P.matvec_x(gpu(x, dt)).cpu().numpy()
    ref = Z.imag @ x
    assert rel(y.real, ref) < 1e-3, rel(y.real, ref)
    assert np.linalg.norm(y.imag) < 1e-4 * np.linalg.norm(ref)


def test_expansion_error_sits_in_the_cos_half():
    """Quarter-wavelength leaves: Section V's point test reproduces
    sin(kr)/r to ~1e-10 but cos(kr)/r only to ~1e-2 at such sizes.  In the
    whole product the same split shows: the sin-kernel R product is an order
    of magnitude more accurate than the Z product, and the cos-kernel X
    product carries the Z product's expansion error."""
    P, Z = case("sphere")
    x = workloads.rhs(P.n, 4, 1414)
    xd = gpu(x, torch.float64)
    ex = rel(P.matvec_x(xd).cpu().numpy().real, Z.imag @ x)
    er = rel(P.matvec_r(xd).cpu().numpy().real, Z.real @ x)
    ez = rel(P.matvec(xd).cpu().numpy(), Z @ x)
    assert er < 0.1 * ez, (er, ez)
    assert 0.5 * ez < ex < 2 * ez, (ex, ez)


def test_r_plus_i_x_is_z_on_wavelength_leaves():
    P, Z = case("plate")
    x = workloads.rhs(P.n, 3, 1415)
    xd = gpu(x, torch.float64)
    z = P.matvec(xd).cpu().numpy()
    rx = P.matvec_r(xd).cpu().numpy() + 1j * P.matvec_x(xd).cpu().numpy()
    assert rel(rx, z) < 2e-3


def test_complex_input():
    P, Z = case("sphere")
    x = workloads.rhs_complex(P.n, 2, 1416)
    y = P.matvec_r(gpu(x, torch.complex128)).cpu().numpy()
    assert rel(y, Z.real @ x) < 1e-3


def test_sin_kernel_needs_three_levels():
    v, t = workloads.icosphere(2, 0.5)
    P = M.MlfmaPlan(v, t, K0, 2, 3.0)
    with pytest.raises(M.MlfmaError) as ei:
        P.matvec_r(gpu(workloads.rhs(P.n, 1, 1), torch.float64))
    assert ei.value.status == 6
