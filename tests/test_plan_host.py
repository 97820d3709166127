"""Host-side plan logic of the C-ABI library, on CPU (host_only plans: no GPU
is touched).  Checked against the oracle's independent RWG list, against the
addition theorem (Section III-A, Eqs. (7)-(8)) and the E1 point test of
Section V, and against exactness properties of the interpolation and
anterpolation (Section III-C)."""
import math
import os

import numpy as np
import pytest

import workloads
from oracle.rwg import rwg_list
from paper_1412_1756_gb300 import mlfma as M


def host_plan(name, **kw):
    W = workloads.get(name)
    v, t = W.mesh()
    return W, v, t, M.MlfmaPlan(v, t, W.k, W.levels, W.digits, host_only=True, **kw)


def test_library_exports_every_declared_symbol():
    import ctypes
    import re
    import os
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "mlfma.h")).read()
    declared = set(re.findall(r"^(?:mlfma_status|void|const char \*)\s*((?:mlfma|cm)_\w+)\(", hdr, re.M))
    assert declared == set(M.EXPORTED)
    lib = ctypes.CDLL(M.library_path())
    for name in declared:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("name", ["sphere-r0.5m-ico3", "sphere-r2m-ico5", "plate6m-strips"])
def test_rwg_list_matches_oracle(name):
    W, v, t, P = host_plan(name)
    ev, tp = P.rwg_edges()
    r = rwg_list(v, t)
    assert P.n == W.n_expected
    assert np.array_equal(ev, r["edge_v"]) and np.array_equal(tp, r["tri"])


def test_bad_meshes_rejected():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1]], float)
    for tris in ([[0, 1, 2], [1, 0, 3], [0, 1, 4]], [[0, 1, 2], [0, 1, 3]], [[0, 1, 7]], [[0, 1, 1]]):
        with pytest.raises(M.MlfmaError) as e:
            M.MlfmaPlan(v, np.array(tris), 2 * math.pi, 3, host_only=True)
        assert e.value.status == 1
    with pytest.raises(M.MlfmaError):
        M.MlfmaPlan(v, np.array([[0, 1, 2], [1, 0, 3]]), -1.0, 3, host_only=True)
    with pytest.raises(M.MlfmaError):
        M.MlfmaPlan(v, np.array([[0, 1, 2], [1, 0, 3]]), 1.0, 1, host_only=True)
    with pytest.raises(M.MlfmaError):
        M.MlfmaPlan(v, np.array([[0, 1, 2], [1, 0, 3]]), 1.0, 3, interp_order=5, host_only=True)


def test_tree_and_lists_sphere_r2():
    """Sizes of the five-level tree on the 30,720-unknown sphere: every
    unknown in exactly one leaf box, a box-pair near structure, and
    interaction lists that, with the near lists, cover every leaf pair once."""
    W, v, t, P = host_plan("sphere-r2m-ico5")
    inf = P.info()
    assert inf["box_count"] == [1, 8, 56, 272, 1160]
    assert inf["trunc_L"][2:] == [20, 13, 8]
    assert inf["samples_K"][2:] == [882, 392, 162]
    assert inf["translations"][2:] == [2504, 12216, 54000]
    perm = P.export(M.X_PERM)
    assert np.array_equal(np.sort(perm), np.arange(P.n))
    assert inf["near_nnz"] == P.export(M.X_NEAR_COUNT)[0]


def test_truncation_number_eq9():
    """L = ceil(kd + 1.8 d0^(2/3) (kd)^(1/3)), d = sqrt(3) a (Section V)."""
    W, v, t, P = host_plan("cube8m")
    inf = P.info()
    for l in range(2, inf["levels"]):
        a = inf["root_side"] / 2 ** l
        kd = W.k * math.sqrt(3) * a
        assert inf["trunc_L"][l] == math.ceil(kd + 1.8 * 3.0 ** (2 / 3) * kd ** (1 / 3))
        assert inf["samples_K"][l] == 2 * (inf["trunc_L"][l] + 1) ** 2


def _grid(P, l):
    g = P.export(M.X_GRID, l)
    st = np.sqrt(1 - g[:, 0] ** 2)
    kh = np.stack([st * np.cos(g[:, 1]), st * np.sin(g[:, 1]), g[:, 0]], 1)
    th = np.stack([g[:, 0] * np.cos(g[:, 1]), g[:, 0] * np.sin(g[:, 1]), -st], 1)
    ph = np.stack([-np.sin(g[:, 1]), np.cos(g[:, 1]), 0 * st], 1)
    return g, kh, th, ph


def test_grid_integrates_band_limited_exactly():
    """(L+1) Gauss-Legendre nodes in cos(theta) x 2(L+1) uniform phi integrate
    spherical polynomials of degree <= 2L+1 exactly: int exp(i k k.d) = 4 pi j0(k|d|)
    for small |d|, and sum of weights = 4 pi."""
    W, v, t, P = host_plan("sphere-r2m-ico5")
    g, kh, _, _ = _grid(P, 2)
    assert abs(g[:, 2].sum() - 4 * math.pi) < 1e-12
    d = np.array([0.1, -0.2, 0.15])
    val = np.sum(g[:, 2] * np.exp(1j * W.k * (kh @ d)))
    x = W.k * np.linalg.norm(d)
    assert abs(val - 4 * math.pi * math.sin(x) / x) < 1e-12


def _point_test(a, d0, ri, rm, rj, rmp, offset=(2, 0, 0), kernel="exp"):
    """Relative error of the plane-wave form of one kernel between two points
    through the library's own translation table at level 2:
    exp(ikr)/r by Eq. (7) with Eq. (8) ("exp"); cos(kr)/r by Eq. (CosKer)
    ("cos"), whose alpha is i x the exported y_l table, so the prefactor
    ik/4pi becomes -k/4pi; sin(kr)/r by Eq. (SinKer) ("sin"), alpha = -i x the
    exported j_l table, prefactor k/4pi; "sin-sib" uses the sibling table of
    Eq. (RI) (nearby offsets)."""
    k = 2 * math.pi
    v, t = workloads.cube(4 * a, 8)
    P = M.MlfmaPlan(v, t, k, 3, d0, host_only=True)
    g, kh, _, _ = _grid(P, 2)
    what, offs_what, pref = {"exp": (M.X_ALPHA, M.X_ALPHA_OFFS, 1j * k / (4 * math.pi)),
                             "cos": (M.X_ALPHA_Y, M.X_ALPHA_OFFS, -k / (4 * math.pi)),
                             "sin": (M.X_ALPHA_J, M.X_ALPHA_OFFS, k / (4 * math.pi)),
                             "sin-sib": (M.X_SIB_ALPHA, M.X_SIB_OFFS, k / (4 * math.pi))}[kernel]
    al = P.export(what, 2).reshape(-1, g.shape[0])
    offs = P.export(offs_what, 2)
    ti = [i for i, o in enumerate(offs) if tuple(o) == offset][0]
    ri, rm, rj, rmp = (np.asarray(z) * a for z in (ri, rm, rj, rmp))
    assert np.allclose(rm - rmp, np.array(offset) * a)
    r = np.linalg.norm(ri - rj)
    exact = {"exp": np.exp(1j * k * r), "cos": np.cos(k * r), "sin": np.sin(k * r),
             "sin-sib": np.sin(k * r)}[kernel] / r
    approx = pref * np.sum(g[:, 2] * np.exp(1j * k * (kh @ ((ri - rm) + (rmp - rj)))) * al[ti])
    return abs(approx - exact) / abs(exact)


def test_addition_theorem_benign_points():
    """Points close to their group centres: the truncated Gegenbauer series
    converges like (|d|/|r|)^L, so Eq. (7) with the table of Eq. (8) must
    reproduce exp(ikr)/r to ~1e-10."""
    for a in (0.5, 1.0, 2.0):
        err = _point_test(a, 3.0, (2.55, 0.45, 0.52), (2.5, 0.5, 0.5), (0.47, 0.53, 0.5), (0.5, 0.5, 0.5))
        assert err < 1e-9, (a, err)


def test_e1_point_test_case1():
    """Section V, Case 1 geometry: source (0.9999a, a, 0) in the group centred
    at (a/2, a/2, a/2); observer (2.9999a, 0, a) in the group centred at
    (2.5a, a/2, a/2); L from Eq. (9) with d0 = 3.  Error falls with a/lambda
    and reaches the 3-digit level from a = lambda on."""
    errs = []
    for a in (0.25, 0.5, 1.0, 2.0, 4.0):
        errs.append(_point_test(a, 3.0, (2.9999, 0, 1.0), (2.5, 0.5, 0.5), (0.9999, 1.0, 0.0), (0.5, 0.5, 0.5)))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[0] < 1e-2 and errs[1] < 3e-3 and max(errs[2:]) < 1e-3, errs


CASE1 = ((2.9999, 0, 1.0), (2.5, 0.5, 0.5), (0.9999, 1.0, 0.0), (0.5, 0.5, 0.5))
CASE2 = ((1.0001, 0, 0), (1.5, 0.5, 0.5), (0.9999, 1.0, 0.0), (0.5, 0.5, 0.5))


def test_e1_point_test_cos_sin_case1():
    """Section V, Case 1 (the addition theorem holds): the sin(kr)/r kernel
    is reproduced at every box size; the cos(kr)/r kernel only from about
    half a wavelength up, its error growing as the box shrinks (the y_l
    terms of Eq. (CosKer)); both halves add up to the exp kernel's table."""
    es, ec = [], []
    for a in (0.125, 0.25, 0.5, 1.0, 2.0):
        es.append(_point_test(a, 3.0, *CASE1, kernel="sin"))
        ec.append(_point_test(a, 3.0, *CASE1, kernel="cos"))
    assert max(es) < 1e-8, es
    assert ec[0] > ec[2] and ec[1] > ec[3], ec
    assert max(ec[3:]) < 1e-3, ec
    v, t = workloads.cube(2.0, 8)
    P = M.MlfmaPlan(v, t, 2 * math.pi, 3, 3.0, host_only=True)
    al, aj, ay = (P.export(w, 2) for w in (M.X_ALPHA, M.X_ALPHA_J, M.X_ALPHA_Y))
    assert np.abs(al - (aj + 1j * ay)).max() < 1e-12 * np.abs(al).max()


def test_e1_point_test_sin_case2_nearby_groups():
    """Section V, Case 2: observer and source in touching groups (the
    addition theorem for exp(ikr)/r is violated, |r_im + r_m'j| > |r_mm'|);
    the regular sin(kr)/r kernel is still reproduced, through the sibling
    table that Eq. (RI) uses for nearby groups."""
    for a in (0.25, 0.5, 1.0, 2.0):
        err = _point_test(a, 3.0, *CASE2, offset=(1, 0, 0), kernel="sin-sib")
        assert err < 1e-6, (a, err)


@pytest.mark.parametrize("order,tol", [(6, 3e-3), (8, 1e-3), (10, 5e-4)])
def test_interpolation_band_limited(order, tol):
    """Local Lagrange interpolation (Section III-C) of the pattern of a point
    current inside a child box to the parent grid, theta and phi components,
    converging with the order; anterpolation is exactly
    W_child^-1 Interp^T W_parent."""
    W, v, t, P = host_plan("sphere-r2m-ico5", interp_order=order)
    for l in (2, 3):
        gp, khp, thp, php = _grid(P, l)
        gc, khc, thc, phc = _grid(P, l + 1)
        Mx = P.export(M.X_INTERP, l).reshape(gp.shape[0], gc.shape[0])
        A = P.export(M.X_ANTERP, l).reshape(gc.shape[0], gp.shape[0])
        assert np.abs(A - (Mx.T * gp[None, :, 2]) / gc[:, 2, None]).max() < 1e-14
        ac = P.info()["root_side"] / 2 ** (l + 1)
        rng = np.random.default_rng(l)
        for _ in range(10):
            d = rng.uniform(-0.5, 0.5, 3) * ac * 1.2
            pol = rng.standard_normal(3)
            for tc, tp in ((thc, thp), (phc, php)):
                fc = (tc @ pol) * np.exp(1j * W.k * (khc @ d))
                fp = (tp @ pol) * np.exp(1j * W.k * (khp @ d))
                assert np.abs(Mx @ fc - fp).max() < tol * np.abs(fp).max()


@pytest.mark.parametrize("name", ["sphere-r2m-ico5", "cube8m-6lv", "plate6m-strips"])
@pytest.mark.parametrize("order", [6, 10])
def test_windowed_tables_rebuild_the_stencils(name, order):
    """The FP32 windowed kernels' tables (stencil rows in groups of four on
    one window of consecutive positions each; pole reflections placed at
    -i-1 / 2n-i-1, phi positions modulo the grid), expanded the way the
    kernels read them, give the same interpolation and anterpolation
    matrices as the row stencils (Section III-C), entry for entry; each
    window is no wider than the union of four rows of its stencil can be."""
    W, v, t, P = host_plan(name, interp_order=order)
    for l in range(2, P.info()["leaf_level"]):
        sh = P.export(M.X_WIN_SHAPE, l)
        assert (sh[:, 0] > 0).all(), sh
        # up: order taps per row, rows at most ~1 source step apart; down: the
        # transposes, at most ~2 source steps apart per row
        assert sh[0, 1] <= order + 4 and sh[1, 1] <= order + 4, sh
        assert sh[2, 1] <= 2 * order + 8 and sh[3, 1] <= 2 * order + 8, sh
        for wi, plain in ((M.X_WIN_INTERP, M.X_INTERP), (M.X_WIN_ANTERP, M.X_ANTERP)):
            a, b = P.export(wi, l), P.export(plain, l)
            assert np.abs(a - b).max() <= 1e-15 * np.abs(b).max()


@pytest.mark.parametrize("name", ["sphere-r2m-ico5", "cube8m-6lv"])
def test_aggregation_shift_and_its_z_split(name):
    """The phase shift of the aggregation from a child box to its parent
    (Section III-C: a child's pattern about its own centre, times
    exp(i k khat . (r_parent - r_child)), is its pattern about the parent's
    centre) matches each child's offset taken from the plan's box centres at
    every parent sample; it factors into an x-y part and a theta-row z part,
    and the x-y part is the same for the two children that differ only in z
    (the sharing the z-pair up and down kernels rely on)."""
    W, v, t, P = host_plan(name)
    leaf = P.info()["leaf_level"]
    for l in range(2, leaf):
        g, kh, _, _ = _grid(P, l)
        nth = len(np.unique(g[:, 0]))
        nph = g.shape[0] // nth
        S, Sxy, Sz = (P.export(w, l) for w in (M.X_SHIFT, M.X_SHIFT_XY, M.X_SHIFT_Z))
        assert S.shape == (8, g.shape[0]) and Sxy.shape == (8, g.shape[0]) and Sz.shape == (8, nth)
        # every child's offset from its parent, from the exported centres
        cp, cc = P.export(M.X_BOX_CENTERS, l), P.export(M.X_BOX_CENTERS, l + 1)
        h = P.info()["root_side"] / 2 ** (l + 2)
        seen = set()
        for c in np.random.default_rng(l).choice(len(cc), min(len(cc), 200), replace=False):
            p = np.argmin(np.abs(cp - cc[c]).sum(1))
            d = cp[p] - cc[c]                                   # r_parent - r_child
            assert np.allclose(np.abs(d), h, rtol=1e-12, atol=0)
            o = 4 * (d[0] < 0) + 2 * (d[1] < 0) + (d[2] < 0)    # the child lies at +x / +y / +z
            seen.add(o)
            ref = np.exp(1j * W.k * (kh @ d))
            assert np.abs(S[o] - ref).max() < 1e-12, (l, o)
        assert len(seen) >= 2
        assert np.abs(np.abs(S) - 1).max() < 1e-14
        assert np.abs(S - Sxy * np.repeat(Sz, nph, axis=1)).max() < 1e-14
        for o in range(0, 8, 2):
            assert np.array_equal(Sxy[o], Sxy[o + 1])
            assert np.array_equal(Sz[o], Sz[0]) and np.array_equal(Sz[o + 1], Sz[1])
        assert np.abs(Sz[0] * Sz[1] - 1).max() < 1e-14     # the two z parts are conjugate
    for bad in (0, leaf):   # no aggregation into the root or into the leaf level
        with pytest.raises(M.MlfmaError):
            P.export(M.X_SHIFT, bad)


def test_tune_cache_key_and_file(tmp_path):
    """The tuned-shape cache: keys separate GPUs, trees, columns and
    precisions; the file round-trips and a damaged file reads as empty."""
    W, v, t, P = host_plan("sphere-r2m-ico5")
    inf = P.info()
    k1 = M.tune_cache_key("GPU A", inf, 10, 64, M.FP32, False)
    assert k1 == M.tune_cache_key("GPU A", inf, 10, 64, M.FP32, False)
    others = [M.tune_cache_key("GPU B", inf, 10, 64, M.FP32, False), M.tune_cache_key("GPU A", inf, 8, 64, M.FP32, False),
              M.tune_cache_key("GPU A", inf, 10, 32, M.FP32, False), M.tune_cache_key("GPU A", inf, 10, 64, M.FP64, False),
              M.tune_cache_key("GPU A", inf, 10, 64, M.FP32, True)]
    assert len(set(others + [k1])) == 6
    W2, v2, t2, P2 = host_plan("sphere-r0.5m-ico3")
    assert M.tune_cache_key("GPU A", P2.info(), 10, 64, M.FP32, False) != k1
    path = str(tmp_path / "tune.json")
    assert M._read_tune_cache(path) == {}
    M._write_tune_cache(path, {k1: list(range(M.TUNE_FIELDS))})
    assert M._read_tune_cache(path)[k1] == list(range(M.TUNE_FIELDS))
    with open(path, "w") as f:
        f.write("{not json")
    assert M._read_tune_cache(path) == {}


def test_header_is_plain_c(tmp_path):
    """include/mlfma.h is a C ABI: it compiles as strict C99 (no C++ in the
    declarations) and as C++."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "use_header.c"
    src.write_text('#include "mlfma.h"\nint main(void) { mlfma_cm_opts o; mlfma_info i; (void)o; (void)i; '
                   'return (int)sizeof(&cm_block_solve) == 0; }\n')
    for cmd in ([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                [gcc, "-x", "c++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, str(src)]):
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr



def test_overlapping_x_and_y_rejected():
    """x and y may not share a byte: a y equal to x, starting inside x or
    ending inside x is MLFMA_EINVAL before anything else is looked at; a y
    that only touches x passes that check (and then fails for the host-only
    plan with another message)."""
    import ctypes
    W, v, t, P = host_plan("sphere-r0.5m-ico2")
    lib = M.load()
    n, B = P.n, 2
    xbytes, ybytes = n * B * 8, n * B * 16      # FP64 real x, complex128 y
    buf = np.zeros((xbytes + 2 * ybytes) // 8, np.float64)
    x = buf.ctypes.data + ybytes
    for fn in (lib.mlfma_matvec_host, lib.mlfma_matvec_noalloc):
        for y in (x, x + 8, x + xbytes - 8, x - ybytes + 8):
            st = fn(P._h, ctypes.c_void_p(x), 0, ctypes.c_void_p(y), B, M.FP64, None)
            assert st == 1 and b"overlap" in lib.mlfma_last_error(), (fn, y - x)
        for y in (x + xbytes, x - ybytes):
            st = fn(P._h, ctypes.c_void_p(x), 0, ctypes.c_void_p(y), B, M.FP64, None)
            assert st == 1 and b"overlap" not in lib.mlfma_last_error(), (fn, y - x)


def test_host_only_plan_refuses_device_work():
    """A host-only plan (tables, no device memory) answers every product,
    the tuner and the field export with MLFMA_EINVAL and a message naming
    the reason, before any CUDA call; so do a NULL plan, a NULL buffer and
    B < 1.  Waiting on it (mlfma_sync) has nothing to wait for."""
    import ctypes
    W, v, t, P = host_plan("sphere-r0.5m-ico2")
    lib = M.load()
    n, B = P.n, 2
    x, y = np.zeros((n, B)), np.zeros((n, B), complex)
    xp, yp = ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(y.ctypes.data)
    for fn in (lib.mlfma_matvec, lib.mlfma_matvec_adjoint, lib.mlfma_matvec_dk, lib.mlfma_matvec_dk_adjoint,
               lib.mlfma_matvec_x, lib.mlfma_matvec_r, lib.mlfma_matvec_host, lib.mlfma_matvec_noalloc):
        assert fn(P._h, xp, 0, yp, B, M.FP64, None) == 1 and b"host-only" in lib.mlfma_last_error(), fn
        assert fn(None, xp, 0, yp, B, M.FP64, None) == 1, fn
        assert fn(P._h, None, 0, yp, B, M.FP64, None) == 1 and b"NULL" in lib.mlfma_last_error(), fn
        assert fn(P._h, xp, 0, yp, 0, M.FP64, None) == 1 and b"B must be" in lib.mlfma_last_error(), fn
    ms = (ctypes.c_double * 64)()
    assert lib.mlfma_profile_stages(P._h, xp, 0, yp, B, M.FP64, None, ms) == 1
    d0, d1 = ctypes.c_double(), ctypes.c_double()
    assert lib.mlfma_tune(P._h, B, 0, M.FP64, None, ctypes.byref(d0), ctypes.byref(d1)) == 1
    assert b"host-only" in lib.mlfma_last_error()
    need = ctypes.c_int64()
    assert lib.mlfma_export_field(P._h, M.FP64, 0, 2, 1, None, 0, ctypes.byref(need)) == 1
    assert lib.mlfma_sync(P._h, None) == 0


def test_tune_set_keeps_documented_shapes_only():
    """mlfma_tune_set / mlfma_tune_get (host logic): every documented value
    of each field round-trips per (columns, precision), other column counts
    keep the built-in shapes, and a value outside a field's documented set is
    MLFMA_EINVAL (include/mlfma.h lists the sets)."""
    W, v, t, P = host_plan("sphere-r2m-ico5")
    L = M.MAX_LEVELS
    up = [0, 1, 2, 4, 8, 16, 202, 204, 208, 216, 304, 308, 316, 404, 408, 704, 708, 716]
    down = [0, 1, 2, 4, 8, 16, 104, 108, 204, 208, 216, 304, 308, 316, 404, 408, 504, 508, 804, 808]
    fields = [(0, range(4)), (1, range(6)), (2, range(7)), (3 + 2, up), (3 + L + 3, down), (3 + 2 * L + 4, range(12))]
    for f, values in fields:
        for val in values:
            ch = np.zeros(M.TUNE_FIELDS, np.int32)
            ch[f] = val
            P.tune_set(16, ch, M.FP32)
            assert np.array_equal(P.tune_get(16, M.FP32), ch), (f, val)
    assert not P.tune_get(32, M.FP32).any() and not P.tune_get(16, M.FP64).any()
    for f, bad in ((0, 4), (1, 6), (2, 7), (3 + 2, 3), (3 + 2, 416), (3 + 2, 804), (3 + L + 3, 416),
                   (3 + L + 3, 704), (3 + 2 * L + 4, 12), (3 + 2 * L + 4, -1)):
        ch = np.zeros(M.TUNE_FIELDS, np.int32)
        ch[f] = bad
        with pytest.raises(M.MlfmaError):
            P.tune_set(16, ch, M.FP32)
    with pytest.raises(M.MlfmaError):
        P.tune_set(0, np.zeros(M.TUNE_FIELDS, np.int32), M.FP32)


def test_translation_tables_match_scipy_series():
    """Eq. (8)'s translation function, its j_l and y_l halves (the sin- and
    cos-kernel tables of Section V, Eqs. (SinKer), (CosKer)) and the sibling
    sin-kernel table, as the library builds them with its own spherical
    Bessel and Legendre recurrences, against SciPy's spherical_jn,
    spherical_yn and eval_legendre at every sample of each level.  The r = 8 m
    sphere puts L = 57 on 4-wavelength boxes, so the nearest offsets reach
    orders well above kr (where an upward j_l recurrence would fail)."""
    from scipy.special import eval_legendre, spherical_jn, spherical_yn
    v, t = workloads.icosphere(3, 8.0)
    k = 2 * math.pi
    P = M.MlfmaPlan(v, t, k, 4, 3.0, host_only=True)
    inf = P.info()
    assert inf["trunc_L"][2] == 57
    for l in range(2, inf["leaf_level"] + 1):
        _, kh, _, _ = _grid(P, l)
        L = inf["trunc_L"][l]
        a = inf["root_side"] / 2 ** l
        ls = np.arange(L + 1)
        il = (1j ** ls) * (2 * ls + 1)
        tables = [(M.X_ALPHA_OFFS, M.X_ALPHA_J, M.X_ALPHA_Y, M.X_ALPHA), (M.X_SIB_OFFS, M.X_SIB_ALPHA, None, None)]
        for offs_code, jcode, ycode, full in tables:
            offs = P.export(offs_code, l)
            aj = P.export(jcode, l).reshape(len(offs), -1)
            ay = P.export(ycode, l).reshape(len(offs), -1) if ycode else None
            al = P.export(full, l).reshape(len(offs), -1) if full else None
            order = np.argsort(np.linalg.norm(offs, axis=1))
            pick = np.unique(np.concatenate([order[:6], order[-4:],
                                             np.random.default_rng(l).choice(len(offs), min(6, len(offs)), False)]))
            for ti in pick:
                r = a * offs[ti]
                rn = np.linalg.norm(r)
                Pl = eval_legendre(ls[:, None], (kh @ r / rn)[None, :])
                jl, yl = spherical_jn(ls, k * rn), spherical_yn(ls, k * rn)
                sj = np.sum((2 * ls + 1) * np.abs(jl))
                assert np.abs(aj[ti] - (il * jl) @ Pl).max() <= 1e-11 * sj, (l, offs[ti])
                if ay is not None:
                    sy = np.sum((2 * ls + 1) * np.abs(yl))
                    assert np.abs(ay[ti] - (il * yl) @ Pl).max() <= 1e-11 * sy, (l, offs[ti])
                    assert np.abs(al[ti] - (aj[ti] + 1j * ay[ti])).max() <= 1e-14 * (sj + sy)


@pytest.mark.parametrize("case", ["nan vertex", "inf vertex", "digits 0", "digits nan", "k nan", "k inf", "levels 23",
                                  "max_batch 0", "interp 0", "interp 2", "interp 40", "negative index", "empty", "zero area", "eta inf", "eta 0"])
def test_plan_arguments_rejected(case):
    """mlfma_plan answers each invalid argument with MLFMA_EINVAL (status 1)
    and a message, before any device work: non-finite coordinates or
    wavenumber, digits outside 1..15, levels outside 2..21, max_batch
    outside 1..4096, an odd interpolation order or one outside 4..12, a vertex
    index out of range, an empty mesh, a triangle of zero area, a wave
    impedance that is not positive and finite."""
    v, t = workloads.icosphere(2, 0.5)
    k, kw, levels, digits = 2 * math.pi, {}, 3, 3.0
    if case in ("nan vertex", "inf vertex"):
        v = v.copy()
        v[0, 0] = np.nan if case == "nan vertex" else np.inf
    elif case == "digits 0":
        digits = 0.0
    elif case == "digits nan":
        digits = float("nan")
    elif case in ("k nan", "k inf"):
        k = float("nan") if case == "k nan" else float("inf")
    elif case == "levels 23":
        levels = 23
    elif case == "max_batch 0":
        kw["max_batch"] = 0
    elif case in ("interp 0", "interp 2", "interp 40"):
        kw["interp_order"] = int(case.split()[1])
    elif case == "negative index":
        t = np.where(t == 0, -1, t)
    elif case == "empty":
        t = t[:0]
    elif case in ("eta inf", "eta 0"):
        kw["eta"] = float("inf") if case == "eta inf" else 0.0
    elif case == "zero area":
        v = np.vstack([v, v[:1]])
        t = np.vstack([t, [[0, len(v) - 1, t[0, 1]]]])
    with pytest.raises(M.MlfmaError) as e:
        M.MlfmaPlan(v, t, k, levels, digits, host_only=True, **kw)
    assert e.value.status == 1 and str(e.value)


@pytest.mark.parametrize("bad", [dict(nev=0), dict(nev=10, ncv=11), dict(ncv=10 ** 6), dict(op=7), dict(prec=2),
                                 dict(tol=0.0), dict(gmres_tol=-1.0), dict(gmres_restart=1), dict(max_inner=0),
                                 dict(max_restarts=0)])
def test_cm_solve_options_checked_before_device_work(bad):
    """cm_ira_solve refuses each invalid option with EINVAL on a host-only
    plan, before it looks for the device; valid options on that plan are
    refused for the plan itself.  cm_block_solve refuses a host-only plan."""
    W, v, t, P = host_plan("sphere-r0.5m-ico2")
    with pytest.raises(M.MlfmaError) as e:
        P.cm_solve(**bad, vectors=False)
    assert e.value.status == 1 and "host-only" not in str(e.value), str(e.value)
    with pytest.raises(M.MlfmaError) as e:
        P.cm_solve(vectors=False)
    assert e.value.status == 1 and "host-only" in str(e.value)
    with pytest.raises(M.MlfmaError) as e:
        P.cm_block_solve(nev=4, block=8, vectors=False)
    assert e.value.status == 1 and "device plan" in str(e.value)


def test_export_refuses_unknown_tables_levels_and_short_buffers():
    """mlfma_export: an unknown table code or a level the table does not
    have is EINVAL; a destination smaller than the table is EINVAL with
    *needed still set to the table's size; asking with dst = NULL only
    reports the size."""
    import ctypes
    W, v, t, P = host_plan("sphere-r2m-ico5")
    lib = M.load()
    for code in (0, 99):
        with pytest.raises(M.MlfmaError):
            P.export(code, 2)
    for code, level in ((M.X_ALPHA, 1), (M.X_INTERP, P.info()["leaf_level"]), (M.X_BOX_CENTERS, 9)):
        with pytest.raises(M.MlfmaError):
            P.export(code, level)
    need = ctypes.c_int64(-1)
    assert lib.mlfma_export(P._h, M.X_GRID, 2, None, 0, ctypes.byref(need)) == 0
    assert need.value == 4 * 8 * P.info()["samples_K"][2]
    buf = np.zeros(need.value // 8 - 1)
    need2 = ctypes.c_int64(-1)
    assert lib.mlfma_export(P._h, M.X_GRID, 2, buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes,
                            ctypes.byref(need2)) == 1
    assert b"too small" in lib.mlfma_last_error() and need2.value == need.value


def test_sweep_admission_refusals_are_host_logic():
    """mlfma_set_create (frequency sweeps): the memory admission compares each
    plan's estimate, made from its host tables, with the budget before any
    device allocation; a plan above the budget is ENOMEM with both sizes in
    the message.  An empty wavenumber list and a non-positive wavenumber are
    EINVAL."""
    v, t = workloads.icosphere(2, 0.5)
    with pytest.raises(M.MlfmaError) as e:
        M.MlfmaPlanSet(v, t, [2 * math.pi, 2.2 * math.pi], 3, device=0, budget_bytes=1 << 20)
    assert e.value.status == 2 and "admission budget is 1 MiB" in str(e.value)
    for ks in ([], [2 * math.pi, -1.0]):
        with pytest.raises(M.MlfmaError) as e:
            M.MlfmaPlanSet(v, t, ks, 3, device=0, budget_bytes=1 << 30)
        assert e.value.status == 1


def test_binding_refuses_host_buffers_for_device_products():
    """The binding's argument checks before any library call: device
    products take CUDA tensors for x and y (a host buffer would be accessed by
    the kernels as device memory), matvec_host takes a y array of the right
    dtype, layout and size (the device-to-host copy fills N*B values), and
    plans and sweep sets take [nv, 3] vertices and [nt, 3] triangles."""
    import types
    torch = pytest.importorskip("torch")
    W, v, t, P = host_plan("sphere-r0.5m-ico2")
    with pytest.raises(ValueError, match="x must be a CUDA tensor"):
        P.matvec(torch.zeros(P.n, 2))
    fake_x = types.SimpleNamespace(is_cuda=True, device="cuda:0")
    with pytest.raises(ValueError, match="y must be a CUDA tensor"):
        M._check_device_pair(fake_x, torch.zeros(4))
    M._check_device_pair(fake_x, None)
    x = np.zeros((P.n, 2), np.float32)
    for y in (np.zeros((P.n, 2), np.complex128), np.zeros((P.n, 1), np.complex64),
              np.zeros((2, P.n), np.complex64).T):
        with pytest.raises(ValueError, match="y must be"):
            P.matvec_host(x, M.FP32, y=y)
    with pytest.raises(M.MlfmaError):   # well-formed buffers: refused by the host-only plan itself
        P.matvec_host(x, M.FP32, y=np.zeros((P.n, 2), np.complex64))
    for vv, tt in ((v[:, :2], t), (v, t[:, :2]), (v.reshape(-1), t)):
        with pytest.raises(ValueError, match="verts must be"):
            M.MlfmaPlan(vv, tt, W.k, 3, host_only=True)
        with pytest.raises(ValueError, match="verts must be"):
            M.MlfmaPlanSet(vv, tt, [W.k], 3, device=0)


def test_c_abi_null_arguments():
    """NULL where the header asks for a plan, set or output pointer is
    MLFMA_EINVAL with a message; destroying NULL is a no-op; the RWG list
    copies only the arrays it is given (either may be NULL)."""
    import ctypes
    W, v, t, P = host_plan("sphere-r0.5m-ico2")
    L = M.load()
    vp, tp = v.ctypes.data_as(ctypes.c_void_p), np.ascontiguousarray(t, np.int32)
    calls = [lambda: L.mlfma_plan_info(P._h, None), lambda: L.mlfma_num_unknowns(P._h, None),
             lambda: L.mlfma_default_opts(None), lambda: L.mlfma_cm_default_opts(None),
             lambda: L.mlfma_plan_info(None, None), lambda: L.mlfma_export(None, M.X_GRID, 2, None, 0, None),
             lambda: L.mlfma_sync(None, None), lambda: L.mlfma_set_info(None, None, None, None, None, None),
             lambda: L.mlfma_set_plan(None, 0, None),
             lambda: L.mlfma_plan(vp, len(v), tp.ctypes.data_as(ctypes.c_void_p), len(t), W.k, 3, 3.0, None, None)]
    for c in calls:
        assert c() == 1 and L.mlfma_last_error()
    L.mlfma_destroy(None)
    L.mlfma_set_destroy(None)
    ev = np.full((P.n, 2), -1, np.int32)
    assert L.mlfma_rwg_edges(P._h, ev.ctypes.data_as(ctypes.c_void_p), None) == 0
    assert (ev >= 0).all() and (ev[:, 0] < ev[:, 1]).all()
    assert L.mlfma_rwg_edges(P._h, None, None) == 0
