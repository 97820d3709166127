"""Planted mistakes in the oracle.  Each plausible slip in the oracle's C
source (a wrong sign, a dropped term, a wrong index, a transposed operand, a
wrong power of k) is written into a copy of efie_oracle.c.  The copy is
compiled on the CPU, and at least one of the oracle's own pins
(test_oracle_matrix, test_oracle_quadrature, test_oracle_dk: symmetry, the
semidefinite resistance, the plane-wave identity for Re Z, the sphere's
closed-form characteristic values, brute-force quadrature of the 1/R and
exp(ikR)/R potentials, central differences in k) must fail against it.  The
unchanged source passes all of them.  The eigen half of the oracle
(oracle/cm.py: the pencil of Eq. (GEP), its symmetric reduction and the
first-order slopes) gets the same treatment with a planted copy of the
module, against the sphere's closed-form values and slopes, and so does the
RWG list (oracle/rwg.py), against its counts, order, orientation, the RWG
identities and the library's own list."""
import importlib.util
import math
import re

import pytest

import workloads
from oracle import build as obuild
from oracle import efie
from tests import test_oracle_dk as td
from tests import test_oracle_matrix as tm
from tests import test_oracle_quadrature as tq
from tests import test_plan_host as th

# (slip, function it goes into, text there, planted text)
PLANTS = [
    ("scalar-potential term with the wrong sign", "z_raw",
     "(vec - Di * Dj * P0 / (k * k))", "(vec + Di * Dj * P0 / (k * k))"),
    ("scalar-potential term over k instead of k^2", "z_raw",
     "(vec - Di * Dj * P0 / (k * k))", "(vec - Di * Dj * P0 / k)"),
    ("test function's free vertex taken from its other triangle", "z_raw",
     "B->vfree[2 * i + a]", "B->vfree[2 * i + 1 - a]"),
    ("test function pointing the wrong way", "z_raw", "(r[c] - vi[c])", "(vi[c] - r[c])"),
    ("Green's function exp(-ikR) / R", "g_full", "cexp(I * k * R)", "cexp(-I * k * R)"),
    ("closed-form 1/R integral dropped", "tri_potential", "p0 += I0;", "p0 += 0.0;"),
    ("linear-density term with the wrong sign", "tri_potential", "I1[c] + rho[c] * I0", "I1[c] - rho[c] * I0"),
    ("quadrature weight read from a barycentric column", "tri_potential", "A * Q7[q][3] * g", "A * Q7[q][2] * g"),
    ("edge normal from a transposed cross product", "static_potential",
     "cross3(lhat, n, uhat);", "cross3(n, lhat, uhat);"),
    ("solid-angle term with the wrong sign", "static_potential",
     "*I0 += t * f - ah * beta;", "*I0 += t * f + ah * beta;"),
    ("dZ/dk scalar-potential term with the wrong sign", "dz_raw",
     "+ I * eta / (k * k) * Phi", "- I * eta / (k * k) * Phi"),
]


def _scope(src, fname):
    """[start, end) of the top-level C function `fname` in src."""
    m = re.search(r"^static [^\n(]*\b%s\(" % fname, src, re.M)
    assert m, fname
    nxt = re.search(r"^(static |int |typedef )", src[m.end():], re.M)
    return m.start(), (m.end() + nxt.start()) if nxt else len(src)


def _pins(stop_at_first=True):
    """Names of the pins that fail with the oracle library now loaded
    (cheap pins first; with stop_at_first only the first failure)."""
    failed = []

    def check(name, fn, *args):
        if failed and stop_at_first:
            return
        try:
            fn(*args)
        except Exception:   # an assertion, or a solver that breaks on a wrong matrix
            failed.append(name)

    v, t = workloads.icosphere(2, 0.5)
    P = efie.Problem(v, t, 2 * math.pi)
    sphere = (P, P.dense())
    check("Z symmetric", tm.test_symmetric, sphere)
    check("-Re Z semidefinite", tm.test_resistance_psd, sphere)
    for idx in (0, 9, 10, 11):
        check("1/R potentials vs Duffy quadrature (point %d)" % idx, tq.test_static_potential_matches_duffy, idx)
    for idx in (0, 10):
        check("extracted potentials vs the full kernel (point %d)" % idx,
              tq.test_extracted_potential_matches_full_kernel, idx)
    check("far potentials vs the full kernel", tq.test_far_potential_plain_rule_matches_full_kernel)
    check("sphere characteristic values vs the closed form", tm.test_sphere_cm_values_coarse, sphere)
    check("Re Z vs its plane-wave identity", tm.test_re_z_spectral_identity, sphere)
    check("dZ/dk vs central differences", td.test_dk_matches_central_differences,
          lambda: workloads.icosphere(1, 0.5), 2 * math.pi * 0.4)
    return failed


def test_unchanged_oracle_passes_every_pin():
    assert _pins(stop_at_first=False) == []


@pytest.mark.parametrize("slip,fname,old,new", PLANTS, ids=[p[0] for p in PLANTS])
def test_planted_mistake_fails_a_pin(tmp_path, monkeypatch, slip, fname, old, new):
    src = open(obuild.SRC).read()
    a, b = _scope(src, fname)
    body = src[a:b]
    assert body.count(old) == 1, (fname, old)
    (tmp_path / "planted.c").write_text(src[:a] + body.replace(old, new) + src[b:])
    lib = efie.load(obuild.compile_source(str(tmp_path / "planted.c"), str(tmp_path / "libplanted.so")))
    monkeypatch.setattr(efie, "_lib", lib)
    assert _pins(), slip


# (slip, function of oracle/cm.py it goes into, text there, planted text)
CM_PLANTS = [
    ("resistance taken as +Re Z", "cm_values", "R = -Z.real", "R = Z.real"),
    ("pencil inverted (mu returned as lambda)", "cm_values", "lam = 1.0 / mu[idx]", "lam = mu[idx]"),
    ("values farthest from zero selected", "cm_values", "np.argsort(-np.abs(mu))[:nev]", "np.argsort(np.abs(mu))[:nev]"),
    ("R factored as U D instead of U D^1/2", "cm_values_symmetric",
     "np.sqrt(np.clip(d, 0.0, None))", "np.clip(d, 0.0, None)"),
    ("X^-1 dropped from the reduction", "cm_values_symmetric",
     "M = U.T @ scipy.linalg.lu_solve(lu, U, check_finite=False)", "M = U.T @ U"),
    ("slope: wrong sign of lambda R'", "cm_derivatives", "- lam[m] * (v @ (Rd @ v))", "+ lam[m] * (v @ (Rd @ v))"),
    ("slope: normalised by J^T X J", "cm_derivatives", "/ (v @ (R @ v))", "/ (v @ (X @ v))"),
    ("slope: real part of dZ/dk as X'", "cm_derivatives", "Xd = dZ.imag", "Xd = dZ.real"),
]


def _py_scope(src, fname):
    m = re.search(r"^def %s\(" % fname, src, re.M)
    assert m, fname
    nxt = re.search(r"^def ", src[m.end():], re.M)
    return m.start(), (m.end() + nxt.start()) if nxt else len(src)


def _cm_pins(stop_at_first=True):
    from oracle import cm  # noqa: F401  (the pins look their functions up on the module)
    failed = []

    def check(name, fn, *args):
        if failed and stop_at_first:
            return
        try:
            fn(*args)
        except Exception:
            failed.append(name)

    v, t = workloads.icosphere(2, 0.5)
    P = efie.Problem(v, t, 2 * math.pi)
    sphere = (P, P.dense())
    check("symmetric reduction on a random semidefinite pencil", tm.test_symmetric_reduction_random_semidefinite_pencil)
    check("sphere characteristic values vs the closed form", tm.test_sphere_cm_values_coarse, sphere)
    check("symmetric reduction equals the QZ route", tm.test_symmetric_reduction_equals_qz, sphere)
    check("sphere slopes vs the closed form", td.test_sphere_dlambda_dk_against_closed_form,
          2, (0.05, 0.03, 0.16), "dense")
    return failed


def test_unchanged_eigen_oracle_passes_every_pin():
    assert _cm_pins(stop_at_first=False) == []


@pytest.mark.parametrize("slip,fname,old,new", CM_PLANTS, ids=[p[0] for p in CM_PLANTS])
def test_planted_eigen_mistake_fails_a_pin(tmp_path, monkeypatch, slip, fname, old, new):
    from oracle import cm
    src = open(cm.__file__).read()
    a, b = _py_scope(src, fname)
    body = src[a:b]
    assert body.count(old) == 1, (fname, old)
    path = tmp_path / "planted_cm.py"
    path.write_text(src[:a] + body.replace(old, new) + src[b:])
    spec = importlib.util.spec_from_file_location("planted_cm", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    for name in ("cm_values", "cm_values_arnoldi", "cm_values_symmetric", "cm_derivatives"):
        monkeypatch.setattr(cm, name, getattr(mod, name))
    assert _cm_pins(), slip


# (slip, text in oracle/rwg.py's rwg_list, planted text)
RWG_PLANTS = [
    ("edges sorted by the larger vertex first", "np.lexsort((~fwd, hi, lo))", "np.lexsort((~fwd, lo, hi))"),
    ("free vertex taken from the edge itself", "opp = tris[:, [2, 0, 1]]", "opp = tris[:, [1, 2, 0]]"),
    ("T+ and T- swapped (free vertices not)", "tp, tm = tid[two], tid[two + 1]", "tp, tm = tid[two + 1], tid[two]"),
    ("edges that share their smaller vertex merged", "(lo[1:] != lo[:-1]) | (hi[1:] != hi[:-1])", "(lo[1:] != lo[:-1])"),
    ("edge length halved", "axis=1)\n    return", "axis=1) / 2\n    return"),
]


def _rwg_pins():
    failed = []

    def check(name, fn, *args):
        if failed:
            return
        try:
            fn(*args)
        except Exception:
            failed.append(name)

    check("counts", tm.test_rwg_counts, lambda: workloads.icosphere(3, 1.0), 1920)
    check("canonical order and orientation", tm.test_rwg_canonical_order_and_orientation)
    check("RWG identities", tm.test_rwg_normal_continuity_and_divergence, lambda: workloads.icosphere(2, 0.5))
    check("the library's own list", th.test_rwg_list_matches_oracle, "sphere-r0.5m-ico3")
    return failed


@pytest.mark.parametrize("slip,old,new", RWG_PLANTS, ids=[p[0] for p in RWG_PLANTS])
def test_planted_rwg_mistake_fails_a_pin(tmp_path, monkeypatch, slip, old, new):
    from oracle import rwg
    src = open(rwg.__file__).read()
    assert src.count(old) == 1, old
    path = tmp_path / "planted_rwg.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("planted_rwg", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    for m in (rwg, tm, th, efie):
        monkeypatch.setattr(m, "rwg_list", mod.rwg_list)
    assert _rwg_pins(), slip


def test_unchanged_rwg_list_passes_every_pin():
    assert _rwg_pins() == []
