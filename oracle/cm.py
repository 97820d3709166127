"""Dense characteristic-mode eigensolve.  Test infrastructure.

Section II, Eq. (GEP): X J_n = lambda_n R J_n with Z = R + iX (Eq. (6)).
Sign reading: taken literally with exp(ikR)/R and the prefactor +ik eta,
Re Z is negative semidefinite and the literal pencil gives characteristic
values of the opposite sign to Table I and to the physical reading of
Section II (lambda < 0 stores electric energy).  This oracle therefore
uses R := -Re Z (positive semidefinite) and X := +Im Z.  Characteristic
values do not depend on the overall scale of Z.

Solved as the pencil (R, X): R J = mu X J, mu = 1 / lambda, so the values
nearest zero are those with the largest |mu| (the same selection the paper
makes with IRA on Eq. (SEP)).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def cm_values(Z: np.ndarray, nev: int = 10) -> np.ndarray:
    """The nev characteristic values nearest zero, sorted by magnitude."""
    R = -Z.real
    X = Z.imag
    mu = scipy.linalg.eigvals(R, X)
    mu = mu[np.isfinite(mu)]
    idx = np.argsort(-np.abs(mu))[:nev]
    lam = 1.0 / mu[idx]
    return lam.real[np.argsort(np.abs(lam.real))]


def cm_values_arnoldi(Z: np.ndarray, nev: int = 10, seed: int = 0) -> np.ndarray:
    """Same selection as ``cm_values`` through a dense LU of X and Arnoldi
    iteration (ARPACK, as in Section IV) on X^-1 R, largest |1/lambda|."""
    import scipy.sparse.linalg as sla

    R = -Z.real
    X = Z.imag
    lu = scipy.linalg.lu_factor(X)
    n = Z.shape[0]
    op = sla.LinearOperator((n, n), matvec=lambda v: scipy.linalg.lu_solve(lu, R @ v), dtype=np.float64)
    v0 = np.random.Generator(np.random.PCG64(seed)).standard_normal(n)
    mu = sla.eigs(op, k=nev, which="LM", v0=v0, ncv=max(2 * nev + 1, 40), tol=1e-12,
                  return_eigenvectors=False)
    lam = (1.0 / mu).real
    return lam[np.argsort(np.abs(lam))]


def cm_values_symmetric(R: np.ndarray, X: np.ndarray, nev: int = 10, overwrite: bool = False) -> np.ndarray:
    """Same selection as ``cm_values`` for large N, by reducing the pencil of
    Eq. (GEP) to one dense symmetric eigenproblem (no iteration).

    R is symmetric positive semidefinite, so R = L L^T with L = U D^1/2 from
    its eigendecomposition R = U D U^T (rounding-level negative D taken as
    0).  For mu != 0, X^-1 R J = mu J holds exactly when L^T X^-1 L u = mu u
    with u = L^T J / mu: the nonzero eigenvalues mu = 1 / lambda of X^-1 R
    are those of the symmetric matrix M = L^T X^-1 L, and the zero ones
    (the null space of R, lambda infinite) are not wanted.  Returns the nev
    values nearest zero (largest |mu|), sorted by magnitude.  With
    overwrite, R and X are used as work space."""
    d, U = scipy.linalg.eigh(R, overwrite_a=overwrite, check_finite=False)
    del R
    U *= np.sqrt(np.clip(d, 0.0, None))[None, :]            # L, in place
    lu = scipy.linalg.lu_factor(X, overwrite_a=overwrite, check_finite=False)
    del X
    M = U.T @ scipy.linalg.lu_solve(lu, U, check_finite=False)
    del lu, U
    M = 0.5 * (M + M.T)
    mu = scipy.linalg.eigh(M, eigvals_only=True, overwrite_a=True, check_finite=False)
    mu = mu[np.argsort(-np.abs(mu))[:nev]]
    lam = 1.0 / mu
    return lam[np.argsort(np.abs(lam))]


def cm_derivatives(Z: np.ndarray, dZ: np.ndarray, nev: int = 10, method: str = "dense", seed: int = 0):
    """Characteristic values nearest zero and their wavenumber derivatives.

    First-order perturbation of the pencil of Eq. (GEP), X J = lambda R J,
    with R = -Re Z and X = Im Z: for an eigenpair (lambda, J),
    d lambda / dk = J^T (X' - lambda R') J / (J^T R J), where R' = -Re dZ/dk
    and X' = Im dZ/dk.  The eigenpairs come from the dense pencil (method
    "dense") or, with the same selection, from Arnoldi iteration on X^-1 R
    as in ``cm_values_arnoldi`` ("arnoldi"; eigenvectors rotated to real).
    Returns (lambda, dlambda) sorted by |lambda|."""
    R = -Z.real
    X = Z.imag
    Rd = -dZ.real
    Xd = dZ.imag
    if method == "dense":
        mu, J = scipy.linalg.eig(R, X)
        ok = np.isfinite(mu)
        mu, J = mu[ok], J[:, ok]
        idx = np.argsort(-np.abs(mu))[:nev]
        mu, J = mu[idx], J[:, idx]
    else:
        import scipy.sparse.linalg as sla
        lu = scipy.linalg.lu_factor(X)
        n = Z.shape[0]
        op = sla.LinearOperator((n, n), matvec=lambda v: scipy.linalg.lu_solve(lu, R @ v), dtype=np.float64)
        v0 = np.random.Generator(np.random.PCG64(seed)).standard_normal(n)
        mu, J = sla.eigs(op, k=nev, which="LM", v0=v0, ncv=max(2 * nev + 1, 40), tol=1e-12)
        piv = np.argmax(np.abs(J), axis=0)
        J = J * np.exp(-1j * np.angle(J[piv, np.arange(J.shape[1])]))
    lam = (1.0 / mu).real
    J = J.real
    dl = np.empty(len(lam))
    for m in range(len(lam)):
        v = J[:, m]
        dl[m] = (v @ (Xd @ v) - lam[m] * (v @ (Rd @ v))) / (v @ (R @ v))
    order = np.argsort(np.abs(lam))
    return lam[order], dl[order]
