"""The host Rayleigh-Ritz step of the block characteristic-mode solver
(cm_rayleigh_ritz), on CPU: Ritz pairs of T = X^-1 R on span Y in the R inner
product, from Y, R Y and W = T Y.  Checked against scipy's generalized
symmetric eigensolver of the projected pencil, the exact pairs of an
invariant subspace, the interlacing bound (no Ritz |mu| above the pencil's
largest, with X indefinite), and the dropped directions (a repeated basis
column, a direction without R energy)."""
import numpy as np
import pytest
import scipy.linalg

from paper_1412_1756_gb300 import mlfma as M


def pencil(n, seed, null=0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    X = A + A.T                # symmetric, indefinite
    Bf = rng.standard_normal((n, n - null))
    R = Bf @ Bf.T / n          # positive semidefinite, rank n - null
    return X, R, rng


def ritz_inputs(X, R, Y):
    RY = R @ Y
    return Y, RY, np.linalg.solve(X, RY)


def test_matches_projected_generalized_eigh():
    X, R, rng = pencil(120, 1)
    Y, RY, W = ritz_inputs(X, R, rng.standard_normal((120, 12)))
    mu, coef = M.rayleigh_ritz(Y, RY, W)
    A, B = RY.T @ W, Y.T @ RY
    A = 0.5 * (A + A.T)
    ref = scipy.linalg.eigh(A, B, eigvals_only=True)
    ref = ref[np.argsort(-np.abs(ref))]
    assert mu.shape == (12,) and coef.shape == (12, 12)
    assert np.allclose(mu, ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())
    assert np.all(np.diff(np.abs(mu)) <= 0)
    assert np.allclose(coef.T @ B @ coef, np.eye(12), atol=1e-9)                 # B-orthonormal
    assert np.allclose(A @ coef, B @ coef * mu, atol=1e-9 * np.abs(A).max())


def test_invariant_subspace_gives_exact_pairs():
    X, R, rng = pencil(80, 2)
    lam, V = scipy.linalg.eig(X, R)
    lam, V = lam.real, V.real
    pick = np.argsort(np.abs(lam))[:6]                  # values nearest zero: largest |mu|
    Y, RY, W = ritz_inputs(X, R, V[:, pick] @ rng.standard_normal((6, 6)))
    mu, coef = M.rayleigh_ritz(Y, RY, W)
    want = 1.0 / lam[pick]
    assert np.allclose(mu, want[np.argsort(-np.abs(want))], rtol=1e-8)
    Z = Y @ coef
    assert np.abs(X @ Z - (R @ Z) / mu).max() < 1e-7 * np.abs(X @ Z).max()


@pytest.mark.parametrize("seed", range(5))
def test_ritz_values_never_exceed_the_largest_mu(seed):
    """Interlacing: with X indefinite, no Ritz |mu| (1 / |lambda|) exceeds
    the pencil's largest, so no spurious value nearer zero than the true
    nearest can appear."""
    X, R, rng = pencil(90, 10 + seed)
    mu_true = np.linalg.eigvals(np.linalg.solve(X, R)).real
    Y, RY, W = ritz_inputs(X, R, rng.standard_normal((90, 10)))
    mu, _ = M.rayleigh_ritz(Y, RY, W)
    assert np.abs(mu).max() <= np.abs(mu_true).max() * (1 + 1e-9)


def test_rank_loss_and_null_energy_are_dropped():
    X, R, rng = pencil(60, 3)
    Y0 = rng.standard_normal((60, 5))
    Y, RY, W = ritz_inputs(X, R, np.concatenate([Y0, Y0[:, :1]], axis=1))   # a repeated column: rank 5
    mu, coef = M.rayleigh_ritz(Y, RY, W)
    assert mu.shape == (5,)
    Yr, RYr, Wr = ritz_inputs(X, R, Y0)
    ref = scipy.linalg.eigh(0.5 * (RYr.T @ Wr + Wr.T @ RYr), Yr.T @ RYr, eigvals_only=True)
    assert np.allclose(mu, ref[np.argsort(-np.abs(ref))], rtol=1e-8)
    # a basis direction in the null space of R carries no R energy: dropped
    X2, R2, rng = pencil(60, 4, null=1)
    nul = scipy.linalg.null_space(R2)[:, 0]
    Y2, RY2, W2 = ritz_inputs(X2, R2, np.concatenate([rng.standard_normal((60, 4)), nul[:, None]], axis=1))
    mu2, _ = M.rayleigh_ritz(Y2, RY2, W2)
    assert mu2.shape == (4,) and np.all(np.isfinite(mu2))


def test_bad_arguments():
    with pytest.raises(ValueError):
        M.rayleigh_ritz(np.zeros((5, 2)), np.zeros((5, 3)), np.zeros((5, 2)))


def test_degenerate_cluster_is_returned_whole():
    """A 5-fold and a 3-fold eigenvalue of the pencil (the shape of the
    sphere's clusters): a basis of their joint invariant subspace gives both
    values with their multiplicities, and R-orthonormal Ritz vectors."""
    rng = np.random.default_rng(9)
    n = 50
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([[0.056] * 5, [-0.077] * 3, rng.uniform(0.5, 3.0, n - 8) * rng.choice([-1, 1], n - 8)])
    d = rng.uniform(0.5, 2.0, n)                       # R = Q diag(d) Q^T, X = Q diag(lam d) Q^T
    R = (Q * d) @ Q.T
    X = (Q * (lam * d)) @ Q.T
    Y, RY, W = ritz_inputs(X, R, Q[:, :8] @ rng.standard_normal((8, 8)))
    mu, coef = M.rayleigh_ritz(Y, RY, W)
    assert np.allclose(np.sort(1.0 / mu), np.sort(lam[:8]), rtol=1e-9)
    Z = Y @ coef
    assert np.allclose(Z.T @ R @ Z, np.eye(8), atol=1e-9)
