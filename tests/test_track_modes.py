"""cm_track_modes (following characteristic modes over frequency, Section
V's sweeps), on CPU with synthetic modes whose correct pairing is known:
orthonormal currents, values in clusters, the second set permuted, mixed by
a random rotation inside each cluster (as an eigensolver may return any
basis of a degenerate subspace), slightly perturbed, with one mode that has
no counterpart."""
import numpy as np

from paper_1412_1756_gb300 import mlfma as M


def _sets(seed=0):
    rng = np.random.default_rng(seed)
    n = 300
    Q, _ = np.linalg.qr(rng.standard_normal((n, 9)))
    lam_a = np.array([-1.0, -1.00005, -1.00008, 0.5, 0.50001, 2.0, 3.1, 0.9])
    Ja = Q[:, :8]
    # set b: clusters rotated inside, values moved a little, order shuffled;
    # mode 7 of set a (0.9) is gone and a new one (Q[:, 8]) appears
    Jb = Ja.copy()
    for cl in ([0, 1, 2], [3, 4]):
        R, _ = np.linalg.qr(rng.standard_normal((len(cl), len(cl))))
        Jb[:, cl] = Ja[:, cl] @ R
    Jb[:, 7] = Q[:, 8]
    lam_b = lam_a * 1.001 + np.array([0, 1e-6, 2e-6, 0, 1e-6, 0, 0, 0])
    lam_b[7] = 7.5
    Jb = Jb + 1e-3 * rng.standard_normal(Jb.shape)
    perm = rng.permutation(8)
    return lam_a, Ja, lam_b[perm], Jb[:, perm] * rng.uniform(0.5, 2.0, 8), perm


def test_clusters_and_single_modes_are_paired():
    lam_a, Ja, lam_b, Jb, perm = _sets()
    match, ov = M.track_modes(lam_a, Ja, lam_b, Jb, cluster_tol=1e-3)
    cluster_of = {0: 0, 1: 0, 2: 0, 3: 1, 4: 1, 5: 2, 6: 3, 7: 4}
    for j, src in enumerate(perm):
        if src == 7:          # the new mode: nothing to continue
            assert match[j] == -1 and ov[j] == 0.0
            continue
        assert match[j] >= 0
        assert cluster_of[match[j]] == cluster_of[src], (j, src, match[j])
        assert ov[j] > 0.99
        if src in (5, 6):     # single modes: exact pairing
            assert match[j] == src
    # every mode of set a is used at most once
    used = match[match >= 0]
    assert len(set(used.tolist())) == len(used)


def test_bad_arguments():
    import pytest
    lam_a, Ja, lam_b, Jb, _ = _sets()
    with pytest.raises(M.MlfmaError):
        M.track_modes(lam_a, Ja, lam_b, Jb, cluster_tol=-1.0)
    with pytest.raises(ValueError):
        M.track_modes(lam_a, Ja[:, :3], lam_b, Jb)
