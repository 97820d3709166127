"""Frequency sweeps on one mesh (mlfma_set_*): one plan per wavenumber,
admitted to the device by an estimate of its memory, the products of a wave
as parallel branches of one CUDA graph.  Each wavenumber's result must be
bit-identical to a standalone plan's (same kernels, same tables, no
atomics), whatever the admission waves; the plan of each wavenumber must
match the dense oracle at that wavenumber."""
import numpy as np
import pytest

import workloads
from oracle import efie

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1412_1756_gb300 import mlfma as M  # noqa: E402

KS = 2 * np.pi * np.array([0.9, 1.0, 1.1])


def mesh():
    return workloads.icosphere(3, 0.5)


def gpu(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


_standalone = {}


def standalone(f, x, dt):
    if f not in _standalone:
        v, t = mesh()
        _standalone[f] = M.MlfmaPlan(v, t, KS[f], 3, 3.0, max_batch=8)
    return _standalone[f].matvec(gpu(x, dt)).cpu().numpy()


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_one_wave_matches_standalone_plans(dt):
    v, t = mesh()
    S = M.MlfmaPlanSet(v, t, KS, 3, 3.0, max_batch=8)
    assert S.info()["waves"] == 1
    x = np.stack([workloads.rhs(S.n, 4, 100 + f) for f in range(len(KS))])
    y = S.matvec(gpu(x, dt)).cpu().numpy()
    for f in range(len(KS)):
        assert np.array_equal(y[f], standalone(f, x[f], dt))
    y2 = S.matvec(gpu(x, dt)).cpu().numpy()      # the captured graph replayed
    assert np.array_equal(y, y2)
    ys = S.matvec(gpu(x[1], dt)).cpu().numpy()   # one block shared by every wavenumber
    assert np.array_equal(ys[1], y[1])
    assert np.array_equal(S.plan(2).matvec(gpu(x[2], dt)).cpu().numpy(), y[2])
    S.close()


def test_each_plan_has_its_own_wavenumber():
    v, t = mesh()
    S = M.MlfmaPlanSet(v, t, KS[[0, 2]], 3, 3.0, max_batch=8)
    x = workloads.rhs(S.n, 2, 7)
    y = S.matvec(gpu(x, torch.float64)).cpu().numpy()
    for i, k in enumerate(KS[[0, 2]]):
        ref = efie.Problem(v, t, k).dense() @ x
        assert np.linalg.norm(y[i] - ref) / np.linalg.norm(ref) < 1e-3
    S.close()


def test_small_budget_runs_in_waves():
    v, t = mesh()
    S = M.MlfmaPlanSet(v, t, KS, 3, 3.0, max_batch=8)
    est = S.info()["est_bytes"]
    S.close()
    S = M.MlfmaPlanSet(v, t, KS, 3, 3.0, max_batch=8, budget_bytes=max(est) + 1)
    inf = S.info()
    assert inf["waves"] == 3 and inf["wave_of"] == [0, 1, 2]
    assert inf["device_bytes"][0] > 0 and inf["device_bytes"][1] == 0
    for f, d in enumerate(inf["device_bytes"][:1]):
        assert d <= est[f]          # the estimate bounds what setup allocates
    x = np.stack([workloads.rhs(S.n, 3, 200 + f) for f in range(len(KS))])
    for _ in range(2):
        y = S.matvec(gpu(x, torch.float32)).cpu().numpy()
        for f in range(len(KS)):
            assert np.array_equal(y[f], standalone(f, x[f], torch.float32))
    S.close()


def test_budget_below_one_plan_is_enomem():
    v, t = mesh()
    S = M.MlfmaPlanSet(v, t, KS[:1], 3, 3.0, max_batch=8)
    est = S.info()["est_bytes"][0]
    S.close()
    with pytest.raises(M.MlfmaError) as ei:
        M.MlfmaPlanSet(v, t, KS, 3, 3.0, max_batch=8, budget_bytes=est - 1)
    assert ei.value.status == 2
