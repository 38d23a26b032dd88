"""The kernel replay used for the roofline: it times the last FP32 block solve's
level-0 launches on their live workspace (stream launches and a captured CUDA graph,
row and TMA-tiled kernels) without changing the solver's results, and it refuses to
run before such a solve exists."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_replay_times_kernels_and_keeps_results():
    from paper_1909_03948_gb300 import Problem, HPError
    w = W.make_workload(2, 64, 50, seed=31)
    dr = W.draws(w)
    P = Problem(2, 64, w.gamma, w.delta, 0.01, dr.obs_xyz, rtol=1e-8)
    flush = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with pytest.raises(HPError):
        P.replay_kernel("smooth", 3, flush)              # no point, no solve yet
    with pytest.raises(HPError):
        P.replay_kernel_graph("smooth", 3)
    P.set_point(torch.zeros(P.n, dtype=torch.float64, device="cuda"))
    X = torch.tensor(np.random.default_rng(1).standard_normal((8, P.n)), device="cuda")
    Y0, _ = P.hessian_apply(X)
    for fam in P.REPLAY_FAMILIES:
        warm, cold = P.replay_kernel(fam, 10, flush)
        assert 0.0 < warm < 1e4 and cold is not None and 0.0 < cold < 1e4, (fam, warm, cold)
        warm2, none = P.replay_kernel(fam, 10)
        assert warm2 > 0.0 and none is None
        for tt in (0, 1):                                 # row and TMA-tiled kernels in a graph
            P.set_tuning(tma_tiles=tt)
            g = P.replay_kernel_graph(fam, 20)
            assert 0.0 < g < 1e4, (fam, tt, g)
        P.set_tuning()
    Y1, _ = P.hessian_apply(X)
    assert torch.equal(Y0, Y1)
    with pytest.raises(ValueError):
        P.replay_kernel("matvec", 3)
    P.close()
