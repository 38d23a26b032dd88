"""Batched problems: running independent problems of different sizes concurrently (one
stream each) gives the same MAP points, eigenpairs and Hessian actions as running them
one at a time, and the Hessian actions match the oracle."""
import numpy as np
import pytest

import workloads as W
from oracle.inverse import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _make(ws):
    from paper_1909_03948_gb300 import Problem
    out = []
    for w in ws:
        orc, m_true, _ = make_problem(w, W.draws(w))
        out.append((orc, Problem(2, w.N, w.gamma, w.delta, orc.sigma, orc.obs_xyz, d_obs=orc.d_obs, rtol=1e-10)))
    return out


def test_batch_matches_one_at_a_time():
    from paper_1909_03948_gb300 import Batch
    ws = [W.Workload(f"b{i}", 2, N, q, g, d, 6, 4, seed=W.SEED_BASE + 400 + i)
          for i, (N, q, g, d) in enumerate([(32, 30, 0.1, 0.5), (64, 60, 0.07, 0.8), (96, 40, 0.15, 0.3)])]
    pairs_a, pairs_b = _make(ws), _make(ws)
    Om = [torch.tensor(np.ascontiguousarray(W.omega(w).T), device=DEV) for w in ws]
    B = Batch([p for _, p in pairs_a], nthreads=3)
    ms, lams, Vs, nst = B.map_and_eig([p.zeros() for _, p in pairs_a], 6, 4, Om)
    B.set_point(ms)
    Ys = B.hessian_apply(Om)
    B.close()
    for i, ((orc, P), w) in enumerate(zip(pairs_b, ws)):
        m, st = P.newton_cg_map()
        lam, V, _ = P.lowrank_eig(m, 6, 4, Om[i])
        P.set_point(m)
        Y, _ = P.hessian_apply(Om[i])
        assert nst[i]["iterations"] == st["iterations"]
        assert torch.allclose(ms[i], m, rtol=1e-12, atol=1e-14)
        assert torch.allclose(lams[i], lam, rtol=1e-12)
        assert torch.allclose(Ys[i], Y, rtol=1e-12, atol=1e-14 * float(Y.abs().max()))
        # and against the oracle at the batched MAP point
        mm = ms[i].cpu().numpy()
        ref = orc.hessian_misfit(mm, orc.forward(mm), W.omega(w))
        got = Ys[i].cpu().numpy().T
        assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref)
    for _, p in pairs_a + pairs_b:
        p.close()
