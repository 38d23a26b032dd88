"""The learned warm start on the GPU: the recorder writes the solves it sees in the
network's scaling, a useless guess falls back to the zero start (results unchanged
bit for bit), and a network trained on the method's own solves guesses held-out
solves well below the zero start's relative residual while the Hessian actions stay
within the solve tolerance (relative 1e-8 per solve; 1e-6 on the Hessian action)."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda"


def _problem(N, nobs=100, seed=21):
    from paper_1909_03948_gb300 import Problem
    w = W.make_workload(2, N, nobs, seed=seed)
    dr = W.draws(w)
    return Problem(2, N, w.gamma, w.delta, 0.01, dr.obs_xyz, rtol=1e-8)


def test_recorder_writes_inputs_and_loss_data():
    """Recorded samples against the oracle's assembled P1 stiffness for the same m."""
    from oracle import unet as OU
    from oracle.fem import Mesh
    from paper_1909_03948_gb300.warmstart import prior_draws
    N = 24
    P = _problem(N)
    H, Wd = P.warmstart_grid()
    assert (H, Wd) == (32, 32)
    m = prior_draws(P, 1, seed=3)[0].contiguous()
    P.set_point(m)
    X = torch.zeros((4, 3, H, Wd), device=DEV)
    A = torch.zeros((4, 4, H, Wd), device=DEV)
    T = torch.zeros((4, 1, H, Wd), device=DEV)
    P.warmstart_record(X, A, T)
    B = torch.tensor(np.random.default_rng(4).standard_normal((2, P.n)), device=DEV)
    Y, st = P.state_solve(B)
    P.warmstart_record()
    assert P.warmstart_counts()["recorded"] == 2
    np1 = N + 1
    mesh = Mesh(2, N)
    mh = m.cpu().numpy()
    K = mesh.stiffness(mesh.elem_mean(np.exp(mh)))
    ch = OU.stencil_channels(K, np1, np1, np1)
    free = (~mesh.dirichlet_mask).reshape(np1, np1)
    pair_x = free & np.roll(free, -1, axis=1)
    pair_x[:, -1] = False
    pair_y = free & np.roll(free, -1, axis=0)
    pair_y[-1, :] = False
    grid = lambda v: v.reshape(np1, np1).cpu().numpy()            # row iy, column ix
    nfree = free.sum()
    close = lambda a, b: np.allclose(a, b, rtol=2e-6, atol=1e-6 * np.abs(b).max())
    for j in range(2):
        b = grid(B[j]) * free
        z = np.where(free, b / ch[0], 0.0)
        c = np.linalg.norm(z) / np.sqrt(nfree)
        Xj, Aj = X[j].cpu().numpy(), A[j].cpu().numpy()
        assert np.array_equal(Xj[0, :np1, :np1], grid(m).astype(np.float32))
        assert close(Xj[1, :np1, :np1], z / c)
        assert np.array_equal(Xj[2, :np1, :np1], free.astype(np.float32))
        assert close(Aj[0, :np1, :np1], b / c)
        assert close(Aj[1, :np1, :np1][free], ch[0][free])
        assert close(Aj[2, :np1, :np1] * pair_x, ch[1] * pair_x)
        assert close(Aj[3, :np1, :np1] * pair_y, ch[2] * pair_y)
        assert not Xj[:, np1:, :].any() and not Xj[:, :, np1:].any() and not Aj[:, np1:, :].any()
        assert close(T[j, 0, :np1, :np1].cpu().numpy(), grid(Y[j]) * free / c)
    # the recorded exact solution has (almost) zero relative residual under the oracle's loss
    L, _ = OU.residual_loss(T[:2].cpu().numpy().astype(np.float64), X[:2].cpu().numpy().astype(np.float64),
                            A[:2].cpu().numpy().astype(np.float64))
    assert L < 1e-7
    P.close()


def test_useless_guess_falls_back_to_zero_start():
    from paper_1909_03948_gb300 import UNet
    from paper_1909_03948_gb300.warmstart import prior_draws
    P = _problem(32)
    # solves with a learned guess refine with FP64 instructions; the zero start does the same
    # here (refine_df 0), so that the two must agree bit for bit
    P.set_tuning(refine_df=0)
    H, Wd = P.warmstart_grid()
    m = prior_draws(P, 1, seed=5)[0].contiguous()
    D = torch.tensor(np.random.default_rng(6).standard_normal((5, P.n)), device=DEV)
    P.set_point(m)
    Y0, st0 = P.hessian_apply(D)
    net = UNet(H, Wd, batch_cap=4)
    net.set_params(np.zeros(net.nparam, dtype=np.float32))       # guess = 0: residual = |b|
    P.warmstart_attach(net)
    Y1, st1 = P.hessian_apply(D)
    c = P.warmstart_counts()
    assert c["guesses"] == 10 and c["fallbacks"] == 10
    assert torch.equal(Y0, Y1) and st0["iterations"] == st1["iterations"]
    P.warmstart_attach(None)
    P.close()


def test_trained_network_guesses_held_out_solves():
    """Train on the method's own solves at 40 prior draws, then check the network on
    held-out ones: (1) under the oracle's relative-residual loss its guesses for solves at
    other prior draws and other directions have relative residual well below 1 (the zero
    start has exactly 1); (2) attached to the solver it is tried in every stiffness solve,
    never falls back, and the Hessian actions equal the zero-start ones within 1e-6.
    The PCG iterations with and without it are printed for damped-Jacobi (nu 2, omega 0.8)
    and the default Chebyshev smoothing: the geometric multigrid converges so fast that a
    guess with relative residual ~0.1 saves at most about one iteration of a solve, and
    with the Chebyshev V-cycle none (a few more), so the zero start stays the default and the
    iteration difference is only bounded (two per held-out point either way)."""
    from oracle import unet as OU
    from paper_1909_03948_gb300.warmstart import generate, prior_draws, train
    P = _problem(64, nobs=200)
    m_train = prior_draws(P, 40, seed=101)
    X, A = generate(P, m_train, ncols=16, seed=202)
    assert X.shape[0] == 40 * 33
    net, losses = train(X, A, epochs=30, batch=16, lr=1e-3, seed=3)
    assert np.all(np.isfinite(losses)) and losses[-1] < 0.5 * losses[0], losses
    m_test = prior_draws(P, 6, seed=303)                          # held out: other prior draws
    Xt, At = generate(P, m_test[:2], ncols=4, seed=606)           # ... and other directions
    rel_res = []
    for j in range(Xt.shape[0]):
        y = net.forward(Xt[j:j + 1].contiguous())
        L, _ = OU.residual_loss(y.cpu().numpy().astype(np.float64), Xt[j:j + 1].cpu().numpy().astype(np.float64),
                                At[j:j + 1].cpu().numpy().astype(np.float64))
        rel_res.append(np.sqrt(2.0 * L))
    rel_res = np.array(rel_res)
    assert np.all(rel_res < 1.0) and np.median(rel_res) < 0.3, rel_res
    D = torch.tensor(np.random.default_rng(404).standard_normal((16, P.n)), device=DEV)
    P.warmstart_attach(net)
    c0 = P.warmstart_counts()
    report = {}
    for name, tune in (("jacobi", dict(nu=2, omega=0.8, smoother=0)), ("chebyshev", {})):
        P.set_tuning(**tune)
        its = {False: 0, True: 0}
        for i in range(m_test.shape[0]):
            Y = {}
            for on in (False, True):
                P.warmstart_enable(on)
                P.set_point(m_test[i].contiguous())
                Y[on], st = P.hessian_apply(D)
                its[on] += st["iterations"]
            rel = float(torch.linalg.norm(Y[True] - Y[False]) / torch.linalg.norm(Y[False]))
            assert rel <= 1e-6, rel
        report[name] = its
    c = P.warmstart_counts()
    print(f"guess relative residual median {np.median(rel_res):.3g} (max {rel_res.max():.3g}); "
          f"PCG iterations (zero start, learned start): damped Jacobi {report['jacobi'][False]}, "
          f"{report['jacobi'][True]}; Chebyshev {report['chebyshev'][False]}, {report['chebyshev'][True]}; "
          f"guesses {c['guesses'] - c0['guesses']}, fallbacks {c['fallbacks'] - c0['fallbacks']}; "
          f"loss {losses[0]:.3g} -> {losses[-1]:.3g}")
    # every stiffness solve with the network on took a guess: per point the 2 Hessian solves of
    # 16 columns (the state at the point was solved just before, with the network off, and
    # set_point at an unchanged point keeps it)
    assert c["guesses"] - c0["guesses"] == 2 * m_test.shape[0] * (2 * 16)
    assert c["fallbacks"] == c0["fallbacks"]
    for name in report:  # a sanity bound: a broken guess path would cost many more
        assert abs(report[name][True] - report[name][False]) <= 2 * m_test.shape[0], report
    P.set_tuning()
    P.warmstart_attach(None)
    P.close()
