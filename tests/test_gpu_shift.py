"""GPU tests of the learned diagonal shift: the feature kernel, the MLP's forward,
gradient and Adam kernels against the FP64 oracle (oracle/shift.py), the shift-doubling
retry against the oracle's rule and factorization, and the gain of the trained network
over the plain retry on held-out elasticity matrices."""
import numpy as np
import pytest

import synth
from oracle import shift as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ick():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_05871_gb300.build import build
    build()
    import paper_1601_05871_gb300 as m
    m.load()
    return m


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dtype is None else t.to(dtype)).cuda()


def _elasticity(ne, nu, ick, k=0, dtype=0, exact=0, block_rows=256):
    p = synth.elasticity3d_q1(ne, nu=nu)
    perm, ranges = ick.ic_nd_grid(*p.grid, 3, block_rows, p.keep)
    h = ick.ic_symbolic(p.rowptr, p.colind, k, perm, ranges, block_rows=block_rows, dtype=dtype, exact=exact)
    return p, perm, h


def test_features_match_oracle(ick):
    cases = [(synth.elasticity3d_q1(5, nu=0.47), 0, 0.47), (synth.laplace3d_27pt(10), 2, 0.0),
             (synth.poisson2d_5pt(13, 9), 1, 0.0), (synth.random_spd(300, 0.05, seed=4), 1, 0.0),
             (synth.diffusion3d_7pt(9, seed=3), 1, 0.0)]
    for p, k, nu in cases:
        h = ick.ic_symbolic(p.rowptr, p.colind, k, block_rows=512)
        f = ick.ic_shift_features(h, dev(p.vals), nu)
        fo = S.features(p.n, p.rowptr, p.colind, p.vals, k, nu)
        assert np.allclose(f, fo, rtol=1e-12, atol=0), (p.name if hasattr(p, "name") else p.n, f, fo)


def test_features_reject_bad_diagonal(ick):
    p = synth.poisson2d_5pt(6, 6)
    v = p.vals.copy()
    diag = [e for i in range(p.n) for e in range(p.rowptr[i], p.rowptr[i + 1]) if p.colind[e] == i]
    v[diag[7]] = -1.0
    h = ick.ic_symbolic(p.rowptr, p.colind, 0)
    with pytest.raises(ick.IckError):
        ick.ic_shift_features(h, dev(v))


def _net(seed, n=300):
    rng = np.random.default_rng(seed)
    theta = synth.mlp_init(32, seed)
    theta[S.NFEAT * 32:S.NFEAT * 32 + 32] += rng.normal(0, 0.2, 32)
    X = rng.normal(0, 1, (n, S.NFEAT)) * rng.uniform(0.1, 3, S.NFEAT) + rng.normal(0, 2, S.NFEAT)
    t = rng.normal(-1.5, 1, n)
    return theta.astype(np.float32), X.astype(np.float32), t.astype(np.float32), X.mean(0).astype(np.float32), \
        (X.std(0) + 0.1).astype(np.float32)


def test_mlp_forward_matches_oracle(ick):
    import torch
    theta, X, t, mean, std = _net(1, 1000)
    m = ick.Mlp(theta)
    ick.ic_mlp_set_scaling(m, mean, std)
    y = torch.empty(len(X), dtype=torch.float32, device="cuda")
    ick.ic_mlp_forward(m, dev(X), y)
    yo, _ = S.forward(theta.astype(np.float64), 32, mean.astype(np.float64), std.astype(np.float64), X)
    assert np.abs(y.cpu().numpy() - yo).max() <= 1e-5 * max(1.0, np.abs(yo).max())
    assert np.array_equal(ick.ic_mlp_get_params(m), theta)


def test_mlp_forward_hand_derived_golden(ick):
    """The hand-derived 2-unit network of tests/golden/mlp_forward_h2.txt, embedded in
    the library's 32-unit layout with zero extra units: every value is a short dyadic
    fraction, so the FP32 kernel must give the derived outputs exactly."""
    import torch
    from test_shift_oracle import pad_network, read_mlp_golden
    H, theta, mean, std, X, y = read_mlp_golden()
    m = ick.Mlp(pad_network(theta, H, 32).astype(np.float32))
    ick.ic_mlp_set_scaling(m, mean.astype(np.float32), std.astype(np.float32))
    out = torch.empty(len(X), dtype=torch.float32, device="cuda")
    ick.ic_mlp_forward(m, dev(X.astype(np.float32)), out)
    assert np.array_equal(out.cpu().numpy(), y.astype(np.float32))


@pytest.mark.parametrize("n", [1, 7, 300, 5000])
def test_mlp_gradient_matches_oracle(ick, n):
    theta, X, t, mean, std = _net(2 + n, n)
    m = ick.Mlp(theta)
    ick.ic_mlp_set_scaling(m, mean, std)
    g, L = ick.ic_mlp_gradient(m, dev(X), dev(t))
    Lo, go = S.loss_and_grad(theta.astype(np.float64), 32, mean.astype(np.float64), std.astype(np.float64), X, t)
    assert abs(L - Lo) <= 1e-5 * Lo
    assert np.abs(g - go).max() <= 1e-5 * np.abs(go).max()
    # the gradient call leaves the parameters alone
    assert np.array_equal(ick.ic_mlp_get_params(m), theta)


def test_adam_trajectory_matches_oracle(ick):
    theta, X, t, mean, std = _net(9, 200)
    m = ick.Mlp(theta)
    ick.ic_mlp_set_scaling(m, mean, std)
    Xd, td = dev(X), dev(t)
    th = theta.astype(np.float64)
    mm = np.zeros_like(th)
    vv = np.zeros_like(th)
    for step in range(1, 21):
        L = ick.ic_mlp_train_step(m, Xd, td, 3e-3)
        Lo, go = S.loss_and_grad(th, 32, mean.astype(np.float64), std.astype(np.float64), X, t)
        assert abs(L - Lo) <= 1e-4 * Lo
        th, mm, vv = S.adam_step(th, go, mm, vv, step, 3e-3)
    assert np.abs(ick.ic_mlp_get_params(m) - th).max() <= 1e-4 * np.abs(th).max()


def test_retry_matches_oracle_decisions(ick, orc):
    """Exact-mode FP64 factors are bit-identical to the oracle's, so the retry makes
    the same breakdown decisions and stops at the same shift."""
    for ne, nu in ((5, 0.48), (6, 0.49), (5, 0.45)):
        p, perm, h = _elasticity(ne, nu, ick, exact=1)
        o = orc.OracleIC.from_problem(p, perm, 0)
        a_o, t_o = S.first_success(lambda a: o.numeric(p.vals, a) != 0, 0.0, 1e-3, 20)
        a, t = ick.ic_numeric_shifted(h, dev(p.vals), 0.0, 1e-3, 20)
        assert t == t_o and a == a_o, (ne, nu, a, t, a_o, t_o)
        assert o.numeric(p.vals, a) == 0
        assert np.array_equal(ick.ic_get_factor(h)[2], o.values())


def test_retry_reports_exhaustion(ick):
    p, perm, h = _elasticity(5, 0.49, ick)
    with pytest.raises(ick.IckError) as e:
        ick.ic_numeric_shifted(h, dev(p.vals), 0.0, 1e-6, 3)
    assert e.value.status == ick.IC_ERR_BREAKDOWN and e.value.attempts == 3


NUS_TRAIN = (0.40, 0.44, 0.46, 0.47, 0.475, 0.48, 0.485, 0.49, 0.493, 0.496, 0.499)
NUS_TEST = (0.4725, 0.4875, 0.4965)
ALPHAS = [0.0] + [1e-3 * 2 ** j for j in range(13)]


def test_learned_shift_beats_doubling(ick):
    """Train on shift sweeps of elasticity matrices (FP32 IC(0) factors), then on
    held-out Poisson ratios compare the plain retry (0, then 1e-3 doubling) with the
    retry started at the network's prediction: fewer attempts and less time to 1e-8."""
    import torch
    from paper_1601_05871_gb300 import shift_train as T
    X, y = [], []
    for ne in (6, 8):
        for nu in NUS_TRAIN:
            p, perm, h = _elasticity(ne, nu, ick, dtype=ick.IC_F32)
            av = dev(p.vals)
            b = dev(synth.rhs(p.n, 11))
            x = torch.empty_like(b)
            lab = T.label(T.sweep(h, av, b, x, ALPHAS))
            assert lab is not None
            X.append(ick.ic_shift_features(h, av, nu))
            y.append(lab)
    m, loss = T.train(np.array(X), np.array(y), steps=1500, lr=1e-2, seed=1)
    assert loss < 0.05
    rows = []
    for ne in (7, 8):
        for nu in NUS_TEST:
            p, perm, h = _elasticity(ne, nu, ick, dtype=ick.IC_F32)
            av = dev(p.vals)
            b = dev(synth.rhs(p.n, 12))
            x = torch.empty_like(b)
            T.solve(h, av, b, x)  # warm-up of both paths
            plain = T.solve(h, av, b, x)
            learned = T.solve(h, av, b, x, mlp=m, nu=nu)
            assert plain["relres"] <= 1e-8 and learned["relres"] <= 1e-8
            rows.append((ne, nu, plain, learned))
            print(f"ne {ne} nu {nu}: plain attempts {plain['attempts']} alpha {plain['alpha']:.3g} "
                  f"it {plain['iterations']} {plain['seconds'] * 1e3:.1f} ms | learned first {learned['first']:.3g} "
                  f"attempts {learned['attempts']} it {learned['iterations']} {learned['seconds'] * 1e3:.1f} ms")
    pa = np.mean([r[2]["attempts"] for r in rows])
    la = np.mean([r[3]["attempts"] for r in rows])
    pt = sum(r[2]["seconds"] for r in rows)
    lt = sum(r[3]["seconds"] for r in rows)
    pi = sum(r[2]["iterations"] for r in rows)
    li = sum(r[3]["iterations"] for r in rows)
    print(f"mean attempts plain {pa:.2f} learned {la:.2f}; iterations {pi} vs {li}; time {pt:.3f} s vs {lt:.3f} s")
    assert la < pa and la <= 1.5
    assert li <= 1.25 * pi
    assert lt < pt
