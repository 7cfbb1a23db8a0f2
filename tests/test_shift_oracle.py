"""Pins of the learned-shift oracle (oracle/shift.py) against facts fixed outside it:
hand-derived features of a small matrix, closed forms of the 5-point Laplacian,
central finite differences of the loss, the zero-weight network, the first Adam step
and the doubling rule against a known threshold.  CPU only."""
import os

import numpy as np
import pytest

import synth
from oracle import shift as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden_matrix(name):
    rows, cols, vals, k, nu, n = [], [], [], None, None, None
    for ln in open(os.path.join(GOLD, name)):
        ln = ln.split("#")[0].split()
        if not ln:
            continue
        if ln[0] == "matrix":
            n = int(ln[1])
        elif ln[0] == "k":
            k = int(ln[1])
        elif ln[0] == "nu":
            nu = float(ln[1])
        else:
            rows.append(int(ln[0])); cols.append(int(ln[1])); vals.append(float(ln[2]))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    for r in rows:
        rowptr[r + 1] += 1
    rowptr = np.cumsum(rowptr)
    return n, rowptr, np.array(cols, dtype=np.int32), np.array(vals), k, nu


def test_features_hand_derived_3x3():
    n, rp, ci, v, k, nu = _read_golden_matrix("features_3x3.txt")
    f = S.features(n, rp, ci, v, k, nu)
    want = [2.0, 7.0 / 3.0, (np.sqrt(18) / 4 + np.sqrt(10) / 3 + np.sqrt(5) / 2) / 3, np.sqrt(5) / 2, 0.5, 1.0,
            np.log10(3.0), 0.3]
    assert np.allclose(f, want, rtol=1e-14, atol=0)


def test_features_poisson_closed_form():
    m = 9
    p = synth.poisson2d_5pt(m, m)
    f = S.features(p.n, p.rowptr, p.colind, p.vals, 0, 0.0)
    # interior rows: 4 neighbours (dd = 1), edge rows 3 (dd = 4/3), corners 2 (dd = 2)
    ni, ne, nc = (m - 2) ** 2, 4 * (m - 2), 4
    dd_mean = (ni * 1.0 + ne * 4.0 / 3.0 + nc * 2.0) / m ** 2
    rn = lambda deg: np.sqrt(16.0 + deg) / 4.0
    rn_mean = (ni * rn(4) + ne * rn(3) + nc * rn(2)) / m ** 2
    assert np.allclose(f, [1.0, dd_mean, rn_mean, rn(4), 0.0, 0.0, np.log10(m * m), 0.0], rtol=1e-14)


def test_features_diagonal_matrix_hits_cap():
    n = 5
    rp = np.arange(n + 1, dtype=np.int64)
    f = S.features(n, rp, np.arange(n, dtype=np.int32), np.full(n, 2.0), 2, 0.0)
    assert f[0] == S.DD_CAP and f[1] == S.DD_CAP and f[2] == 1.0 and f[3] == 1.0 and f[4] == 0.0


def test_features_reject_nonpositive_diagonal():
    rp = np.array([0, 1], dtype=np.int64)
    with pytest.raises(ValueError):
        S.features(1, rp, np.array([0], dtype=np.int32), np.array([-1.0]), 0)


def _random_net(hidden, seed, nsamp=17):
    rng = np.random.default_rng(seed)
    theta = synth.mlp_init(hidden, seed)
    # non-zero biases in both hidden layers, so that no pre-activation sits exactly on
    # the ReLU kink (where a central difference averages the two one-sided slopes)
    theta[NB1(hidden)] += rng.normal(0, 0.3, hidden)
    theta[NB2(hidden)] += rng.normal(0, 0.3, hidden)
    X = rng.normal(0, 1, (nsamp, S.NFEAT)) * np.array([0.3, 1, 2, 1, 0.2, 1, 1, 0.1]) + 1.0
    mean, std = X.mean(axis=0), X.std(axis=0) + 0.5
    t = rng.normal(-2, 1, nsamp)
    return theta, X, mean, std, t


def NB1(hidden):
    return slice(S.NFEAT * hidden, S.NFEAT * hidden + hidden)


def NB2(hidden):
    o = S.NFEAT * hidden + hidden + hidden * hidden
    return slice(o, o + hidden)


@pytest.mark.parametrize("hidden", [4, 16, 32])
def test_gradient_matches_central_differences(hidden):
    theta, X, mean, std, t = _random_net(hidden, 11 + hidden)
    L, g = S.loss_and_grad(theta, hidden, mean, std, X, t)
    assert g.shape == (S.n_params(hidden),)
    h = 1e-6
    rng = np.random.default_rng(5)
    idx = rng.choice(len(theta), size=min(60, len(theta)), replace=False)
    for q in idx:
        e = np.zeros_like(theta)
        e[q] = h
        Lp, _ = S.loss_and_grad(theta + e, hidden, mean, std, X, t)
        Lm, _ = S.loss_and_grad(theta - e, hidden, mean, std, X, t)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[q]) <= 1e-7 + 1e-5 * abs(fd), (q, fd, g[q])


def test_zero_network_closed_form():
    hidden = 8
    theta = np.zeros(S.n_params(hidden))
    theta[-1] = 0.7  # b3
    X = np.random.default_rng(1).normal(size=(5, S.NFEAT))
    t = np.array([0.0, 1.0, 2.0, -1.0, 0.5])
    y, _ = S.forward(theta, hidden, np.zeros(S.NFEAT), np.ones(S.NFEAT), X)
    assert np.all(y == 0.7)
    L, g = S.loss_and_grad(theta, hidden, np.zeros(S.NFEAT), np.ones(S.NFEAT), X, t)
    assert np.isclose(L, 0.5 * np.mean((0.7 - t) ** 2))
    assert np.isclose(g[-1], np.mean(0.7 - t)) and np.all(g[:-1] == 0.0)


def test_first_adam_step_is_signed_learning_rate():
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    th, m, v = S.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    # step 1: mhat = g, vhat = g^2, so the update is lr * g / (|g| + eps)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_retry_rule_against_a_known_threshold():
    assert S.retry_sequence(0.0, 1e-3, 5) == [0.0, 1e-3, 2e-3, 4e-3, 8e-3]
    a, tries = S.first_success(lambda x: x < 0.01, 0.0)
    assert np.isclose(a, 0.016) and tries == 6
    a, tries = S.first_success(lambda x: x < 0.01, 0.012)
    assert a == 0.012 and tries == 1
    a, tries = S.first_success(lambda x: True, 0.0, max_tries=4)
    assert a is None and tries == 4


def test_retry_rule_resolves_the_golden_breakdown(orc):
    """The 4x4 matrix whose IC(0) breaks down (tests/golden/ic0_breakdown_4x4.txt) factors
    once shifted: the doubling rule finds a shift."""
    A = np.array([[2.0, 0.75, 0.25, -1.0], [0.75, 1.0, 1.0, 0.0], [0.25, 1.0, 1.5, 0.75], [-1.0, 0.0, 0.75, 2.0]])
    rows, cols = np.nonzero(A)
    rp = np.zeros(5, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    o = orc.OracleIC(4, rp, cols.astype(np.int32), None, 0)
    vals = A[rows, cols]
    a, tries = S.first_success(lambda x: o.numeric(vals, x) != 0, 0.0)
    assert tries > 1 and a > 0.0
    assert o.numeric(vals, a) == 0 and o.numeric(vals, 0.0) != 0


# ------------------------------------------------ the shifted factorization


def _csr_from_dense(A):
    rows, cols = np.nonzero(A)
    rp = np.zeros(A.shape[0] + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp), cols.astype(np.int32), A[rows, cols]


def test_shifted_factor_hand_derived_3x3(orc):
    """B = [[2,2,4],[2,5,0],[4,0,4]], identity order, IC(0): the fill (2,1) has level 1
    and is dropped.  The shift multiplies the diagonal of B by (1 + alpha) before any
    elimination.  alpha = 1: B_00 -> 4, L_00 = 2, L_10 = 1, L_20 = 2, L_11 = sqrt(10 - 1)
    = 3, L_22 = sqrt(8 - 4) = 2 (the dropped fill is discarded, not added to the
    diagonal).  alpha = 0: L_22^2 = 4 - 8 < 0, so row 2 breaks down.  An additive
    shift, a shift applied after elimination or a compensated drop all give other
    numbers."""
    A = np.array([[2.0, 2.0, 4.0], [2.0, 5.0, 0.0], [4.0, 0.0, 4.0]])
    rp, ci, v = _csr_from_dense(A)
    o = orc.OracleIC(3, rp, ci, None, 0)
    lptr, lcol, _ = o.pattern()
    assert list(lptr) == [0, 1, 3, 5] and list(lcol) == [0, 0, 1, 0, 2]
    assert o.numeric(v, 1.0) == 0
    assert list(o.values()) == [2.0, 1.0, 3.0, 2.0, 2.0]
    assert o.numeric(v, 0.0) == orc.ERR_BREAKDOWN and o.breakdown_row == 2
    # with the fill kept (k = 1): L_21 = (0 - L_20 L_10) / L_11 = -2/3 and
    # L_22 = sqrt(8 - 4 - 4/9) = sqrt(32)/3
    o1 = orc.OracleIC(3, rp, ci, None, 1)
    assert o1.numeric(v, 1.0) == 0
    assert np.allclose(o1.values(), [2.0, 1.0, 3.0, 2.0, -2.0 / 3.0, np.sqrt(32.0) / 3.0], rtol=1e-15, atol=0)


def test_shifted_diagonal_matrix_closed_form(orc):
    d = np.array([1.0, 2.0, 0.5, 7.0, 3.25])
    n = len(d)
    rp = np.arange(n + 1, dtype=np.int64)
    o = orc.OracleIC(n, rp, np.arange(n, dtype=np.int32), None, 2)
    for alpha in (0.0, 1e-3, 0.3, 5.0):
        assert o.numeric(d, alpha) == 0
        assert np.allclose(o.values(), np.sqrt((1.0 + alpha) * d), rtol=2e-16, atol=0), alpha


@pytest.mark.parametrize("alpha,k", [(1e-3, 0), (0.05, 1), (0.4, 2)])
def test_shift_equals_factor_of_preshifted_matrix(orc, alpha, k):
    """Shifting inside the factorization gives the factor of the matrix whose diagonal
    was scaled beforehand, under a nested-dissection order (the shift lands on B_ii =
    A_perm(i),perm(i), whichever row that is in A's order)."""
    p = synth.laplace3d_27pt(9)
    perm, _ = orc.nd_grid(9, 9, 9, 1, 100)
    diag = np.zeros(len(p.vals), dtype=bool)
    for i in range(p.n):
        s, e = p.rowptr[i], p.rowptr[i + 1]
        diag[s:e] = p.colind[s:e] == i
    pre = p.vals.copy()
    pre[diag] = pre[diag] + alpha * pre[diag]
    o = orc.OracleIC.from_problem(p, perm, k)
    assert o.numeric(p.vals, alpha) == 0
    shifted = o.values()
    assert o.numeric(pre, 0.0) == 0
    assert np.array_equal(shifted, o.values())
    assert o.numeric(p.vals, 0.0) == 0
    assert not np.array_equal(shifted, o.values())


# ------------------------------------------------ a hand-derived network


def read_mlp_golden():
    g = {"x": []}
    for ln in open(os.path.join(GOLD, "mlp_forward_h2.txt")):
        ln = ln.split("#")[0].split()
        if not ln:
            continue
        if ln[0] == "x":
            g["x"].append([float(t) for t in ln[1:]])
        else:
            g[ln[0]] = [float(t) for t in ln[1:]]
    H = int(g["hidden"][0])
    theta = np.concatenate([g["W1"], g["b1"], g["W2"], g["b2"], g["w3"], g["b3"]])
    return H, theta, np.array(g["mean"]), np.array(g["std"]), np.array(g["x"]), np.array(g["y"])


def pad_network(theta, hidden, to):
    """The same function with `to` hidden units per layer: the extra units have zero
    weights and biases, so they output ReLU(0) = 0 and feed nothing."""
    W1, b1, W2, b2, w3, b3 = S.unpack(theta, hidden)
    P1 = np.zeros((S.NFEAT, to)); P1[:, :hidden] = W1
    P2 = np.zeros((to, to)); P2[:hidden, :hidden] = W2
    pad = lambda v: np.concatenate([v, np.zeros(to - hidden)])
    return np.concatenate([P1.ravel(), pad(b1), P2.ravel(), pad(b2), pad(w3), [b3]])


def test_mlp_forward_hand_derived():
    H, theta, mean, std, X, y = read_mlp_golden()
    assert len(theta) == S.n_params(H)
    out, (Z, a1, h1, a2, h2) = S.forward(theta, H, mean, std, X)
    assert np.array_equal(out, y)
    # every ReLU unit of both layers is inactive for at least one input
    assert np.all((a1 <= 0).any(axis=0)) and np.all((a2 <= 0).any(axis=0))
    padded = pad_network(theta, H, 32)
    assert np.array_equal(S.forward(padded, 32, mean, std, X)[0], y)
