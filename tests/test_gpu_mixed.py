"""GPU tests of the mixed-precision factorization (dtype IC_F32): FP32 factor values
and FP32 triangular solves, with FP64 diagonal pivots (accumulation, square root and
breakdown test) and FP64 PCG.

Bound on the factor: every entry of L is a sum of at most (row length) products formed
and accumulated in FP32 (unit roundoff 2^-24 ~ 6e-8), so its error against the FP64
oracle is about (number of updates) * 6e-8 * |partial sums|; for the matrices here
(<= ~100 updates per entry, partial sums <= max|A|) that is <= ~1e-5 * max|A|.  The
test asserts 2e-5 * max|A| and reports the measured value.  The pivots are FP64, so a
breakdown row must agree with the oracle's exactly.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

F32_TOL = 2e-5


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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def mixed_vs_oracle(ick, orc, prob, perm, ranges, k, **opts):
    h = ick.ic_symbolic(prob.rowptr, prob.colind, k, perm, ranges, dtype=ick.IC_F32, **opts)
    ick.ic_numeric(h, dev(prob.vals))
    rp, ci, lv, levels = ick.ic_get_factor(h)
    o = orc.OracleIC.from_problem(prob, perm, k)
    assert o.numeric(prob.vals) == 0
    orp, oci, olev = o.pattern()
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci) and np.array_equal(levels, olev)
    err = np.abs(lv - o.values()).max() / np.abs(prob.vals).max()
    return h, o, err


@pytest.mark.parametrize("case", ["c1", "27pt", "aniso", "elast"])
def test_f32_factor_within_bound(ick, orc, case):
    if case == "c1":
        prob = synth.config_problem(1)
        perm, ranges = ick.ic_nd_grid(64, 64, 1, 1, 256)
        k, br = 1, 256
    elif case == "27pt":
        prob = synth.laplace3d_27pt(14)
        perm, ranges = ick.ic_nd_grid(14, 14, 14, 1, 300)
        k, br = 2, 300
    elif case == "aniso":
        prob = synth.diffusion3d_7pt(17, sigma=2.0, zscale=100.0, seed=5002)
        perm, ranges = ick.ic_nd_grid(17, 17, 17, 1, 400)
        k, br = 3, 257
    else:
        prob = synth.elasticity3d_q1(5, seed=4006)
        perm, ranges = ick.ic_nd_grid(6, 6, 6, 3, 120, keep=prob.keep)
        k, br = 2, 100
    h, o, err = mixed_vs_oracle(ick, orc, prob, perm, ranges, k, block_rows=br)
    print(f"{prob.name}: max|L32 - L64| / max|A| = {err:.3e}")
    assert err <= F32_TOL, err


def test_f32_tasks_split_over_ctas(ick, orc):
    prob = synth.laplace3d_27pt(24)
    perm, ranges = ick.ic_nd_grid(24, 24, 24, 1, 1024)
    h, o, err = mixed_vs_oracle(ick, orc, prob, perm, ranges, 2, block_rows=1024)
    assert ick.ic_stats(h)["nsplit"] > 0
    assert err <= F32_TOL, err


def test_f32_long_rows(ick, orc):
    prob = synth.random_spd(300, 1.0, 12, kind="dense_spd")
    h, o, err = mixed_vs_oracle(ick, orc, prob, None, None, 300, block_rows=100)
    assert err <= F32_TOL, err


def test_f32_breakdown_row_from_fp64_pivots(ick, orc):
    A = np.array([[2.0, 0.75, 0.25, -1.0], [0.75, 1.0, 1.0, 0.0], [0.25, 1.0, 1.5, 0.75],
                  [-1.0, 0.0, 0.75, 2.0]])
    rows, cols = np.nonzero(A)
    prob = synth.matrices._from_coo("brk4", 4, rows, cols, A[rows, cols], 0)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 0, dtype=ick.IC_F32, block_rows=2)
    with pytest.raises(ick.IckError) as e:
        ick.ic_numeric(h, dev(prob.vals))
    assert e.value.status == 3 and e.value.row == 3


def test_f32_pcg_reaches_fp64_tolerance(ick, orc):
    import torch
    prob = synth.laplace3d_27pt(24)
    perm, ranges = ick.ic_nd_grid(24, 24, 24, 1, 1000)
    av = dev(prob.vals)
    b = dev(synth.rhs(prob.n, 2))
    its = {}
    for dt in (ick.IC_F64, ick.IC_F32):
        h = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, dtype=dt, block_rows=1000)
        ick.ic_numeric(h, av)
        x = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        it, rel = ick.pcg_solve(h, av, b, x, 1e-10, 2000)
        xh = x.cpu().numpy()
        true_rel = np.linalg.norm(prob.scipy() @ xh - b.cpu().numpy()) / np.linalg.norm(b.cpu().numpy())
        assert rel <= 1e-10 and true_rel <= 2e-10, (dt, rel, true_rel)
        its[dt] = it
    assert its[ick.IC_F32] <= its[ick.IC_F64] + 3, its


def test_f32_apply_close_to_f64_apply(ick, orc):
    import torch
    prob = synth.diffusion3d_7pt(16, sigma=1.0, seed=3002)
    perm, ranges = ick.ic_nd_grid(16, 16, 16, 1, 256)
    r = dev(np.random.default_rng(4).standard_normal(prob.n))
    out = {}
    for dt in (ick.IC_F64, ick.IC_F32):
        h = ick.ic_symbolic(prob.rowptr, prob.colind, 1, perm, ranges, dtype=dt, block_rows=256)
        ick.ic_numeric(h, dev(prob.vals))
        z = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        ick.ic_apply(h, r, z)
        torch.cuda.synchronize()
        out[dt] = z.cpu().numpy()
    rel = np.abs(out[ick.IC_F32] - out[ick.IC_F64]).max() / np.abs(out[ick.IC_F64]).max()
    assert rel <= 1e-4, rel
