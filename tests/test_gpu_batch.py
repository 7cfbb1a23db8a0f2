"""GPU tests of batched factorization: many independent uneven SPD systems as one
block-diagonal handle factored by one persistent launch, batched PCG replayed from a
captured CUDA graph, the numeric phase captured in a CUDA graph, and the autotuner.
Each system is compared with the oracle on its own matrix."""
import numpy as np
import pytest

import synth

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


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_batch(orc, count, smin, smax, seed, leaf=64):
    probs = synth.diffusion_batch(count, smin, smax, seed=seed)
    nd = [orc.nd_grid(*p.grid, 1, leaf) for p in probs]
    return probs, [x[0] for x in nd], [x[1] for x in nd]


def split_factor(ick, h, probs):
    """Per-system (rowptr, colind, values) of L taken out of the union's factor."""
    rp, ci, lv, _ = ick.ic_get_factor(h)
    off = ick.ic_batch_info(h)
    out = []
    for s in range(len(probs)):
        a, b = off[s], off[s + 1]
        out.append((rp[a:b + 1] - rp[a], ci[rp[a]:rp[b]] - a, lv[rp[a]:rp[b]]))
    return out


def test_batch_factor_bitwise_per_system(ick, orc):
    probs, perms, ranges = make_batch(orc, 24, 4, 12, 3200)
    vals = np.concatenate([p.vals for p in probs])
    h = ick.ic_symbolic_batch([(p.rowptr, p.colind) for p in probs], 1, perms, ranges, exact=1,
                              block_rows=128)
    ick.ic_numeric(h, dev(vals))
    for s, (lrp, lci, lv) in enumerate(split_factor(ick, h, probs)):
        o = orc.OracleIC.from_problem(probs[s], perms[s], 1)
        assert o.numeric(probs[s].vals) == 0
        orp, oci, _ = o.pattern()
        assert np.array_equal(lrp, orp) and np.array_equal(lci, oci), s
        assert np.array_equal(lv, o.values()), s


def test_batch_f32_within_bound(ick, orc):
    probs, perms, ranges = make_batch(orc, 16, 5, 14, 3300)
    vals = np.concatenate([p.vals for p in probs])
    h = ick.ic_symbolic_batch([(p.rowptr, p.colind) for p in probs], 1, perms, ranges, dtype=ick.IC_F32,
                              block_rows=256)
    ick.ic_numeric(h, dev(vals))
    for s, (lrp, lci, lv) in enumerate(split_factor(ick, h, probs)):
        o = orc.OracleIC.from_problem(probs[s], perms[s], 1)
        o.numeric(probs[s].vals)
        assert np.abs(lv - o.values()).max() <= 2e-5 * np.abs(probs[s].vals).max(), s


def test_batch_breakdown_in_one_system_reports_its_row(ick, orc):
    A = np.array([[2.0, 0.75, 0.25, -1.0], [0.75, 1.0, 1.0, 0.0], [0.25, 1.0, 1.5, 0.75],
                  [-1.0, 0.0, 0.75, 2.0]])
    rows, cols = np.nonzero(A)
    bad = synth.matrices._from_coo("brk4", 4, rows, cols, A[rows, cols], 0)
    good = synth.poisson2d_5pt(5, 5)
    probs = [good, bad, good]
    h = ick.ic_symbolic_batch([(p.rowptr, p.colind) for p in probs], 0, block_rows=8)
    with pytest.raises(ick.IckError) as e:
        ick.ic_numeric(h, dev(np.concatenate([p.vals for p in probs])))
    off = ick.ic_batch_info(h)
    assert e.value.status == 3 and e.value.row == off[1] + 3


def test_batch_pcg_matches_oracle_per_system(ick, orc):
    import torch
    probs, perms, ranges = make_batch(orc, 20, 4, 12, 3400)
    vals = dev(np.concatenate([p.vals for p in probs]))
    bs = [synth.rhs(p.n, 3400 + s) for s, p in enumerate(probs)]
    b = dev(np.concatenate(bs))
    h = ick.ic_symbolic_batch([(p.rowptr, p.colind) for p in probs], 1, perms, ranges, block_rows=128)
    ick.ic_numeric(h, vals)
    x = torch.empty_like(b)
    its, rels = ick.pcg_solve_batch(h, vals, b, x, 1e-8, 500)
    xh = x.cpu().numpy()
    off = ick.ic_batch_info(h)
    for s, p in enumerate(probs):
        o = orc.OracleIC.from_problem(p, perms[s], 1)
        o.numeric(p.vals)
        xo, ito, relo, st = orc.pcg(p, bs[s], o, tol=1e-8)
        assert st == 0 and abs(int(its[s]) - ito) <= 1 and rels[s] <= 1e-8, (s, its[s], ito)
        xs = xh[off[s]:off[s + 1]]
        assert np.linalg.norm(p.scipy() @ xs - bs[s]) / np.linalg.norm(bs[s]) <= 2e-8, s


def test_numeric_phase_captured_in_cuda_graph(ick, orc):
    import torch
    probs, perms, ranges = make_batch(orc, 12, 4, 10, 3500)
    vals = dev(np.concatenate([p.vals for p in probs]))
    h = ick.ic_symbolic_batch([(p.rowptr, p.colind) for p in probs], 1, perms, ranges, block_rows=128)
    ick.ic_numeric(h, vals)
    ref = ick.ic_get_factor(h)[2]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ick.ic_numeric_async(h, vals, s)  # warm-up outside capture
    s.synchronize()
    ick.ic_numeric_status(h)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        ick.ic_numeric_async(h, vals, s)
    for _ in range(3):
        g.replay()
        torch.cuda.synchronize()
        ick.ic_numeric_status(h)
        assert np.array_equal(ick.ic_get_factor(h)[2], ref)


def test_autotune_choice_factors_correctly(ick, orc):
    probs, perms, ranges = make_batch(orc, 10, 6, 12, 3600)
    vals = dev(np.concatenate([p.vals for p in probs]))
    pats = [(p.rowptr, p.colind) for p in probs]
    opts, (tn, ta) = ick.ic_autotune(pats, 1, vals, perms, ranges, reps=2, exact=1)
    assert opts["block_rows"] in (1024, 2048, 4096, 8192) and opts["warps_per_cta"] in (8, 16, 32)
    assert opts["solve_lanes"] in (8, 16, 32) and tn > 0 and ta > 0
    h = ick.ic_symbolic_batch(pats, 1, perms, ranges, **opts)
    ick.ic_numeric(h, vals)
    for s, (lrp, lci, lv) in enumerate(split_factor(ick, h, probs)):
        o = orc.OracleIC.from_problem(probs[s], perms[s], 1)
        o.numeric(probs[s].vals)
        assert np.array_equal(lv, o.values()), s


@pytest.mark.slow
def test_c3_batch_512_systems_one_launch(ick, orc):
    """The batched workload: 512 cubes of side U{8..32}, kappa ~ LogNormal(0,1), IC(1),
    FP32 factors, one persistent launch; FP64 batched PCG to 1e-8.  Sampled systems are
    compared with the oracle; every system must converge."""
    import torch
    probs = synth.config_problem(3)
    nd = [orc.nd_grid(*p.grid, 1, 4096) for p in probs]
    perms, ranges = [x[0] for x in nd], [x[1] for x in nd]
    vals = dev(np.concatenate([p.vals for p in probs]))
    h = ick.ic_symbolic_batch([(p.rowptr, p.colind) for p in probs], 1, perms, ranges,
                              dtype=ick.IC_F32, block_rows=4096)
    st = ick.ic_stats(h)
    ick.ic_set_timing(h, True)
    ick.ic_numeric(h, vals)
    t = ick.ic_get_timing(h)
    assert t["launches"] >= 2
    bs = np.concatenate([synth.rhs(p.n, 3000 + s) for s, p in enumerate(probs)])
    b = dev(bs)
    x = torch.empty_like(b)
    its, rels = ick.pcg_solve_batch(h, vals, b, x, 1e-8, 1000)
    assert np.all(rels <= 1e-8)
    print(f"C3: n={st['n']} tasks={st['ntasks']} factor {t['prepare_ms'] + t['numeric_ms']:.2f} ms, "
          f"PCG iterations {its.min()}..{its.max()}")
    parts = split_factor(ick, h, probs)
    for s in (0, 1, 255, 511):
        o = orc.OracleIC.from_problem(probs[s], perms[s], 1)
        o.numeric(probs[s].vals)
        assert np.abs(parts[s][2] - o.values()).max() <= 2e-5 * np.abs(probs[s].vals).max(), s
