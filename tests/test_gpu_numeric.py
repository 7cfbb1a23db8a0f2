"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Pattern and levels must match bit for bit; FP64 values within 1e-12 * max|A| (the
bound the workload sets for FP64); with exact=1 (separately rounded multiply and
subtract, the oracle's operation sequence) the factor must match bit for bit.
Breakdown rows must match the oracle's first failing row.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def factor_both(ick, orc, prob, perm, ranges, k, **opts):
    h = ick.ic_symbolic(prob.rowptr, prob.colind, k, perm, ranges, **opts)
    vals = dev(prob.vals)
    gpu_brk = -1
    try:
        ick.ic_numeric(h, vals)
    except ick.IckError as e:
        if e.status != 3:
            raise
        gpu_brk = e.row
    o = orc.OracleIC.from_problem(prob, perm, k)
    st = o.numeric(prob.vals)
    return h, o, gpu_brk, st


def check_parity(ick, orc, prob, perm, ranges, k, exact=0, **opts):
    h, o, gpu_brk, st = factor_both(ick, orc, prob, perm, ranges, k, exact=exact, **opts)
    assert st == 0 and gpu_brk == -1, (prob.name, st, gpu_brk)
    rp, ci, lv, levels = ick.ic_get_factor(h)
    orp, oci, olev = o.pattern()
    assert np.array_equal(rp, orp) and np.array_equal(ci, oci) and np.array_equal(levels, olev)
    ref = o.values()
    amax = np.abs(prob.vals).max()
    err = np.abs(lv - ref).max() / amax
    if exact:
        assert np.array_equal(lv, ref), (prob.name, err)
    else:
        assert err <= TOL, (prob.name, err)
    return h, o, lv


def test_c1_uniform_blocks_exact_and_fma(ick, orc):
    """2-D Poisson 64x64, IC(1), 16 uniform 256-row blocks of the ND-ordered matrix."""
    prob = synth.config_problem(1)
    perm, _ = ick.ic_nd_grid(64, 64, 1, 1, 256)
    check_parity(ick, orc, prob, perm, None, 1, exact=1, block_rows=256)
    check_parity(ick, orc, prob, perm, None, 1, exact=0, block_rows=256)


def test_c1_nd_ranges(ick, orc):
    prob = synth.config_problem(1)
    perm, ranges = ick.ic_nd_grid(64, 64, 1, 1, 256)
    check_parity(ick, orc, prob, perm, ranges, 1, exact=1, block_rows=256)


@pytest.mark.parametrize("warps", [8, 16, 32])
def test_27pt_ic2(ick, orc, warps):
    prob = synth.laplace3d_27pt(14)
    perm, ranges = ick.ic_nd_grid(14, 14, 14, 1, 300)
    check_parity(ick, orc, prob, perm, ranges, 2, exact=1, block_rows=300, warps_per_cta=warps)
    check_parity(ick, orc, prob, perm, ranges, 2, exact=0, block_rows=300, warps_per_cta=warps)


@pytest.mark.parametrize("warps", [16, 32])
def test_tasks_split_over_ctas(ick, orc, warps):
    """Chol/Trsm tasks expected to run with little else in flight are spread over
    several CTAs, rows claimed from a global counter and published in a shadow array:
    the factor is the one CTA would give (bit-exact in exact mode)."""
    prob = synth.laplace3d_27pt(24)
    perm, ranges = ick.ic_nd_grid(24, 24, 24, 1, 1024)
    for exact in (1, 0):
        h, o, lv = check_parity(ick, orc, prob, perm, ranges, 2, exact=exact, block_rows=1024,
                                warps_per_cta=warps)
        assert ick.ic_stats(h)["nsplit"] > 0
        # whichever CTA takes a row, every entry sees the same operations: same bits
        v = dev(prob.vals)
        for _ in range(2):
            ick.ic_numeric(h, v)
            assert np.array_equal(ick.ic_get_factor(h)[2], lv)


def test_rows_wider_than_the_column_map(ick, orc):
    """Natural order of a 5000 x 3 grid in two 7500-row blocks: a row's segment in a
    block reaches 5000 columns past its diagonal, so a target row is cut into chunks
    whose columns each span at most 4096."""
    prob = synth.poisson2d_5pt(5000, 3)
    for exact in (1, 0):
        check_parity(ick, orc, prob, None, None, 1, exact=exact, block_rows=8192)


def test_anisotropic_ic3_ragged_blocks(ick, orc):
    prob = synth.diffusion3d_7pt(19, 17, 13, sigma=2.0, zscale=100.0, seed=5001)
    perm, ranges = ick.ic_nd_grid(19, 17, 13, 1, 333)
    check_parity(ick, orc, prob, perm, ranges, 3, exact=1, block_rows=257, rows_per_item=7)


def test_elasticity_ic1(ick, orc):
    prob = synth.elasticity3d_q1(5, seed=4004)
    perm, ranges = ick.ic_nd_grid(6, 6, 6, 3, 120, keep=prob.keep)
    h, o, brk, st = factor_both(ick, orc, prob, perm, ranges, 1, block_rows=100)
    assert brk == (o.breakdown_row if st else -1)
    if st == 0:
        check_parity(ick, orc, prob, perm, ranges, 1, exact=1, block_rows=100)


@pytest.mark.parametrize("block_rows", [1, 3, 8192])
def test_extreme_block_sizes(ick, orc, block_rows):
    prob = synth.poisson2d_5pt(23, 19)
    perm, _ = ick.ic_nd_grid(23, 19, 1, 1, 30)
    check_parity(ick, orc, prob, perm, None, 2, exact=1, block_rows=block_rows)


def test_long_rows_chunked(ick, orc):
    """Complete fill of a dense SPD matrix: rows of 300 entries exceed one staged chunk."""
    prob = synth.random_spd(300, 1.0, 11, kind="dense_spd")
    check_parity(ick, orc, prob, None, None, 300, exact=1, block_rows=64)
    check_parity(ick, orc, prob, None, None, 300, exact=0, block_rows=100)


@pytest.mark.parametrize("seed", range(4))
def test_random_signed(ick, orc, seed):
    prob = synth.random_spd(200, 0.03, 50 + seed, kind="signed")
    for k in (0, 2):
        h, o, brk, st = factor_both(ick, orc, prob, None, None, k, block_rows=37, exact=1)
        if st:
            assert brk == o.breakdown_row
        else:
            assert brk == -1
            rp, ci, lv, _ = ick.ic_get_factor(h)
            assert np.array_equal(lv, o.values())


def test_breakdown_row_hand_computed(ick, orc):
    A = np.array([[2.0, 0.75, 0.25, -1.0], [0.75, 1.0, 1.0, 0.0], [0.25, 1.0, 1.5, 0.75],
                  [-1.0, 0.0, 0.75, 2.0]])
    rows, cols = np.nonzero(A)
    prob = synth.matrices._from_coo("brk4", 4, rows, cols, A[rows, cols], 0)
    for br in (1, 2, 4):
        h, o, brk, st = factor_both(ick, orc, prob, None, None, 0, block_rows=br)
        assert st == orc.ERR_BREAKDOWN and o.breakdown_row == 3 and brk == 3


def test_tiny_and_empty(ick, orc):
    prob = synth.matrices._from_coo("one", 1, [0], [0], [4.0], 0)
    h, o, lv = check_parity(ick, orc, prob, None, None, 0, exact=1)
    assert lv[0] == 2.0
    h = ick.ic_symbolic(np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), 1)
    import torch
    ick.ic_numeric(h, torch.zeros(1, dtype=torch.float64, device="cuda"))
    s = ick.ic_stats(h)
    assert s["n"] == 0


def test_repeat_calls_bitwise_and_shift(ick, orc):
    prob = synth.laplace3d_27pt(10)
    perm, ranges = ick.ic_nd_grid(10, 10, 10, 1, 100)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=128)
    v = dev(prob.vals)
    ick.ic_numeric(h, v)
    a = ick.ic_get_factor(h)[2]
    for _ in range(3):
        ick.ic_numeric(h, v)
        assert np.array_equal(ick.ic_get_factor(h)[2], a)
    hs = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=128,
                         shift_alpha=0.25, exact=1)
    ick.ic_numeric(hs, v)
    o = orc.OracleIC.from_problem(prob, perm, 2)
    assert o.numeric(prob.vals, 0.25) == 0
    assert np.array_equal(ick.ic_get_factor(hs)[2], o.values())


def test_timeout_when_a_task_is_never_released(ick, orc):
    """Host-side fault injection: one task's in-degree is raised so that no
    predecessor ever releases it.  Every device wait is bounded, so the call returns
    IC_ERR_TIMEOUT; afterwards the restored plan factors correctly."""
    prob = synth.poisson2d_5pt(30, 30)
    perm, ranges = ick.ic_nd_grid(30, 30, 1, 1, 60)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 1, perm, ranges, block_rows=64, timeout_s=0.5)
    ntasks = ick.ic_stats(h)["ntasks"]
    ick.ic_test_hold_task(h, ntasks // 2, 1)
    v = dev(prob.vals)
    with pytest.raises(ick.IckError) as e:
        ick.ic_numeric(h, v)
    assert e.value.status == 4
    ick.ic_test_hold_task(h, ntasks // 2, 0)
    ick.ic_numeric(h, v)
    o = orc.OracleIC.from_problem(prob, perm, 1)
    o.numeric(prob.vals)
    assert np.abs(ick.ic_get_factor(h)[2] - o.values()).max() <= TOL * np.abs(prob.vals).max()


def test_apply_matches_oracle(ick, orc):
    import torch
    prob = synth.diffusion3d_7pt(16, sigma=1.0, seed=3001)
    perm, ranges = ick.ic_nd_grid(16, 16, 16, 1, 256)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 1, perm, ranges, block_rows=256)
    ick.ic_numeric(h, dev(prob.vals))
    o = orc.OracleIC.from_problem(prob, perm, 1)
    o.numeric(prob.vals)
    r = np.random.default_rng(1).standard_normal(prob.n)
    z = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ick.ic_apply(h, dev(r), z)
    torch.cuda.synchronize()
    zr = o.apply(r)
    assert np.abs(z.cpu().numpy() - zr).max() <= 1e-11 * np.abs(zr).max()
    with pytest.raises(ick.IckError):
        ick.ic_apply(h, z, z)


def test_solve_timeout_is_reported_and_later_applies_recover(ick, orc):
    """Host-side fault injection into the block-DAG solve: one forward task's in-degree
    is raised so that nothing releases it.  The wait gives up after timeout_s; the
    timeout is recorded, ic_apply_status and pcg_solve report it, and once the plan is
    restored the next applications are correct again (each one clears the abort word
    of the previous)."""
    import torch
    prob = synth.diffusion3d_7pt(14, sigma=1.0, seed=3002)
    perm, ranges = ick.ic_nd_grid(14, 14, 14, 1, 256)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 1, perm, ranges, block_rows=256, timeout_s=0.5)
    av = dev(prob.vals)
    ick.ic_numeric(h, av)
    o = orc.OracleIC.from_problem(prob, perm, 1)
    o.numeric(prob.vals)
    nt = len(ick.ic_get_solve_tasks(h)["tasks"])
    rh = np.random.default_rng(4).standard_normal(prob.n)
    r = dev(rh)
    z = torch.empty_like(r)
    ick.ic_test_hold_solve_task(h, nt // 2, 1)
    ick.ic_apply(h, r, z)
    with pytest.raises(ick.IckError) as e:
        ick.ic_apply_status(h)
    assert e.value.status == 4
    ick.ic_apply_status(h)  # the record was cleared by the read
    b = dev(synth.rhs(prob.n, 5))
    x = torch.empty_like(b)
    with pytest.raises(ick.IckError) as e:
        ick.pcg_solve(h, av, b, x, 1e-8, 3)
    assert e.value.status == 4
    ick.ic_test_hold_solve_task(h, nt // 2, 0)
    zr = o.apply(rh)
    for _ in range(2):
        ick.ic_apply(h, r, z)
        ick.ic_apply_status(h)
        assert np.abs(z.cpu().numpy() - zr).max() <= 1e-11 * np.abs(zr).max()
    it, rel = ick.pcg_solve(h, av, b, x, 1e-8, 500)
    assert rel <= 1e-8


@pytest.mark.parametrize("dtype", [0, 1])
def test_row_level_and_block_dag_solves_agree(ick, orc, dtype):
    """Both triangular-solve implementations (solve_mode 1: every row a unit in global
    level order; 0: block-DAG) apply the same factor: each matches the oracle's apply
    within the precision's bound, and they agree with each other."""
    import torch
    prob = synth.laplace3d_27pt(18)
    perm, ranges = ick.ic_nd_grid(18, 18, 18, 1, 512)
    o = orc.OracleIC.from_problem(prob, perm, 2)
    o.numeric(prob.vals)
    r = np.random.default_rng(7).standard_normal(prob.n)
    zr = o.apply(r)
    out = []
    for mode in (1, 0):
        h = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=512, dtype=dtype,
                            solve_mode=mode)
        ick.ic_numeric(h, dev(prob.vals))
        z = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        ick.ic_apply(h, dev(r), z)
        torch.cuda.synchronize()
        out.append(z.cpu().numpy())
    tol = 1e-11 if dtype == 0 else 2e-4
    for z in out:
        assert np.abs(z - zr).max() <= tol * np.abs(zr).max()
    assert np.abs(out[0] - out[1]).max() <= tol * np.abs(zr).max()


def test_pcg_matches_oracle(ick, orc):
    import torch
    prob = synth.config_problem(1)
    perm, _ = ick.ic_nd_grid(64, 64, 1, 1, 256)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 1, perm, None, block_rows=256)
    av = dev(prob.vals)
    ick.ic_numeric(h, av)
    b = synth.rhs(prob.n, prob.seed)
    x = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    it, rel = ick.pcg_solve(h, av, dev(b), x, 1e-8, 1000)
    o = orc.OracleIC.from_problem(prob, perm, 1)
    o.numeric(prob.vals)
    xo, ito, relo, st = orc.pcg(prob, b, o, tol=1e-8)
    assert st == 0 and abs(it - ito) <= 1 and rel <= 1e-8
    xg = x.cpu().numpy()
    true_rel = np.linalg.norm(prob.scipy() @ xg - b) / np.linalg.norm(b)
    assert true_rel <= 2e-8
    assert np.abs(xg - xo).max() <= 1e-6 * np.abs(xo).max()


def test_coloured_separators_parity(ick, orc):
    """Separator strips numbered in 2x2 colour classes (the oracle's own ordering):
    the factor is bit-exact in exact mode and within TOL with FMAs, and the
    block-DAG solves match the oracle's substitutions."""
    import torch
    prob = synth.laplace3d_27pt(20)
    perm, ranges = orc.nd_grid(20, 20, 20, 1, 256, sep_colours=2)
    check_parity(ick, orc, prob, perm, ranges, 2, exact=1, block_rows=256)
    h, o, _ = check_parity(ick, orc, prob, perm, ranges, 2, exact=0, block_rows=256)
    r = synth.rhs(prob.n, 9)
    z = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ick.ic_apply(h, dev(r), z)
    ick.ic_apply_status(h)
    zr = o.apply(r)
    assert np.abs(z.cpu().numpy() - zr).max() <= 1e-11 * np.abs(zr).max()


def test_repeated_applies_are_identical(ick):
    """Two hundred preconditioner applications in a row give the same bits and no
    timeout: the solves are deterministic, so a CTA whose warps disagreed on the task
    at hand (a race on the shared task slot between a release and the next claim)
    would show here as a changed result or a wait that gives up."""
    import torch
    prob = synth.laplace3d_27pt(24)
    perm, ranges = ick.ic_nd_grid(24, 24, 24, 1, 1024)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=1024)
    ick.ic_numeric(h, dev(prob.vals))
    r = dev(synth.rhs(prob.n, 5))
    z = torch.empty_like(r)
    ick.ic_apply(h, r, z)
    torch.cuda.synchronize()
    z0 = z.cpu().numpy()
    outs = torch.empty((200, prob.n), dtype=torch.float64, device="cuda")
    for k in range(200):
        ick.ic_apply(h, r, outs[k])
    ick.ic_apply_status(h)  # raises if a wait gave up
    assert bool((outs == torch.from_numpy(z0).cuda()).all())


def test_pcg_graph_matches_host_loop(ick):
    """pcg_solve as one graph (timing off: the loop runs on the device) and as a host
    loop (timing on) take the same steps: the same iterations and the same x, on a
    repeated call (the graph kept) and after a change of tol (the graph rebuilt); a
    maxit that stops the loop early gives IC_ERR_NOCONV after exactly maxit
    iterations in both."""
    import torch
    prob = synth.laplace3d_27pt(20)
    perm, ranges = ick.ic_nd_grid(20, 20, 20, 1, 1024)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 1, perm, ranges, block_rows=1024)
    av = dev(prob.vals)
    ick.ic_numeric(h, av)
    b = dev(synth.rhs(prob.n, 77))

    x = torch.empty(prob.n, dtype=torch.float64, device="cuda")  # the same x every call

    def solve(timing, tol, maxit=1000):
        ick.ic_set_timing(h, timing)
        x.fill_(7.0)
        it, rel = ick.pcg_solve(h, av, b, x, tol, maxit, raise_noconv=False)
        torch.cuda.synchronize()
        return it, rel, x.cpu().numpy()

    for tol in (1e-8, 1e-8, 1e-11):
        ig, rg, xg = solve(False, tol)
        ih, rh, xh = solve(True, tol)
        assert ig == ih and ig > 3 and rg <= tol
        assert rg == rh
        assert np.array_equal(xg, xh)
    # new values behind the same pointer (the kept graph reads them): 2A x = b
    av.mul_(2.0)
    ick.ic_numeric(h, av)
    ig, rg, x2 = solve(False, 1e-11)
    ih, rh, x2h = solve(True, 1e-11)
    assert ig == ih and np.array_equal(x2, x2h)
    assert np.abs(2.0 * x2 - xg).max() <= 1e-8 * np.abs(xg).max()
    for timing in (False, True):
        ick.ic_set_timing(h, timing)
        with pytest.raises(ick.IckError) as e:
            ick.pcg_solve(h, av, b, x, 1e-14, 3)
        assert e.value.status == ick.IC_ERR_NOCONV
        it, rel = ick.pcg_solve(h, av, b, x, 1e-14, 3, raise_noconv=False)
        assert it == 3 and rel > 1e-14
    ick.ic_set_timing(h, False)


@pytest.mark.slow
def test_full_size_27pt_96_ic2(ick, orc):
    """The bench workload at full size (96^3 27-point, IC(2), ND ranges of <= 4096 rows,
    16 warps per CTA): every entry of L against the oracle, plus the defining identity
    on sampled pattern entries."""
    prob = synth.config_problem(2)
    perm, ranges = ick.ic_nd_grid(96, 96, 96, 1, 4096)
    h, o, lv = check_parity(ick, orc, prob, perm, ranges, 2, exact=0, block_rows=4096)
    rp, ci, _, _ = ick.ic_get_factor(h)
    g = np.random.default_rng(0)
    n = prob.n
    pinv = np.empty(n, dtype=np.int64)
    pinv[perm] = np.arange(n)
    A = prob.scipy()
    for i in g.integers(0, n, size=200):
        row_i = dict(zip(ci[rp[i]:rp[i + 1]].tolist(), lv[rp[i]:rp[i + 1]].tolist()))
        for j in ci[rp[i]:rp[i + 1]]:
            row_j = dict(zip(ci[rp[j]:rp[j + 1]].tolist(), lv[rp[j]:rp[j + 1]].tolist()))
            s = sum(row_i[c] * row_j[c] for c in row_i if c in row_j and c <= j)
            bij = A[perm[i], perm[j]]
            assert abs(s - bij) <= 1e-12 * 26
