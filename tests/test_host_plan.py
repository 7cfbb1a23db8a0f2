"""CPU tests of libick.so's host logic: exports, nested dissection, the level-k
symbolic pass, the 2D block matrix, the Cholesky-by-blocks DAG and the per-task work
lists.  No GPU is used: handles are built with host_only=1.

The plan executor below runs the work lists of every task on the CPU, in random
topological orders of the DAG, with each update a separately rounded multiply then
subtract.  It is a test of the plan only (DAG edges and target lists), never a
product path.  With exact=1 the DAG serialises every update to a block in k order and
a task applies its pivots in ascending order, so every entry sees the same operation
sequence as the oracle's up-looking order: the result must match the oracle bit for
bit in any valid order.  Without it the updates of a block are chained in another
order (their inputs' estimated readiness): the result is the oracle's within rounding
and the same bits in every valid order.
"""
import os
import subprocess

import numpy as np
import pytest

import synth
import paper_1601_05871_gb300 as ick
from paper_1601_05871_gb300.build import build, lib_path

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()
    ick.load()


def test_library_exports_declared_symbols():
    names = ick.ick.declared_symbols()
    assert "ic_symbolic" in names and "ic_numeric" in names and "pcg_solve" in names
    L = ick.load()
    for nm in names:
        assert hasattr(L, nm), nm
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path()], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(names) <= exported


def test_strerror_and_last_error():
    L = ick.load()
    for st in range(9):
        assert L.ic_strerror(st)
    with pytest.raises(ick.IckError) as e:
        ick.ic_symbolic(np.array([0, 1, 2], dtype=np.int64), np.array([1, 0], dtype=np.int32), 0,
                        host_only=1)
    assert e.value.status == ick.ick.IC_ERR_PATTERN and "diagonal" in str(e.value)


# ------------------------------------------------------------------ worked example

def _read_worked_example():
    pattern, iters = {}, {}
    for ln in open(os.path.join(GOLD, "worked_example_tasks.txt")):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        if ln.startswith("pattern"):
            head, tail = ln.split(":")
            pattern[int(head.split()[1])] = [int(x) for x in tail.split()]
        else:
            head, tail = ln.split(":")
            iters[int(head)] = [tuple(t.split()) for t in tail.split(",")]
    return pattern, iters


def test_worked_example_task_sequence():
    """Section 3.3's 5x5 example: 19 tasks in the printed order."""
    pattern, iters = _read_worked_example()
    bptr = [0]
    bcol = []
    for b in range(len(pattern)):
        bcol += pattern[b]
        bptr.append(len(bcol))
    d = ick.ic_block_dag(bptr, bcol)
    got = []
    for t in range(len(d["type"])):
        name = ick.TASK_NAMES[d["type"][t]]
        k, i, j = int(d["k"][t]), int(d["i"][t]), int(d["j"][t])
        if name == "Chol":
            got.append((k + 1, (name, str(k), str(k))))
        elif name == "Trsm":
            got.append((k + 1, (name, str(k), str(j))))
        else:
            got.append((k + 1, (name, str(i), str(j))))
    want = [(it, t) for it in sorted(iters) for t in iters[it]]
    assert got == want and len(got) == 19
    # Chol(A22) has no predecessor; Trsm(A04)'s only predecessor is Chol(A00)
    idx = {(ick.TASK_NAMES[d["type"][t]], int(d["k"][t]), int(d["i"][t]), int(d["j"][t])): t
           for t in range(len(d["type"]))}
    pp, pr = d["pred_ptr"], d["pred"]
    t22 = idx[("Chol", 2, 2, 2)]
    assert pp[t22 + 1] == pp[t22]
    t04 = idx[("Trsm", 0, 0, 4)]
    assert list(pr[pp[t04]:pp[t04 + 1]]) == [idx[("Chol", 0, 0, 0)]]
    # dependence rule Chol -> Trsm -> Herk/Gemm: Herk44 at k=0 needs Trsm04
    h44 = idx[("Herk", 0, 4, 4)]
    assert list(pr[pp[h44]:pp[h44 + 1]]) == [t04]


def test_block_dag_rejects_bad_patterns():
    with pytest.raises(ick.IckError):
        ick.ic_block_dag([0, 1, 2], [1, 1])  # block row 0 lacks its diagonal
    with pytest.raises(ick.IckError):
        ick.ic_block_dag([0, 2, 3], [0, 5, 1])  # column out of range


# ------------------------------------------------------------------ ND and symbolic vs oracle

@pytest.mark.parametrize("colours", [(0, 0), (2, 0), (3, 0), (0, 2), (2, 2), (3, 4)])
@pytest.mark.parametrize("grid", [(64, 64, 1, 1, 256), (17, 9, 5, 1, 40), (6, 6, 6, 3, 50),
                                  (12, 12, 12, 1, 1), (1, 1, 1, 1, 1), (31, 30, 29, 1, 700)])
def test_nd_matches_oracle(orc, grid, colours):
    nx, ny, nz, dof, leaf = grid
    sep, lc = colours
    p1, r1 = ick.ic_nd_grid(nx, ny, nz, dof, leaf, sep_colours=sep, leaf_colours=lc)
    p2, r2 = orc.nd_grid(nx, ny, nz, dof, leaf, sep_colours=sep, leaf_colours=lc)
    assert np.array_equal(p1, p2) and np.array_equal(r1, r2)


@pytest.mark.parametrize("colours", [(0, 0), (2, 0), (2, 2)])
def test_nd_keep_matches_oracle(orc, colours):
    p = synth.elasticity3d_q1(4, seed=4002)
    sep, lc = colours
    p1, r1 = ick.ic_nd_grid(5, 5, 5, 3, 30, keep=p.keep, sep_colours=sep, leaf_colours=lc)
    p2, r2 = orc.nd_grid(5, 5, 5, 3, 30, keep=p.keep, sep_colours=sep, leaf_colours=lc)
    assert np.array_equal(p1, p2) and np.array_equal(r1, r2) and len(p1) == p.n


def test_nd_rejects_bad_colours():
    for c in (-1, 17):
        with pytest.raises(ick.IckError):
            ick.ic_nd_grid(8, 8, 8, 1, 40, sep_colours=c)
    for c in (-1, 5):
        with pytest.raises(ick.IckError):
            ick.ic_nd_grid(8, 8, 8, 1, 40, leaf_colours=c)


def test_coloured_separators_shorten_the_solve_dag():
    """Colour classes of a separator strip hold no 27-point neighbours, so the
    triangular solves' dependence DAG gets shallower (both directions); the strips are
    the blocks the lexicographic plane is cut into, so the level-k pattern, the block
    pattern and the task DAG keep their size."""
    p = synth.laplace3d_27pt(24)
    st, parts = [], []
    for c in (0, 2):
        perm, ranges = ick.ic_nd_grid(24, 24, 24, 1, 256, sep_colours=c)
        parts.append(len(ranges) - 1)
        h = ick.ic_symbolic(p.rowptr, p.colind, 2, perm, ranges, block_rows=256, host_only=1)
        st.append(ick.ic_stats(h))
    for key in ("nnz_l", "flops", "nranges", "nblocks", "ntasks", "critical_path"):
        assert st[1][key] == st[0][key], key
    assert parts[1] > parts[0]  # planes of more than 256 rows come as strips
    assert all(d1 < d0 for d0, d1 in zip(st[0]["solve_depth"], st[1]["solve_depth"]))


def _cases(orc):
    out = []
    p = synth.poisson2d_5pt(20, 17)
    out.append((p, ick.ic_nd_grid(20, 17, 1, 1, 40), 2))
    p = synth.laplace3d_27pt(7)
    out.append((p, ick.ic_nd_grid(7, 7, 7, 1, 30), 2))
    p = synth.diffusion3d_7pt(8, sigma=2.0, zscale=100.0, seed=5005)
    out.append((p, ick.ic_nd_grid(8, 8, 8, 1, 50), 3))
    p = synth.elasticity3d_q1(3, seed=4003)
    out.append((p, ick.ic_nd_grid(4, 4, 4, 3, 40, keep=p.keep), 0))
    p = synth.random_spd(40, 0.1, 9, kind="signed")
    out.append((p, (None, None), 1))
    return out


def _lower_sets(rp, ci, lv):
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    return rows, ci, lv


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_symbolic_matches_oracle(orc, k):
    """Pattern and levels from the per-row BFS equal the oracle's row-wise sum rule."""
    for prob, (perm, ranges), _ in _cases(orc):
        h = ick.ic_symbolic(prob.rowptr, prob.colind, k, perm, ranges, block_rows=64, host_only=1)
        rp, ci, _, lv = ick.ic_get_factor(h, values=False)
        o = orc.OracleIC.from_problem(prob, perm, k)
        orp, oci, olv = o.pattern()
        assert np.array_equal(rp, orp) and np.array_equal(ci, oci) and np.array_equal(lv, olv), prob.name
        st = o.numeric(prob.vals)
        if st == 0:
            assert ick.ic_stats(h)["flops"] == o.flops, prob.name


def test_pattern_errors():
    rp = np.array([0, 2, 3], dtype=np.int64)
    for ci, why in [(np.array([0, 1, 1], dtype=np.int32), "asymmetric"),
                    (np.array([1, 0, 1], dtype=np.int32), "unsorted"),
                    (np.array([0, 2, 1], dtype=np.int32), "range")]:
        with pytest.raises(ick.IckError) as e:
            ick.ic_symbolic(rp, ci, 1, host_only=1)
        assert e.value.status == ick.ick.IC_ERR_PATTERN, why
    p = synth.poisson2d_5pt(3, 3)
    with pytest.raises(ick.IckError) as e:
        ick.ic_symbolic(p.rowptr, p.colind, 1, perm=np.zeros(9, dtype=np.int32), host_only=1)
    assert e.value.status == ick.ick.IC_ERR_ARG
    with pytest.raises(ick.IckError):
        ick.ic_symbolic(p.rowptr, p.colind, 1, block_rows=9000, host_only=1)
    with pytest.raises(ick.IckError) as e:
        ick.ic_symbolic(p.rowptr, p.colind, 1, warps_per_cta=24, host_only=1)
    assert e.value.status == ick.ick.IC_ERR_ARG


def test_launch_shape_defaults():
    """One system: 32-warp CTAs; a batch: 16-warp CTAs; rows per Herk/Gemm item follow
    the warps unless given."""
    p = synth.poisson2d_5pt(6, 5)
    one = ick.ic_stats(ick.ic_symbolic(p.rowptr, p.colind, 1, host_only=1))
    assert (one["warps_per_cta"], one["rows_per_item"]) == (32, 32)
    batch = ick.ic_stats(ick.ic_symbolic_batch([(p.rowptr, p.colind)] * 3, 1, host_only=1))
    assert (batch["warps_per_cta"], batch["rows_per_item"]) == (16, 16)
    given = ick.ic_stats(ick.ic_symbolic(p.rowptr, p.colind, 1, warps_per_cta=8, rows_per_item=5, host_only=1))
    assert (given["warps_per_cta"], given["rows_per_item"]) == (8, 5)
    only_warps = ick.ic_stats(ick.ic_symbolic(p.rowptr, p.colind, 1, warps_per_cta=16, host_only=1))
    assert only_warps["rows_per_item"] == 16


def test_split_tasks_plan():
    """Only Chol/Trsm tasks of at least 512 target rows are split (several work items);
    their blocks' row-flag ranges are disjoint; the item total adds up."""
    prob = synth.laplace3d_27pt(24)
    perm, ranges = ick.ic_nd_grid(24, 24, 24, 1, 1024)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=1024, host_only=1)
    s = ick.ic_stats(h)
    d = ick.ic_get_tasks(h)
    nt = len(d["type"])
    items = 0
    split = 0
    for t in range(nt):
        ntg = len(ick.ic_get_task_targets(h, t))
        if d["type"][t] >= 2:
            items += max(1, -(-ntg // s["rows_per_item"]))
        elif ntg >= 512:
            split += 1
    assert 0 < s["nsplit"] <= split
    assert s["nitems"] == items + (sum(d["type"] < 2) - s["nsplit"]) + 8 * s["nsplit"]


def test_split_tasks_shadow_layout():
    """The published copy of every target segment of a split task lies inside the
    shadow array with 4 values of margin (16-byte copies may reach 3 past either end),
    is congruent to its U position modulo 4 (so the copies stay 16-byte aligned), and
    no two overlap."""
    prob = synth.laplace3d_27pt(24)
    perm, ranges = ick.ic_nd_grid(24, 24, 24, 1, 1024)
    for dtype in (ick.IC_F64, ick.IC_F32):
        h = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=1024, host_only=1,
                            dtype=dtype)
        lay = ick.ic_get_split_layout(h)
        rng, _, _ = ick.ic_get_blocks(h)
        d = ick.ic_get_tasks(h)
        fo, so, nsh = lay["flag_off"], lay["soff"], lay["nshadow"]
        split = np.nonzero(fo >= 0)[0]
        assert len(split) == ick.ic_stats(h)["nsplit"] > 0
        assert all(d["type"][t] in (0, 1) for t in split)
        spans = []
        for t in split:
            k = int(d["k"][t])
            for r, ca, cb, tb, te in ick.ic_get_task_targets(h, t):
                off = int(so[fo[t] + r - rng[k]])
                assert (tb + off) % 4 == tb % 4
                spans.append((tb + off, te + off))
        spans.sort()
        assert spans[0][0] >= 4 and spans[-1][1] <= nsh - 4
        assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    # no split tasks: an empty layout
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=300, host_only=1)
    lay = ick.ic_get_split_layout(h)
    assert (lay["flag_off"] < 0).all() == (ick.ic_stats(h)["nsplit"] == 0)


def test_empty_matrix():
    h = ick.ic_symbolic(np.zeros(1, dtype=np.int64), np.zeros(0, dtype=np.int32), 2, host_only=1)
    s = ick.ic_stats(h)
    assert s["n"] == 0 and s["ntasks"] == 0 and s["nitems"] == 0


# ------------------------------------------------------------------ DAG properties on real plans

def _plan(h):
    urp, ucol, cptr, cp, cpos = ick.ic_get_upper(h)
    ranges, bptr, bcol = ick.ic_get_blocks(h)
    d = ick.ic_get_tasks(h)
    tg = [ick.ic_get_task_targets(h, t) for t in range(len(d["type"]))]
    return urp, ucol, cp, cpos, ranges, bptr, bcol, d, tg


def test_block_pattern_and_dag_invariants():
    prob = synth.laplace3d_27pt(8)
    perm, ranges = ick.ic_nd_grid(8, 8, 8, 1, 40)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=48, host_only=1, exact=1)
    urp, ucol, cp, cpos, rng, bptr, bcol, d, tg = _plan(h)
    n = prob.n
    blk = np.searchsorted(rng, np.arange(n), side="right") - 1
    # a block exists iff S has an entry in it
    rows = np.repeat(np.arange(n), np.diff(urp))
    want = set(zip(blk[rows].tolist(), blk[ucol].tolist()))
    got = {(b, int(c)) for b in range(len(bptr) - 1) for c in bcol[bptr[b]:bptr[b + 1]]}
    assert got == want
    # predecessors come earlier; each block's writers form a chain in k order
    pp, pr = d["pred_ptr"], d["pred"]
    writers = {}
    for t in range(len(d["type"])):
        assert all(pr[pp[t]:pp[t + 1]] < t)
        ty, k, i, j = (int(d[x][t]) for x in ("type", "k", "i", "j"))
        key = (k, k) if ty == 0 else (k, j) if ty == 1 else (i, j)
        if key in writers:
            assert writers[key] in pr[pp[t]:pp[t + 1]]
        writers[key] = t
    s = ick.ic_stats(h)
    assert s["critical_path"] >= 1 and s["ntasks"] == sum(s["ntasks_type"])


def _execute_plan(prob, perm, h, order):
    """Run every task's work list on the CPU in `order` (a topological order)."""
    urp, ucol, cp, cpos, rng, bptr, bcol, d, tg = _plan(h)
    n = prob.n
    pinv = np.empty(n, dtype=np.int64)
    pm = np.arange(n) if perm is None else perm
    pinv[pm] = np.arange(n)
    # U := B on S (zero on fill)
    U = np.zeros(len(ucol))
    for o in range(n):
        i = pinv[o]
        for e in range(prob.rowptr[o], prob.rowptr[o + 1]):
            j = pinv[prob.colind[e]]
            if j >= i:
                pos = urp[i] + np.searchsorted(ucol[urp[i]:urp[i + 1]], j)
                U[pos] = prob.vals[e]
    for t in order:
        ty, k, i, j = (int(d[x][t]) for x in ("type", "k", "i", "j"))
        src = k if ty == 0 else j
        start_at_r = ty in (0, 2)
        lo, hi = rng[src], rng[src + 1]
        for r, ca, cb, tb, te in tg[t]:
            tcols = ucol[tb:te]
            for q in range(ca, cb):
                p, pos = int(cp[q]), int(cpos[q])
                row = ucol[urp[p]:urp[p + 1]]
                sb = urp[p] + np.searchsorted(row, lo)
                se = urp[p] + np.searchsorted(row, hi)
                if start_at_r:
                    sb = pos
                if se <= sb:
                    continue
                cols = ucol[sb:se]
                idx = np.searchsorted(tcols, cols)
                ok = (idx < len(tcols))
                ok[ok] &= tcols[idx[ok]] == cols[ok]
                tpos = tb + idx[ok]
                U[tpos] = U[tpos] - U[pos] * U[sb:se][ok]
            if ty == 0:
                U[tb] = np.sqrt(U[tb])
                U[tb + 1:te] = U[tb + 1:te] / U[tb]
            elif ty == 1:
                U[tb:te] = U[tb:te] / U[urp[r]]
    return urp, ucol, U


def _random_topo(d, rng):
    nt = len(d["type"])
    pp, pr = d["pred_ptr"], d["pred"]
    indeg = np.diff(pp).astype(int)
    succ = [[] for _ in range(nt)]
    for t in range(nt):
        for p in pr[pp[t]:pp[t + 1]]:
            succ[p].append(t)
    ready = [t for t in range(nt) if indeg[t] == 0]
    order = []
    while ready:
        t = ready.pop(rng.integers(len(ready)))
        order.append(t)
        for s in succ[t]:
            indeg[s] -= 1
            if indeg[s] == 0:
                ready.append(s)
    assert len(order) == nt
    return order


@pytest.mark.parametrize("case", range(4))
def test_plan_in_random_orders_matches_oracle_bitwise(orc, case):
    if case == 0:
        prob = synth.poisson2d_5pt(16, 16)
        perm, ranges = ick.ic_nd_grid(16, 16, 1, 1, 20)
        k, br = 1, 16
    elif case == 1:
        prob = synth.laplace3d_27pt(6)
        perm, ranges = ick.ic_nd_grid(6, 6, 6, 1, 20)
        k, br = 2, 24
    elif case == 2:
        prob = synth.diffusion3d_7pt(7, sigma=2.0, zscale=100.0, seed=77)
        perm, ranges = None, None
        k, br = 3, 40
    else:
        prob = synth.elasticity3d_q1(4, seed=4004)
        perm, ranges = ick.ic_nd_grid(5, 5, 5, 3, 90, keep=prob.keep)
        k, br = 1, 70
    o = orc.OracleIC.from_problem(prob, perm, k)
    assert o.numeric(prob.vals) == 0
    lref = o.values()
    lrp, lci, _ = o.pattern()
    amax = np.abs(prob.vals).max()
    g = np.random.default_rng(case)
    for exact in (1, 0):
        h = ick.ic_symbolic(prob.rowptr, prob.colind, k, perm, ranges, block_rows=br, host_only=1, exact=exact)
        d = ick.ic_get_tasks(h)
        first = None
        for trial in range(2):
            order = _random_topo(d, g)
            urp, ucol, U = _execute_plan(prob, perm, h, order)
            # L_ij = U_ji: map the oracle's lower entries onto U positions
            n = prob.n
            rows = np.repeat(np.arange(n), np.diff(lrp))
            upos = urp[lci] + np.array([np.searchsorted(ucol[urp[c]:urp[c + 1]], r) for r, c in zip(rows, lci)])
            if exact:
                # the task generator's k order per block: the oracle's operation sequence
                assert np.array_equal(U[upos], lref), (case, trial)
            else:
                # chains ordered by readiness: the same sums in another order, and one
                # fixed order per entry whatever the topological order of the run
                assert np.abs(U[upos] - lref).max() <= 1e-12 * amax, (case, trial)
                if first is None:
                    first = U.copy()
                assert np.array_equal(U, first), (case, trial)


def _chains(d):
    """Per written block: (Chol/Trsm task, updates in generation order); pred sets."""
    nt = len(d["type"])
    pp, pr = d["pred_ptr"], d["pred"]
    preds = [set(pr[pp[t]:pp[t + 1]].tolist()) for t in range(nt)]
    ups, final = {}, {}
    for t in range(nt):
        ty, k, i, j = (int(d[x][t]) for x in ("type", "k", "i", "j"))
        if ty >= 2:
            ups.setdefault((i, j), []).append(t)
        else:
            final[(k, k) if ty == 0 else (k, j)] = t
    return preds, ups, final


def test_fma_plan_reorders_update_chains():
    """Without exact, the updates into a block form one chain in the order of their
    inputs' estimated readiness: the same tasks and data dependencies as the task
    generator's plan, each block's updates a permutation of its k-ordered chain, ending
    in the block's Chol/Trsm; on an ND-ordered grid some chains leave k order."""
    prob = synth.laplace3d_27pt(12)
    perm, ranges = ick.ic_nd_grid(12, 12, 12, 1, 60)
    he = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=64, host_only=1, exact=1)
    hf = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=64, host_only=1)
    de, df = ick.ic_get_tasks(he), ick.ic_get_tasks(hf)
    for x in ("type", "k", "i", "j"):
        assert np.array_equal(de[x], df[x])
    nt = len(df["type"])
    _random_topo(df, np.random.default_rng(0))  # acyclic, every task reachable
    preds, ups, final = _chains(df)
    trsm = {(int(df["k"][t]), int(df["j"][t])): t for t in range(nt) if df["type"][t] == 1}
    chol = {int(df["k"][t]): t for t in range(nt) if df["type"][t] == 0}
    moved = 0
    for blk, us in ups.items():
        inset = set(us)
        # each update: its inputs Trsm(k,i), Trsm(k,j) and at most one update of the block
        prev = {}
        for u in us:
            k, i, j = (int(df[x][u]) for x in ("k", "i", "j"))
            src = {trsm[(k, i)], trsm[(k, j)]}
            assert src <= preds[u]
            rest = preds[u] - src
            assert rest <= inset and len(rest) <= 1
            prev[u] = next(iter(rest)) if rest else None
        # one chain through all of them, ending in the block's Chol/Trsm
        heads = [u for u in us if prev[u] is None]
        assert len(heads) == 1
        nxt = {p: u for u, p in prev.items() if p is not None}
        chain = [heads[0]]
        while chain[-1] in nxt:
            chain.append(nxt[chain[-1]])
        assert sorted(chain) == sorted(us)
        f = final[blk]
        assert preds[f] & inset == {chain[-1]}
        moved += chain != sorted(us)
    for t in range(nt):
        if df["type"][t] == 1:
            assert chol[int(df["k"][t])] in preds[t]
    assert moved > 0
    s_e, s_f = ick.ic_stats(he), ick.ic_stats(hf)
    assert s_e["ntasks"] == s_f["ntasks"] and s_e["nitems"] == s_f["nitems"]
    assert 1 <= s_f["critical_path"] <= nt


# ------------------------------------------------------------------ batches (block-diagonal unions)

def _batch(orc, count=6, seed=3000):
    probs = synth.diffusion_batch(count, 3, 7, seed=seed)
    perms = [orc.nd_grid(*p.grid, 1, 40)[0] for p in probs]
    return probs, perms


def test_batch_plan_is_union_of_independent_plans(orc):
    probs, perms = _batch(orc)
    h = ick.ic_symbolic_batch([(p.rowptr, p.colind) for p in probs], 1, perms, host_only=1, block_rows=64)
    off = ick.ic_batch_info(h)
    assert list(np.diff(off)) == [p.n for p in probs]
    rp, ci, _, lv = ick.ic_get_factor(h, values=False)
    for s, (p, pm) in enumerate(zip(probs, perms)):
        o = orc.OracleIC.from_problem(p, pm, 1)
        orp, oci, olv = o.pattern()
        a, b = off[s], off[s + 1]
        assert np.array_equal(rp[a:b + 1] - rp[a], orp)
        assert np.array_equal(ci[rp[a]:rp[b]] - a, oci) and np.array_equal(lv[rp[a]:rp[b]], olv)
    # no task depends on a task of another system
    rng, bptr, bcol = ick.ic_get_blocks(h)
    sys_of_block = np.searchsorted(off, rng[:-1], side="right") - 1
    d = ick.ic_get_tasks(h)
    pp, pr = d["pred_ptr"], d["pred"]
    for t in range(len(d["type"])):
        for q in pr[pp[t]:pp[t + 1]]:
            assert sys_of_block[d["k"][t]] == sys_of_block[d["k"][q]]


def test_batch_plan_executes_bitwise_per_system(orc):
    probs, perms = _batch(orc, count=4, seed=3100)
    rows, cols, vals = [], [], []
    off = 0
    for p in probs:
        r = np.repeat(np.arange(p.n), np.diff(p.rowptr)) + off
        rows.append(r); cols.append(p.colind + off); vals.append(p.vals)
        off += p.n
    union = synth.matrices._from_coo("union", off, np.concatenate(rows), np.concatenate(cols),
                                     np.concatenate(vals), 0)
    uperm = np.concatenate([pm + o for pm, o in zip(perms, np.cumsum([0] + [p.n for p in probs])[:-1])])
    h = ick.ic_symbolic_batch([(p.rowptr, p.colind) for p in probs], 1, perms, host_only=1, block_rows=48,
                              exact=1)
    d = ick.ic_get_tasks(h)
    urp, ucol, U = _execute_plan(union, uperm, h, _random_topo(d, np.random.default_rng(5)))
    offs = ick.ic_batch_info(h)
    for s, (p, pm) in enumerate(zip(probs, perms)):
        o = orc.OracleIC.from_problem(p, pm, 1)
        assert o.numeric(p.vals) == 0
        lrp, lci, _ = o.pattern()
        a = offs[s]
        rws = np.repeat(np.arange(p.n), np.diff(lrp))
        upos = urp[lci + a] + np.array([np.searchsorted(ucol[urp[c + a]:urp[c + a + 1]], r + a)
                                        for r, c in zip(rws, lci)])
        assert np.array_equal(U[upos], o.values()), s


@pytest.mark.parametrize("exact", [0, 1])
def test_claim_order_covers_every_item_after_its_predecessors(orc, exact):
    """The persistent numeric kernel's CTAs claim the work items in this order and wait
    for each item's predecessors: every item must appear exactly once and after every
    item of its task's predecessors (so a waiting CTA waits only for items held by
    running CTAs).  Executing the tasks in the order their last items are claimed
    reproduces the oracle (bit for bit in exact mode)."""
    for prob, (perm, ranges), k in _cases(orc)[:4]:
        h = ick.ic_symbolic(prob.rowptr, prob.colind, k, perm, ranges, block_rows=32, host_only=1, exact=exact)
        st = ick.ic_stats(h)
        d = ick.ic_get_tasks(h)
        task, chunk = ick.ic_get_claim_order(h)
        assert len(task) == st["nitems"]
        nt = len(d["type"])
        nitems = np.bincount(task, minlength=nt)
        assert np.all(nitems >= 1)
        pairs = set(zip(task.tolist(), chunk.tolist()))
        assert len(pairs) == st["nitems"]
        assert all(0 <= c < nitems[t] for t, c in pairs)
        last = np.zeros(nt, dtype=np.int64)
        firstpos = np.full(nt, -1, dtype=np.int64)
        for q, t in enumerate(task):
            last[t] = q
            if firstpos[t] < 0:
                firstpos[t] = q
        pp, pr = d["pred_ptr"], d["pred"]
        for t in range(nt):
            for p in pr[pp[t]:pp[t + 1]]:
                assert last[p] < firstpos[t], (t, p)
        o = orc.OracleIC.from_problem(prob, perm, k)
        assert o.numeric(prob.vals) == 0
        lref = o.values()
        lrp, lci, _ = o.pattern()
        urp, ucol, U = _execute_plan(prob, perm, h, np.argsort(last))
        rows = np.repeat(np.arange(prob.n), np.diff(lrp))
        upos = urp[lci] + np.array([np.searchsorted(ucol[urp[c]:urp[c + 1]], r) for r, c in zip(rows, lci)])
        if exact:
            assert np.array_equal(U[upos], lref)
        else:
            assert np.abs(U[upos] - lref).max() <= 1e-12 * np.abs(prob.vals).max()
