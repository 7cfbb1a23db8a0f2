"""CPU tests of the block-DAG triangular solves' plan (host_only handles, no GPU).

The plan splits every block row (range) into E tasks, which sum the entries reaching
outside the range, and one L task, which solves the range's rows in its own local
level order.  The tests check the plan's invariants (split points, padded local
orders, counters) and that running its tasks one after another in claim order never
meets an unmet counter: the condition under which the persistent solve grid, which
claims tasks in that order, cannot deadlock.  Executing the tasks with the oracle's
factor values, in exactly the kernels' arithmetic order, must give the triangular
solves that scipy computes with the same factor.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular

import synth
import paper_1601_05871_gb300 as ick
from paper_1601_05871_gb300.build import build

PAD = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    build()
    ick.load()


def _cases(orc):
    p = synth.laplace3d_27pt(14)
    perm, ranges = orc.nd_grid(14, 14, 14, 1, 256)
    yield "27pt-14-nd", p, perm, ranges, 2, 128
    perm, ranges = orc.nd_grid(14, 14, 14, 1, 256, sep_colours=2)
    yield "27pt-14-nd-coloured-separators", p, perm, ranges, 2, 128
    perm, ranges = orc.nd_grid(14, 14, 14, 1, 256, sep_colours=2, leaf_colours=2)
    yield "27pt-14-nd-coloured-leaves", p, perm, ranges, 2, 128
    p = synth.poisson2d_5pt(40, 40)
    yield "5pt-40-natural", p, None, None, 1, 100
    p = synth.elasticity3d_q1(5, nu=0.3)
    perm, ranges = orc.nd_grid(*p.grid, 3, 96, p.keep)
    yield "elasticity-5", p, perm, ranges, 1, 64
    p = synth.random_spd(60, 0.15, seed=5)
    yield "random-60-tiny-ranges", p, None, None, 2, 7
    p = synth.poisson2d_5pt(12, 12)
    yield "one-range", p, None, None, 1, 4096


def _plan(case):
    name, p, perm, ranges, k, br = case
    h = ick.ic_symbolic(p.rowptr, p.colind, k, perm, ranges, block_rows=br, host_only=1)
    return h


def _check_direction(h, backward):
    urp, ucol, cptr, cp, cpos = ick.ic_get_upper(h)
    rg, _, _ = ick.ic_get_blocks(h)
    n, nr = len(urp) - 1, len(rg) - 1
    d = ick.ic_get_solve_tasks(h, backward)
    split, optr, order = d["split"], d["order_ptr"], d["order"]
    blk = np.searchsorted(rg, np.arange(n), side="right") - 1
    # split points: external entries first (forward) / last (backward)
    deps = []
    for i in range(n):
        s, e = rg[blk[i]], rg[blk[i] + 1]
        if not backward:
            ps = cp[cptr[i]:cptr[i + 1]]
            q = split[i] - cptr[i]
            assert 0 <= q <= len(ps)
            assert np.all(ps[:q] < s) and np.all((ps[q:] >= s) & (ps[q:] < i))
            deps.append(ps[q:])
        else:
            cs = ucol[urp[i] + 1:urp[i + 1]]
            q = split[i]
            assert 0 <= q <= len(cs)
            assert np.all((cs[:q] > i) & (cs[:q] < e)) and np.all(cs[q:] >= e)
            deps.append(cs[:q])
    # padded local orders: each range's rows once, every internal dependence in an
    # earlier aligned group of PAD positions
    for k in range(nr):
        seg = order[optr[k]:optr[k + 1]]
        assert len(seg) % PAD == 0 and optr[k] % PAD == 0
        rows = seg[seg >= 0]
        assert np.array_equal(np.sort(rows), np.arange(rg[k], rg[k + 1]))
        pos = {int(r): q for q, r in enumerate(seg) if r >= 0}
        for r in rows:
            for dd in deps[r]:
                assert pos[int(dd)] // PAD < pos[int(r)] // PAD, (k, r, dd)
        # need: rows of the lower levels, constant over each aligned group, and every
        # dependence of a row lies among the rows counted by its need
        need = d["need"][optr[k]:optr[k + 1]]
        assert np.all(np.diff(need) >= 0)
        for g0 in range(0, len(seg), PAD):
            assert np.all(need[g0:g0 + PAD] == need[g0])
            assert need[g0] <= np.sum(seg[:g0] >= 0)
        real_before = np.cumsum(seg >= 0) - (seg >= 0)
        for r in rows:
            for dd in deps[r]:
                assert real_before[pos[int(dd)]] < need[pos[int(r)]], (k, r, dd)
        # the kernels' rule, replayed with rows finishing in a random admissible order:
        # a row may run once `done >= need`; its dependences must then be complete
        rng = np.random.default_rng(k)
        done, fin = 0, set()
        waiting = [q for q in range(len(seg)) if seg[q] >= 0]
        while waiting:
            ready = [q for q in waiting if need[q] <= done]
            assert ready
            q = ready[rng.integers(len(ready))]
            assert all(int(dd) in fin for dd in deps[seg[q]])
            fin.add(int(seg[q]))
            done += 1
            waiting.remove(q)
    # contiguous layout: exactly the internal entries of each row, with their values'
    # positions in U
    x = ick.ic_get_solve_entries(h, backward)
    for i in range(n):
        s = rg[blk[i]]
        a, c = x["ptr"][i], x["ptr"][i + 1]
        assert np.array_equal(np.sort(x["j"][a:c] + s), np.sort(deps[i]))
        if not backward:
            want_pos = np.sort(cpos[split[i]:cptr[i + 1]])
        else:
            want_pos = np.arange(urp[i] + 1, urp[i] + 1 + split[i])
        assert np.array_equal(np.sort(x["pos"][a:c]), want_pos)
    # tasks: per range, L parts cover its order positions contiguously and in order; E
    # tasks cover exactly the rows with external entries, each inside one part
    tasks, indeg = d["tasks"], d["counters"]
    sptr, succ = d["succ_ptr"], d["succ"]
    has_ext = np.array([(split[i] > cptr[i]) if not backward else (split[i] < urp[i + 1] - urp[i] - 1)
                        for i in range(n)])
    part_of = np.full(n, -1)
    for k in range(nr):
        Ls = sorted([t for t in range(len(tasks)) if tasks[t, 0] == 1 and tasks[t, 1] == k], key=lambda t: tasks[t, 2])
        assert Ls and tasks[Ls[0], 2] == optr[k] and tasks[Ls[-1], 3] == optr[k + 1]
        for a_, b_ in zip(Ls, Ls[1:]):
            assert tasks[a_, 3] == tasks[b_, 2]
        for t in Ls:
            lo, hi = tasks[t, 2], tasks[t, 3]
            rows = order[lo:hi]
            part_of[rows[rows >= 0]] = t
            if lo > optr[k]:   # a part starts on a level boundary
                assert d["need"][lo] == np.sum(order[optr[k]:lo] >= 0)
        if not has_ext[rg[k]:rg[k + 1]].any():
            assert len(Ls) == 1
    covered = np.zeros(n, dtype=int)
    for t in range(len(tasks)):
        if tasks[t, 0] == 0:
            lo, hi = tasks[t, 2], tasks[t, 3]
            rows = order[lo:hi]
            rows = rows[rows >= 0]
            covered[rows[has_ext[rows]]] += 1
            assert len(set(part_of[rows])) == 1
    assert np.array_equal(covered, has_ext.astype(int))
    # sequential execution in claim order never meets an unmet counter, and every
    # dependence of the data is ordered before its use
    cnt = indeg.copy()
    done_t = np.zeros(len(tasks), dtype=bool)
    for t in range(len(tasks)):
        assert cnt[t] == 0, t
        lo, hi = tasks[t, 2], tasks[t, 3]
        rows = order[lo:hi]
        rows = rows[rows >= 0]
        if tasks[t, 0] == 0:
            for i in rows[has_ext[rows]]:
                srcs = cp[cptr[i]:split[i]] if not backward else ucol[urp[i] + 1 + split[i]:urp[i + 1]]
                assert done_t[part_of[srcs]].all(), (t, i)
        else:
            k = tasks[t, 1]
            earlier = order[optr[k]:lo]
            assert done_t[part_of[earlier[earlier >= 0]]].all()
            mine = [u for u in range(len(tasks)) if tasks[u, 0] == 0 and tasks[u, 1] == k and lo <= tasks[u, 2] < hi]
            assert done_t[mine].all(), (t, mine)
        done_t[t] = True
        for s_ in succ[sptr[t]:sptr[t + 1]]:
            cnt[s_] -= 1
    assert np.all(cnt == 0)
    return d


def test_solve_plan_invariants(orc):
    for case in _cases(orc):
        h = _plan(case)
        for backward in (False, True):
            _check_direction(h, backward)


def _execute(h, uval, b, backward, rhs):
    """The kernels' arithmetic, task by task in claim order, in FP64 on the host."""
    urp, ucol, cptr, cp, cpos = ick.ic_get_upper(h)
    d = ick.ic_get_solve_tasks(h, backward)
    lay = ick.ic_get_solve_entries(h, backward)
    rg, _, _ = ick.ic_get_blocks(h)
    split, optr, order = d["split"], d["order_ptr"], d["order"]
    n = len(urp) - 1
    x = np.full(n, np.nan)
    w = np.zeros(n)
    for t in d["tasks"]:
        if t[0] == 0:
            for i in order[t[2]:t[3]]:
                if i < 0 or not ((split[i] > cptr[i]) if not backward else (split[i] < urp[i + 1] - urp[i] - 1)):
                    continue
                if not backward:
                    q = np.arange(cptr[i], split[i])
                    vals = x[cp[q]]
                    assert not np.isnan(vals).any()
                    w[i] = np.dot(uval[cpos[q]], vals)
                else:
                    q = np.arange(urp[i] + 1 + split[i], urp[i + 1])
                    vals = x[ucol[q]]
                    assert not np.isnan(vals).any()
                    w[i] = np.dot(uval[q], vals)
        else:
            s = rg[t[1]]
            for i in order[t[2]:t[3]]:
                if i < 0:
                    continue
                a, c = lay["ptr"][i], lay["ptr"][i + 1]
                vals = x[lay["j"][a:c] + s]
                assert not np.isnan(vals).any()
                ext = (split[i] > cptr[i]) if not backward else (split[i] < urp[i + 1] - urp[i] - 1)
                v = rhs[i] - (w[i] if ext else 0.0)
                x[i] = (v - np.dot(uval[lay["pos"][a:c]], vals)) / uval[urp[i]]
    return x


def test_solve_plan_executes_to_triangular_solves(orc):
    for name, p, perm, ranges, k, br in _cases(orc):
        h = ick.ic_symbolic(p.rowptr, p.colind, k, perm, ranges, block_rows=br, host_only=1)
        o = orc.OracleIC.from_problem(p, perm if perm is not None else np.arange(p.n, dtype=np.int32), k)
        assert o.numeric(p.vals) == 0
        Lf = o.factor_csr()
        U = sp.csr_matrix(Lf.T)
        U.sort_indices()
        urp, ucol, _, _, _ = ick.ic_get_upper(h)
        assert np.array_equal(U.indptr, urp) and np.array_equal(U.indices, ucol), name
        r = synth.rhs(p.n, 77)
        y = _execute(h, U.data, None, False, r)
        y_ref = spsolve_triangular(Lf.tocsr(), r, lower=True)
        assert np.allclose(y, y_ref, rtol=1e-12, atol=1e-12 * np.abs(y_ref).max()), name
        z = _execute(h, U.data, None, True, y)
        z_ref = spsolve_triangular(U, y, lower=False)
        assert np.allclose(z, z_ref, rtol=1e-12, atol=1e-12 * np.abs(z_ref).max()), name


def test_solve_plan_batch_union(orc):
    probs = synth.diffusion_batch(6, 4, 8, seed=55)
    nd = [orc.nd_grid(*q.grid, 1, 64) for q in probs]
    h = ick.ic_symbolic_batch([(q.rowptr, q.colind) for q in probs], 1, [x[0] for x in nd], [x[1] for x in nd],
                              block_rows=48, host_only=1)
    for backward in (False, True):
        d = _check_direction(h, backward)
        # the systems are independent: no task releases a task of another system
        rg, _, _ = ick.ic_get_blocks(h)
        off = ick.ic_batch_info(h)
        sys_of = np.searchsorted(off, rg[:-1], side="right") - 1
        tk = d["tasks"]
        for t in range(len(tk)):
            for u in d["succ"][d["succ_ptr"][t]:d["succ_ptr"][t + 1]]:
                assert sys_of[tk[u, 1]] == sys_of[tk[t, 1]]
