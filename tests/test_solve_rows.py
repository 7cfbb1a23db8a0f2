"""CPU tests of the block-row triangular solves' plan (solve_mode 2; host_only
handles, no GPU).

One CTA solves a whole block row, its rows in ascending level of the solve's row
dependence DAG, each level padded to a multiple of 8 positions so that one warp's
rows never depend on each other; the CTAs take the block rows in a claim order that
must be a topological order of the block-row graph (a CTA waits only for rows of
block rows claimed before its own).  The tests check those invariants, and that
executing the plan -- block rows in claim order, rows in their order, the external
entries and then the internal ones in their stored order -- gives the triangular
solves scipy computes with the oracle's factor.
"""
import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular

import synth
import paper_1601_05871_gb300 as ick
from test_solve_dag import _cases, _built  # noqa: F401  (fixture: builds the library)

PAD = 8


def _sources(urp, ucol, cptr, cp, i, backward):
    return ucol[urp[i] + 1:urp[i + 1]] if backward else cp[cptr[i]:cptr[i + 1]]


def _levels(urp, ucol, cptr, cp, n, backward):
    lev = np.zeros(n, dtype=np.int64)
    rows = range(n - 1, -1, -1) if backward else range(n)
    for i in rows:
        s = _sources(urp, ucol, cptr, cp, i, backward)
        lev[i] = lev[s].max() + 1 if len(s) else 0
    return lev


def _check(h, backward):
    urp, ucol, cptr, cp, cpos = ick.ic_get_upper(h)
    rg, _, _ = ick.ic_get_blocks(h)
    n, nr = len(urp) - 1, len(rg) - 1
    blk = np.searchsorted(rg, np.arange(n), side="right") - 1
    lev = _levels(urp, ucol, cptr, cp, n, backward)
    st = ick.ic_stats(h)
    assert st["solve_depth"][int(backward)] == (lev.max() + 1 if n else 0)
    d = ick.ic_get_solve_rows(h, backward)
    claim, ptr, order = d["claim"], d["ptr"], d["ord"]
    # the claim order is a permutation of the block rows and a topological order
    assert np.array_equal(np.sort(claim), np.arange(nr))
    at = np.empty(nr, dtype=np.int64)
    at[claim] = np.arange(nr)
    for i in range(n):
        src = _sources(urp, ucol, cptr, cp, i, backward)
        other = blk[src][blk[src] != blk[i]]
        assert np.all(at[other] < at[blk[i]]), (i, other)
    # each block row's rows once, levels ascending, each level's run padded to PAD,
    # so the rows of an aligned group of PAD positions share one level
    assert ptr[0] == 0 and ptr[-1] == len(order)
    for k in range(nr):
        seg = order[ptr[k]:ptr[k + 1]]
        assert len(seg) % PAD == 0 and ptr[k] % PAD == 0
        rows = seg[seg >= 0]
        assert np.array_equal(np.sort(rows), np.arange(rg[k], rg[k + 1]))
        assert np.all(np.diff(lev[rows]) >= 0)
        for g0 in range(0, len(seg), PAD):
            g = seg[g0:g0 + PAD]
            g = g[g >= 0]
            assert len(set(lev[g])) <= 1, (k, g0)
        # need: the range's rows of lower levels, so every internal source of a row is
        # among the rows counted before it may run
        need = d["need"][ptr[k]:ptr[k + 1]]
        real_before = np.cumsum(seg >= 0) - (seg >= 0)
        for q, r in enumerate(seg):
            if r < 0:
                continue
            assert need[q] == np.sum(lev[rows] < lev[r])
            src = _sources(urp, ucol, cptr, cp, r, backward)
            inside = src[blk[src] == k]
            pos = {int(x): qq for qq, x in enumerate(seg) if x >= 0}
            assert all(real_before[pos[int(x)]] < need[q] for x in inside), (k, r)
    return d


def test_block_row_plan_invariants(orc):
    for case in _cases(orc):
        name, p, perm, ranges, k, br = case
        h = ick.ic_symbolic(p.rowptr, p.colind, k, perm, ranges, block_rows=br, host_only=1)
        for backward in (False, True):
            _check(h, backward)


def _execute(h, uval, rhs, backward):
    """The kernels' arithmetic, block row by block row in claim order, in FP64."""
    urp, ucol, cptr, cp, cpos = ick.ic_get_upper(h)
    rg, _, _ = ick.ic_get_blocks(h)
    d = ick.ic_get_solve_rows(h, backward)
    t = ick.ic_get_solve_tasks(h, backward)
    lay = ick.ic_get_solve_entries(h, backward)
    split = t["split"]
    x = np.full(len(urp) - 1, np.nan)
    for k in d["claim"]:
        s = rg[k]
        for i in d["ord"][d["ptr"][k]:d["ptr"][k + 1]]:
            if i < 0:
                continue
            if backward:
                q = np.arange(urp[i] + 1 + split[i], urp[i + 1])
                ext_w, ext_v = uval[q], x[ucol[q]]
            else:
                q = np.arange(cptr[i], split[i])
                ext_w, ext_v = uval[cpos[q]], x[cp[q]]
            a, c = lay["ptr"][i], lay["ptr"][i + 1]
            int_v = x[lay["j"][a:c] + s]
            assert not np.isnan(ext_v).any() and not np.isnan(int_v).any(), (k, i)
            acc = np.dot(ext_w, ext_v) + np.dot(uval[lay["pos"][a:c]], int_v)
            x[i] = (rhs[i] - acc) / uval[urp[i]]
    return x


def test_block_row_plan_executes_to_triangular_solves(orc):
    for name, p, perm, ranges, k, br in _cases(orc):
        h = ick.ic_symbolic(p.rowptr, p.colind, k, perm, ranges, block_rows=br, host_only=1)
        o = orc.OracleIC.from_problem(p, perm if perm is not None else np.arange(p.n, dtype=np.int32), k)
        assert o.numeric(p.vals) == 0
        Lf = o.factor_csr()
        U = sp.csr_matrix(Lf.T)
        U.sort_indices()
        r = synth.rhs(p.n, 78)
        y = _execute(h, U.data, r, False)
        y_ref = spsolve_triangular(Lf.tocsr(), r, lower=True)
        assert np.allclose(y, y_ref, rtol=1e-12, atol=1e-12 * np.abs(y_ref).max()), name
        z = _execute(h, U.data, y, True)
        z_ref = spsolve_triangular(U, y, lower=False)
        assert np.allclose(z, z_ref, rtol=1e-12, atol=1e-12 * np.abs(z_ref).max()), name


def test_block_row_plan_internal_entries_lowest_level_first(orc):
    """Each row's internal entries are stored by ascending level of their source, so
    the sources that finish last are summed last."""
    p = synth.laplace3d_27pt(12)
    perm, ranges = orc.nd_grid(12, 12, 12, 1, 200)
    h = ick.ic_symbolic(p.rowptr, p.colind, 2, perm, ranges, block_rows=200, host_only=1)
    urp, ucol, cptr, cp, _ = ick.ic_get_upper(h)
    rg, _, _ = ick.ic_get_blocks(h)
    n = len(urp) - 1
    blk = np.searchsorted(rg, np.arange(n), side="right") - 1
    for backward in (False, True):
        lev = _levels(urp, ucol, cptr, cp, n, backward)
        lay = ick.ic_get_solve_entries(h, backward)
        for i in range(n):
            src = lay["j"][lay["ptr"][i]:lay["ptr"][i + 1]] + rg[blk[i]]
            assert np.all(np.diff(lev[src]) >= 0), (backward, i)
