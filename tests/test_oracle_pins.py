"""Pins of the CPU oracle to facts fixed outside the oracle itself.

Each test checks the oracle against mathematics or a hand-derived fixture, never
against a re-typing of its own formulas:
  * complete fill (k >= n-1) is the Cholesky factor (LAPACK via numpy);
  * the defining identity (L L^T)_ij = B_ij on the pattern S, for every k;
  * IC(0) of a tridiagonal matrix is exact; a diagonal matrix gives sqrt(diag);
  * the level-k pattern equals a brute-force enumeration of fill paths
    (level definition: Section 1 footnote; fill-path rule of Hysom and Pothen
    cited in Section 3.1);
  * S_0 = pattern(B), S_k grows with k and is bounded by the complete pattern
    (the trend of Table 2);
  * M-matrices never break down (Meijerink and van der Vorst);
  * a hand-computed 4x4 breakdown (tests/golden/ic0_breakdown_4x4.txt);
  * hand-derived nested-dissection orders (tests/golden/nd_small.txt);
  * PCG with the complete factor converges in one iteration, and CG work on the
    2-D Poisson problem grows like sqrt(condition number).
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def permuted_dense(prob, perm):
    A = prob.to_dense()
    if perm is None:
        return A
    return A[np.ix_(perm, perm)]


def oracle_factor(orc, prob, perm, k, shift=0.0):
    h = orc.OracleIC.from_problem(prob, perm, k)
    st = h.numeric(prob.vals, shift)
    return h, st


def small_problems():
    out = []
    for seed in range(4):
        out.append((synth.random_spd(9 + seed, 0.35, seed, kind="mmatrix"), None))
        out.append((synth.random_spd(10, 0.3, 10 + seed, kind="signed"), None))
    out.append((synth.random_spd(7, 1.0, 3, kind="dense_spd"), None))
    return out


def grid_problems(orc):
    probs = []
    p = synth.poisson2d_5pt(7, 6)
    probs.append((p, orc.nd_grid(7, 6, 1, 1, 4)[0]))
    p = synth.laplace3d_27pt(4)
    probs.append((p, orc.nd_grid(4, 4, 4, 1, 8)[0]))
    p = synth.diffusion3d_7pt(5, sigma=2.0, zscale=100.0, seed=11)
    probs.append((p, orc.nd_grid(5, 5, 5, 1, 10)[0]))
    p = synth.elasticity3d_q1(2, seed=4001)
    probs.append((p, orc.nd_grid(3, 3, 3, 3, 6, keep=p.keep)[0]))
    return probs


# --------------------------------------------------------------- numeric pins

def test_complete_fill_is_cholesky(orc):
    """k >= n-1 keeps every fill entry: L must be LAPACK's Cholesky factor of B."""
    for prob, perm in small_problems() + grid_problems(orc):
        h, st = oracle_factor(orc, prob, perm, prob.n)
        assert st == 0
        B = permuted_dense(prob, perm)
        Lref = np.linalg.cholesky(B)
        L = h.factor_csr().toarray()
        scale = np.abs(Lref).max()
        assert np.abs(L - Lref).max() <= 1e-13 * scale, prob.name
        # entries outside the symbolic pattern are exact zeros in the dense factor
        outside = (L == 0) & (np.tril(np.ones_like(L)) == 1)
        lptr, lcol, _ = h.pattern()
        inpat = np.zeros_like(L, dtype=bool)
        for i in range(prob.n):
            inpat[i, lcol[lptr[i]:lptr[i + 1]]] = True
        assert np.all(Lref[~inpat & (np.tril(np.ones_like(L)) == 1)] == 0.0), prob.name
        assert outside.sum() >= 0


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_pattern_identity_every_k(orc, k):
    """(L L^T)_ij = B_ij for every (i,j) in S: the defining property of IC(k)."""
    for prob, perm in small_problems() + grid_problems(orc):
        h, st = oracle_factor(orc, prob, perm, k)
        if st != 0:
            continue  # signed matrices may break down; checked elsewhere
        B = permuted_dense(prob, perm)
        L = h.factor_csr().toarray()
        R = L @ L.T - B
        lptr, lcol, _ = h.pattern()
        rows = np.repeat(np.arange(prob.n), np.diff(lptr))
        assert np.abs(R[rows, lcol]).max() <= 1e-13 * np.abs(B).max(), (prob.name, k)


def test_ic0_tridiagonal_exact(orc):
    """A tridiagonal matrix has no fill in natural order, so IC(0) = Cholesky."""
    for seed in range(5):
        prob = synth.tridiagonal_spd(40, seed)
        h, st = oracle_factor(orc, prob, None, 0)
        assert st == 0
        Lref = np.linalg.cholesky(prob.to_dense())
        assert np.abs(h.factor_csr().toarray() - Lref).max() <= 1e-14 * np.abs(Lref).max()
        assert h.nnz == 2 * prob.n - 1


def test_diagonal_matrix(orc):
    n = 17
    d = np.random.default_rng(5).uniform(0.5, 3.0, size=n)
    prob = synth.matrices._from_coo("diag", n, np.arange(n), np.arange(n), d, 0)
    for k in (0, 3):
        h, st = oracle_factor(orc, prob, None, k)
        assert st == 0 and h.nnz == n
        assert np.array_equal(h.values(), np.sqrt(d))


def test_mmatrix_never_breaks_down(orc):
    """IC(k) of an M-matrix exists for every pattern (Meijerink and van der Vorst)."""
    cases = [synth.poisson2d_5pt(16, 16), synth.diffusion3d_7pt(8, sigma=2.0, zscale=100.0, seed=5),
             synth.laplace3d_27pt(6), synth.random_spd(30, 0.2, 7, kind="mmatrix")]
    for prob in cases:
        if prob.grid is not None:
            perm = orc.nd_grid(*prob.grid, 1, 16)[0]
        else:
            perm = None
        for k in range(5):
            h, st = oracle_factor(orc, prob, perm, k)
            assert st == 0 and h.breakdown_row == -1, (prob.name, k)
            assert np.all(np.isfinite(h.values()))


def _read_golden_breakdown():
    lines = [ln for ln in open(os.path.join(GOLD, "ic0_breakdown_4x4.txt")) if not ln.startswith("#")]
    A = np.array([[float(x) for x in ln.split()] for ln in lines[:4]])
    piv = [Fraction(x) for x in lines[4].split()]
    row, last = lines[5].split()
    return A, piv, int(row), Fraction(last)


def test_breakdown_hand_computed(orc):
    A, piv, row, last = _read_golden_breakdown()
    assert np.linalg.eigvalsh(A).min() > 0  # SPD: the complete factor exists
    rows, cols = np.nonzero(A)
    prob = synth.matrices._from_coo("brk4", 4, rows, cols, A[rows, cols], 0)
    h, st = oracle_factor(orc, prob, None, 0)
    assert st == orc.ERR_BREAKDOWN and h.breakdown_row == row
    L = h.values()
    lptr, _, _ = h.pattern()
    for i, p in enumerate(piv):
        assert abs(L[lptr[i + 1] - 1] ** 2 - float(p)) <= 1e-14 * float(p)
    # the dropped fill (3,1) has level 1: IC(1) and complete fill both succeed
    for k in (1, 3):
        h1, st1 = oracle_factor(orc, prob, None, k)
        assert st1 == 0
    assert float(last) < 0


# --------------------------------------------------------------- symbolic pins

def brute_force_levels(n, adj):
    """lev[(i,j)], i > j: (edges - 1) of the shortest simple path i -> j whose interior
    vertices are all < j, found by enumerating every simple path (tiny n only)."""
    lev = {}
    for i in range(n):
        for j in range(i):
            best = None
            lim = j  # interior < min(i, j) = j
            allowed = [v for v in range(lim)]
            # enumerate interior sequences over allowed vertices (simple paths)
            for L in range(0, len(allowed) + 1):
                if best is not None and L + 1 > best:
                    break
                for seq in itertools.permutations(allowed, L):
                    path = (i,) + seq + (j,)
                    if all(adj[path[t]][path[t + 1]] for t in range(len(path) - 1)):
                        best = L + 1 if best is None else min(best, L + 1)
                        break
            if best is not None:
                lev[(i, j)] = best - 1
    return lev


@pytest.mark.parametrize("seed", range(6))
def test_symbolic_matches_fill_paths(orc, seed):
    rng = np.random.default_rng(100 + seed)
    n = 8
    density = [0.2, 0.3, 0.4][seed % 3]
    prob = synth.random_spd(n, density, 100 + seed, kind="mmatrix")
    A = prob.to_dense()
    adj = (A != 0) & ~np.eye(n, dtype=bool)
    truth = brute_force_levels(n, adj)
    for k in range(0, n):
        h = orc.OracleIC.from_problem(prob, None, k)
        lptr, lcol, llev = h.pattern()
        got = {}
        for i in range(n):
            for e in range(lptr[i], lptr[i + 1]):
                j = int(lcol[e])
                if j != i:
                    got[(i, j)] = int(llev[e])
            assert lcol[lptr[i + 1] - 1] == i
        want = {ij: l for ij, l in truth.items() if l <= k}
        assert got == want, (seed, k)
    del rng


def test_symbolic_patterns_nest_and_bound(orc):
    """S_0 = pattern(B); S_k is a subset of S_k+1; complete fill bounds every S_k."""
    prob = synth.laplace3d_27pt(6)
    perm = orc.nd_grid(6, 6, 6, 1, 16)[0]
    B = permuted_dense(prob, perm)
    prev = None
    sizes = []
    full = orc.OracleIC.from_problem(prob, perm, prob.n)
    fptr, fcol, _ = full.pattern()
    fullset = {(i, int(c)) for i in range(prob.n) for c in fcol[fptr[i]:fptr[i + 1]]}
    for k in range(6):
        h = orc.OracleIC.from_problem(prob, perm, k)
        lptr, lcol, _ = h.pattern()
        s = {(i, int(c)) for i in range(prob.n) for c in lcol[lptr[i]:lptr[i + 1]]}
        if k == 0:
            rows, cols = np.nonzero(np.tril(B))
            assert s == set(zip(rows.tolist(), cols.tolist()))
        if prev is not None:
            assert prev <= s
        assert s <= fullset
        sizes.append(len(s))
        prev = s
    assert sizes == sorted(sizes) and sizes[0] < sizes[2] < len(fullset)


# --------------------------------------------------------------- ND pins

def test_nd_hand_derived(orc):
    for ln in open(os.path.join(GOLD, "nd_small.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        head, tail = ln.split(":")
        nx, ny, nz, dof, leaf = map(int, head.split())
        want = [int(x) for x in tail.split()]
        perm, ranges = orc.nd_grid(nx, ny, nz, dof, leaf)
        assert perm.tolist() == want


def test_nd_is_permutation_and_separates(orc):
    """Every cut plane separates its halves: no 27-point edge joins the two halves."""
    nx, ny, nz = 9, 7, 5
    perm, ranges = orc.nd_grid(nx, ny, nz, 1, 20)
    assert sorted(perm.tolist()) == list(range(nx * ny * nz))
    assert ranges[0] == 0 and ranges[-1] == nx * ny * nz
    # In ND order every edge (u, v) joins a vertex to one in its own part or a later
    # part; a leaf never touches another leaf.  Leaves: parts whose vertices are not
    # a single plane of the grid spanning a cut -- test the weaker, exact property
    # that the complete factor has no fill between the two halves of the top cut.
    prob = synth.laplace3d_27pt(nx, ny, nz)
    h = orc.OracleIC.from_problem(prob, perm, prob.n)
    lptr, lcol, _ = h.pattern()
    iperm = np.empty_like(perm)
    iperm[perm] = np.arange(len(perm))
    x = perm % nx
    # top cut is along x (longest axis) at m = 4: low x<4 numbered first, then high x>4
    low = x < 4
    high = x > 4
    for i in range(prob.n):
        for c in lcol[lptr[i]:lptr[i + 1]]:
            assert not (low[i] and high[c]) and not (high[i] and low[c])


def test_nd_keep_mask(orc):
    """Eliminated dofs are skipped.  Leaf tests count kept rows only, so with
    leaf_rows = 1 (where a part of <= 1 kept row orders the same whether or not it is
    split further) the kept order is exactly the full order restricted."""
    nx, ny, nz, dof = 5, 4, 3, 3
    keep = np.ones(nx * ny * nz * dof, dtype=np.uint8)
    keep[::7] = 0
    perm_full, _ = orc.nd_grid(nx, ny, nz, dof, 1)
    perm_kept, _ = orc.nd_grid(nx, ny, nz, dof, 1, keep=keep)
    newidx = np.cumsum(keep) - 1
    want = [int(newidx[p]) for p in perm_full if keep[p]]
    assert perm_kept.tolist() == want


def _consecutive_independent_segments(rows, adjacent):
    """Fewest consecutive segments of `rows` with no two rows of a segment adjacent
    (greedy is optimal: a sub-run of an independent run is independent)."""
    segs, cur = 0, []
    for r in rows:
        if not cur or any(adjacent(r, q) for q in cur):
            segs += 1
            cur = []
        cur.append(r)
    return segs


@pytest.mark.parametrize("colours,reach", [(2, 1), (3, 2)])
def test_nd_coloured_separators(orc, colours, reach):
    """With C x C colour classes a separator plane of R rows becomes ceil(R/leaf_rows)
    even strips of its lexicographic order, each a part of its own, numbered as at
    most C*C runs, each an independent set of the plane's nodes at Chebyshev
    distance <= reach (reach 1: the 27-point stencil; C = 3 keeps nodes up to
    distance 2 apart), classes in ascending key order, rows ascending inside each;
    boxes keep their order and their part."""
    nx, ny, nz, leaf = 11, 9, 7, 20
    plain, r0 = orc.nd_grid(nx, ny, nz, 1, leaf)
    perm, r1 = orc.nd_grid(nx, ny, nz, 1, leaf, sep_colours=colours)
    assert set(r0.tolist()) <= set(r1.tolist())
    assert np.array_equal(orc.nd_grid(nx, ny, nz, 1, leaf, sep_colours=1)[0], plain)

    def xyz(v):
        return v % nx, (v // nx) % ny, v // (nx * ny)

    def adjacent(u, v):
        return max(abs(a - b) for a, b in zip(xyz(u), xyz(v))) <= reach

    planes = strips_total = 0
    lex_runs = []
    for a, b in zip(r0[:-1], r0[1:]):
        subs = r1[(r1 >= a) & (r1 <= b)].tolist()
        if len(subs) == 2 and perm[a:b].tolist() == plain[a:b].tolist():
            continue  # a box, or a plane that colouring leaves as it was
        planes += 1
        got_all = perm[a:b].tolist()
        const = [ax for ax in range(3) if len({xyz(v)[ax] for v in got_all}) == 1]
        assert const, "only separator planes are recoloured"
        rows = b - a
        m = -(-rows // leaf)
        assert subs == [a + rows * q // m for q in range(m + 1)]
        strips_total += m
        for lo, hi in zip(subs[:-1], subs[1:]):
            got, lex = perm[lo:hi].tolist(), plain[lo:hi].tolist()
            assert sorted(got) == sorted(lex)
            assert _consecutive_independent_segments(got, adjacent) <= colours * colours
            lex_runs.append(_consecutive_independent_segments(lex, adjacent))
            cls = [tuple(c % colours for i, c in enumerate(xyz(v)) if i != const[0]) for v in got]
            for k in set(cls):
                run = [v for v, c in zip(got, cls) if c == k]
                assert run == sorted(run)
            # classes in ascending (u mod C) + C (v mod C), u the lower-numbered free axis
            keys = [c[0] + colours * c[1] for c in cls]
            assert keys == sorted(keys)
    assert planes >= 3 and strips_total > planes
    # the lexicographic strips are not independent runs of that count
    assert max(lex_runs) > colours * colours


@pytest.mark.parametrize("colours,reach", [(2, 1), (3, 2)])
def test_nd_coloured_leaves(orc, colours, reach):
    """With C x C x C colour classes every leaf box is numbered as at most C^3 runs,
    each an independent set of nodes at Chebyshev distance <= reach (reach 1: the
    27-point stencil), classes in ascending (x mod C) + C (y mod C) + C^2 (z mod C),
    rows ascending inside each; the parts, and the separators' order, do not change."""
    nx, ny, nz, leaf = 12, 10, 8, 120
    plain, r0 = orc.nd_grid(nx, ny, nz, 1, leaf)
    perm, r1 = orc.nd_grid(nx, ny, nz, 1, leaf, leaf_colours=colours)
    assert np.array_equal(r0, r1)
    assert np.array_equal(orc.nd_grid(nx, ny, nz, 1, leaf, leaf_colours=1)[0], plain)

    def xyz(v):
        return v % nx, (v // nx) % ny, v // (nx * ny)

    def adjacent(u, v):
        return max(abs(a - b) for a, b in zip(xyz(u), xyz(v))) <= reach

    boxes = 0
    lex_runs = []
    for a, b in zip(r0[:-1], r0[1:]):
        got, lex = perm[a:b].tolist(), plain[a:b].tolist()
        assert sorted(got) == sorted(lex)
        if any(len({xyz(v)[ax] for v in lex}) == 1 for ax in range(3)) and b - a > 1:
            assert got == lex  # a separator plane keeps its lexicographic order
            continue
        boxes += 1
        assert _consecutive_independent_segments(got, adjacent) <= colours ** 3
        lex_runs.append(_consecutive_independent_segments(lex, adjacent))
        keys = [x % colours + colours * (y % colours) + colours * colours * (z % colours)
                for x, y, z in map(xyz, got)]
        assert keys == sorted(keys)
        for k in set(keys):
            run = [v for v, kk in zip(got, keys) if kk == k]
            assert run == sorted(run)
    assert boxes >= 4
    assert max(lex_runs) > colours ** 3


# --------------------------------------------------------------- apply / PCG pins

def test_apply_with_complete_factor_inverts(orc):
    prob = synth.laplace3d_27pt(5)
    perm = orc.nd_grid(5, 5, 5, 1, 10)[0]
    h, st = oracle_factor(orc, prob, perm, prob.n)
    assert st == 0
    r = np.random.default_rng(3).standard_normal(prob.n)
    z = h.apply(r)
    A = prob.scipy()
    assert np.abs(A @ z - r).max() <= 1e-12 * np.abs(r).max()
    b = synth.rhs(prob.n, 1)
    x, it, rel, st = orc.pcg(prob, b, h, tol=1e-10)
    assert st == 0 and it == 1 and rel <= 1e-10


def test_cg_iterations_grow_like_sqrt_kappa(orc):
    """Unpreconditioned CG on 2-D Poisson: doubling the grid side doubles sqrt(kappa);
    the iteration count should roughly double (plausibility, not an exact law)."""
    its = []
    for s in (32, 64):
        prob = synth.poisson2d_5pt(s, s)
        b = synth.rhs(prob.n, 1)
        x, it, rel, st = orc.pcg(prob, b, None, tol=1e-8)
        assert st == 0
        its.append(it)
    assert 1.5 <= its[1] / its[0] <= 2.5


def test_ick_preconditioner_reduces_iterations(orc):
    prob = synth.poisson2d_5pt(64, 64)
    perm = orc.nd_grid(64, 64, 1, 1, 256)[0]
    b = synth.rhs(prob.n, prob.seed)
    its = []
    for k in (None, 0, 1, 2):
        h = None
        if k is not None:
            h, st = oracle_factor(orc, prob, perm, k)
            assert st == 0
        x, it, rel, st = orc.pcg(prob, b, h, tol=1e-8)
        assert st == 0
        res = np.linalg.norm(prob.scipy() @ x - b) / np.linalg.norm(b)
        assert res <= 1.01e-8
        its.append(it)
    assert its[0] > its[1] > its[2] >= its[3]


def test_flop_count_closed_form(orc):
    """Dense SPD with complete fill: divides n(n-1)/2, sqrt n, and 2 flops for each of
    the sum_j (n-j-1)(n-j)/2 landing updates (pairs r <= c after pivot j)."""
    n = 9
    prob = synth.random_spd(n, 1.0, 2, kind="dense_spd")
    h, st = oracle_factor(orc, prob, None, n)
    assert st == 0
    upd = sum((n - j - 1) * (n - j) // 2 for j in range(n))
    assert h.flops == n * (n - 1) / 2 + n + 2 * upd


def test_generators_exactly_symmetric():
    """Every generated matrix is symmetric bit for bit, so reading either triangle of
    B = P^T A P gives the same values (the oracle reads the lower, the library the upper)."""
    probs = [synth.poisson2d_5pt(9, 7), synth.laplace3d_27pt(6), synth.elasticity3d_q1(4, seed=4005),
             synth.diffusion3d_7pt(7, sigma=2.0, zscale=100.0, seed=5),
             synth.random_spd(30, 0.2, 1, kind="signed"), synth.tridiagonal_spd(20, 3)]
    probs += synth.diffusion_batch(3, 4, 6, seed=3000)
    for p in probs:
        assert synth.is_exactly_symmetric(p), p.name
