"""Seeded SPD test matrices shaped like the paper's workloads.

The paper evaluates on SuiteSparse matrices (Table 1 of Section 4): four
low-degree matrices with nnz/n of 5 to 7 (ecology2, G3_circuit,
parabolic_fem, thermal2) and two structural matrices with nnz/n of 53 to 72
(bmwcra_1, pwtk).  Those files are not available, so the generators below
stand in for them: 5- and 7-point diffusion stencils for the low-degree
family, a 27-point Laplacian and trilinear-hex elasticity for the structural
family.

Every matrix is returned as a full symmetric CSR pattern on a structured
grid with the node index ``x + nx*(y + ny*z)`` (x fastest) and, for
``dof > 1``, the dof index ``dof*node + component``.  Columns are sorted in
every row, ``rowptr`` is int64, ``colind`` int32 and the values float64.
Randomness comes only from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    name: str
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    vals: np.ndarray
    grid: tuple | None = None      # (nx, ny, nz) grid nodes
    dof: int = 1
    keep: np.ndarray | None = None  # uint8 over grid dofs; None: all kept
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            a[i, self.colind[s:e]] = self.vals[s:e]
        return a

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colind, self.rowptr), shape=(self.n, self.n))


def rhs(n: int, seed: int) -> np.ndarray:
    """Right-hand side b ~ N(0, 1) drawn from ``default_rng(seed + 7)``."""
    return np.random.default_rng(seed + 7).standard_normal(n)


def _coords(nx, ny, nz):
    idx = np.arange(nx * ny * nz, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    return x, y, z


def _offsets(radius_box: bool):
    """Stencil offsets sorted by (dz, dy, dx) so that columns come out sorted."""
    if radius_box:
        offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    else:
        offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    return offs


def _stencil_csr(nx, ny, nz, offs, values):
    """values[t] is an (n,) array (or scalar) for offset t; invalid neighbours dropped."""
    n = nx * ny * nz
    x, y, z = _coords(nx, ny, nz)
    m = len(offs)
    cols = np.empty((n, m), dtype=np.int64)
    vals = np.empty((n, m), dtype=np.float64)
    mask = np.empty((n, m), dtype=bool)
    for t, (dx, dy, dz) in enumerate(offs):
        xx, yy, zz = x + dx, y + dy, z + dz
        valid = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        cols[:, t] = xx + nx * (yy + ny * zz)
        vals[:, t] = values[t]
        mask[:, t] = valid
    counts = mask.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, cols[mask].astype(np.int32), vals[mask].astype(np.float64)


def poisson2d_5pt(nx: int = 64, ny: int = 64) -> Problem:
    """5-point Laplacian on an nx-by-ny grid with Dirichlet boundary (diag 4, off -1)."""
    offs = [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    vals = [-1.0 if o != (0, 0, 0) else 4.0 for o in offs]
    rp, ci, va = _stencil_csr(nx, ny, 1, offs, vals)
    return Problem(f"poisson2d_5pt_{nx}x{ny}", nx * ny, rp, ci, va, grid=(nx, ny, 1), seed=1000)


def laplace3d_27pt(nx: int = 96, ny: int | None = None, nz: int | None = None) -> Problem:
    """27-point constant Laplacian (diag 26, all 26 neighbours -1), Dirichlet truncation."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    offs = _offsets(True)
    vals = [26.0 if o == (0, 0, 0) else -1.0 for o in offs]
    rp, ci, va = _stencil_csr(nx, ny, nz, offs, vals)
    return Problem(f"laplace3d_27pt_{nx}x{ny}x{nz}", nx * ny * nz, rp, ci, va,
                   grid=(nx, ny, nz), seed=2000)


def diffusion3d_7pt(nx: int, ny: int | None = None, nz: int | None = None, *, sigma: float = 1.0,
                    zscale: float = 1.0, seed: int = 0) -> Problem:
    """7-point variable-coefficient diffusion with node conductivities kappa ~ LogNormal(0, sigma).

    The coefficient of an interior face is the harmonic mean of its two nodes' kappa; a
    Dirichlet boundary face uses the node's own kappa.  Faces normal to z are multiplied by
    ``zscale`` (anisotropy).  The diagonal is the sum of the six face coefficients, so the
    matrix is a symmetric M-matrix, strictly diagonally dominant on boundary rows.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    n = nx * ny * nz
    rng = np.random.default_rng(seed)
    kappa = rng.lognormal(mean=0.0, sigma=sigma, size=n)
    x, y, z = _coords(nx, ny, nz)
    offs = _offsets(False)
    diag = np.zeros(n)
    values = []
    for (dx, dy, dz) in offs:
        if (dx, dy, dz) == (0, 0, 0):
            values.append(None)
            continue
        xx, yy, zz = x + dx, y + dy, z + dz
        valid = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        j = np.where(valid, xx + nx * (yy + ny * zz), 0)
        kj = kappa[j]
        # 2*(ki*kj)/(ki+kj): both products and the sum commute, so the face
        # coefficient is bitwise the same from either side (exact symmetry)
        c = np.where(valid, 2.0 * (kappa * kj) / (kappa + kj), kappa)
        if dz != 0:
            c = c * zscale
        diag += c
        values.append(-c)
    values[offs.index((0, 0, 0))] = diag
    rp, ci, va = _stencil_csr(nx, ny, nz, offs, values)
    return Problem(f"diffusion3d_7pt_{nx}x{ny}x{nz}_s{sigma:g}_z{zscale:g}", n, rp, ci, va,
                   grid=(nx, ny, nz), seed=seed, meta={"sigma": sigma, "zscale": zscale})


def _hex_stiffness(h: float, E: float, nu: float) -> np.ndarray:
    """24x24 stiffness of a trilinear cube of side h, 2x2x2 Gauss, isotropic linear elasticity."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    g = 1.0 / np.sqrt(3.0)
    signs = np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1]
                      for a in range(8)], dtype=np.float64)
    K = np.zeros((24, 24))
    for xi in (-g, g):
        for eta in (-g, g):
            for zeta in (-g, g):
                sx, sy, sz = signs[:, 0], signs[:, 1], signs[:, 2]
                dxi = 0.125 * sx * (1 + eta * sy) * (1 + zeta * sz)
                deta = 0.125 * sy * (1 + xi * sx) * (1 + zeta * sz)
                dzeta = 0.125 * sz * (1 + xi * sx) * (1 + eta * sy)
                dN = np.stack([dxi, deta, dzeta]) * (2.0 / h)  # (3, 8)
                B = np.zeros((6, 24))
                for a in range(8):
                    nx_, ny_, nz_ = dN[:, a]
                    c = 3 * a
                    B[0, c] = nx_
                    B[1, c + 1] = ny_
                    B[2, c + 2] = nz_
                    B[3, c] = ny_
                    B[3, c + 1] = nx_
                    B[4, c + 1] = nz_
                    B[4, c + 2] = ny_
                    B[5, c] = nz_
                    B[5, c + 2] = nx_
                K += B.T @ D @ B * (h / 2) ** 3
    return K


def elasticity3d_q1(ne: int = 48, *, nu: float | None = None, E: float = 1.0, seed: int = 4000,
                    clamp: bool = True) -> Problem:
    """Trilinear-hex linear elasticity on an ne^3 element cube of side 1, 3 dof per node.

    Poisson ratio nu ~ U[0.25, 0.45] from ``default_rng(seed)`` unless given.  The face x = 0
    is clamped: its dofs are eliminated (rows and columns removed).  Node-major dof order;
    the structural pattern keeps the full 3x3 block of every pair of nodes sharing an
    element.  The result is SPD but not an M-matrix.
    """
    if nu is None:
        nu = float(np.random.default_rng(seed).uniform(0.25, 0.45))
    nn = ne + 1
    nnode = nn ** 3
    Ke = _hex_stiffness(1.0 / ne, E, nu)
    Kb = Ke.reshape(8, 3, 8, 3).transpose(0, 2, 1, 3)  # [la, lb, a, b]
    x, y, z = _coords(nn, nn, nn)
    offs = _offsets(True)
    blocks = np.zeros((nnode, 27, 3, 3))
    for t, (dx, dy, dz) in enumerate(offs):
        for cz in (-1, 0):
            for cy in (-1, 0):
                for cx in (-1, 0):
                    li = (-cx, -cy, -cz)
                    lj = (-cx + dx, -cy + dy, -cz + dz)
                    if min(lj) < 0 or max(lj) > 1:
                        continue
                    ex, ey, ez = x + cx, y + cy, z + cz
                    ok = (ex >= 0) & (ex < ne) & (ey >= 0) & (ey < ne) & (ez >= 0) & (ez < ne)
                    la = li[0] + 2 * li[1] + 4 * li[2]
                    lb = lj[0] + 2 * lj[1] + 4 * lj[2]
                    blocks[ok, t] += Kb[la, lb]
    # rows (node, a), columns (offset t, b): sorted since offsets are sorted and b innermost
    cols = np.empty((nnode, 27), dtype=np.int64)
    valid = np.empty((nnode, 27), dtype=bool)
    for t, (dx, dy, dz) in enumerate(offs):
        xx, yy, zz = x + dx, y + dy, z + dz
        valid[:, t] = (xx >= 0) & (xx < nn) & (yy >= 0) & (yy < nn) & (zz >= 0) & (zz < nn)
        cols[:, t] = xx + nn * (yy + nn * zz)
    n_full = 3 * nnode
    dcols = (3 * cols[:, None, :, None] + np.arange(3)[None, None, None, :])  # (node,1,27,3)
    dcols = np.broadcast_to(dcols, (nnode, 3, 27, 3))
    dvalid = np.broadcast_to(valid[:, None, :, None], (nnode, 3, 27, 3))
    dvals = blocks.transpose(0, 2, 1, 3)  # (node, a, t, b)
    keep = np.ones(n_full, dtype=np.uint8)
    if clamp:
        keep[np.repeat(x == 0, 3)] = 0
    newidx = np.cumsum(keep, dtype=np.int64) - 1
    newidx[keep == 0] = -1
    rowkeep = keep.reshape(nnode, 3).astype(bool)
    safe = np.where(dvalid, dcols, 0)
    m = dvalid & (keep[safe] == 1) & rowkeep[:, :, None, None]
    m2 = m.reshape(n_full, 81)
    counts = m2.sum(axis=1)[keep == 1]
    n = int(keep.sum())
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = newidx[safe.reshape(n_full, 81)[m2]].astype(np.int32)
    vals = np.ascontiguousarray(dvals).reshape(n_full, 81)[m2].astype(np.float64)
    vals = _symmetrize(n, rowptr, colind, vals)
    return Problem(f"elasticity3d_q1_{ne}^3_nu{nu:.4f}", n, rowptr, colind, vals,
                   grid=(nn, nn, nn), dof=3, keep=keep, seed=seed, meta={"nu": nu, "E": E})


def _symmetrize(n, rowptr, colind, vals):
    """(A + A^T) / 2 on a symmetric pattern: a + b commutes, so the result is exactly
    symmetric even where the assembly summed element contributions in different orders."""
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    key = rows * n + colind
    tkey = colind.astype(np.int64) * n + rows
    order = np.argsort(key)
    tpos = order[np.searchsorted(key[order], tkey)]
    assert np.array_equal(key[tpos], tkey), "pattern is not symmetric"
    return (vals + vals[tpos]) * 0.5


def is_exactly_symmetric(prob) -> bool:
    """True when the pattern is symmetric and A_ij == A_ji bit for bit."""
    n = prob.n
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(prob.rowptr))
    key = rows * n + prob.colind
    tkey = prob.colind.astype(np.int64) * n + rows
    order = np.argsort(key)
    idx = np.searchsorted(key[order], tkey)
    if np.any(idx >= len(key)):
        return False
    tpos = order[idx]
    return bool(np.array_equal(key[tpos], tkey) and np.array_equal(prob.vals, prob.vals[tpos]))


def diffusion_batch(count: int = 512, smin: int = 8, smax: int = 32, *, sigma: float = 1.0,
                    seed: int = 3000) -> list[Problem]:
    """``count`` independent 7-point diffusion cubes with side s ~ U{smin..smax}."""
    sides = np.random.default_rng(seed).integers(smin, smax + 1, size=count)
    return [diffusion3d_7pt(int(s), sigma=sigma, seed=seed + 1 + i) for i, s in enumerate(sides)]


def tridiagonal_spd(n: int, seed: int = 0, *, sign_mix: bool = True) -> Problem:
    """Random strictly diagonally dominant tridiagonal SPD matrix."""
    rng = np.random.default_rng(seed)
    off = rng.uniform(0.1, 1.0, size=n - 1)
    if sign_mix:
        off *= rng.choice([-1.0, 1.0], size=n - 1)
    diag = np.zeros(n)
    diag[:-1] += np.abs(off)
    diag[1:] += np.abs(off)
    diag += rng.uniform(0.1, 1.0, size=n)
    rows, cols, vals = [], [], []
    for i in range(n):
        if i > 0:
            rows.append(i); cols.append(i - 1); vals.append(off[i - 1])
        rows.append(i); cols.append(i); vals.append(diag[i])
        if i < n - 1:
            rows.append(i); cols.append(i + 1); vals.append(off[i])
    return _from_coo(f"tridiag_{n}", n, rows, cols, vals, seed)


def _from_coo(name, n, rows, cols, vals, seed, grid=None):
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return Problem(name, n, rowptr, cols.astype(np.int32), vals, grid=grid, seed=seed)


def random_spd(n: int, density: float = 0.2, seed: int = 0, *, kind: str = "mmatrix") -> Problem:
    """Small random sparse SPD matrix with a random symmetric pattern.

    kind = "mmatrix": negative off-diagonals, strictly diagonally dominant (an M-matrix);
    kind = "signed": off-diagonals of random sign, strictly diagonally dominant;
    kind = "dense_spd": every entry present, A = R^T R + n I with R ~ N(0,1).
    """
    rng = np.random.default_rng(seed)
    if kind == "dense_spd":
        R = rng.standard_normal((n, n))
        A = R.T @ R + n * np.eye(n)
        rows, cols = np.nonzero(np.ones((n, n)))
        return _from_coo(f"dense_spd_{n}", n, rows, cols, A[rows, cols], seed)
    upper = np.triu(rng.random((n, n)) < density, 1)
    off = np.zeros((n, n))
    mag = rng.uniform(0.1, 1.0, size=(n, n))
    if kind == "mmatrix":
        off[upper] = -mag[upper]
    elif kind == "signed":
        off[upper] = mag[upper] * rng.choice([-1.0, 1.0], size=(n, n))[upper]
    else:
        raise ValueError(kind)
    off = off + off.T
    A = off.copy()
    A[np.arange(n), np.arange(n)] = np.abs(off).sum(axis=1) + rng.uniform(0.1, 1.0, size=n)
    mask = (A != 0)
    rows, cols = np.nonzero(mask)
    return _from_coo(f"random_{kind}_{n}_{seed}", n, rows, cols, A[rows, cols], seed)


def config_problem(config: int, *, scale: int | None = None, instance: int = 0):
    """The five workload shapes (C1..C5); ``scale`` shrinks the grid side for quick tests.

    C1: 2-D 5-point Poisson 64x64.            C2: 27-point Laplacian 96^3.
    C3: batch of 512 7-point diffusion cubes.  C4: Q1 elasticity 48^3 elements.
    C5: 7-point diffusion 160^3, sigma 2, z-faces x100.
    Seeds are 1000*config + instance.
    """
    seed = 1000 * config + instance
    if config == 1:
        s = scale or 64
        p = poisson2d_5pt(s, s)
    elif config == 2:
        p = laplace3d_27pt(scale or 96)
    elif config == 3:
        return diffusion_batch(512 if scale is None else scale, seed=seed)
    elif config == 4:
        p = elasticity3d_q1(scale or 48, seed=seed)
    elif config == 5:
        p = diffusion3d_7pt(scale or 160, sigma=2.0, zscale=100.0, seed=seed)
    else:
        raise ValueError(config)
    p.seed = seed
    return p
