"""Python face of the CPU oracle (oracle.c) -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py may
import this package.  It loads ``oracle/_build/liboracle.so`` (built by
``oracle.build.build()`` with plain gcc, ``-ffp-contract=off``) and shares no code
with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build, lib_path

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_nd_grid.restype = C.c_int64
        L.orc_nd_grid.argtypes = [C.c_int] * 7 + [P, P, P, P]
        L.orc_ic_create.restype = P
        L.orc_ic_create.argtypes = [C.c_int64, P, P, P, C.c_int, P]
        L.orc_ic_free.argtypes = [P]
        L.orc_ic_nnz.restype = C.c_int64
        L.orc_ic_nnz.argtypes = [P]
        L.orc_ic_flops.restype = C.c_double
        L.orc_ic_flops.argtypes = [P]
        L.orc_ic_pattern.argtypes = [P, P, P, P]
        L.orc_ic_values.argtypes = [P, P]
        L.orc_ic_numeric.restype = C.c_int
        L.orc_ic_numeric.argtypes = [P, P, C.c_double, P]
        L.orc_ic_apply.restype = C.c_int
        L.orc_ic_apply.argtypes = [P, P, P]
        L.orc_pcg.restype = C.c_int
        L.orc_pcg.argtypes = [P, C.c_int64, P, P, P, P, P, C.c_double, C.c_int, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


OK, ERR_ARG, ERR_BREAKDOWN, ERR_NOMEM, ERR_NOCONV = 0, 1, 3, 6, 7


def nd_grid(nx, ny, nz, dof=1, leaf_rows=64, keep=None, sep_colours=0, leaf_colours=0):
    """Geometric nested dissection: returns (perm, ranges); perm[new] = old.
    sep_colours >= 2 cuts each separator plane into strips sorted by their nodes' colour
    key; leaf_colours >= 2 sorts each leaf box by its nodes' 3D colour key."""
    L = _load()
    nfull = nx * ny * nz * dof
    perm = np.empty(nfull, dtype=np.int32)
    ranges = np.empty(nfull + 1, dtype=np.int64)
    nr = np.zeros(1, dtype=np.int64)
    keep_a = None if keep is None else np.ascontiguousarray(keep, dtype=np.uint8)
    n = L.orc_nd_grid(nx, ny, nz, dof, leaf_rows, sep_colours, leaf_colours, _p(keep_a), _p(perm), _p(ranges),
                      _p(nr))
    if n < 0:
        raise ValueError("orc_nd_grid: bad arguments")
    return perm[:n].copy(), ranges[: nr[0] + 1].copy()


class OracleIC:
    """Permuted matrix B = P^T A P with its level-k pattern; numeric IC(k) on demand."""

    def __init__(self, n, rowptr, colind, perm, k):
        L = _load()
        self.n = int(n)
        self.k = int(k)
        self._rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self._colind = np.ascontiguousarray(colind, dtype=np.int32)
        self._perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
        st = np.zeros(1, dtype=np.int32)
        self._h = L.orc_ic_create(self.n, _p(self._rowptr), _p(self._colind), _p(self._perm),
                                  self.k, _p(st))
        if not self._h:
            raise ValueError(f"orc_ic_create failed with status {int(st[0])}")
        self.nnz = int(L.orc_ic_nnz(self._h))
        self.status = None
        self.breakdown_row = -1

    @classmethod
    def from_problem(cls, prob, perm, k):
        return cls(prob.n, prob.rowptr, prob.colind, perm, k)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_ic_free(self._h)
            self._h = None

    def pattern(self):
        """(lptr, lcol, llev) of L: lower CSR, rows sorted, diagonal last."""
        lptr = np.empty(self.n + 1, dtype=np.int64)
        lcol = np.empty(self.nnz, dtype=np.int32)
        llev = np.empty(self.nnz, dtype=np.int32)
        _load().orc_ic_pattern(self._h, _p(lptr), _p(lcol), _p(llev))
        return lptr, lcol, llev

    def numeric(self, vals, shift_alpha=0.0):
        v = np.ascontiguousarray(vals, dtype=np.float64)
        brk = np.zeros(1, dtype=np.int64)
        self.status = int(_load().orc_ic_numeric(self._h, _p(v), float(shift_alpha), _p(brk)))
        self.breakdown_row = int(brk[0])
        return self.status

    @property
    def flops(self):
        return float(_load().orc_ic_flops(self._h))

    def values(self):
        out = np.empty(self.nnz, dtype=np.float64)
        _load().orc_ic_values(self._h, _p(out))
        return out

    def factor_csr(self):
        """scipy CSR of L (permuted order)."""
        import scipy.sparse as sp
        lptr, lcol, _ = self.pattern()
        return sp.csr_matrix((self.values(), lcol, lptr), shape=(self.n, self.n))

    def apply(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty_like(r)
        st = _load().orc_ic_apply(self._h, _p(r), _p(z))
        if st:
            raise RuntimeError(f"orc_ic_apply status {st}")
        return z


def pcg(prob, b, ic=None, tol=1e-8, maxit=10000):
    """Textbook PCG with M = L L^T from ``ic`` (None: M = I).  Returns (x, iters, relres, status)."""
    L = _load()
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty_like(b)
    it = np.zeros(1, dtype=np.int32)
    rel = np.zeros(1, dtype=np.float64)
    rp = np.ascontiguousarray(prob.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(prob.colind, dtype=np.int32)
    av = np.ascontiguousarray(prob.vals, dtype=np.float64)
    st = L.orc_pcg(ic._h if ic is not None else None, prob.n, _p(rp), _p(ci), _p(av), _p(b), _p(x),
                   float(tol), int(maxit), _p(it), _p(rel))
    return x, int(it[0]), float(rel[0]), int(st)
