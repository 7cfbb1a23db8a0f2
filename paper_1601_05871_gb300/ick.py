"""Thin ctypes binding of libick.so (include/ick.h): the same names, argument
marshalling only.  Device arrays are torch CUDA tensors (their data_ptr() is passed
through); host arrays are numpy arrays.  Every compute step runs in the library's
CUDA kernels: when the library is not built, loading it raises instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import lib_path

IC_OK, IC_ERR_ARG, IC_ERR_PATTERN, IC_ERR_BREAKDOWN, IC_ERR_TIMEOUT = 0, 1, 2, 3, 4
IC_ERR_CUDA, IC_ERR_NOMEM, IC_ERR_NOCONV, IC_ERR_STATE = 5, 6, 7, 8
IC_F64, IC_F32 = 0, 1
TASK_NAMES = ("Chol", "Trsm", "Herk", "Gemm")

_lib = None


class IckError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class ic_csr_pattern(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p)]


class ic_opts(C.Structure):
    _fields_ = [("block_rows", C.c_int), ("dtype", C.c_int), ("warps_per_cta", C.c_int),
                ("rows_per_item", C.c_int), ("timeout_s", C.c_double), ("shift_alpha", C.c_double),
                ("exact", C.c_int), ("threads", C.c_int), ("host_only", C.c_int),
                ("solve_ctas_per_sm", C.c_int), ("solve_lanes", C.c_int), ("solve_mode", C.c_int),
                ("reserved", C.c_int * 2)]


class ic_stats_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz_a", C.c_int64), ("nnz_l", C.c_int64), ("nranges", C.c_int64),
                ("nblocks", C.c_int64), ("ntasks", C.c_int64), ("ntasks_type", C.c_int64 * 4),
                ("nitems", C.c_int64), ("critical_path", C.c_int64), ("max_level", C.c_int64),
                ("flops", C.c_double), ("bytes", C.c_double), ("symbolic_s", C.c_double),
                ("grid_ctas", C.c_int64), ("solve_depth", C.c_int64 * 2), ("warps_per_cta", C.c_int64),
                ("rows_per_item", C.c_int64), ("nsplit", C.c_int64)]


def load():
    """Load libick.so; raises when it is missing (build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libick.so is not built ({path}); run paper_1601_05871_gb300.build.build()")
    L = C.CDLL(path)
    P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
    sig = {
        "ic_nd_grid": (I, [I, I, I, I, I, I, I, P, P, P, P, P]),
        "ic_symbolic": (I, [P, I, P, P, I64, P, P]),
        "ic_numeric": (I, [P, P, P, P]),
        "ic_apply": (I, [P, P, P, P]),
        "ic_apply_status": (I, [P, P]),
        "ic_apply_static": (I, [P, P, P, P]),
        "ic_apply_static_status": (I, [P]),
        "pcg_solve": (I, [P, P, P, P, D, I, P, P, P]),
        "ic_get_factor": (I, [P, P, P, P, P]),
        "ic_stats": (I, [P, P]),
        "ic_get_tasks": (I, [P, P, P, P, P, P, P, P, P]),
        "ic_block_dag": (I, [I64, P, P, P, P, P, P, P, P, P, P]),
        "ic_get_task_targets": (I, [P, I64, P, P]),
        "ic_get_upper": (I, [P, P, P, P, P, P]),
        "ic_get_blocks": (I, [P, P, P, P]),
        "ic_get_solve_tasks": (I, [P, I, P, P, P, P, P, P, P, P, P]),
        "ic_set_timing": (I, [P, I]),
        "ic_reset_timing": (I, [P]),
        "ic_get_timing": (I, [P, P]),
        "ic_fma_peak": (I, [I, P, P]),
        "ic_test_hold_task": (I, [P, I64, I]),
        "ic_test_hold_solve_task": (I, [P, I, I64, I]),
        "ic_symbolic_batch": (I, [I64, P, I, P, P, P, P, P]),
        "ic_batch_info": (I, [P, P, P]),
        "pcg_solve_batch": (I, [P, P, P, P, D, I, P, P, P]),
        "ic_numeric_async": (I, [P, P, P]),
        "ic_numeric_status": (I, [P, P]),
        "ic_autotune": (I, [I64, P, I, P, P, P, P, P, I, P, P, P]),
        "ic_set_trace": (I, [P, I]),
        "ic_get_trace": (I, [P, P]),
        "ic_get_solve_trace": (I, [P, I, P]),
        "ic_get_solve_entries": (I, [P, I, P, P, P]),
        "ic_get_split_layout": (I, [P, P, P, P, P]),
        "ic_get_claim_order": (I, [P, P, P]),
        "ic_shift_features": (I, [P, P, D, P, P]),
        "ic_numeric_shifted": (I, [P, P, D, D, I, P, P, P]),
        "ic_mlp_n_params": (I, []),
        "ic_mlp_create": (I, [P, P]),
        "ic_mlp_set_params": (I, [P, P]),
        "ic_mlp_get_params": (I, [P, P]),
        "ic_mlp_set_scaling": (I, [P, P, P]),
        "ic_mlp_get_scaling": (I, [P, P, P]),
        "ic_mlp_forward": (I, [P, P, I64, P, P]),
        "ic_mlp_gradient": (I, [P, P, P, I64, P, P, P]),
        "ic_mlp_train_step": (I, [P, P, P, I64, C.c_float, P, P]),
        "ic_mlp_predict_shift": (I, [P, P, P, P]),
        "ic_mlp_destroy": (None, [P]),
        "ic_destroy": (None, [P]),
        "ic_strerror": (C.c_char_p, [I]),
        "ic_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def declared_symbols():
    """Names of the functions include/ick.h declares (parsed from the header text)."""
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ick.h")
    text = open(hdr).read()
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*((?:ic|pcg)_\w+)\s*\(", text, re.M)
    return sorted(set(names))


def _p(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())  # torch tensor


def _check(st):
    if st != IC_OK:
        L = load()
        raise IckError(st, f"{L.ic_strerror(st).decode()}: {L.ic_last_error().decode()}")


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def ic_nd_grid(nx, ny, nz, dof=1, leaf_rows=4096, keep=None, sep_colours=0, leaf_colours=0):
    """Geometric nested dissection; returns (perm, ranges) with perm[new] = old.
    sep_colours >= 2 numbers separator planes in block-sized strips, each colour class
    by colour class; leaf_colours >= 2 numbers each leaf box colour class by class."""
    L = load()
    nfull = nx * ny * nz * dof
    perm = np.empty(nfull, dtype=np.int32)
    ranges = np.empty(nfull + 1, dtype=np.int64)
    nr = np.zeros(1, dtype=np.int64)
    n = np.zeros(1, dtype=np.int64)
    keep_a = None if keep is None else np.ascontiguousarray(keep, dtype=np.uint8)
    _check(L.ic_nd_grid(nx, ny, nz, dof, leaf_rows, sep_colours, leaf_colours, _p(keep_a), _p(perm),
                        _p(ranges), _p(nr), _p(n)))
    return perm[: n[0]].copy(), ranges[: nr[0] + 1].copy()


class Handle:
    """Owns an ic_handle; ic_destroy runs when the object is collected."""

    def __init__(self, ptr, n, nnz_a):
        self._h = ptr
        self.n = n
        self.nnz_a = nnz_a

    @property
    def ptr(self):
        return self._h

    def close(self):
        if self._h:
            load().ic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # convenience methods mirroring the module functions
    def numeric(self, values, stream=None):
        return ic_numeric(self, values, stream)

    def apply(self, r, z, stream=None):
        return ic_apply(self, r, z, stream)

    def pcg(self, A_vals, b, x, tol=1e-8, maxit=10000, stream=None):
        return pcg_solve(self, A_vals, b, x, tol, maxit, stream)

    def factor(self, values=True):
        return ic_get_factor(self, values)

    def stats(self):
        return ic_stats(self)


def ic_symbolic(rowptr, colind, k, perm=None, ranges=None, *, block_rows=0, dtype=IC_F64,
                warps_per_cta=0, rows_per_item=0, timeout_s=0.0, shift_alpha=0.0, exact=0,
                threads=0, host_only=0, solve_ctas_per_sm=0, solve_lanes=0, solve_mode=0):
    L = load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    n = len(rowptr) - 1
    pat = ic_csr_pattern(n, _p(rowptr), _p(colind))
    o = ic_opts(block_rows, dtype, warps_per_cta, rows_per_item, timeout_s, shift_alpha, exact, threads,
                host_only, solve_ctas_per_sm, solve_lanes, solve_mode)
    perm_a = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    ranges_a = None if ranges is None else np.ascontiguousarray(ranges, dtype=np.int64)
    nr = 0 if ranges_a is None else len(ranges_a) - 1
    out = C.c_void_p()
    _check(L.ic_symbolic(C.byref(pat), int(k), _p(perm_a), _p(ranges_a), nr, C.byref(o), C.byref(out)))
    return Handle(out.value, n, int(rowptr[-1]))


def ic_numeric(h, values, stream=None):
    """Numeric IC(k); values: CUDA float64 tensor in A's CSR order.  Returns -1, or raises
    IckError (status IC_ERR_BREAKDOWN carries .row)."""
    L = load()
    brk = np.zeros(1, dtype=np.int64)
    st = L.ic_numeric(h.ptr, _p(values), _stream(stream), _p(brk))
    if st == IC_ERR_BREAKDOWN:
        e = IckError(st, f"breakdown at row {int(brk[0])}")
        e.row = int(brk[0])
        raise e
    _check(st)
    return -1


def ic_apply(h, r, z, stream=None):
    _check(load().ic_apply(h.ptr, _p(r), _p(z), _stream(stream)))


def ic_apply_status(h, stream=None):
    """Raises IckError(IC_ERR_TIMEOUT) if a solve wait of an earlier ic_apply expired
    (synchronises the stream; clears the record)."""
    _check(load().ic_apply_status(h.ptr, _stream(stream)))


def ic_apply_static_status(stream=None):
    """Raises IckError(IC_ERR_TIMEOUT) if a solve wait of an earlier ic_apply_static on
    the current device expired (synchronises the stream; clears the record)."""
    _check(load().ic_apply_static_status(_stream(stream)))


def ic_apply_static(h, r, z, stream=None):
    """ic_apply without any allocation: scratch in the library's static device array
    (at most 1,048,576 rows; calls must not overlap on the GPU)."""
    _check(load().ic_apply_static(h.ptr, _p(r), _p(z), _stream(stream)))


def pcg_solve(h, A_vals, b, x, tol=1e-8, maxit=10000, stream=None, raise_noconv=True):
    """Returns (iters, relres); x (CUDA float64) receives the solution."""
    it = np.zeros(1, dtype=np.int32)
    rel = np.zeros(1, dtype=np.float64)
    st = load().pcg_solve(h.ptr, _p(A_vals), _p(b), _p(x), float(tol), int(maxit), _p(it), _p(rel),
                          _stream(stream))
    if st != IC_ERR_NOCONV or raise_noconv:
        _check(st)
    return int(it[0]), float(rel[0])


def ic_stats(h):
    s = ic_stats_t()
    _check(load().ic_stats(h.ptr, C.byref(s)))
    d = {f: getattr(s, f) for f, _ in s._fields_}
    d["ntasks_type"] = list(s.ntasks_type)
    d["solve_depth"] = list(s.solve_depth)
    return d


def ic_get_factor(h, values=True):
    """(rowptr, colind, vals or None, levels) of L in lower CSR, permuted order."""
    st = ic_stats(h)
    n, nnz = st["n"], st["nnz_l"]
    rp = np.empty(n + 1, dtype=np.int64)
    ci = np.empty(nnz, dtype=np.int32)
    lv = np.empty(nnz, dtype=np.int32)
    va = np.empty(nnz, dtype=np.float64) if values else None
    _check(load().ic_get_factor(h.ptr, _p(rp), _p(ci), _p(va), _p(lv)))
    return rp, ci, va, lv


def _dag_out(call):
    nt = np.zeros(1, dtype=np.int64)
    npr = np.zeros(1, dtype=np.int64)
    _check(call(None, None, None, None, None, None, _p(nt), _p(npr)))
    t = int(nt[0])
    arr = [np.empty(t, dtype=np.int32) for _ in range(4)]
    pp = np.empty(t + 1, dtype=np.int64)
    pr = np.empty(max(1, int(npr[0])), dtype=np.int32)
    _check(call(*[_p(a) for a in arr], _p(pp), _p(pr), _p(nt), _p(npr)))
    return {"type": arr[0], "k": arr[1], "i": arr[2], "j": arr[3], "pred_ptr": pp,
            "pred": pr[: int(npr[0])]}


def ic_get_tasks(h):
    L = load()
    return _dag_out(lambda *a: L.ic_get_tasks(h.ptr, *a))


def ic_block_dag(bptr, bcol):
    L = load()
    bptr = np.ascontiguousarray(bptr, dtype=np.int64)
    bcol = np.ascontiguousarray(bcol, dtype=np.int32)
    nb = len(bptr) - 1
    return _dag_out(lambda *a: L.ic_block_dag(nb, _p(bptr), _p(bcol), *a))


def ic_get_task_targets(h, t):
    L = load()
    cnt = np.zeros(1, dtype=np.int64)
    _check(L.ic_get_task_targets(h.ptr, int(t), None, _p(cnt)))
    out = np.empty((int(cnt[0]), 5), dtype=np.int32)
    _check(L.ic_get_task_targets(h.ptr, int(t), _p(out), _p(cnt)))
    return out


def ic_get_upper(h):
    st = ic_stats(h)
    n, nnz = st["n"], st["nnz_l"]
    urp = np.empty(n + 1, dtype=np.int64)
    ucol = np.empty(nnz, dtype=np.int32)
    cptr = np.empty(n + 1, dtype=np.int64)
    cp = np.empty(max(1, nnz - n), dtype=np.int32)
    cpos = np.empty(max(1, nnz - n), dtype=np.int32)
    _check(load().ic_get_upper(h.ptr, _p(urp), _p(ucol), _p(cptr), _p(cp), _p(cpos)))
    return urp, ucol, cptr, cp[: nnz - n], cpos[: nnz - n]


def ic_get_blocks(h):
    """(ranges, bptr, bcol) of the 2D block matrix."""
    st = ic_stats(h)
    nr, nbk = st["nranges"], st["nblocks"]
    ranges = np.empty(nr + 1, dtype=np.int64)
    bptr = np.empty(nr + 1, dtype=np.int64)
    bcol = np.empty(max(1, nbk), dtype=np.int32)
    _check(load().ic_get_blocks(h.ptr, _p(ranges), _p(bptr), _p(bcol)))
    return ranges, bptr, bcol[:nbk]


def ic_get_solve_tasks(h, backward=False):
    """Block-DAG solve plan of one direction: dict with tasks (ntasks x 4: type 0 = E /
    1 = L, range, first and end order position) in claim order, counters (in-degree of
    each task), succ_ptr/succ (tasks each task releases), split (per row),
    order_ptr/order and need."""
    L = load()
    st = ic_stats(h)
    n, nr = st["n"], st["nranges"]
    nt = np.zeros(1, dtype=np.int64)
    _check(L.ic_get_solve_tasks(h.ptr, int(bool(backward)), _p(nt), None, None, None, None, None, None, None,
                                None))
    ntk = int(nt[0])
    tasks = np.empty((max(1, ntk), 4), dtype=np.int32)
    cnt = np.empty(max(1, ntk), dtype=np.int32)
    sptr = np.empty(ntk + 1, dtype=np.int32)
    optr = np.empty(nr + 1, dtype=np.int32)
    split = np.empty(max(1, n), dtype=np.int32)
    _check(L.ic_get_solve_tasks(h.ptr, int(bool(backward)), None, None, _p(cnt), _p(sptr), None, None, _p(optr),
                                None, None))
    succ = np.empty(max(1, int(sptr[-1])), dtype=np.int32)
    order = np.empty(max(1, int(optr[-1])), dtype=np.int32)
    need = np.empty(max(1, int(optr[-1])), dtype=np.int32)
    _check(L.ic_get_solve_tasks(h.ptr, int(bool(backward)), None, _p(tasks), None, None, _p(succ), _p(split), None,
                                _p(order), _p(need)))
    return {"tasks": tasks[:ntk], "counters": cnt[:ntk], "succ_ptr": sptr, "succ": succ[: int(sptr[-1])],
            "split": split[:n], "order_ptr": optr, "order": order[: int(optr[-1])], "need": need[: int(optr[-1])]}


def ic_get_solve_entries(h, backward=False):
    """Internal entries of the rows as the L tasks apply them: dict with ptr (n+1),
    j and pos (ptr[-1] each)."""
    L = load()
    n = ic_stats(h)["n"]
    ptr = np.empty(n + 1, dtype=np.int32)
    _check(L.ic_get_solve_entries(h.ptr, int(bool(backward)), _p(ptr), None, None))
    m = int(ptr[-1])
    j = np.empty(max(1, m), dtype=np.int32)
    pos = np.empty(max(1, m), dtype=np.int32)
    _check(L.ic_get_solve_entries(h.ptr, int(bool(backward)), None, _p(j), _p(pos)))
    return {"ptr": ptr, "j": j[:m], "pos": pos[:m]}


def ic_get_claim_order(h):
    """(task, chunk) of every numeric work item, in the order the kernel's CTAs claim them."""
    n = ic_stats(h)["nitems"]
    task = np.empty(max(1, n), dtype=np.int32)
    chunk = np.empty(max(1, n), dtype=np.int32)
    _check(load().ic_get_claim_order(h.ptr, _p(task), _p(chunk)))
    return task[:n], chunk[:n]


def ic_get_split_layout(h):
    """Split Chol/Trsm tasks' published-row layout: dict with flag_off (ntasks), soff,
    nshadow."""
    L = load()
    nt = ic_stats(h)["ntasks"]
    ns = np.zeros(1, dtype=np.int64)
    nsh = np.zeros(1, dtype=np.int64)
    _check(L.ic_get_split_layout(h.ptr, None, None, _p(ns), _p(nsh)))
    fo = np.empty(max(1, nt), dtype=np.int32)
    so = np.empty(max(1, int(ns[0])), dtype=np.int32)
    _check(L.ic_get_split_layout(h.ptr, _p(fo), _p(so), None, None))
    return {"flag_off": fo[:nt], "soff": so[:int(ns[0])], "nshadow": int(nsh[0])}


def ic_get_solve_trace(h, backward=False):
    """(ntasks, 4) uint64 of the last block-DAG solve: claim ns, wait end ns, end ns,
    task | SM << 32 (tasks in ic_get_solve_tasks' claim order)."""
    nt = np.zeros(1, dtype=np.int64)
    _check(load().ic_get_solve_tasks(h.ptr, int(bool(backward)), _p(nt), None, None, None, None, None, None, None,
                                     None))
    out = np.zeros((max(1, int(nt[0])), 4), dtype=np.uint64)
    _check(load().ic_get_solve_trace(h.ptr, int(bool(backward)), _p(out)))
    return out[: int(nt[0])]


class ic_timing_t(C.Structure):
    _fields_ = [("prepare_ms", C.c_double), ("numeric_ms", C.c_double), ("apply_ms", C.c_double),
                ("apply_calls", C.c_int64), ("launches", C.c_int64), ("fwd_ms", C.c_double),
                ("bwd_ms", C.c_double)]


def ic_set_timing(h, on=True):
    _check(load().ic_set_timing(h.ptr, int(bool(on))))


def ic_reset_timing(h):
    _check(load().ic_reset_timing(h.ptr))


def ic_get_timing(h):
    t = ic_timing_t()
    _check(load().ic_get_timing(h.ptr, C.byref(t)))
    return {f: getattr(t, f) for f, _ in t._fields_}


def ic_fma_peak(dtype=IC_F64, stream=None):
    """Measured FMA throughput (GFLOP/s) of the current GPU for IC_F64 or IC_F32."""
    g = np.zeros(1, dtype=np.float64)
    _check(load().ic_fma_peak(int(dtype), _p(g), _stream(stream)))
    return float(g[0])


def ic_test_hold_solve_task(h, t, extra=1, backward=False):
    _check(load().ic_test_hold_solve_task(h.ptr, int(bool(backward)), int(t), int(extra)))


def ic_test_hold_task(h, t, extra=1):
    _check(load().ic_test_hold_task(h.ptr, int(t), int(extra)))


def ic_set_trace(h, on=True):
    _check(load().ic_set_trace(h.ptr, int(bool(on))))


def ic_get_trace(h):
    """(nitems, 4) uint64: start ns, end ns, task | chunk << 32, SM id per queue slot."""
    n = ic_stats(h)["nitems"]
    out = np.zeros((n, 4), dtype=np.uint64)
    _check(load().ic_get_trace(h.ptr, _p(out)))
    return out


def _opts(block_rows=0, dtype=IC_F64, warps_per_cta=0, rows_per_item=0, timeout_s=0.0, shift_alpha=0.0,
          exact=0, threads=0, host_only=0, solve_ctas_per_sm=0, solve_lanes=0, solve_mode=0):
    return ic_opts(block_rows, dtype, warps_per_cta, rows_per_item, timeout_s, shift_alpha, exact, threads,
                   host_only, solve_ctas_per_sm, solve_lanes, solve_mode)


def _batch_args(patterns, perms, ranges):
    """ctypes arrays for a batch: patterns is a list of (rowptr, colind)."""
    count = len(patterns)
    keep = []
    pats = (ic_csr_pattern * count)()
    for s, (rp, ci) in enumerate(patterns):
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        keep += [rp, ci]
        pats[s] = ic_csr_pattern(len(rp) - 1, _p(rp), _p(ci))
    pp = None
    if perms is not None:
        pp = (C.c_void_p * count)()
        for s, pm in enumerate(perms):
            if pm is not None:
                pm = np.ascontiguousarray(pm, dtype=np.int32)
                keep.append(pm)
                pp[s] = pm.ctypes.data
    rr, nr = None, None
    if ranges is not None:
        rr = (C.c_void_p * count)()
        nr = np.zeros(count, dtype=np.int64)
        keep.append(nr)
        for s, rg in enumerate(ranges):
            if rg is not None:
                rg = np.ascontiguousarray(rg, dtype=np.int64)
                keep.append(rg)
                rr[s] = rg.ctypes.data
                nr[s] = len(rg) - 1
    return count, pats, pp, rr, nr, keep


def ic_symbolic_batch(patterns, k, perms=None, ranges=None, **opts):
    """One handle over independent systems; patterns: list of (rowptr, colind)."""
    L = load()
    count, pats, pp, rr, nr, keep = _batch_args(patterns, perms, ranges)
    o = _opts(**opts)
    out = C.c_void_p()
    _check(L.ic_symbolic_batch(count, pats, int(k), pp, rr, _p(nr), C.byref(o), C.byref(out)))
    n = sum(len(p[0]) - 1 for p in patterns)
    nnz = sum(int(np.asarray(p[0])[-1]) for p in patterns)
    del keep
    return Handle(out.value, n, nnz)


def ic_batch_info(h):
    """Row offsets (count+1) of the handle's systems."""
    L = load()
    cnt = np.zeros(1, dtype=np.int64)
    _check(L.ic_batch_info(h.ptr, _p(cnt), None))
    off = np.empty(int(cnt[0]) + 1, dtype=np.int64)
    _check(L.ic_batch_info(h.ptr, _p(cnt), _p(off)))
    return off


def pcg_solve_batch(h, A_vals, b, x, tol=1e-8, maxit=10000, stream=None, raise_noconv=True):
    """Independent PCG per system; returns (iters, relres) arrays."""
    count = len(ic_batch_info(h)) - 1
    it = np.zeros(count, dtype=np.int32)
    rel = np.zeros(count, dtype=np.float64)
    st = load().pcg_solve_batch(h.ptr, _p(A_vals), _p(b), _p(x), float(tol), int(maxit), _p(it), _p(rel),
                                _stream(stream))
    if st != IC_ERR_NOCONV or raise_noconv:
        _check(st)
    return it, rel


def ic_numeric_async(h, values, stream=None):
    _check(load().ic_numeric_async(h.ptr, _p(values), _stream(stream)))


def ic_numeric_status(h):
    brk = np.zeros(1, dtype=np.int64)
    st = load().ic_numeric_status(h.ptr, _p(brk))
    if st == IC_ERR_BREAKDOWN:
        e = IckError(st, f"breakdown at row {int(brk[0])}")
        e.row = int(brk[0])
        raise e
    _check(st)
    return -1


def ic_autotune(patterns, k, values, perms=None, ranges=None, reps=3, stream=None, **base):
    """Returns (opts dict, (numeric_ms, apply_ms)) chosen by timing on the device."""
    L = load()
    count, pats, pp, rr, nr, keep = _batch_args(patterns, perms, ranges)
    b = _opts(**base)
    best = ic_opts()
    times = np.zeros(2, dtype=np.float64)
    _check(L.ic_autotune(count, pats, int(k), pp, rr, _p(nr), _p(values), C.byref(b), int(reps),
                         C.byref(best), _p(times), _stream(stream)))
    del keep
    d = {f: getattr(best, f) for f, _ in best._fields_ if f != "reserved"}
    return d, (float(times[0]), float(times[1]))


def ic_destroy(h):
    h.close()


# ------------------------------------------------------------- diagonal shift


def ic_shift_features(h, values, nu=0.0, stream=None):
    """The 8 matrix features of the shift predictor (numpy float64)."""
    out = np.zeros(8, dtype=np.float64)
    _check(load().ic_shift_features(h.ptr, _p(values), float(nu), _p(out), _stream(stream)))
    return out


def ic_numeric_shifted(h, values, alpha_first=0.0, alpha0=1e-3, max_tries=20, stream=None):
    """Numeric IC(k) with the shift-doubling retry; returns (alpha used, attempts)."""
    a = np.zeros(1, dtype=np.float64)
    t = np.zeros(1, dtype=np.int32)
    st = load().ic_numeric_shifted(h.ptr, _p(values), float(alpha_first), float(alpha0), int(max_tries), _p(a),
                                   _p(t), _stream(stream))
    if st == IC_ERR_BREAKDOWN:
        e = IckError(st, f"all {int(t[0])} shift attempts broke down")
        e.attempts = int(t[0])
        raise e
    _check(st)
    return float(a[0]), int(t[0])


def ic_mlp_n_params():
    return int(load().ic_mlp_n_params())


class Mlp:
    """The shift-predictor network (owns an ic_mlp)."""

    def __init__(self, params=None):
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        out = C.c_void_p()
        _check(load().ic_mlp_create(_p(p), C.byref(out)))
        self._m = out.value

    @property
    def ptr(self):
        return self._m

    def close(self):
        if self._m:
            load().ic_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ic_mlp_create(params=None):
    return Mlp(params)


def ic_mlp_set_params(m, params):
    _check(load().ic_mlp_set_params(m.ptr, _p(np.ascontiguousarray(params, dtype=np.float32))))


def ic_mlp_get_params(m):
    out = np.empty(ic_mlp_n_params(), dtype=np.float32)
    _check(load().ic_mlp_get_params(m.ptr, _p(out)))
    return out


def ic_mlp_set_scaling(m, mean, std):
    _check(load().ic_mlp_set_scaling(m.ptr, _p(np.ascontiguousarray(mean, dtype=np.float32)),
                                     _p(np.ascontiguousarray(std, dtype=np.float32))))


def ic_mlp_get_scaling(m):
    mean = np.empty(8, dtype=np.float32)
    std = np.empty(8, dtype=np.float32)
    _check(load().ic_mlp_get_scaling(m.ptr, _p(mean), _p(std)))
    return mean, std


def ic_mlp_forward(m, X, y, stream=None):
    """X: CUDA float32 tensor (n, 8); y: CUDA float32 tensor (n,)."""
    _check(load().ic_mlp_forward(m.ptr, _p(X), int(X.shape[0]), _p(y), _stream(stream)))


def ic_mlp_gradient(m, X, t, stream=None):
    """(gradient as numpy float32, loss) of (1/2n) sum (y - t)^2; no update."""
    g = np.empty(ic_mlp_n_params(), dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _check(load().ic_mlp_gradient(m.ptr, _p(X), _p(t), int(X.shape[0]), _p(g), _p(loss), _stream(stream)))
    return g, float(loss[0])


def ic_mlp_train_step(m, X, t, lr, stream=None, want_loss=True):
    """One Adam step; returns the loss before the step (None when want_loss is false:
    the call then does not synchronise)."""
    loss = np.zeros(1, dtype=np.float32) if want_loss else None
    _check(load().ic_mlp_train_step(m.ptr, _p(X), _p(t), int(X.shape[0]), float(lr), _p(loss), _stream(stream)))
    return float(loss[0]) if want_loss else None


def ic_mlp_predict_shift(m, features, stream=None):
    a = np.zeros(1, dtype=np.float64)
    _check(load().ic_mlp_predict_shift(m.ptr, _p(np.ascontiguousarray(features, dtype=np.float64)), _p(a),
                                       _stream(stream)))
    return float(a[0])

