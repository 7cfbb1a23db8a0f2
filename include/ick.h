/*
 * ick.h -- C ABI of the GB300 level-of-fill incomplete Cholesky library (libick.so).
 *
 * The library computes IC(k) on the 2D sparse partitioned-block layout of
 * Kim, Rajamanickam, Stelle, Edwards and Olivier, "Task Parallel Incomplete
 * Cholesky Factorization using 2D Partitioned-Block Layout" (arXiv:1601.05871):
 * symbolic factorization (Algorithm 1, Section 3.1), the 2D block matrix
 * (Section 3.2) and the numeric Cholesky-by-blocks task DAG (Section 3.3, the
 * Chol / Trsm / Herk / Gemm task generator figure) executed by one persistent
 * CUDA kernel.  The factor is used as a PCG preconditioner (Section 1).
 *
 * Conventions shared by every call:
 *   - A is symmetric positive definite, given as a FULL symmetric CSR pattern
 *     (both triangles) with sorted, duplicate-free columns and a structural
 *     diagonal in every row; rowptr is int64, colind int32, values float64.
 *   - perm[new] = old.  B = P^T A P is the reordered matrix, B_ij = A_perm[i],perm[j].
 *     Only the upper triangle of B is read (B_ij with i <= j, wherever it lies in A),
 *     so A's values must be symmetric bit for bit.
 *   - The factor is kept as U = L^T (upper CSR, diagonal first in each row) so that
 *     B ~= U^T U = L L^T; ic_get_factor returns L in lower CSR (diagonal last).
 *   - "host" pointers are CPU memory; "device" pointers are CUDA global memory on the
 *     current device; "stream" is a cudaStream_t (NULL: the legacy default stream).
 *   - Every call returns an ic_status; no call aborts the process or traps on the GPU.
 *     Device waits are bounded by ic_opts.timeout_s and end in IC_ERR_TIMEOUT.
 *   - Inputs are borrowed for the duration of the call and copied where kept.
 *     The handle owns every device allocation it makes; ic_destroy frees them.
 */
#ifndef ICK_H
#define ICK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IC_OK = 0,
    IC_ERR_ARG = 1,       /* bad argument (NULL, size, range, option)                  */
    IC_ERR_PATTERN = 2,   /* malformed CSR: unsorted, duplicate, out of range,
                             asymmetric, or missing diagonal                           */
    IC_ERR_BREAKDOWN = 3, /* a pivot <= 0 or not finite; *breakdown_row = first row    */
    IC_ERR_TIMEOUT = 4,   /* a bounded device wait expired; the factor is invalid      */
    IC_ERR_CUDA = 5,      /* a CUDA runtime call failed                                */
    IC_ERR_NOMEM = 6,     /* host or device allocation failed                          */
    IC_ERR_NOCONV = 7,    /* PCG reached maxit before the tolerance                    */
    IC_ERR_STATE = 8      /* call out of order (e.g. ic_apply before ic_numeric)       */
} ic_status;

enum { IC_F64 = 0, IC_F32 = 1 };

typedef struct {
    int64_t n;
    const int64_t* rowptr; /* host, n+1 */
    const int32_t* colind; /* host, rowptr[n]; full symmetric, sorted */
} ic_csr_pattern;

/* Options.  A zero-initialised struct selects the defaults given in brackets. */
typedef struct {
    int block_rows;    /* [4096] largest block; longer ranges are split evenly; <= 8192 */
    int dtype;         /* [IC_F64] factor precision                                      */
    int warps_per_cta; /* [32 for one system, 16 for a batch] warps in each CTA of the
                          persistent numeric kernel: 8|16|32 (32: one CTA per SM,
                          16: two)                                                      */
    int rows_per_item; /* [warps_per_cta] target rows per work item of a Herk/Gemm task */
    double timeout_s;  /* [10] bound on every device wait of one call                    */
    double shift_alpha;/* [0] factor B + alpha * diag(B) instead of B                    */
    int exact;         /* [0] 1: each update is a separately rounded multiply then
                          subtract (no FMA), and the updates of a block are applied in
                          ascending k: the same operation sequence per entry as the
                          up-looking row order, so the FP64 factor is reproducible
                          bit for bit; 0: fused multiply-add, and the updates of a block
                          chained in the order of their inputs' estimated readiness
                          (deterministic: one fixed order per entry)                    */
    int threads;       /* [0 = all] host threads for the symbolic phase                  */
    int host_only;     /* [0] 1: ic_symbolic builds the plan in host memory only (no GPU
                          needed); such a handle serves the ic_get_* and ic_stats calls   */
    int solve_ctas_per_sm; /* [2 block-DAG, 3 row-level] CTAs per SM for the triangular-
                              solve kernels (capped by occupancy)                    */
    int solve_lanes;   /* [8 block-DAG, 32 row-level] lanes per row in the ic_apply /
                          pcg_solve solves: 4|8|16|32                                 */
    int solve_mode;    /* [0] triangular solves of ic_apply / pcg_solve: 0 block-DAG (block
                        * rows as tasks, one CTA per block row's local chain), 1 row-level
                        * (every row a unit, claimed in dependence-level order)           */
    int reserved[2];
} ic_opts;

typedef struct {
    int64_t n;            /* rows                                                    */
    int64_t nnz_a;        /* nonzeros of A (both triangles)                          */
    int64_t nnz_l;        /* nonzeros of L (= of U), diagonal included               */
    int64_t nranges;      /* block rows/columns of the 2D block matrix               */
    int64_t nblocks;      /* existing blocks (i <= j) of the 2D block matrix         */
    int64_t ntasks;       /* Chol + Trsm + Herk + Gemm tasks                         */
    int64_t ntasks_type[4];/* per type: Chol, Trsm, Herk, Gemm                       */
    int64_t nitems;       /* work items the persistent kernel drains                 */
    int64_t critical_path;/* tasks on the longest DAG path                           */
    int64_t max_level;    /* largest level of fill kept (<= k)                       */
    double flops;         /* algorithmic flops of one numeric factorization          */
    double bytes;         /* compulsory HBM bytes of one numeric factorization       */
    double symbolic_s;    /* wall time of ic_symbolic                                */
    int64_t grid_ctas;    /* CTAs of the persistent kernel launch                    */
    int64_t solve_depth[2];/* levels of the forward / backward solve's row DAG        */
    int64_t warps_per_cta;/* warps per CTA of the persistent kernel (defaults resolved) */
    int64_t rows_per_item;/* target rows per Herk/Gemm work item (defaults resolved)    */
    int64_t nsplit;       /* Chol/Trsm tasks spread over several CTAs (expected to run
                             with little else in flight; their finished rows published
                             in a shadow array read with no completion flags)          */
} ic_stats_t;

typedef struct ic_handle ic_handle;

/* Geometric nested dissection of a grid (Algorithm 1, steps 1 and 3; Section 3.1,
 * with Scotch replaced by cuts of the grid coordinates).  The box's longest axis
 * (ties: x, y, z) is cut by the one-node plane m = lo + (hi-lo)/2; the low half,
 * the high half and the plane are numbered in that order, recursively.  A part
 * with <= leaf_rows kept rows, or whose longest extent is < 3, is a leaf (this is
 * the pruning of the ND tree, Algorithm 1 step 3).  Inside a part rows are
 * lexicographic with x fastest; dof > 1 keeps a node's dofs together.  The paper
 * takes the order inside a separator from Scotch and does not fix it; with
 * sep_colours = C >= 2 a separator plane of R kept rows cut across axis a is split
 * into m = ceil(R / leaf_rows) strips (strip q: rows [q R / m, (q+1) R / m) of its
 * lexicographic order), each a part of its own, and each strip is numbered colour
 * class by colour class: a node's class is (u mod C) + C (v mod C), u and v its
 * coordinates along the two other axes (u the lower-numbered axis), classes in
 * ascending order, lexicographic inside a class.  With leaf_rows = the block size the
 * strips are the blocks the lexicographic plane would be cut into, so the block
 * pattern and task DAG do not change; the triangular solves' dependence chains get
 * shorter.  On the 27-point grids measured the fill count did not change either.
 *   sep_colours 0 or 1: lexicographic separators; 2..16: C.
 * With leaf_colours = C >= 2 every leaf box is numbered the same way by the classes
 * (x mod C) + C (y mod C) + C^2 (z mod C), as one part: the solves' chains through
 * the leaves get shorter, at the cost of more fill (on the 27-point grids measured
 * with C = 2 and IC(2), 9-12 % more entries of L and 27-34 % more factor flops).
 *   leaf_colours 0 or 1: lexicographic leaves; 2..4: C.
 *   keep      host, nx*ny*nz*dof bytes or NULL: 0 drops that dof (eliminated
 *             boundary conditions); the returned order covers the kept dofs only,
 *             indexed in grid order among the kept ones.
 *   perm_out  host, >= n entries: perm[new] = old.
 *   ranges_out host, >= n+1 entries or NULL: 0 then the end of each part, in order.
 *   nranges_out, n_out: number of parts and of kept rows.
 * Errors: IC_ERR_ARG for non-positive sizes, sep_colours outside 0..16,
 * leaf_colours outside 0..4 or NULL perm_out. */
int ic_nd_grid(int nx, int ny, int nz, int dof, int leaf_rows, int sep_colours, int leaf_colours,
               const uint8_t* keep, int32_t* perm_out, int64_t* ranges_out, int64_t* nranges_out,
               int64_t* n_out);

/* Symbolic factorization (Algorithm 1, steps 2, 4, 5; Sections 3.1-3.3) on the host:
 * reorders A by perm (NULL: identity), finds the level-k fill pattern S by a
 * breadth-first search from every row (the Hysom-Pothen scheme of Section 4.1:
 * entry (i,j) has level = edges - 1 of the shortest path i..j whose interior
 * vertices are all < min(i,j); kept when <= k), builds the 2D block matrix over
 * the ranges (NULL: uniform blocks of opts->block_rows rows), generates the
 * Cholesky-by-blocks task DAG, and uploads everything to the current device.
 *   A       host pattern (values are not needed here).
 *   ranges  host, nranges+1 increasing boundaries from 0 to n, or NULL.
 *   opts    NULL for defaults.
 *   out     receives the handle; *out is NULL on error.
 * Errors: IC_ERR_ARG, IC_ERR_PATTERN, IC_ERR_NOMEM, IC_ERR_CUDA. */
int ic_symbolic(const ic_csr_pattern* A, int k, const int32_t* perm, const int64_t* ranges,
                int64_t nranges, const ic_opts* opts, ic_handle** out);

/* Numeric factorization (Section 3.3): scatters B's values onto S (zero on fill) and
 * runs the Chol / Trsm / Herk / Gemm task DAG in one persistent kernel launch whose
 * CTAs claim the work items in a precomputed order (ic_get_claim_order) and start each
 * once its atomic dependency counter has reached zero.  Updates that
 * fall outside S are discarded.  Blocks until the stream has finished the launch.
 *   values  device, nnz(A) doubles in A's CSR order.
 *   breakdown_row  host out (may be NULL): -1, or the smallest row (permuted order)
 *                  whose pivot was <= 0 or not finite (then IC_ERR_BREAKDOWN).
 * Errors: IC_ERR_ARG, IC_ERR_BREAKDOWN, IC_ERR_TIMEOUT, IC_ERR_CUDA. */
int ic_numeric(ic_handle* h, const void* values, void* stream, int64_t* breakdown_row);

/* Preconditioner application z = (L L^T)^{-1} r = P (U^T U)^{-1} P^T r: forward then
 * backward triangular solves on the device (the use of Section 1; the paper does not
 * describe the solves).  r and z are device vectors of n doubles in the ORIGINAL
 * ordering; they may not alias.  Asynchronous on stream.  The solves share the
 * handle's work vector and completion stamps, so calls on one handle must not overlap
 * on the GPU (issue them on one stream).  Their row dependences are acyclic, so the
 * bounded waits can only expire if the GPU stops the kernel for longer than
 * opts.timeout_s; z is then undefined and the timeout is recorded on the handle:
 * ic_apply_status reports it (and pcg_solve reports a timeout of its own
 * applications).  Each call starts afresh, so one expired wait does not stop later
 * calls.
 * Errors: IC_ERR_ARG, IC_ERR_STATE (no successful ic_numeric yet), IC_ERR_CUDA. */
int ic_apply(ic_handle* h, const void* r, void* z, void* stream);

/* Synchronises stream, then reports whether a triangular-solve wait of an ic_apply on
 * this handle expired since the last ic_apply_status or pcg_solve (IC_ERR_TIMEOUT),
 * and clears that record (pcg_solve and pcg_solve_batch clear it too: they report the
 * timeouts of their own applications).  Errors: IC_ERR_ARG, IC_ERR_TIMEOUT, IC_ERR_CUDA. */
int ic_apply_status(ic_handle* h, void* stream);

/* The same preconditioner application as ic_apply, for callers that cannot allocate
 * GPU memory where they apply it: a plugin running inside another framework that owns
 * the device's memory budget and gives its plugins no allocator, or a loop with a hard
 * latency limit in which a cudaMalloc (which may synchronise the device) is not
 * allowed.  The paper has no counterpart; this is an interface convenience of this
 * library.  The call allocates nothing and calls no allocating routine: the solves'
 * scratch (the permuted work vector, per-row completion stamps, claim counters, abort
 * word and timeout record) lives in one file-scope device array for at most 1,048,576
 * rows (about 12 MB), which every GPU that loads the library keeps until the process
 * exits.  It runs the row-level solves (every row a unit, ic_opts.solve_mode = 1),
 * whatever the handle's solve_mode: they need no per-handle task state, and they are
 * 1.3-1.7x slower than the default block-DAG solves of ic_apply on large 3D problems.
 * The first call on a device looks up that array's device address (once per device,
 * with the device current), so make it before any stream capture begins.  All calls
 * share the array and it keeps the last call's contents (counters are cleared at the
 * start of each call): calls that overlap on the GPU -- on different streams or from
 * different threads, for any handle -- race, and the caller must serialise them.  A
 * wait that expires leaves z undefined; the call cannot report it (it does not wait
 * for the GPU), ic_apply_static_status does.  r and z: as for ic_apply.
 * Errors: IC_ERR_ARG (NULL or aliased vectors, n above 1,048,576 rows, or an IC_F32
 * factor), IC_ERR_STATE (no successful ic_numeric yet), IC_ERR_CUDA. */
int ic_apply_static(ic_handle* h, const void* r, void* z, void* stream);

/* Synchronises stream, then reports whether a solve wait of an ic_apply_static call on
 * the current device expired since the last ic_apply_static_status (IC_ERR_TIMEOUT),
 * and clears that record.  Allocates nothing.  Errors: IC_ERR_TIMEOUT, IC_ERR_CUDA. */
int ic_apply_static_status(void* stream);

/* Preconditioned conjugate gradients on A x = b with M = L L^T (textbook PCG, x0 = 0,
 * stop when ||r||_2 / ||b||_2 <= tol).  A's pattern is the one given to ic_symbolic.
 *   A_vals  device, nnz(A) doubles in A's CSR order.
 *   b, x    device, n doubles, original ordering; x is overwritten.
 *   iters, relres  host out (may be NULL): iterations done and the final recursive
 *                  relative residual.
 * With kernel timing off (the default) the whole solve is one CUDA graph launch: the
 * loop runs on the device (a WHILE conditional node, its test computed by a kernel) and
 * the host synchronises once, at the end.  The graph is captured and instantiated on
 * a stream of the handle at the first call with a given (A_vals, b, x, tol, maxit) and
 * kept until a call with other arguments.  With timing on (ic_set_timing) the loop
 * runs on the host with one synchronisation per iteration, so that every kernel can be
 * timed.  Both take the same arithmetic steps in the same order.
 * Errors: IC_ERR_ARG, IC_ERR_STATE, IC_ERR_NOCONV (x holds the last iterate), IC_ERR_CUDA. */
int pcg_solve(ic_handle* h, const void* A_vals, const double* b, double* x, double tol, int maxit,
              int* iters, double* relres, void* stream);

/* Host copy of L = U^T in lower CSR, permuted order, rows sorted, diagonal last.
 * rowptr (n+1), colind and vals (nnz_l) are host buffers; any may be NULL to skip.
 * levels (host, nnz_l int32 or NULL) receives each entry's level of fill.
 * vals require a successful ic_numeric.
 * Errors: IC_ERR_ARG, IC_ERR_STATE, IC_ERR_CUDA. */
int ic_get_factor(ic_handle* h, int64_t* rowptr, int32_t* colind, double* vals, int32_t* levels);

/* Sizes, flop and byte counts and DAG statistics of the handle. */
int ic_stats(const ic_handle* h, ic_stats_t* out);

/* Task list of the handle in generation order (the loop of Section 3.3's task
 * generator figure).  type: 0 Chol, 1 Trsm, 2 Herk, 3 Gemm; (tk, ti, tj) block
 * indices: Chol (k,k,k), Trsm (k,k,j), Herk (k,i,i), Gemm (k,i,j).  pred_ptr
 * (ntasks+1) and pred list the distinct predecessors.  With exact = 1 these are the
 * generator's (the updates of a block chained in k order, every predecessor earlier
 * in the list); with exact = 0 the updates of a block are chained in another order
 * (see ic_opts.exact), so an update's predecessor may come later in the list.  The
 * dependencies on data (Trsm on Chol, an update on its two Trsm inputs, a block's
 * Chol/Trsm on its last update) are the same in both.  Call with NULL arrays to get
 * *ntasks and *npred, then again with buffers of at least those sizes.
 * Errors: IC_ERR_ARG. */
int ic_get_tasks(const ic_handle* h, int32_t* type, int32_t* tk, int32_t* ti, int32_t* tj,
                 int64_t* pred_ptr, int32_t* pred, int64_t* ntasks, int64_t* npred);

/* The same task generator on a bare block pattern: nb block rows, block pattern in
 * upper CSR (bptr: nb+1, bcol sorted, each row containing its diagonal block).
 * Same outputs and two-call protocol as ic_get_tasks.
 * Errors: IC_ERR_ARG, IC_ERR_PATTERN. */
int ic_block_dag(int64_t nb, const int64_t* bptr, const int32_t* bcol, int32_t* type, int32_t* tk,
                 int32_t* ti, int32_t* tj, int64_t* pred_ptr, int32_t* pred, int64_t* ntasks,
                 int64_t* npred);

/* Work-item targets of one task, for inspection: for each target row r of task t,
 * (r, first and one-past-last index into the column lists of U, first and
 * one-past-last position of the target segment in U).  Two-call protocol on *count.
 * Also returns (when not NULL) U's upper pattern and column lists:
 * urp (n+1), ucol (nnz_l), cptr (n+1), cp (nnz_l - n: pivot row p of each entry),
 * cpos (nnz_l - n: position of U_pr).
 * Errors: IC_ERR_ARG. */
int ic_get_task_targets(const ic_handle* h, int64_t t, int32_t* tgt5, int64_t* count);
int ic_get_upper(const ic_handle* h, int64_t* urp, int32_t* ucol, int64_t* cptr, int32_t* cp,
                 int32_t* cpos);

/* The 2D block matrix of the handle (Section 3.2): ranges (nranges+1 row boundaries
 * after splitting to at most block_rows rows) and the upper block pattern bptr
 * (nranges+1), bcol (nblocks; diagonal block first in each block row).  Sizes come
 * from ic_stats.  Errors: IC_ERR_ARG. */
int ic_get_blocks(const ic_handle* h, int64_t* ranges, int64_t* bptr, int32_t* bcol);

/* The block-DAG triangular solves of ic_apply (solve_mode 0), for inspection and
 * tests.  Each block row (range) has its rows in local dependence-level order
 * (order); a range with entries reaching outside it is cut into parts of a few
 * levels.  Per part, task L (one CTA) solves the part's rows after the range's
 * previous part, and tasks E sum, for chunks of the part's rows, the entries that
 * reach outside the range, once the parts holding those source rows have finished.
 * backward = 0: L y = r; 1: L^T z = y.  Every pointer may be NULL (output skipped).
 *   ntasks      receives the number of tasks.
 *   tasks       4 per task in claim order: type (0 = E, 1 = L), range, first and end
 *               position in order (a position may hold -1: padding).
 *   counters    ntasks: the number of tasks each task waits for.
 *   succ_ptr, succ  ntasks + 1 offsets and the tasks each task releases (size
 *               succ_ptr[ntasks]).
 *   split       n: forward, the column-list index (into ic_get_upper's cp) where
 *               the entries inside the row's range begin; backward, the number of
 *               entries after the diagonal of the row that lie inside its range.
 *   order_ptr, order  nranges + 1 offsets and the rows of each range in claim order,
 *               every level padded with -1 to a multiple of 8 (size order_ptr[nranges]).
 *   need        order_ptr[nranges]: per order position, the number of the range's rows
 *               in lower levels; the row there runs once that many rows are complete.
 * Errors: IC_ERR_ARG. */
int ic_get_solve_tasks(const ic_handle* h, int backward, int64_t* ntasks, int32_t* tasks, int32_t* counters,
                       int32_t* succ_ptr, int32_t* succ, int32_t* split, int32_t* order_ptr, int32_t* order,
                       int32_t* need);

/* The internal entries of each row as the L tasks apply them (same direction
 * convention; any pointer may be NULL).  ptr (n + 1): row i's entries are
 * [ptr[i], ptr[i+1]); j (ptr[n]): the source row minus the range's first row; pos
 * (ptr[n]): the position of the value in ic_get_upper's row-major storage.
 * Errors: IC_ERR_ARG. */
int ic_get_solve_entries(const ic_handle* h, int backward, int32_t* ptr, int32_t* j, int32_t* pos);

/* The order in which the persistent numeric kernel's CTAs claim the work items (ic_stats
 * nitems of them), for inspection: task[q] and chunk[q] (host buffers of nitems
 * entries, either may be NULL) of the q-th item claimed.  The symbolic phase computes
 * it as a list schedule of the task DAG (Section 3.3) on the kernel's CTAs, under a
 * duration model of the items, running first the ready item whose task has the
 * longest remaining path; every item comes after all items of its task's
 * predecessors, so a CTA waiting for a claimed item's predecessors waits only for
 * items held by running CTAs.  A host-only handle's order assumes 152 CTAs.
 * Errors: IC_ERR_ARG. */
int ic_get_claim_order(const ic_handle* h, int32_t* task, int32_t* chunk);

/* Layout of the split Chol/Trsm tasks (ic_stats nsplit), for inspection.  A split
 * task's finished rows are published in a shadow array of *nshadow values: the target
 * segment [tb, te) of row r of such a task (ic_get_task_targets) sits at shadow
 * positions [tb + soff[flag_off[t] + r - ranges[k]], te + ...), k the task's block
 * row, at a position congruent to tb modulo 4.  flag_off (ntasks): the task's first
 * entry in soff, -1 for tasks that are not split.  soff (*nsoff): one per row of each
 * split task's block.  Call with NULL arrays to get *nsoff and *nshadow.
 * Errors: IC_ERR_ARG. */
int ic_get_split_layout(const ic_handle* h, int32_t* flag_off, int32_t* soff, int64_t* nsoff,
                        int64_t* nshadow);

/* Kernel timing of the handle's calls, from CUDA events recorded on the launching
 * stream while timing is on (ic_set_timing(h, 1); it adds no synchronisation beyond
 * what the calls already do).  launches counts the library's own kernel launches
 * since the last ic_reset_timing. */
typedef struct {
    double prepare_ms;     /* value scatter + scheduler reset of the last ic_numeric       */
    double numeric_ms;     /* persistent task-DAG kernel of the last ic_numeric            */
    double apply_ms;       /* triangular-solve kernels, summed since the last reset        */
    int64_t apply_calls;   /* ic_apply calls (direct, or inside pcg_solve while timing is
                              on) since the reset                                          */
    int64_t launches;      /* kernels launched by the library since the reset              */
    double fwd_ms;         /* forward-solve kernel alone, summed since the last reset      */
    double bwd_ms;         /* backward-solve kernel alone, summed since the last reset     */
} ic_timing_t;
int ic_set_timing(ic_handle* h, int on);
int ic_reset_timing(ic_handle* h);
int ic_get_timing(const ic_handle* h, ic_timing_t* out);

/* Fused multiply-add throughput of the current GPU in GFLOP/s for dtype IC_F64 or
 * IC_F32 (2 flops per FMA): a kernel of independent register FMA chains, 8 CTAs of 256
 * threads per SM, best of three timed launches (CUDA events on stream, which is
 * synchronised).  It is the arithmetic roof against which the numeric factorization's
 * GFLOP/s (Section 3.3's Chol/Trsm/Herk/Gemm flops) is compared; the paper has no
 * counterpart.  Allocates and frees a buffer of 8 bytes per thread.
 * Errors: IC_ERR_ARG, IC_ERR_CUDA. */
int ic_fma_peak(int dtype, double* gflops, void* stream);

/* Fault injection for tests, done on the host: adds `extra` to task t's initial
 * in-degree, so with extra = 1 the task is never released and the next ic_numeric
 * ends in IC_ERR_TIMEOUT once opts.timeout_s has passed (every device wait is
 * bounded; nothing traps).  extra = 0 restores the plan.  Errors: IC_ERR_ARG, IC_ERR_CUDA. */
int ic_test_hold_task(ic_handle* h, int64_t t, int extra);

/* The same for the block-DAG solves (solve_mode 0): adds `extra` to the initial
 * in-degree of task t (claim order of ic_get_solve_tasks) of the forward (backward = 0)
 * or backward (1) solve, so with extra = 1 every later ic_apply gives up that task's
 * wait after opts.timeout_s and records a timeout (ic_apply_status, pcg_solve report
 * it).  extra = 0 restores the plan.  Errors: IC_ERR_ARG, IC_ERR_STATE, IC_ERR_CUDA. */
int ic_test_hold_solve_task(ic_handle* h, int backward, int64_t t, int extra);

/* Batched symbolic factorization: count independent SPD matrices (different sizes
 * allowed) become one block-diagonal system whose task DAG is the union of the
 * systems' independent DAGs, so one ic_numeric launch factors all of them.  System s
 * occupies rows [row_off[s], row_off[s+1]) of the union in the original ordering;
 * its values are the concatenation of every system's CSR values in order.
 *   A        host, count patterns.
 *   perms    host, NULL or count entries (each NULL = identity) of the systems' orders.
 *   ranges, nranges  host, NULL or count entries: each system's ranges (NULL entry: the
 *            whole system as one range, split by block_rows).
 * Errors: as ic_symbolic. */
int ic_symbolic_batch(int64_t count, const ic_csr_pattern* A, int k, const int32_t* const* perms,
                      const int64_t* const* ranges, const int64_t* nranges, const ic_opts* opts,
                      ic_handle** out);

/* Number of systems of the handle (1 for ic_symbolic) and, when row_off is not NULL,
 * their count+1 row offsets.  Errors: IC_ERR_ARG. */
int ic_batch_info(const ic_handle* h, int64_t* count, int64_t* row_off);

/* Independent PCG on every system of the handle (textbook PCG per system, x0 = 0, each
 * system stops when its own ||r||/||b|| <= tol; a converged system's iterate no longer
 * changes while the others continue).  One iteration over all systems is captured
 * into a CUDA graph and replayed; convergence is read from the device every 4
 * iterations.  b and x: device, the union's rows.  iters, relres: host, count entries
 * or NULL.  Errors: IC_ERR_ARG, IC_ERR_STATE, IC_ERR_NOCONV (some system reached maxit),
 * IC_ERR_TIMEOUT, IC_ERR_CUDA. */
int pcg_solve_batch(ic_handle* h, const void* A_vals, const double* b, double* x, double tol, int maxit,
                    int* iters, double* relres, void* stream);

/* ic_numeric without the final synchronisation: enqueues the value scatter, the task
 * kernel and the copies of the status words on stream, so it can be captured into a
 * CUDA graph.  After the stream (or graph) has completed, ic_numeric_status returns
 * what ic_numeric would have (IC_OK, IC_ERR_BREAKDOWN with *breakdown_row,
 * IC_ERR_TIMEOUT).  Until then the factor is treated as valid by ic_apply.
 * Errors: IC_ERR_ARG, IC_ERR_STATE, IC_ERR_CUDA. */
int ic_numeric_async(ic_handle* h, const void* values, void* stream);
int ic_numeric_status(ic_handle* h, int64_t* breakdown_row);

/* Autotuner for the task granularity trade-offs of Section 4 (block size and the work
 * per task) and the solve launch shape.  For the given matrix or batch (count = 1 for
 * one matrix; arguments as ic_symbolic_batch), it times ic_numeric (median of reps)
 * over block_rows in {1024, 2048, 4096, 8192}, then warps_per_cta in {8, 16, 32}, then
 * rows_per_item in {16, 32, 64} (coordinate search, each best kept), and ic_apply over
 * solve_lanes in {8, 16, 32} (8 only for the block-DAG solves) x solve_ctas_per_sm in
 * {2, 3, 4, 6} (within occupancy) on the chosen plan.
 * values: device, the (concatenated) values.  base: other options (NULL: defaults).
 * best: receives the chosen options; times (host, 2 doubles or NULL): numeric ms and
 * apply ms of the choice.  The stream is synchronised.
 * Errors: as ic_symbolic and ic_numeric. */
int ic_autotune(int64_t count, const ic_csr_pattern* A, int k, const int32_t* const* perms,
                const int64_t* const* ranges, const int64_t* nranges, const void* values,
                const ic_opts* base, int reps, ic_opts* best, double* times, void* stream);

/* Task trace of the numeric kernel.  ic_set_trace(h, 1) allocates 4 uint64 words per
 * work item; every later ic_numeric records, per queue slot, the %globaltimer start
 * and end (ns) of the item, task | chunk << 32, and the SM that ran it.
 * ic_get_trace copies nitems * 4 words (nitems from ic_stats) to the host buffer out.
 * Errors: IC_ERR_ARG, IC_ERR_STATE (host-only handle or tracing off), IC_ERR_CUDA. */
int ic_set_trace(ic_handle* h, int on);
int ic_get_trace(const ic_handle* h, uint64_t* out);

/* Task trace of the block-DAG solves (solve_mode 0), recorded while ic_set_trace is
 * on: per task of ic_get_solve_tasks' claim order, 4 uint64 words: %globaltimer (ns)
 * at the claim, when its wait ended, and when it finished; task index | SM id << 32.
 * ic_get_solve_trace copies ntasks * 4 words of the last ic_apply's forward
 * (backward = 0) or backward (1) solve.  Errors: IC_ERR_ARG, IC_ERR_STATE, IC_ERR_CUDA. */
int ic_get_solve_trace(const ic_handle* h, int backward, uint64_t* out);

/* ----------------------------------------------------------------------------
 * Diagonal shift.  IC(k) of a matrix that is not an M-matrix can break down (a pivot
 * <= 0 once fill is dropped; Section 1 motivates IC(k) for SPD matrices, which does
 * not guarantee positive incomplete pivots).  Factoring B + alpha * diag(B) restores
 * positive pivots for a large enough alpha, at the price of a weaker preconditioner.
 * ------------------------------------------------------------------------- */

/* Features of the handle's matrix with the given values (device, CSR order of A),
 * computed on the GPU in FP64 with deterministic reductions: for row i with d = A_ii,
 * s = sum_{j != i} |A_ij| and r = ||row i||_2, dd_i = d / max(s, d / 1000) and
 * rn_i = r / d; out (host, 8 doubles) = [min dd, mean dd, mean rn, max rn, fraction
 * of off-diagonal entries > 0, k, log10 n, nu].  nu: a material parameter supplied by
 * the caller (0 when none applies).  Errors: IC_ERR_ARG (also when a diagonal entry
 * is missing or not positive), IC_ERR_CUDA. */
int ic_shift_features(const ic_handle* h, const void* A_vals, double nu, double* out, void* stream);

/* Numeric factorization with the shift-doubling retry: attempts are made with
 * alpha = alpha_first, then twice the previous alpha (alpha0 after a zero alpha),
 * until one has no breakdown or max_tries attempts have broken down.  The handle's
 * own shift_alpha is not changed.  alpha_used and attempts (host, may be NULL)
 * receive the successful alpha and the number of attempts made.  Returns IC_OK, or
 * IC_ERR_BREAKDOWN when every attempt broke down (the handle then holds no factor),
 * or the error of a failing attempt. */
int ic_numeric_shifted(ic_handle* h, const void* A_vals, double alpha_first, double alpha0, int max_tries,
                       double* alpha_used, int* attempts, void* stream);

/* Shift-predictor MLP (8 standardised features -> 32 ReLU -> 32 ReLU -> log10 alpha),
 * FP32 parameters on the device of creation, trained and evaluated by the library's
 * kernels.  Parameters (ic_mlp_n_params() floats) in the order W1 (8 x 32 row-major,
 * feature f to unit h at f*32 + h), b1 (32), W2 (32 x 32 row-major, unit g to unit h
 * at g*32 + h), b2 (32), w3 (32), b3.  The paper has no counterpart: this is the
 * learned part of the shift retry. */
typedef struct ic_mlp ic_mlp;
int ic_mlp_n_params(void);
/* params (host, NULL: zeros) are copied; Adam moments start at zero. */
int ic_mlp_create(const float* params, ic_mlp** out);
int ic_mlp_set_params(ic_mlp* m, const float* params);
int ic_mlp_get_params(const ic_mlp* m, float* params);
/* Feature standardisation z = (x - mean) / std (host, 8 floats each; std > 0). */
int ic_mlp_set_scaling(ic_mlp* m, const float* mean, const float* std);
int ic_mlp_get_scaling(const ic_mlp* m, float* mean, float* std);
/* y[i] = network(X[i]) for n samples; X (device, n x 8 row-major), y (device, n). */
int ic_mlp_forward(ic_mlp* m, const float* X, int64_t n, float* y, void* stream);
/* Loss (1 / 2n) sum (y_i - t_i)^2 and its gradient with respect to the parameters,
 * without an update; X, t device; grad (host, n_params floats) and loss (host) may be
 * NULL.  The stream is synchronised. */
int ic_mlp_gradient(ic_mlp* m, const float* X, const float* t, int64_t n, float* grad, float* loss, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected; the handle counts the
 * steps) on the loss above with learning rate lr; loss (host, may be NULL) receives
 * the loss before the step (the stream is then synchronised). */
int ic_mlp_train_step(ic_mlp* m, const float* X, const float* t, int64_t n, float lr, float* loss, void* stream);
/* alpha = 10^network(features) for one feature vector (host, 8 doubles). */
int ic_mlp_predict_shift(ic_mlp* m, const double* features, double* alpha, void* stream);
void ic_mlp_destroy(ic_mlp* m);

void ic_destroy(ic_handle* h);

/* Static English text for a status code. */
const char* ic_strerror(int status);

/* Detail text of the last failing call made by the calling thread ("" if none).
 * Valid until that thread's next failing call. */
const char* ic_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ICK_H */
