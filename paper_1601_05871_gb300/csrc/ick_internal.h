// Internal declarations shared by the host C++ (symbolic phase, C ABI) and the CUDA
// kernels of libick.so.  Not part of the public interface (include/ick.h is).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ick.h"

namespace ick {

// Block task types of the Cholesky-by-blocks generator (Section 3.3).
enum TaskType : int { T_CHOL = 0, T_TRSM = 1, T_HERK = 2, T_GEMM = 3 };

constexpr int kMaxBlockRows = 8192;  // per-row completion flags of one block live in shared memory
constexpr int kSegCap = 128;         // target-segment entries staged per warp in shared memory
constexpr int kClaimPad = 8;         // level runs of the padded solve orders are multiples of this

// Internal entries of the rows of a block-DAG solve (host_solve.cpp): per row i the
// entries [ptr[i], ptr[i+1]); j = source row - range start, pos = position of the
// value in U's row-major storage.
struct SolveLayout {
    std::vector<int32_t> ptr, j, pos;
};

// Tasks of one direction of the block-DAG solves, in claim order: (type 0 = E /
// 1 = L, range, first order position, end order position), in-degrees, successors.
struct SolveTasks {
    std::vector<int4> task;
    std::vector<int32_t> indeg0, succ_ptr, succ;
    std::vector<int32_t> next;  // per L task: the same range's next part (-1: none; E tasks -1)
};

// Everything the symbolic phase produces, in host memory.
struct HostPlan {
    int64_t n = 0, nnz_a = 0, nnz_u = 0;
    int k = 0;
    std::vector<int32_t> perm, iperm;
    std::vector<int64_t> arp;       // A pattern (original order), for SpMV in PCG
    std::vector<int32_t> acol;
    // U = L^T, upper CSR in permuted order, diagonal first in every row
    std::vector<int64_t> urp;
    std::vector<int32_t> ucol;
    std::vector<int32_t> ulev;      // level of fill of each entry
    std::vector<int32_t> gsrc;      // per U position: A value index; -1 fill; -2-idx diagonal
    std::vector<int32_t> udiag_src; // per row: index of A's diagonal entry
    // 2D block matrix: block ranges and per-row block segments
    std::vector<int32_t> ranges;    // nb + 1 boundaries
    std::vector<int32_t> blk_of;    // block of each row
    std::vector<int32_t> rseg_ptr;  // n + 1
    std::vector<int32_t> rseg_blk;  // block column of each segment
    std::vector<int2> rseg_se;      // [begin, end) positions of each segment in U
    // column lists of U (strictly upper): for column r, pivot rows p < r ascending
    std::vector<int32_t> cptr;      // n + 1
    std::vector<int2> csc;          // (p, position of U_pr)
    std::vector<int32_t> cseg_end;  // per column-list entry: end of row p's segment in block(r)
    // block pattern (upper), bptr: nb + 1
    std::vector<int64_t> bptr;
    std::vector<int32_t> bcol;
    // tasks in generation order
    std::vector<int4> task;         // (type, k, i, j)
    std::vector<int64_t> pred_ptr;
    std::vector<int32_t> pred;
    std::vector<int32_t> succ_ptr, succ;
    std::vector<int32_t> indeg0, nitems;
    // Chol/Trsm tasks spread over several CTAs (nitems > 1): offset of their block's
    // rows in soff, -1 for the others (completion flags in shared memory).  A split
    // task's finished rows are published in a shadow array: row r's target segment
    // [tb, te) sits at shadow positions tb + soff[...], congruent to tb modulo 4
    std::vector<int32_t> flag_off, soff;
    int64_t nflags = 0, nsplit = 0, nshadow = 0;
    std::vector<int32_t> tgt_ptr;   // ntasks + 1
    std::vector<int4> tgt;          // (r, csc_a, csc_b, seg_begin)
    std::vector<int32_t> tgt_end;   // seg_end
    std::vector<int2> claim;        // (task, chunk) of every work item in claim order
    std::vector<int32_t> fwd_order, bwd_order;  // claim orders of the triangular solves
    std::vector<int32_t> fwd_pad, bwd_pad;      // the same, each level padded with -1
    int64_t fwd_depth = 0, bwd_depth = 0;        // levels of the row dependence DAGs
    // block-DAG solves (host_solve.cpp): per row the start of the internal entries
    // (forward: absolute column-list index; backward: count after the diagonal), per
    // range the padded local orders, and each direction's tasks
    std::vector<int32_t> sf_split, sb_nint;
    std::vector<int32_t> lf_ptr, lf_ord, lb_ptr, lb_ord;
    std::vector<int32_t> lf_need, lb_need;  // per order position: rows of lower levels
    SolveLayout xf, xb;                     // forward / backward internal entries
    SolveTasks fs, bs;
    int32_t max_range_rows = 0;
    int64_t total_items = 0;
    int64_t critical_path = 0;
    int64_t max_level = 0;
    int64_t ntype[4] = {0, 0, 0, 0};
    double flops = 0.0, bytes = 0.0;
    int rows_per_item = 32;
};

// Plain pointers handed to the kernels by value.
struct DevPlan {
    int n, nnz_u, nb, ntasks, total_items, rows_per_item;
    const long long* urp;
    const int* ucol;
    const int* gsrc;
    const int* ranges;
    const int* rseg_ptr;
    const int* rseg_blk;
    const int2* rseg_se;
    const int* cptr;
    const int2* csc;
    const int* cseg_end;
    const int4* task;
    const int* tgt_ptr;
    const int4* tgt;
    const int* tgt_end;
    const int* nitems;
    const int* succ_ptr;
    const int* succ;
    const int* indeg0;
    const int2* claim;     // work items (task, chunk) in the order the CTAs claim them
    const int* flag_off;   // per task: its block's rows in soff (split Chol/Trsm) or -1
    const int* soff;       // per row of a split task's block: shadow position - U position
    long long nshadow;
    // mutable state
    void* uval;            // factor values (double for IC_F64)
    int* indeg;
    int* items_left;
    int* counters;         // [0] claim counter, [1] unused, [2] status bits, [3] abort
    long long* brk_row;    // smallest breakdown row
    int* diag;             // [0] items completed, [1] timeout site
    unsigned long long* trace;  // NULL, or 4 words per queue slot: start ns, end ns,
                                // task | chunk << 32, SM id
    double* udiag;         // IC_F32: FP64 diagonal pivots (U_ii) of the factor
    double* urcp;          // FMA mode: 1/U_ii of every row, kept by its Chol for Trsm
    const int* diag_src;   // IC_F32: index of A's diagonal value of each row
    void* shadow;          // finished rows of split Chol/Trsm tasks, else the sentinel
    int* row_next;         // per task: next target to claim (split Chol/Trsm)
};

// Status bits written by the kernels into counters[2].
constexpr int kStBreakdown = 1;
constexpr int kStTimeout = 2;

// Device-side buffers of the triangular solves and PCG.
struct SolvePlan {
    int n;
    long long nnz_a;
    const long long* urp;
    const int* ucol;
    const int* cptr;
    const int2* csc;
    const double* uval;
    const int* perm;
    const long long* arp;
    const int* acol;
    double* y;       // permuted work vector
    int* flag;       // per-row completion stamps of the solves
    int* counter;    // [0] forward row claim, [1] backward row claim, [2] abort word of the
                     // running application (cleared when each one starts), [3] timeout
                     // record (set with the abort word, cleared by the host when read)
    const int* fwd_order;  // rows in forward claim order (by dependence depth)
    const int* bwd_order;  // rows in backward claim order
    const int* fwd_pad;    // padded claim orders (-1: empty slot) and their lengths
    const int* bwd_pad;
    int nfwd_pad, nbwd_pad;
    double* rdiag;         // 1 / U_ii, computed after each numeric factorization
    int lanes_per_row;     // 4, 8, 16 or 32 lanes per row in the ic_apply solves
    int dtype;             // IC_F64 or IC_F32 (factor values and solves in FP32)
    const float* uval32;   // IC_F32 factor values
    const double* udiag;   // IC_F32 FP64 pivots
    float* rdiag32;        // IC_F32 reciprocal pivots
    // block-DAG solves (blocksolve.cu); see HostPlan for the meaning of the arrays
    int solve_mode;        // 0: block-DAG solves, 1: row-level solves in level order
    int nranges, max_range_rows, nftask, nbtask, noff;
    const int* ranges;     // nranges + 1 row boundaries of the block rows
    const int* sf_split;
    const int* sb_nint;
    const int* lf_ptr;
    const int* lf_ord;
    const int* lb_ptr;
    const int* lb_ord;
    const int* lf_need;
    const int* lb_need;
    // internal entries per direction (SolveLayout) and their values (solve type),
    // gathered from the factor after each numeric phase
    const int* xf_ptr;
    const int* xf_j;
    const int* xf_pos;
    void* xf_val;
    const int* xb_ptr;
    const int* xb_j;
    const int* xb_pos;
    void* xb_val;
    int nxf, nxb;
    void* uvt;             // factor values in column-list (csc) order, refreshed after each
                           // numeric phase: the forward solve reads them contiguously
    const int4* ftask;     // tasks in claim order: (0 = E / 1 = L, range, first, end order position)
    const int4* btask;
    const int* f_succ_ptr; // successors of each task (indices into the same direction's list)
    const int* f_succ;
    const int* b_succ_ptr;
    const int* b_succ;
    const int* dag_indeg0; // in-degrees, forward tasks then backward, copied into dag_indeg
    int* dag_indeg;        // before each apply
    const int* f_next;     // per task: the same range's next L part, or -1
    const int* b_next;
    int* dag_taken;        // per task (forward then backward): 1 once a CTA has taken it
    void* dag_w;           // external sums of the rows, n values of the solve type per
                           // direction (forward, then backward); 0 where a row has none
    unsigned long long* trace;  // NULL, or 4 words per task: forward tasks, then backward
};

// Kernel entry points (numeric.cu, solve.cu).
cudaError_t launch_numeric_prepare(const DevPlan& P, const double* avals, double shift_alpha, int dtype,
                                   cudaStream_t s);
cudaError_t launch_numeric(const DevPlan& P, int warps, bool exact, int dtype, int grid,
                           unsigned long long timeout_ns, cudaStream_t s);
cudaError_t numeric_blocks_per_sm(int warps, bool exact, int dtype, int* blocks);

// t0 / t1 (may be NULL): events recorded just before the forward and just before the
// backward solve kernel.
cudaError_t launch_apply(const SolvePlan& S, const double* r, double* z, int epoch,
                         unsigned long long timeout_ns, int grid, cudaStream_t s,
                         cudaEvent_t t0 = nullptr, cudaEvent_t t1 = nullptr);
cudaError_t launch_apply_dag(const SolvePlan& S, const double* r, double* z, unsigned long long timeout_ns,
                             int grid, cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1);
cudaError_t launch_dag_prepare(const SolvePlan& S, cudaStream_t s);
int dag_prepare_launches(const SolvePlan& S);
cudaError_t dag_blocks_per_sm(int lanes, int dtype, int max_range_rows, int* blocks);
cudaError_t launch_spmv(const SolvePlan& S, const double* av, const double* x, double* y,
                        cudaStream_t s);
cudaError_t apply_blocks_per_sm(int* blocks);
cudaError_t launch_solve_prepare(const SolvePlan& S, cudaStream_t s);
// Allocation-free application (solve.cu): scratch in a file-scope device array.
constexpr int kStaticApplyDevices = 64;  // devices whose scratch address is cached
int static_apply_max_rows();
// Reads and clears the timeout record of the current device's scratch (*timed_out = 0
// or 1); synchronises the stream.
cudaError_t static_apply_timeout(int* timed_out, cudaStream_t s);
cudaError_t launch_apply_static(const SolvePlan& S, const double* r, double* z, int epoch,
                                unsigned long long timeout_ns, int grid, cudaStream_t s,
                                bool clear_stamps);

// PCG vector kernels (solve.cu): scalars live in a small device struct.  Reductions
// are two-stage and deterministic: nparts block partials, then one block sums them in
// a fixed order and applies `op` (0: alpha = rz/pq, 1: relres = sqrt(rr)/|b|,
// 2: beta = rz_new/rz and rz = rz_new, 3: rz, 4: |b|).
struct PcgScalars {
    double rz, rz_new, pq, rr, bnorm, alpha, beta, relres;
};
constexpr int kMaxParts = 1024;
int pcg_parts(int n);
cudaError_t pcg_dot(const double* a, const double* b, int n, double* partial, int nparts,
                    cudaStream_t s);
cudaError_t pcg_finish(const double* partial, int nparts, PcgScalars* sc, int op, cudaStream_t s);
cudaError_t pcg_step_x_r(int n, double* x, double* r, const double* p, const double* q,
                         PcgScalars* sc, double* partial, int nparts, cudaStream_t s);
cudaError_t pcg_step_p(int n, double* p, const double* z, PcgScalars* sc, cudaStream_t s);
cudaError_t pcg_init(int n, const double* b, double* x, double* r, cudaStream_t s);
// pcg_solve's device-side loop test: iteration count and the WHILE node's condition.
cudaError_t pcg_loop_step(PcgScalars* sc, int* it, double tol, int maxit, cudaGraphConditionalHandle cond,
                          bool first, cudaStream_t s);

// Batched PCG (batch.cu): per-system scalars of systems stored block-diagonally.
struct BatchScalars {
    double *tmp, *rz, *bnorm, *alpha, *beta, *relres;
    int *active, *iters, *nactive, *iter;
};
cudaError_t batch_dot(const long long* row_off, int count, const double* a, const double* b,
                      double* out, cudaStream_t s);
cudaError_t batch_scalars(const BatchScalars& B, int count, int op, double tol, cudaStream_t s);
cudaError_t batch_bump(const BatchScalars& B, cudaStream_t s);
cudaError_t batch_xr(int n, const int* sys, const double* alpha, double* x, double* r, const double* p,
                     const double* q, cudaStream_t s);
cudaError_t batch_p(int n, const int* sys, const double* beta, const int* active, double* p,
                    const double* z, cudaStream_t s);

// Learned diagonal shift (shift.cu).
constexpr double kShiftDdCap = 1000.0;  // diagonal dominance of a row without off-diagonals
constexpr int kMlpFeatures = 8;
constexpr int kMlpHidden = 32;
constexpr int kMlpParams = kMlpFeatures * kMlpHidden + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden +
                           kMlpHidden + 1;
constexpr int kMlpMaxBlocks = 1024;     // partial-gradient blocks of one gradient evaluation
struct MlpDev {
    float *theta, *m, *v, *grad;  // parameters, Adam moments, last gradient (kMlpParams each)
    float *mean, *rstd;           // feature standardisation: (x - mean) * rstd
    float *part, *loss_part, *loss;  // per-block partial gradients and losses, the loss
};
int mlp_grad_blocks(long long n);
cudaError_t launch_features(int n, const long long* rp, const int* ci, const double* v, int k, double nu,
                            void* scratch, double* out, cudaStream_t s);
size_t features_scratch_bytes();
cudaError_t launch_mlp_forward(const MlpDev& M, const float* X, long long n, float* y, cudaStream_t s);
cudaError_t launch_mlp_grad(const MlpDev& M, const float* X, const float* t, long long n, cudaStream_t s);
cudaError_t launch_mlp_adam(const MlpDev& M, float lr, int step, cudaStream_t s);

// FMA throughput of the current GPU in GFLOP/s (probe.cu); synchronises the stream.
cudaError_t measure_fma_peak(int dtype, double* gflops, cudaStream_t s);

// Host symbolic phase (host.cpp).
// k_order: updates into each block applied in ascending k (the task generator's order,
// which exact mode needs); otherwise ordered by the estimated readiness of their inputs.
// solve_ctas: the CTAs of the block-DAG solves' grid, for their claim order's schedule.
int build_plan(const ic_csr_pattern* A, int k, const int32_t* perm, const int64_t* ranges,
               int64_t nranges, int block_rows, int rows_per_item, int threads, bool k_order,
               int solve_ctas, HostPlan& P, std::string& err);
void build_solve_dag(HostPlan& P, int threads, int ctas);
void build_claim_order(HostPlan& P, int nctas);
int block_dag(int64_t nb, const int64_t* bptr, const int32_t* bcol, std::vector<int4>& task,
              std::vector<int64_t>& pred_ptr, std::vector<int32_t>& pred);
int nd_grid(int nx, int ny, int nz, int dof, int leaf_rows, int sep_colours, int leaf_colours,
            const uint8_t* keep, int32_t* perm, int64_t* ranges, int64_t* nranges, int64_t* n_out);

}  // namespace ick
