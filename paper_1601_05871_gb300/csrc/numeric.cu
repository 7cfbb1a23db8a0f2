// Numeric phase of IC(k) by blocks (Section 3.3) on sm_103a.
//
// One persistent kernel drains a device ready queue of work items.  A work item is a
// block task of the Cholesky-by-blocks DAG (Chol, Trsm, Herk, Gemm) or, for Herk and
// Gemm, a chunk of its target rows.  A task's in-degree counter is decremented by
// each finishing predecessor; the predecessor that brings it to zero pushes the
// task's items onto the queue (the scheduler duties of Section 2.2: track ready and
// waiting tasks, run ready ones, release dependents on completion).
//
// Inside a task every target row r is owned by one warp (data parallelism within a
// task, the remedy Section 6 plans for task granularity).  The warp stages the
// target segment of row r in shared memory and applies, pivot by pivot in ascending
// order, U_rc -= U_pr * U_pc for the columns c of the pivot row's source segment
// that belong to the target segment; other contributions fall outside the IC(k)
// pattern S and are discarded.  Chol and Trsm rows depend on earlier rows of the
// same diagonal block; those waits use per-row completion flags in shared memory.
// Every wait is bounded by a %globaltimer deadline and ends in a status bit.
#include <cstdint>

#include "ick_internal.h"

namespace ick {
namespace {

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

template <bool EXACT>
__device__ __forceinline__ double sub_product(double acc, double a, double b) {
    if (EXACT) return __dsub_rn(acc, __dmul_rn(a, b));
    return fma(-a, b, acc);
}

enum Mode { M_CHOL = 0, M_TRSM = 1, M_UPDATE = 2 };

struct Smem {
    int task, chunk, next, pad;
};

// Segment [b, e) of pivot row p that lies in block column `blk`, or an empty range.
__device__ __forceinline__ int2 row_segment(const DevPlan& P, int p, int blk) {
    const int s0 = __ldg(P.rseg_ptr + p), s1 = __ldg(P.rseg_ptr + p + 1);
    for (int s = s0; s < s1; ++s)
        if (__ldg(P.rseg_blk + s) == blk) return __ldg(P.rseg_se + s);
    return make_int2(0, 0);
}

__device__ __forceinline__ void set_timeout(const DevPlan& P, int site) {
    atomicOr(P.counters + 2, kStTimeout);
    atomicExch(P.counters + 3, 1);
    atomicExch(P.diag + 1, site);
}

// Wait until done[local] is set by another warp of this CTA; false on timeout/abort.
__device__ bool wait_row(const DevPlan& P, volatile unsigned char* done, int local,
                         unsigned long long deadline) {
    unsigned spins = 0;
    while (done[local] == 0) {
        if ((++spins & 255) == 0) {
            if (ld_volatile(P.counters + 3)) return false;
            if (gtimer() > deadline) { set_timeout(P, 2); return false; }
        }
        __nanosleep(20);
    }
    __threadfence_block();
    return true;
}

// One target row: r, pivots csc[ca, cb), target segment [tb, te) of row r.
// MODE: Chol (source = pivot row's block-k segment from column r on; wait on pivot
// rows; finalise with sqrt and scaling), Trsm (source = pivot row's block-j segment;
// wait on pivot rows that have one; finalise by dividing by U_rr), Update (Herk/Gemm:
// all inputs final).  start_at_r: the source segment starts at the pivot's entry in
// column r (target block column == block of r).
template <int MODE, bool EXACT>
__device__ void process_target(const DevPlan& P, double* U, int r, int ca, int cb, int tb, int te,
                               int srcblk, bool start_at_r, int rbase,
                               volatile unsigned char* done, int* tcol, double* tval,
                               unsigned long long deadline) {
    const int lane = threadIdx.x & 31;
    double piv = 1.0;
    if (MODE == M_TRSM) piv = __ldcg(U + __ldg(P.urp + r));
    for (int c0 = tb; c0 < te; c0 += kSegCap) {
        const int m = min(kSegCap, te - c0);
        for (int x = lane; x < m; x += 32) {
            tcol[x] = __ldg(P.ucol + c0 + x);
            tval[x] = __ldcg(U + c0 + x);
        }
        __syncwarp();
        const int cmin = tcol[0], cmax = tcol[m - 1];
        for (int q0 = ca; q0 < cb; q0 += 32) {
            const int nq = min(32, cb - q0);
            int p = 0, pos = 0, sb = 0, se = 0;
            if (lane < nq) {
                const int2 pe = __ldg(P.csc + q0 + lane);
                p = pe.x;
                pos = pe.y;
                const int2 s = row_segment(P, p, srcblk);
                sb = start_at_r ? pos : s.x;
                se = s.y;
            }
            for (int q = 0; q < nq; ++q) {
                const int pq = __shfl_sync(0xffffffffu, p, q);
                const int posq = __shfl_sync(0xffffffffu, pos, q);
                const int sbq = __shfl_sync(0xffffffffu, sb, q);
                const int seq = __shfl_sync(0xffffffffu, se, q);
                if (seq <= sbq) continue;
                if (MODE != M_UPDATE) {
                    int ok = 1;
                    if (lane == 0) ok = wait_row(P, done, pq - rbase, deadline);
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) return;
                }
                const double upr = __ldcg(U + posq);
                for (int e = sbq + lane; e < seq; e += 32) {
                    const int c = __ldg(P.ucol + e);
                    if (c < cmin || c > cmax) continue;
                    int lo = 0, hi = m - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (tcol[mid] < c) lo = mid + 1; else hi = mid;
                    }
                    if (tcol[lo] == c) tval[lo] = sub_product<EXACT>(tval[lo], upr, __ldcg(U + e));
                }
                __syncwarp();
            }
        }
        if (MODE == M_CHOL) {
            if (c0 == tb) {
                if (lane == 0) {
                    const double d = tval[0];
                    if (!(d > 0.0) || !isfinite(d)) {
                        atomicOr(P.counters + 2, kStBreakdown);
                        atomicMin(P.brk_row, (long long)r);
                    }
                    piv = sqrt(d);
                    tval[0] = piv;
                }
                piv = __shfl_sync(0xffffffffu, piv, 0);
                __syncwarp();
                for (int x = 1 + lane; x < m; x += 32) tval[x] = tval[x] / piv;
            } else {
                for (int x = lane; x < m; x += 32) tval[x] = tval[x] / piv;
            }
        } else if (MODE == M_TRSM) {
            for (int x = lane; x < m; x += 32) tval[x] = tval[x] / piv;
        }
        __syncwarp();
        for (int x = lane; x < m; x += 32) __stcg(U + c0 + x, tval[x]);
        __syncwarp();
    }
}

template <int WARPS, bool EXACT>
__global__ void __launch_bounds__(WARPS * 32)
numeric_persistent(DevPlan P, int epoch, unsigned long long timeout_ns) {
    __shared__ Smem sm;
    __shared__ unsigned char s_done[kMaxBlockRows];
    __shared__ int s_tcol[WARPS][kSegCap];
    __shared__ double s_tval[WARPS][kSegCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* U = static_cast<double*>(P.uval);
    const unsigned long long deadline = gtimer() + timeout_ns;
    volatile unsigned char* done = s_done;

    for (;;) {
        if (threadIdx.x == 0) {
            int task = -1, chunk = 0;
            const int slot = atomicAdd(P.counters + 0, 1);
            if (slot < P.total_items) {
                unsigned spins = 0;
                bool ok = true;
                while (ld_volatile(P.qstamp + slot) != epoch) {
                    if ((++spins & 63) == 0) {
                        if (ld_volatile(P.counters + 3)) { ok = false; break; }
                        if (gtimer() > deadline) { set_timeout(P, 1); ok = false; break; }
                    }
                    __nanosleep(64);
                }
                if (ok) {
                    __threadfence();
                    const volatile int* q = reinterpret_cast<const volatile int*>(P.queue + slot);
                    task = q[0];
                    chunk = q[1];
                }
            }
            sm.task = task;
            sm.chunk = chunk;
        }
        __syncthreads();
        const int task = sm.task, chunk = sm.chunk;
        if (task < 0) break;
        const int4 T = __ldg(P.task + task);
        const int t0 = __ldg(P.tgt_ptr + task), nt = __ldg(P.tgt_ptr + task + 1) - t0;

        if (T.x == T_CHOL || T.x == T_TRSM) {
            const int blk = T.y;
            const int rbase = __ldg(P.ranges + blk), nrows = __ldg(P.ranges + blk + 1) - rbase;
            for (int i = threadIdx.x; i < nrows; i += WARPS * 32) s_done[i] = 0;
            if (threadIdx.x == 0) sm.next = 0;
            __syncthreads();
            for (;;) {
                int idx = 0;
                if (lane == 0) idx = atomicAdd(&sm.next, 1);
                idx = __shfl_sync(0xffffffffu, idx, 0);
                if (idx >= nt) break;
                const int4 g = __ldg(P.tgt + t0 + idx);
                const int gend = __ldg(P.tgt_end + t0 + idx);
                if (T.x == T_CHOL)
                    process_target<M_CHOL, EXACT>(P, U, g.x, g.y, g.z, g.w, gend, blk, true, rbase,
                                                  done, s_tcol[warp], s_tval[warp], deadline);
                else
                    process_target<M_TRSM, EXACT>(P, U, g.x, g.y, g.z, g.w, gend, T.w, false, rbase,
                                                  done, s_tcol[warp], s_tval[warp], deadline);
                __threadfence_block();
                __syncwarp();
                if (lane == 0) done[g.x - rbase] = 1;
            }
        } else {
            const int first = chunk * P.rows_per_item;
            const int last = min(nt, first + P.rows_per_item);
            const bool herk = (T.x == T_HERK);
            for (int idx = first + warp; idx < last; idx += WARPS) {
                const int4 g = __ldg(P.tgt + t0 + idx);
                const int gend = __ldg(P.tgt_end + t0 + idx);
                process_target<M_UPDATE, EXACT>(P, U, g.x, g.y, g.z, g.w, gend, T.w, herk, 0, done,
                                                s_tcol[warp], s_tval[warp], deadline);
            }
        }
        __threadfence();
        __syncthreads();

        // release: the CTA that finishes a task's last item decrements its successors
        if (warp == 0) {
            int last = 0;
            if (lane == 0) {
                last = atomicSub(P.items_left + task, 1) == 1;
                atomicAdd(P.diag + 0, 1);
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                const int s0 = __ldg(P.succ_ptr + task), s1 = __ldg(P.succ_ptr + task + 1);
                for (int e = s0 + lane; e < s1; e += 32) {
                    const int s = __ldg(P.succ + e);
                    if (atomicSub(P.indeg + s, 1) == 1) {
                        const int ni = __ldg(P.nitems + s);
                        const int base = atomicAdd(P.counters + 1, ni);
                        for (int c = 0; c < ni; ++c) P.queue[base + c] = make_int2(s, c);
                        __threadfence();
                        for (int c = 0; c < ni; ++c)
                            *reinterpret_cast<volatile int*>(P.qstamp + base + c) = epoch;
                    }
                }
            }
        }
    }
}

// Scatter of B's values onto the pattern S (zero on fill, optional diagonal shift)
// and reset of the scheduler state.  gsrc >= 0: index into A's values; -1: fill;
// <= -2: the diagonal, whose index is -2 - gsrc.
__global__ void numeric_prepare(DevPlan P, const double* __restrict__ av, double alpha, int nnz_u,
                                int epoch) {
    const int stride = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double* U = static_cast<double*>(P.uval);
    for (int pos = tid; pos < nnz_u; pos += stride) {
        const int s = __ldg(P.gsrc + pos);
        double v = 0.0;
        if (s >= 0) {
            v = __ldg(av + s);
        } else if (s <= -2) {
            v = __ldg(av + (-2 - s));
            if (alpha != 0.0) v = __dadd_rn(v, __dmul_rn(alpha, v));
        }
        U[pos] = v;
    }
    for (int t = tid; t < P.ntasks; t += stride) {
        P.indeg[t] = __ldg(P.indeg0 + t);
        P.items_left[t] = __ldg(P.nitems + t);
    }
    for (int s = tid; s < P.nseeds; s += stride) {
        P.queue[s] = __ldg(P.seeds + s);
        P.qstamp[s] = epoch;
    }
    if (tid == 0) {
        P.counters[0] = 0;
        P.counters[1] = P.nseeds;
        P.counters[2] = 0;
        P.counters[3] = 0;
        *P.brk_row = 0x7fffffffffffffffLL;
        P.diag[0] = 0;
        P.diag[1] = 0;
    }
}

template <int WARPS, bool EXACT>
cudaError_t launch_t(const DevPlan& P, int grid, int epoch, unsigned long long timeout_ns,
                     cudaStream_t s) {
    numeric_persistent<WARPS, EXACT><<<grid, WARPS * 32, 0, s>>>(P, epoch, timeout_ns);
    return cudaGetLastError();
}

}  // namespace

cudaError_t numeric_blocks_per_sm(int warps, bool exact, int* blocks) {
    if (warps == 8)
        return exact ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, numeric_persistent<8, true>, 256, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, numeric_persistent<8, false>, 256, 0);
    return exact ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, numeric_persistent<16, true>, 512, 0)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, numeric_persistent<16, false>, 512, 0);
}

cudaError_t launch_numeric_prepare(const DevPlan& P, const double* avals, double shift_alpha,
                                   int epoch, cudaStream_t s) {
    const int work = P.nnz_u > P.ntasks ? P.nnz_u : P.ntasks;
    int pgrid = (work + 255) / 256;
    pgrid = pgrid < 1 ? 1 : (pgrid > 8192 ? 8192 : pgrid);
    numeric_prepare<<<pgrid, 256, 0, s>>>(P, avals, shift_alpha, P.nnz_u, epoch);
    return cudaGetLastError();
}

cudaError_t launch_numeric(const DevPlan& P, int epoch, int warps, bool exact, int grid,
                           unsigned long long timeout_ns, cudaStream_t s) {
    if (warps == 8)
        return exact ? launch_t<8, true>(P, grid, epoch, timeout_ns, s)
                     : launch_t<8, false>(P, grid, epoch, timeout_ns, s);
    return exact ? launch_t<16, true>(P, grid, epoch, timeout_ns, s)
                 : launch_t<16, false>(P, grid, epoch, timeout_ns, s);
}

}  // namespace ick
