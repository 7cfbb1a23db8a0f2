// Block-DAG triangular solves of ic_apply: L y = r (forward) and L^T z = y (backward)
// with L = U^T the incomplete factor.
//
// The 2D block structure of Section 3.2 organises the solve like the factorization's
// task DAG (Section 3.3): a range of rows (a block row), its rows in local
// dependence-level order, is cut into parts of whole levels.  Task E sums, for a chunk
// of a part's rows, the entries whose other index lies in another range, once the
// parts holding those rows have finished; task L is one CTA that solves a part's rows
// with the remaining, internal entries after the range's previous part, the range's
// results kept in shared memory, so a dependence inside a range costs a
// shared-memory round trip rather than an L2 one.  Nested-dissection leaves are
// independent in the forward solve and run concurrently; a separator's first parts
// run while its subdomains are still finishing.
//
// Scheduling: one persistent grid per direction claims tasks in a fixed topological
// order (atomic counter), waits (bounded) until the task's in-degree reaches zero,
// runs it and releases its successors; a CTA that finishes an L part runs the same
// range's next part itself when it is ready, keeping its shared-memory state.  Every
// task a CTA waits for was claimed earlier by a resident CTA (or is running as a
// continuation), so the claims cannot deadlock.  All waits give up at the deadline or
// when another CTA has set the abort word, and the host reports IC_ERR_TIMEOUT.
#include <cstdint>

#include "ick_internal.h"

namespace ick {
namespace {

constexpr int kDagThreads = 512;

__device__ __forceinline__ unsigned long long gclock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool aborted(const int* abort_word) {
    return *reinterpret_cast<const volatile int*>(abort_word) != 0;
}

// Ends the solve after a wait gave up: the abort word stops every other waiting CTA
// of this launch (it is cleared when the next application starts); the word after it
// records the timeout until the host reads it.
__device__ __forceinline__ void raise_abort(int* abort_word) {
    atomicExch(abort_word, 1);
    atomicOr(abort_word + 1, 1);
}

// Thread 0: wait until *c is zero; false on abort or timeout.
__device__ bool await_zero(const int* c, int* abort_word, unsigned long long deadline) {
    const volatile int* p = c;
    unsigned spins = 0;
    while (*p != 0) {
        if ((++spins & 63) == 0 && (aborted(abort_word) || gclock() > deadline)) {
            raise_abort(abort_word);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// Lane 0: wait until the range's count of completed rows reaches need (one shared
// word, read by one lane per waiting warp); false on abort or timeout.
__device__ bool await_count(const int* done, int need, int* abort_word, unsigned long long deadline) {
    const volatile int* p = done;
    unsigned spins = 0;
    int d;
    while ((d = *p) < need) {
        if ((++spins & 255) == 0 && (aborted(abort_word) || gclock() > deadline)) {
            raise_abort(abort_word);
            return false;
        }
        (void)d;
    }
    __threadfence_block();
    return true;
}

template <int G, typename T>
__device__ __forceinline__ T sum_group(T v) {
    const int lane = threadIdx.x & 31;
    const unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// A row's first 64 internal entries are loaded into registers (64 / G per lane)
// before its wait, so the loads overlap the wait and leave the dependence chain.
template <int G>
struct Held {
    static constexpr int M = 64 / G;
};

// Marks the warp's rows complete: every lane's stores precede the count update.
__device__ __forceinline__ void complete_rows(int* done, unsigned rows_mask) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0 && rows_mask) {
        __threadfence_block();
        atomicAdd(done, __popc(rows_mask));
    }
}

// ------------------------------------------------------------------ forward tasks

// E: w_i = sum of U_pi y_p over the column-list entries of row i with p outside the
// row's range (a prefix of the list, pivots ascending), for the rows at order
// positions [lo, hi).  The values come from the column-ordered copy, contiguous with
// the column lists.
template <int G, typename T>
__device__ void fwd_external(const SolvePlan& S, const T* __restrict__ uvt, const T* y, T* w, int lo, int hi) {
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31, sub = lane / G, sl = lane % G;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = lo + warp * R; base < hi; base += nw * R) {
        const int i = base + sub < hi ? __ldg(S.lf_ord + base + sub) : -1;
        T acc = T(0);
        int a = 0, b = 0;
        if (i >= 0) {
            a = __ldg(S.cptr + i);
            b = __ldg(S.sf_split + i);
            for (int q = a + sl; q < b; q += G) acc = fma(__ldg(uvt + q), ldcg(y + __ldg(&S.csc[q].x)), acc);
        }
        acc = sum_group<G>(acc);
        if (sl == 0 && a < b) w[i] = acc;
    }
}

// L of either direction: the rows at order positions [lo, hi) of range k (whole
// levels), G lanes per row and 32/G rows per warp (one level per claim).  The range's
// earlier results (positions before lo, finished by the range's previous parts) are
// first loaded into shared memory and counted as complete; a row runs once every row
// of the lower levels is complete (done >= need); its internal operands come from
// shared memory and its other operands are loaded before the wait.
//   forward:  y_i = (r_perm(i) - w_i - sum) / U_ii, stored to y
//   backward: z_i = (y_i - w_i - sum) / U_ii, stored to zv and to z at perm(i)
template <int G, typename T, bool BW>
__device__ void solve_local(const SolvePlan& S, const T* __restrict__ xv, const T* __restrict__ rd_all,
                            const double* __restrict__ r, const T* y, T* out, double* __restrict__ z, const T* w,
                            int k, int lo, int hi, T* sh, int* done, bool cont,
                            unsigned long long deadline) {
    constexpr int R = 32 / G, M = Held<G>::M;
    const int lane = threadIdx.x & 31, sl = lane % G;
    const int* ord = BW ? S.lb_ord : S.lf_ord;
    const int* need_a = BW ? S.lb_need : S.lf_need;
    const int* xptr = BW ? S.xb_ptr : S.xf_ptr;
    const int* xj = BW ? S.xb_j : S.xf_j;
    const int base = __ldg((BW ? S.lb_ptr : S.lf_ptr) + k);
    const int s = __ldg(S.ranges + k);
    if (!cont) {  // a continuation already holds the range's earlier results and count
        for (int q = base + int(threadIdx.x); q < lo; q += blockDim.x) {
            const int i = __ldg(ord + q);
            if (i >= 0) sh[i - s] = ldcg(out + i);
        }
        if (threadIdx.x == 0) *done = lo > base ? __ldg(need_a + lo) : 0;
        __syncthreads();
    }
    const int len = hi - lo;
    // group g of R positions goes to warp g mod (warps): the groups of one level sit on
    // consecutive warps, i.e. on different SM sub-partitions, whose FP64 units then
    // work in parallel; each warp takes its groups in order, and a group depends only
    // on lower groups, so the waits cannot cycle
    const int nw = blockDim.x >> 5;
    for (int t0 = (threadIdx.x >> 5) * R;; t0 += nw * R) {
        if (t0 >= len) break;
        const int i = __ldg(ord + lo + t0 + lane / G);
        const int need = __ldg(need_a + lo + t0);
        T t = T(0), rd = T(0);
        int a = 0, c = 0, dst = 0;
        if (i >= 0) {
            a = __ldg(xptr + i);
            c = __ldg(xptr + i + 1);
            if (sl == 0) {
                rd = __ldg(rd_all + i);
                bool ext;
                if (BW) {
                    t = ldcg(y + i);
                    dst = __ldg(S.perm + i);
                    ext = __ldg(S.sb_nint + i) < int(__ldg(S.urp + i + 1) - __ldg(S.urp + i)) - 1;
                } else {
                    t = T(__ldg(r + __ldg(S.perm + i)));
                    ext = __ldg(S.cptr + i) < __ldg(S.sf_split + i);
                }
                if (ext) t -= ldcg(w + i);
                t *= rd;  // the row's result is t - rd * (sum of the internal products)
            }
        }
        int j[M];
        T u[M];
        int cnt = 0;
#pragma unroll
        for (int x = 0; x < M; ++x) {
            const int q = a + sl + x * G;
            j[x] = 0;
            u[x] = T(0);
            if (q < c) {
                j[x] = __ldg(xj + q);
                u[x] = __ldg(xv + q);
                cnt = x + 1;
            }
        }
        const unsigned rows = __ballot_sync(0xffffffffu, sl == 0 && i >= 0);
        const int most = __reduce_max_sync(0xffffffffu, cnt);
        int ok = 1;
        if (lane == 0) ok = await_count(done, need, S.counter + 2, deadline);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        // two accumulators halve the dependent FMA chain (64 cycles per FP64 FMA)
        T acc0 = T(0), acc1 = T(0);
#pragma unroll
        for (int x = 0; x < M; x += 2) {
            if (x >= most) break;
            if (x < cnt) acc0 = fma(u[x], sh[j[x]], acc0);
            if (x + 1 < cnt) acc1 = fma(u[x + 1], sh[j[x + 1]], acc1);
        }
        for (int q = a + sl + M * G; q < c; q += G) acc0 = fma(__ldg(xv + q), sh[__ldg(xj + q)], acc0);
        const T acc = sum_group<G>(acc0 + acc1);
        T v = T(0);
        if (sl == 0 && i >= 0) {
            v = fma(-rd, acc, t);
            sh[i - s] = v;
        }
        // the count is raised before the global stores, so its fence waits only for
        // the shared-memory results; later tasks read the global copies after the
        // task's closing fence
        complete_rows(done, rows);
        if (sl == 0 && i >= 0) {
            out[i] = v;
            if (BW) z[dst] = double(v);
        }
    }
}

// ----------------------------------------------------------------- backward tasks

// E (backward): w_i = sum of U_im z_m over the entries of row i with m beyond the
// row's range (a suffix of the row, columns ascending), for the rows at order
// positions [lo, hi).
template <int G, typename T>
__device__ void bwd_external(const SolvePlan& S, const T* __restrict__ uv, const T* zv, T* w, int lo, int hi) {
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31, sub = lane / G, sl = lane % G;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = lo + warp * R; base < hi; base += nw * R) {
        const int i = base + sub < hi ? __ldg(S.lb_ord + base + sub) : -1;
        T acc = T(0);
        long long a = 0, b = 0;
        if (i >= 0) {
            a = __ldg(S.urp + i) + 1 + __ldg(S.sb_nint + i);
            b = __ldg(S.urp + i + 1);
            for (long long q = a + sl; q < b; q += G) acc = fma(__ldg(uv + q), ldcg(zv + __ldg(S.ucol + q)), acc);
        }
        acc = sum_group<G>(acc);
        if (sl == 0 && a < b) w[i] = acc;
    }
}

// ------------------------------------------------------------------ the two grids

__device__ __forceinline__ unsigned smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

// Claims the next task; thread 0 waits until its in-degree is zero.  Returns the task
// index, or -1 when the list is exhausted or the solve was aborted.
__device__ int claim_task(int* claim_ctr, int ntasks, const int* indeg, int* taken, int* abort_word,
                          unsigned long long deadline, int* s_task, int* s_done,
                          unsigned long long* trace) {
    if (threadIdx.x == 0) {
        int t = -1;
        if (!aborted(abort_word)) {
            do {  // tasks already taken as a continuation are skipped
                t = atomicAdd(claim_ctr, 1);
            } while (t < ntasks && atomicExch(taken + t, 1) != 0);
            if (t >= ntasks) {
                t = -1;
            } else {
                const unsigned long long t0 = gclock();
                if (!await_zero(indeg + t, abort_word, deadline)) t = -1;
                if (trace && t >= 0) {
                    trace[4 * t] = t0;
                    trace[4 * t + 1] = gclock();
                    trace[4 * t + 3] = (unsigned long long)t | ((unsigned long long)smid() << 32);
                }
            }
        }
        *s_task = t;
        *s_done = 0;
    }
    __syncthreads();
    return *s_task;
}

// After a task: its results are made visible, then its successors are released.  If
// the task was an L part whose range's next part is now ready and not yet taken, the
// CTA takes it (returned; -1 otherwise) and runs it with the shared-memory state it
// already holds.
__device__ __forceinline__ int release(int t, bool is_l, const int* succ_ptr, const int* succ, const int* next,
                                       int* indeg, int* taken, unsigned long long* trace, int* s_task) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (trace) trace[4 * t + 2] = gclock();
        const int a = __ldg(succ_ptr + t), b = __ldg(succ_ptr + t + 1);
        for (int q = a; q < b; ++q) atomicSub(indeg + __ldg(succ + q), 1);
        int nx = is_l ? __ldg(next + t) : -1;
        if (nx >= 0 && !(*reinterpret_cast<volatile int*>(indeg + nx) == 0 && atomicExch(taken + nx, 1) == 0))
            nx = -1;
        if (nx >= 0) {
            __threadfence();
            if (trace) {
                const unsigned long long now = gclock();
                trace[4 * nx] = now;
                trace[4 * nx + 1] = now;
                trace[4 * nx + 3] = (unsigned long long)nx | ((unsigned long long)smid() << 32);
            }
        }
        *s_task = nx;
    }
    __syncthreads();
    return *s_task;
}

template <int G, typename T>
__global__ void __launch_bounds__(kDagThreads)
forward_dag(SolvePlan S, const T* __restrict__ uvt, const T* __restrict__ rd_all, const double* __restrict__ r,
            T* y, T* w, unsigned long long timeout_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* sh = reinterpret_cast<T*>(smem);
    __shared__ int s_task, s_done;
    const unsigned long long deadline = gclock() + timeout_ns;
    int* indeg = S.dag_indeg;
    int* taken = S.dag_taken;
    int t = -1;
    bool cont = false;
    for (;;) {
        if (t < 0) {
            t = claim_task(S.counter + 0, S.nftask, indeg, taken, S.counter + 2, deadline, &s_task, &s_done,
                           S.trace);
            cont = false;
        }
        if (t < 0) break;
        const int4 tk = S.ftask[t];
        if (tk.x == 0)
            fwd_external<G, T>(S, uvt, y, w, tk.z, tk.w);
        else
            solve_local<G, T, false>(S, static_cast<const T*>(S.xf_val), rd_all, r, nullptr, y, nullptr, w, tk.y,
                                     tk.z, tk.w, sh, &s_done, cont, deadline);
        t = release(t, tk.x == 1, S.f_succ_ptr, S.f_succ, S.f_next, indeg, taken, S.trace, &s_task);
        cont = t >= 0;
    }
}

template <int G, typename T>
__global__ void __launch_bounds__(kDagThreads)
backward_dag(SolvePlan S, const T* __restrict__ uv, const T* __restrict__ rd_all, const T* y, T* zv,
             double* __restrict__ z, T* w, unsigned long long timeout_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* sh = reinterpret_cast<T*>(smem);
    __shared__ int s_task, s_done;
    const unsigned long long deadline = gclock() + timeout_ns;
    int* indeg = S.dag_indeg + S.nftask;
    int* taken = S.dag_taken + S.nftask;
    unsigned long long* tr = S.trace ? S.trace + 4 * size_t(S.nftask) : nullptr;
    int t = -1;
    bool cont = false;
    for (;;) {
        if (t < 0) {
            t = claim_task(S.counter + 1, S.nbtask, indeg, taken, S.counter + 2, deadline, &s_task, &s_done, tr);
            cont = false;
        }
        if (t < 0) break;
        const int4 tk = S.btask[t];
        if (tk.x == 0)
            bwd_external<G, T>(S, uv, zv, w, tk.z, tk.w);
        else
            solve_local<G, T, true>(S, static_cast<const T*>(S.xb_val), rd_all, nullptr, y, zv, z, w, tk.y, tk.z,
                                    tk.w, sh, &s_done, cont, deadline);
        t = release(t, tk.x == 1, S.b_succ_ptr, S.b_succ, S.b_next, indeg, taken, tr, &s_task);
        cont = t >= 0;
    }
}

// ------------------------------------------------------ block-row solves (mode 2)
//
// One CTA solves a whole range (block row) and then claims the next range of the
// claim order.  Its rows run in level order (the level of a row in the dependence DAG
// of the whole solve), R = 32 / G rows of one level per warp group, groups spread over
// the warps round-robin.  A row's sources in other ranges are read from the global
// result vector, which starts as the all-ones bit pattern (a NaN that arithmetic never
// produces, kUnset): a value that is no longer kUnset is final, and the reader spins
// (bounded) on it, with no flag, counter or fence between the ranges.  A row's sources
// inside the range are read from shared memory once the range's count of completed
// rows reaches the rows of the row's lower levels (one shared word, polled by one lane
// of each waiting warp).  A row's sources have lower levels, so they come earlier in
// its range's order or lie in ranges claimed before its range; the waits cannot cycle.
// Each row sums its entries in a fixed order (the other ranges' entries, then its
// range's entries sorted by their source's level), so the result does not depend on
// timing.

template <typename T>
__device__ __forceinline__ bool unset(T v);
template <>
__device__ __forceinline__ bool unset<double>(double v) { return __double_as_longlong(v) == -1LL; }
template <>
__device__ __forceinline__ bool unset<float>(float v) { return __float_as_int(v) == -1; }

// A result that happens to carry the reserved pattern is published as another NaN.
template <typename T>
__device__ __forceinline__ T publishable_value(T v) {
    if (unset(v)) return sizeof(T) == 8 ? T(__longlong_as_double(0x7fffffffffffffffLL)) : T(__int_as_float(0x7fffffff));
    return v;
}

template <typename T>
__device__ __forceinline__ T ld_vol(const T* p) { return *reinterpret_cast<const volatile T*>(p); }
template <typename T>
__device__ __forceinline__ void st_vol(T* p, T v) { *reinterpret_cast<volatile T*>(p) = v; }

// Every wait of the block-row solves also gives up after kRowSpinCap polls, whatever
// the clock says, and the first wait to give up records where: counter[4] = site (1:
// a source in another range, 2: the range's completion count), counter[5] = range,
// counter[6] = row.
constexpr unsigned kRowSpinCap = 1u << 24;

__device__ __forceinline__ void record_give_up(int* abort_word, int site, int k, int i) {
    int* rec = abort_word + 2;  // counter[4..6]
    if (atomicCAS(rec, 0, site) == 0) {
        rec[1] = k;
        rec[2] = i;
    }
    raise_abort(abort_word);
}

// v was loaded from p; while it is still kUnset, reload it (bounded).  ok turns false
// on timeout, at the poll cap, or when another CTA has aborted the solve.
template <typename T>
__device__ __forceinline__ T await_set(const T* p, T v, int* abort_word, unsigned long long deadline, bool& ok,
                                       int k, int i) {
    unsigned spins = 0;
    while (unset(v)) {
        if ((++spins & 127) == 0 &&
            (aborted(abort_word) || gclock() > deadline || spins >= kRowSpinCap)) {
            record_give_up(abort_word, 1, k, i);
            ok = false;
            return T(0);
        }
        v = ld_vol(p);
    }
    return v;
}

// Lane 0: wait until the range's count of completed rows reaches need (bounded).
__device__ bool await_rows(const int* done, int need, int* abort_word, unsigned long long deadline, int k,
                           int i) {
    const volatile int* p = done;
    unsigned spins = 0;
    while (*p < need) {
        if ((++spins & 255) == 0 &&
            (aborted(abort_word) || gclock() > deadline || spins >= kRowSpinCap)) {
            record_give_up(abort_word, 2, k, i);
            return false;
        }
    }
    __threadfence_block();
    return true;
}

constexpr int kExtBatch = 4;  // external entries per lane loaded together

// Internal entries per lane held in registers (loaded before the row's wait): 32 per
// row, fewer than the block-DAG solves hold, so that two CTAs of 16 warps fit on an SM
// beside the registers of the external sums.
template <int G>
struct RowHeld {
    static constexpr int M = 32 / G;
};

// The rows of range k.  Forward (BW false): y_i = (r_perm(i) - sum_p U_pi y_p) / U_ii;
// backward: z_i = (y_i - sum_c U_ic z_c) / U_ii, also stored to z at perm(i).
template <int G, typename T, bool BW>
__device__ void solve_range(const SolvePlan& S, const T* __restrict__ ext_val, const T* __restrict__ int_val,
                            const T* __restrict__ rd_all, const double* __restrict__ r, const T* __restrict__ y,
                            T* out, double* __restrict__ z, int k, T* sh, int* done, unsigned long long deadline) {
    constexpr int R = 32 / G, M = RowHeld<G>::M;
    const int lane = threadIdx.x & 31, sl = lane % G;
    const int* ord = BW ? S.rb_ord : S.rf_ord;
    const int* need_a = BW ? S.rb_need : S.rf_need;
    const int* xptr = BW ? S.xb_ptr : S.xf_ptr;
    const int* xj = BW ? S.xb_j : S.xf_j;
    int* abort_word = S.counter + 2;
    const int base = __ldg((BW ? S.rb_ptr : S.rf_ptr) + k);
    const int len = __ldg((BW ? S.rb_ptr : S.rf_ptr) + k + 1) - base;
    const int s = __ldg(S.ranges + k);
    if (threadIdx.x == 0) *done = 0;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    bool ok = true;
    for (int t0 = (threadIdx.x >> 5) * R; t0 < len; t0 += nw * R) {
        const int i = __ldg(ord + base + t0 + lane / G);
        const int need = __ldg(need_a + base + t0);
        T acc0 = T(0), acc1 = T(0), t = T(0), rd = T(0);
        int a = 0, c = 0, cnt = 0;
        int j[M];
        T u[M];
#pragma unroll
        for (int x = 0; x < M; ++x) {
            j[x] = 0;
            u[x] = T(0);
        }
        if (i >= 0) {
            a = __ldg(xptr + i);
            c = __ldg(xptr + i + 1);
#pragma unroll
            for (int x = 0; x < M; ++x) {
                const int q = a + sl + x * G;
                if (q < c) {
                    j[x] = __ldg(xj + q);
                    u[x] = __ldg(int_val + q);
                    cnt = x + 1;
                }
            }
            long long ea, eb;
            if (BW) {
                ea = __ldg(S.urp + i) + 1 + __ldg(S.sb_nint + i);
                eb = __ldg(S.urp + i + 1);
            } else {
                ea = __ldg(S.cptr + i);
                eb = __ldg(S.sf_split + i);
            }
            if (sl == 0) {
                rd = __ldg(rd_all + i);
                t = BW ? ldcg(y + i) : T(__ldg(r + __ldg(S.perm + i)));
            }
            // entries whose source lies in another range: their values are in global memory
            for (long long q0 = ea + sl; q0 < eb && ok; q0 += G * kExtBatch) {
                T w[kExtBatch], v[kExtBatch];
                int src[kExtBatch];
#pragma unroll
                for (int x = 0; x < kExtBatch; ++x) {
                    const long long q = q0 + x * G;
                    src[x] = 0;
                    w[x] = T(0);
                    if (q < eb) {
                        src[x] = BW ? __ldg(S.ucol + q) : __ldg(&S.csc[q].x);
                        w[x] = __ldg(ext_val + q);
                    }
                }
#pragma unroll
                for (int x = 0; x < kExtBatch; ++x) v[x] = q0 + x * G < eb ? ld_vol(out + src[x]) : T(0);
#pragma unroll
                for (int x = 0; x < kExtBatch; ++x) {
                    if (q0 + x * G < eb) {
                        v[x] = await_set(out + src[x], v[x], abort_word, deadline, ok, k, i);
                        if (x & 1) acc1 = fma(w[x], v[x], acc1);
                        else acc0 = fma(w[x], v[x], acc0);
                    }
                }
            }
        }
        const unsigned rows = __ballot_sync(0xffffffffu, sl == 0 && i >= 0);
        const int most = __reduce_max_sync(0xffffffffu, cnt);
        // entries inside the range: shared memory, once the lower levels are complete
        int w_ok = 1;
        if (lane == 0) w_ok = await_rows(done, need, abort_word, deadline, k, __ldg(ord + base + t0));
        ok = ok && __shfl_sync(0xffffffffu, w_ok, 0);
        if (ok) {
#pragma unroll
            for (int x = 0; x < M; x += 2) {
                if (x >= most) break;
                if (x < cnt) acc0 = fma(u[x], sh[j[x]], acc0);
                if (x + 1 < cnt) acc1 = fma(u[x + 1], sh[j[x + 1]], acc1);
            }
            for (int q = a + sl + M * G; q < c; q += G) acc0 = fma(__ldg(int_val + q), sh[__ldg(xj + q)], acc0);
        }
        const T acc = sum_group<G>(acc0 + acc1);
        T val = T(0);
        if (sl == 0 && i >= 0 && ok) {
            val = fma(-rd, acc, t * rd);
            sh[i - s] = val;
        }
        // the count is raised before the global stores, so its fence waits only for the
        // shared-memory results; a warp with a failed wait counts none of its rows
        const bool all_ok = __all_sync(0xffffffffu, ok);
        complete_rows(done, all_ok ? rows : 0u);
        if (sl == 0 && i >= 0 && all_ok) {
            st_vol(out + i, publishable_value(val));
            if (BW) z[__ldg(S.perm + i)] = double(val);
        }
        if (!all_ok) break;
    }
    __syncthreads();  // sh and the count are reused by the next range
}

template <int G, typename T>
__global__ void __launch_bounds__(kDagThreads)
forward_rows(SolvePlan S, const T* __restrict__ uvt, const T* __restrict__ rd_all, const double* __restrict__ r,
             T* y, unsigned long long timeout_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* sh = reinterpret_cast<T*>(smem);
    __shared__ int s_claim, s_done;
    const unsigned long long deadline = gclock() + timeout_ns;
    for (;;) {
        if (threadIdx.x == 0) s_claim = aborted(S.counter + 2) ? S.nranges : atomicAdd(S.counter + 0, 1);
        __syncthreads();
        const int c = s_claim;
        if (c >= S.nranges) break;
        const int k = __ldg(S.rf_claim + c);  // -1: left out (host-side fault injection)
        if (k >= 0)
            solve_range<G, T, false>(S, uvt, static_cast<const T*>(S.xf_val), rd_all, r, nullptr, y, nullptr, k,
                                     sh, &s_done, deadline);
        else
            __syncthreads();
    }
}

template <int G, typename T>
__global__ void __launch_bounds__(kDagThreads)
backward_rows(SolvePlan S, const T* __restrict__ uv, const T* __restrict__ rd_all, const T* __restrict__ y, T* zv,
              double* __restrict__ z, unsigned long long timeout_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    T* sh = reinterpret_cast<T*>(smem);
    __shared__ int s_claim, s_done;
    const unsigned long long deadline = gclock() + timeout_ns;
    for (;;) {
        if (threadIdx.x == 0) s_claim = aborted(S.counter + 2) ? S.nranges : atomicAdd(S.counter + 1, 1);
        __syncthreads();
        const int c = s_claim;
        if (c >= S.nranges) break;
        const int k = __ldg(S.rb_claim + c);
        if (k >= 0)
            solve_range<G, T, true>(S, uv, static_cast<const T*>(S.xb_val), rd_all, nullptr, y, zv, z, k, sh,
                                    &s_done, deadline);
        else
            __syncthreads();
    }
}

template <int G, typename T>
cudaError_t rows_smem_and_occupancy(size_t smem, int* blocks) {
    const int cap = int(kMaxBlockRows * sizeof(T));
    cudaError_t e = cudaFuncSetAttribute(forward_rows<G, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(backward_rows<G, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e != cudaSuccess) return e;
    int a = 0, b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, forward_rows<G, T>, kDagThreads, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, backward_rows<G, T>, kDagThreads, smem);
    *blocks = a < b ? a : b;
    return e;
}

template <int G, typename T>
void launch_rows(const SolvePlan& S, const T* uv, const T* rd, const double* r, double* z, T* y, int grid,
                 size_t smem, unsigned long long timeout_ns, cudaStream_t s, cudaEvent_t t1) {
    forward_rows<G, T><<<grid, kDagThreads, smem, s>>>(S, static_cast<const T*>(S.uvt), rd, r, y, timeout_ns);
    if (t1) cudaEventRecord(t1, s);
    backward_rows<G, T><<<grid, kDagThreads, smem, s>>>(S, uv, rd, y, y + S.n, z, timeout_ns);
}

template <typename T>
cudaError_t launch_rows_t(const SolvePlan& S, const T* uv, const T* rd, const double* r, double* z, T* y,
                          int grid, unsigned long long timeout_ns, cudaStream_t s, cudaEvent_t t1) {
    const size_t smem = size_t(S.max_range_rows) * sizeof(T);
    if (S.lanes_per_row == 4) launch_rows<4, T>(S, uv, rd, r, z, y, grid, smem, timeout_ns, s, t1);
    else launch_rows<8, T>(S, uv, rd, r, z, y, grid, smem, timeout_ns, s, t1);
    return cudaGetLastError();
}

// The shared-memory cap is a per-function setting shared by all handles, so it is
// always the largest range (kMaxBlockRows rows); the occupancy uses the actual size.
template <int G, typename T>
cudaError_t set_smem_and_occupancy(size_t smem, int* blocks) {
    const int cap = int(kMaxBlockRows * sizeof(T));
    cudaError_t e = cudaFuncSetAttribute(forward_dag<G, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(backward_dag<G, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
    if (e != cudaSuccess) return e;
    int a = 0, b = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, forward_dag<G, T>, kDagThreads, smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, backward_dag<G, T>, kDagThreads, smem);
    *blocks = a < b ? a : b;
    return e;
}

template <int G, typename T>
void launch_dag(const SolvePlan& S, const T* uv, const T* rd, const double* r, double* z, T* y, T* w, int grid,
                size_t smem, unsigned long long timeout_ns, cudaStream_t s, cudaEvent_t t1) {
    forward_dag<G, T><<<grid, kDagThreads, smem, s>>>(S, static_cast<const T*>(S.uvt), rd, r, y, w, timeout_ns);
    if (t1) cudaEventRecord(t1, s);
    backward_dag<G, T><<<grid, kDagThreads, smem, s>>>(S, uv, rd, y, y + S.n, z, w, timeout_ns);
}

template <typename T>
cudaError_t launch_dag_t(const SolvePlan& S, const T* uv, const T* rd, const double* r, double* z, T* y, T* w,
                         int grid, unsigned long long timeout_ns, cudaStream_t s, cudaEvent_t t1) {
    const size_t smem = size_t(S.max_range_rows) * sizeof(T);
    switch (S.lanes_per_row) {
        case 4: launch_dag<4, T>(S, uv, rd, r, z, y, w, grid, smem, timeout_ns, s, t1); break;
        case 8: launch_dag<8, T>(S, uv, rd, r, z, y, w, grid, smem, timeout_ns, s, t1); break;
        case 16: launch_dag<16, T>(S, uv, rd, r, z, y, w, grid, smem, timeout_ns, s, t1); break;
        default: launch_dag<32, T>(S, uv, rd, r, z, y, w, grid, smem, timeout_ns, s, t1); break;
    }
    return cudaGetLastError();
}

// uvt[q] = value of the U entry the column-list entry q refers to.
template <typename T>
__global__ void transpose_values(int noff, const int2* __restrict__ csc, const T* __restrict__ uv,
                                 T* __restrict__ uvt) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < noff; q += gridDim.x * blockDim.x)
        uvt[q] = uv[__ldg(&csc[q].y)];
}

// out[q] = uv[pos[q]].
template <typename T>
__global__ void gather_values(int cnt, const int* __restrict__ pos, const T* __restrict__ uv, T* __restrict__ out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) out[q] = uv[__ldg(pos + q)];
}

template <typename T>
void launch_gathers(const SolvePlan& S, const T* uv, cudaStream_t s) {
    auto grid = [](int cnt) { return (cnt + 255) / 256 < 8192 ? (cnt + 255) / 256 : 8192; };
    if (S.noff > 0) transpose_values<T><<<grid(S.noff), 256, 0, s>>>(S.noff, S.csc, uv, static_cast<T*>(S.uvt));
    if (S.nxf > 0) gather_values<T><<<grid(S.nxf), 256, 0, s>>>(S.nxf, S.xf_pos, uv, static_cast<T*>(S.xf_val));
    if (S.nxb > 0) gather_values<T><<<grid(S.nxb), 256, 0, s>>>(S.nxb, S.xb_pos, uv, static_cast<T*>(S.xb_val));
}

}  // namespace

// Number of kernels launch_dag_prepare launches.
int dag_prepare_launches(const SolvePlan& S) {
    return S.solve_mode == 1 ? 0 : (S.noff > 0) + (S.nxf > 0) + (S.nxb > 0);
}

cudaError_t launch_dag_prepare(const SolvePlan& S, cudaStream_t s) {
    if (S.solve_mode == 1) return cudaSuccess;
    if (S.dtype == IC_F32) launch_gathers<float>(S, S.uval32, s);
    else launch_gathers<double>(S, S.uval, s);
    return cudaGetLastError();
}

cudaError_t rows_blocks_per_sm(int lanes, int dtype, int max_range_rows, int* blocks) {
    const size_t smem = size_t(max_range_rows < 1 ? 1 : max_range_rows) * (dtype == IC_F32 ? 4 : 8);
    if (dtype == IC_F32)
        return lanes == 4 ? rows_smem_and_occupancy<4, float>(smem, blocks)
                          : rows_smem_and_occupancy<8, float>(smem, blocks);
    return lanes == 4 ? rows_smem_and_occupancy<4, double>(smem, blocks)
                      : rows_smem_and_occupancy<8, double>(smem, blocks);
}

cudaError_t launch_apply_rows(const SolvePlan& S, const double* r, double* z, unsigned long long timeout_ns,
                              int grid, cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1) {
    if (S.n == 0) return cudaSuccess;
    // both result vectors start as kUnset (forward then backward, n values each)
    const size_t bytes = 2 * size_t(S.n) * (S.dtype == IC_F32 ? sizeof(float) : sizeof(double));
    cudaError_t e = cudaMemsetAsync(S.y, 0xff, bytes, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(S.counter, 0, 3 * sizeof(int), s);  // range claims and the abort word
    if (e != cudaSuccess) return e;
    if (t0) cudaEventRecord(t0, s);
    if (S.dtype == IC_F32)
        return launch_rows_t<float>(S, S.uval32, S.rdiag32, r, z, reinterpret_cast<float*>(S.y), grid, timeout_ns,
                                    s, t1);
    return launch_rows_t<double>(S, S.uval, S.rdiag, r, z, S.y, grid, timeout_ns, s, t1);
}

cudaError_t dag_blocks_per_sm(int lanes, int dtype, int max_range_rows, int* blocks) {
    const size_t smem = size_t(max_range_rows < 1 ? 1 : max_range_rows) * (dtype == IC_F32 ? 4 : 8);
    if (dtype == IC_F32) {
        switch (lanes) {
            case 4: return set_smem_and_occupancy<4, float>(smem, blocks);
            case 8: return set_smem_and_occupancy<8, float>(smem, blocks);
            case 16: return set_smem_and_occupancy<16, float>(smem, blocks);
            default: return set_smem_and_occupancy<32, float>(smem, blocks);
        }
    }
    switch (lanes) {
        case 4: return set_smem_and_occupancy<4, double>(smem, blocks);
        case 8: return set_smem_and_occupancy<8, double>(smem, blocks);
        case 16: return set_smem_and_occupancy<16, double>(smem, blocks);
        default: return set_smem_and_occupancy<32, double>(smem, blocks);
    }
}

cudaError_t launch_apply_dag(const SolvePlan& S, const double* r, double* z, unsigned long long timeout_ns,
                             int grid, cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1) {
    if (S.n == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(S.dag_indeg, S.dag_indeg0, size_t(S.nftask + S.nbtask) * sizeof(int),
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(S.dag_taken, 0, size_t(S.nftask + S.nbtask) * sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(S.counter, 0, 3 * sizeof(int), s);  // claims and the abort word
    if (e != cudaSuccess) return e;
    if (t0) cudaEventRecord(t0, s);
    if (S.dtype == IC_F32)
        return launch_dag_t<float>(S, S.uval32, S.rdiag32, r, z, reinterpret_cast<float*>(S.y),
                                   reinterpret_cast<float*>(S.dag_w), grid, timeout_ns, s, t1);
    return launch_dag_t<double>(S, S.uval, S.rdiag, r, z, S.y, reinterpret_cast<double*>(S.dag_w), grid,
                                timeout_ns, s, t1);
}

}  // namespace ick
