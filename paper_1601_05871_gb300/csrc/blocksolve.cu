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

// Whole warp: wait until the range's count of completed rows reaches need; false on
// abort or timeout.  The count is one shared word that all lanes read in the same
// load (a broadcast), so every lane sees the same values and takes the same branch:
// no lane has to pass the outcome on to the others.
__device__ bool await_count(const int* done, int need, int* abort_word, unsigned long long deadline) {
    const volatile int* p = done;
    unsigned spins = 0;
    while (*p < need) {
        if ((++spins & 255) == 0 && (aborted(abort_word) || gclock() > deadline)) {
            if ((threadIdx.x & 31) == 0) raise_abort(abort_word);
            return false;
        }
    }
    // one acquire load of the count (lighter than a fence): it reads a value made by
    // the chain of release-adds of the completed rows, so their results are visible
    int v;
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(done));
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    (void)v;
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

// Marks one row complete, by the lane that stored its result: the release orders that
// store before the count update, for the CTA's threads that acquire the count.
__device__ __forceinline__ void complete_row(int* done) {
    const unsigned a = static_cast<unsigned>(__cvta_generic_to_shared(done));
    asm volatile("red.release.cta.shared::cta.add.u32 [%0], 1;" ::"r"(a) : "memory");
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

// Thread 0 waits until task t's in-degree is zero, then the CTA synchronises; false
// (in every thread) on abort or timeout.
__device__ bool wait_ready(int t, const int* indeg, int* abort_word, unsigned long long deadline,
                           unsigned long long* trace, int* s_ok) {
    if (threadIdx.x == 0) {
        const bool ok = await_zero(indeg + t, abort_word, deadline);
        if (trace && ok) trace[4 * t + 1] = gclock();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// L of either direction: the rows at order positions [lo, hi) of range k (whole
// levels), G lanes per row and 32/G rows per warp (one level per claim).  The range's
// earlier results (positions before lo, finished by the range's previous parts) are
// first loaded into shared memory and counted as complete; a row runs once every row
// of the lower levels is complete (done >= need); its internal operands come from
// shared memory and its other operands are loaded before the wait.  For a task just
// claimed (wait_t >= 0), each warp loads its first group's operands (factor values,
// indices, the right-hand side: none is written by an earlier task) before waiting
// for the task's in-degree, so the chain of dependent loads overlaps the wait; only
// the external sum, written by the part's E tasks, is read after it.  Returns false
// when that wait gave up.
//   forward:  y_i = (r_perm(i) - w_i - sum) / U_ii, stored to y
//   backward: z_i = (y_i - w_i - sum) / U_ii, stored to zv and to z at perm(i)
template <int G, typename T, bool BW>
__device__ bool solve_local(const SolvePlan& S, const T* __restrict__ xv, const T* __restrict__ rd_all,
                            const double* __restrict__ r, const T* y, T* out, double* __restrict__ z, const T* w,
                            int k, int lo, int hi, T* sh, int* done, bool cont, int wait_t, const int* indeg,
                            unsigned long long deadline, int* s_ok) {
    constexpr int R = 32 / G, M = Held<G>::M;
    const int lane = threadIdx.x & 31, sl = lane % G;
    const int* ord = BW ? S.lb_ord : S.lf_ord;
    const int* need_a = BW ? S.lb_need : S.lf_need;
    const int* xptr = BW ? S.xb_ptr : S.xf_ptr;
    const int* xj = BW ? S.xb_j : S.xf_j;
    const int len = hi - lo;
    // the warp's current group: row, rows of lower levels it waits for, entry range,
    // permutation entry, reciprocal pivot, right-hand side and its first 64 internal
    // entries (64 / G per lane)
    int i = -1, need = 0, a = 0, c = 0, dst = 0, cnt = 0, most = 0;
    T t = T(0), rd = T(0);
    int j[M];
    T u[M];
    auto load = [&](int t0) {
        i = __ldg(ord + lo + t0 + lane / G);
        need = __ldg(need_a + lo + t0);
        t = T(0);
        rd = T(0);
        a = 0;
        c = 0;
        dst = 0;
        if (i >= 0) {
            a = __ldg(xptr + i);
            c = __ldg(xptr + i + 1);
            if (sl == 0) {
                rd = __ldg(rd_all + i);
                if (BW) {
                    t = ldcg(y + i);
                    dst = __ldg(S.perm + i);
                } else {
                    t = T(__ldg(r + __ldg(S.perm + i)));
                }
            }
        }
        cnt = 0;
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
        most = __reduce_max_sync(0xffffffffu, cnt);
    };
    // group g of R positions goes to warp g mod (warps): the groups of one level sit on
    // consecutive warps, i.e. on different SM sub-partitions, whose FP64 units then
    // work in parallel; each warp takes its groups in order, and a group depends only
    // on lower groups, so the waits cannot cycle
    const int nw = blockDim.x >> 5;
    const int first = (threadIdx.x >> 5) * R;
    if (first < len) load(first);
    unsigned long long* trace = S.trace && BW ? S.trace + 4 * size_t(S.nftask) : S.trace;
    if (wait_t >= 0 && !wait_ready(wait_t, indeg, S.counter + 2, deadline, trace, s_ok)) return false;
    const int base = __ldg((BW ? S.lb_ptr : S.lf_ptr) + k);
    const int s = __ldg(S.ranges + k);
    if (!cont) {  // a continuation already holds the range's earlier results and count
        for (int q = base + int(threadIdx.x); q < lo; q += blockDim.x) {
            const int ii = __ldg(ord + q);
            if (ii >= 0) sh[ii - s] = ldcg(out + ii);
        }
        if (threadIdx.x == 0) *done = lo > base ? __ldg(need_a + lo) : 0;
        __syncthreads();
    }
    for (int t0 = first; t0 < len; t0 += nw * R) {
        if (t0 != first) load(t0);
        // the row's result is rd * t plus the sum of the internal products, whose
        // values hold -rd already (gather_scaled); a row without external entries keeps
        // w = 0 (never written), which leaves t unchanged
        if (i >= 0 && sl == 0) t = (t - ldcg(w + i)) * rd;
        if (!await_count(done, need, S.counter + 2, deadline)) break;
        // the source values first: M independent shared-memory loads issued together
        // (an unused slot reads sh[0], which is never used), so their latency is paid
        // once instead of once per entry; then the FMA chain over interleaved
        // accumulators: two in FP64, whose FMAs issue about 64 cycles apart in a warp
        // anyway (more would only add the additions that combine them), four in FP32
        constexpr int NA = sizeof(T) == 4 ? 4 : 2;
        T sv[M];
#pragma unroll
        for (int x = 0; x < M; ++x) sv[x] = sh[j[x]];
        T acc[NA];
#pragma unroll
        for (int yy = 0; yy < NA; ++yy) acc[yy] = T(0);
        acc[0] = t;  // the scaled right-hand side (0 on the other lanes of the row)
#pragma unroll
        for (int x = 0; x < M; x += NA) {
            if (x >= most) break;
#pragma unroll
            for (int yy = 0; yy < NA; ++yy)
                if (x + yy < M && x + yy < cnt) acc[yy] = fma(u[x + yy], sv[x + yy], acc[yy]);
        }
        for (int q = a + sl + M * G; q < c; q += G) acc[0] = fma(__ldg(xv + q), sh[__ldg(xj + q)], acc[0]);
        T tot = acc[0] + acc[1];
        if constexpr (NA == 4) tot = (acc[0] + acc[1]) + (acc[2] + acc[3]);
        const T accs = sum_group<G>(tot);
        if (sl == 0 && i >= 0) {
            const T v = accs;
            sh[i - s] = v;
            // the count is raised before the global stores, so its release waits only
            // for the shared-memory result; later tasks read the global copies after
            // the task's closing fence
            complete_row(done);
            out[i] = v;
            if (BW) z[dst] = double(v);
        }
    }
    return true;
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

// Claims the next task (its in-degree is awaited by the task itself, with wait_ready).
// Returns the task index, or -1 when the list is exhausted or the solve was aborted.
// s_claim is a shared word of its own, not release's s_task: the barrier at the start of
// release orders every read of its last value before the next write, whereas a warp
// delayed past a claim into s_task could read the new task as a continuation.
__device__ int claim_task(int* claim_ctr, int ntasks, int* taken, int* abort_word, int* s_claim,
                          unsigned long long* trace) {
    if (threadIdx.x == 0) {
        int t = -1;
        if (!aborted(abort_word)) {
            do {  // tasks already taken as a continuation are skipped
                t = atomicAdd(claim_ctr, 1);
            } while (t < ntasks && atomicExch(taken + t, 1) != 0);
            if (t >= ntasks) {
                t = -1;
            } else if (trace) {
                trace[4 * t] = gclock();
                trace[4 * t + 3] = (unsigned long long)t | ((unsigned long long)smid() << 32);
            }
        }
        *s_claim = t;
    }
    __syncthreads();
    return *s_claim;
}

// After a task: its results are made visible, then its successors are released, by
// all threads of the CTA at once (a separator's part can have a hundred successors,
// and released one after another they would wait a memory round trip each).  If the
// task was an L part whose range's next part is now ready and not yet taken, the CTA
// takes it (returned; -1 otherwise) and runs it with the shared-memory state it
// already holds: the thread whose decrement made that part's in-degree zero takes it.
__device__ __forceinline__ int release(int t, bool is_l, const int* succ_ptr, const int* succ, const int* next,
                                       int* indeg, int* taken, unsigned long long* trace, int* s_task) {
    __threadfence();
    __syncthreads();  // the task is done in every thread, and s_task is no longer read
    if (threadIdx.x == 0) {
        if (trace) trace[4 * t + 2] = gclock();
        *s_task = -1;
    }
    __syncthreads();
    const int a = __ldg(succ_ptr + t), b = __ldg(succ_ptr + t + 1);
    const int nx = is_l ? __ldg(next + t) : -1;
    for (int q = a + int(threadIdx.x); q < b; q += blockDim.x) {
        const int sx = __ldg(succ + q);
        if (sx != nx) {
            atomicSub(indeg + sx, 1);
        } else if (atomicSub(indeg + sx, 1) == 1 && atomicExch(taken + sx, 1) == 0) {
            __threadfence();  // acquire: the part's other inputs are visible to this CTA
            if (trace) {
                const unsigned long long now = gclock();
                trace[4 * sx] = now;
                trace[4 * sx + 1] = now;
                trace[4 * sx + 3] = (unsigned long long)sx | ((unsigned long long)smid() << 32);
            }
            *s_task = sx;
        }
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
    __shared__ int s_task, s_claim, s_done, s_ok;
    const unsigned long long deadline = gclock() + timeout_ns;
    int* indeg = S.dag_indeg;
    int* taken = S.dag_taken;
    int t = -1;
    bool cont = false;
    for (;;) {
        if (t < 0) {
            t = claim_task(S.counter + 0, S.nftask, taken, S.counter + 2, &s_claim, S.trace);
            cont = false;
        }
        if (t < 0) break;
        const int4 tk = S.ftask[t];
        if (tk.x == 0) {
            if (!wait_ready(t, indeg, S.counter + 2, deadline, S.trace, &s_ok)) break;
            fwd_external<G, T>(S, uvt, y, w, tk.z, tk.w);
        } else if (!solve_local<G, T, false>(S, static_cast<const T*>(S.xf_val), rd_all, r, nullptr, y, nullptr, w,
                                             tk.y, tk.z, tk.w, sh, &s_done, cont, cont ? -1 : t, indeg, deadline,
                                             &s_ok)) {
            break;
        }
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
    __shared__ int s_task, s_claim, s_done, s_ok;
    const unsigned long long deadline = gclock() + timeout_ns;
    int* indeg = S.dag_indeg + S.nftask;
    int* taken = S.dag_taken + S.nftask;
    unsigned long long* tr = S.trace ? S.trace + 4 * size_t(S.nftask) : nullptr;
    int t = -1;
    bool cont = false;
    for (;;) {
        if (t < 0) {
            t = claim_task(S.counter + 1, S.nbtask, taken, S.counter + 2, &s_claim, tr);
            cont = false;
        }
        if (t < 0) break;
        const int4 tk = S.btask[t];
        if (tk.x == 0) {
            if (!wait_ready(t, indeg, S.counter + 2, deadline, tr, &s_ok)) break;
            bwd_external<G, T>(S, uv, zv, w, tk.z, tk.w);
        } else if (!solve_local<G, T, true>(S, static_cast<const T*>(S.xb_val), rd_all, nullptr, y, zv, z, w, tk.y,
                                            tk.z, tk.w, sh, &s_done, cont, cont ? -1 : t, indeg, deadline, &s_ok)) {
            break;
        }
        t = release(t, tk.x == 1, S.b_succ_ptr, S.b_succ, S.b_next, indeg, taken, tr, &s_task);
        cont = t >= 0;
    }
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
    backward_dag<G, T><<<grid, kDagThreads, smem, s>>>(S, uv, rd, y, y + S.n, z, w + S.n, timeout_ns);
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

template <typename T>
__global__ void gather_scaled(int n, const int* __restrict__ ptr, const int* __restrict__ pos,
                              const T* __restrict__ uv, const T* __restrict__ rd, T* __restrict__ out) {
    const int lane = threadIdx.x & 31, warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const T m = -__ldg(rd + i);
        const int e = __ldg(ptr + i + 1);
        for (int q = __ldg(ptr + i) + lane; q < e; q += 32) out[q] = __ldg(uv + __ldg(pos + q)) * m;
    }
}

template <typename T>
void launch_gathers(const SolvePlan& S, const T* uv, const T* rd, cudaStream_t s) {
    auto grid = [](int cnt) { return (cnt + 255) / 256 < 8192 ? (cnt + 255) / 256 : 8192; };
    if (S.noff > 0) transpose_values<T><<<grid(S.noff), 256, 0, s>>>(S.noff, S.csc, uv, static_cast<T*>(S.uvt));
    const int rows = (S.n + 7) / 8 < 8192 ? (S.n + 7) / 8 : 8192;  // 8 warps of 256 threads per block
    if (S.nxf > 0)
        gather_scaled<T><<<rows, 256, 0, s>>>(S.n, S.xf_ptr, S.xf_pos, uv, rd, static_cast<T*>(S.xf_val));
    if (S.nxb > 0)
        gather_scaled<T><<<rows, 256, 0, s>>>(S.n, S.xb_ptr, S.xb_pos, uv, rd, static_cast<T*>(S.xb_val));
}

}  // namespace

// Number of kernels launch_dag_prepare launches.
int dag_prepare_launches(const SolvePlan& S) {
    return S.solve_mode != 0 ? 0 : (S.noff > 0) + (S.nxf > 0) + (S.nxb > 0);
}

cudaError_t launch_dag_prepare(const SolvePlan& S, cudaStream_t s) {
    if (S.solve_mode != 0) return cudaSuccess;
    if (S.dtype == IC_F32) launch_gathers<float>(S, S.uval32, S.rdiag32, s);
    else launch_gathers<double>(S, S.uval, S.rdiag, s);
    return cudaGetLastError();
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
