// Numeric phase of IC(k) by blocks (Section 3.3) on sm_103a.
//
// One persistent kernel runs every work item of the Cholesky-by-blocks DAG.  A work item
// is a block task (Chol, Trsm, Herk, Gemm), a chunk of a Herk/Gemm task's target rows,
// or one of the CTAs that share a split Chol/Trsm task.  The CTAs claim items in a
// fixed order computed by the symbolic phase (a list schedule that runs first the ready
// items whose tasks have the longest remaining path); a CTA waits (bounded) until the
// claimed item's task has no unfinished predecessor, runs it, and the CTA that finishes
// a task's last item decrements its successors' in-degree counters (the scheduler
// duties of Section 2.2: track waiting tasks, run ready ones, release dependents on
// completion).  Every item comes after all items of its predecessors in the order, so a
// CTA only waits for items that running CTAs hold.
//
// Inside a task every target row r is owned by one warp (data parallelism within a
// task, the remedy Section 6 plans for task granularity).  The warp stages the
// target segment of row r in shared memory, with a bit map of its columns, and
// applies, pivot by pivot in ascending order, U_rc -= U_pr * U_pc for the columns c
// of the pivot row's source segment that belong to the target segment; other
// contributions fall outside the IC(k) pattern S and are discarded.  Chol and Trsm
// rows depend on earlier rows of the same diagonal block: a task on one CTA keeps
// their completion flags in shared memory; a split task (several CTAs claiming its
// rows from a global counter) publishes each finished row in a shadow array that
// holds a sentinel until written, and readers take a value once it is not the
// sentinel.  Every wait is bounded by a %globaltimer deadline and ends in a status bit.
//
// Precision: T = double is the FP64 factorization.  T = float keeps the off-diagonal
// factor values in FP32 while every diagonal pivot is accumulated, square-rooted and
// tested for breakdown in FP64 (array udiag): in Chol and Herk each pivot row's source
// segment starts at column r, so its contribution to U_rr is exactly U_pr^2, which the
// owning warp subtracts in FP64.  EXACT (FP64 only) rounds every multiply and
// subtract separately and finishes a row with the IEEE square root and divisions;
// otherwise updates are fused multiply-adds and a row is scaled by its reciprocal
// pivot.
#include <climits>
#include <cstdint>
#include <type_traits>

#include "ick_internal.h"

namespace ick {
namespace {

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }

template <bool EXACT>
__device__ __forceinline__ double sub_product(double acc, double a, double b) {
    if (EXACT) return __dsub_rn(acc, __dmul_rn(a, b));
    return fma(-a, b, acc);
}
template <bool EXACT>
__device__ __forceinline__ float sub_product(float acc, float a, float b) {
    return fmaf(-a, b, acc);
}

enum Mode { M_CHOL = 0, M_TRSM = 1, M_UPDATE = 2 };

// 1/sqrt(d) by Newton's iteration for the reciprocal square root,
// y <- y + y (1 - d y^2) / 2, started from the single-precision estimate: each step
// about doubles the number of correct bits, so two reach double precision.  Outside
// the single-precision exponent range (and for d <= 0 or NaN) the library's square
// root and division are used.
__device__ __forceinline__ double rsqrt_newton(double d) {
    if (!(d >= 1e-30 && d <= 1e30)) return 1.0 / sqrt(d);
    double y = double(rsqrtf(float(d)));
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const double e = fma(-(d * y), y, 1.0);
        y = fma(0.5 * y, e, y);
    }
    return y;
}

struct Smem {
    int task, chunk, next, slot;
    unsigned long long t0;
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

__device__ __forceinline__ void note_breakdown(const DevPlan& P, int r) {
    atomicOr(P.counters + 2, kStBreakdown);
    atomicMin(P.brk_row, (long long)r);
}

// Wait until done[local] is set by another warp of this CTA (flags in shared memory);
// false on timeout/abort.  The caller fences before it reads the row.
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
    return true;
}

constexpr int kMapWords = 128;  // per-warp column map: 4096 column offsets
constexpr int kMapBits = 32 * kMapWords;

// Per-warp shared-memory work area.  The target chunk's columns, offsets from its first
// column c_0, are a bit map with the rank of each word's first bit: column c sits at
// slot rank[w] + popc(bits[w] below bit b), w = (c - c_0) / 32, b = (c - c_0) % 32.
template <typename T>
struct WarpBuf {
    int4 piv[32];          // pivot row, position of U_pr, source segment start, length
    int psoff[32];         // split tasks: the pivot row's shadow offset
    double dacc;           // FP64 diagonal accumulator (T = float)
    double pad;
    T abuf[32];            // T = float: the batch's multipliers U_pr, for the diagonal
    uint2 cmap[kMapWords]; // (bits, rank) per 32 column offsets
    T tval[kSegCap];       // target segment values (one chunk)
    int tcol[kSegCap];     // target segment columns
};

// Slot of column c in the target chunk, or -1.
template <typename T>
__device__ __forceinline__ int find_col(const WarpBuf<T>& W, int c, int c_0, unsigned span) {
    const unsigned off = unsigned(c - c_0);
    if (off >= span) return -1;
    const uint2 e = W.cmap[off >> 5];
    const unsigned b = off & 31u;
    return ((e.x >> b) & 1u) ? int(e.y) + __popc(e.x & ((1u << b) - 1u)) : -1;
}

template <bool EXACT, typename T>
__device__ __forceinline__ void apply_one(WarpBuf<T>& W, int c, int c_0, unsigned span, T a, T v) {
    const int idx = find_col(W, c, c_0, span);
    if (idx >= 0) W.tval[idx] = sub_product<EXACT>(W.tval[idx], a, v);
}

// Split tasks publish finished rows in a shadow array that holds a signalling NaN
// with a fixed payload until each value is written.  Arithmetic never produces that
// bit pattern (a NaN result is the quiet canonical one), and an aligned 8- or 4-byte
// store is seen whole or not at all, so a value read that is not the sentinel is final.
constexpr unsigned long long kSentinel64 = 0x7FF00000DEADBEEFull;
constexpr unsigned kSentinel32 = 0x7F80BEEFu;
__device__ __forceinline__ bool is_sentinel(double v) {
    return (unsigned long long)__double_as_longlong(v) == kSentinel64;
}
__device__ __forceinline__ bool is_sentinel(float v) { return __float_as_uint(v) == kSentinel32; }
__device__ __forceinline__ double ld_vol(const double* p) {
    return *reinterpret_cast<const volatile double*>(p);
}
__device__ __forceinline__ float ld_vol(const float* p) {
    return *reinterpret_cast<const volatile float*>(p);
}

// One published value of a split task's pivot row (per lane, bounded).
template <typename T>
__device__ T await_value(const DevPlan& P, const T* src, unsigned long long deadline) {
    unsigned spins = 0;
    for (;;) {
        const T t = ld_vol(src);
        if (!is_sentinel(t)) return t;
        if ((++spins & 63) == 0 && (ld_volatile(P.counters + 3) || gtimer() > deadline)) {
            if (!ld_volatile(P.counters + 3)) set_timeout(P, 4);
            return t;
        }
        __nanosleep(20);
    }
}

// One pivot in registers: lane l holds element l of the pivot row's source segment
// (value v and column c), a the multiplier U_pr when it lies outside the segment, st 0
// (empty segment), 1 (loaded) or 2 (the pivot row is not complete yet: it is waited for
// and loaded when it is applied), len and z the segment's length and first position
// (kept here so that the application does not read the batch entry again).
template <typename T>
struct PivReg {
    T v, a;
    int c, st, len, z;
};

// Load pivot j of the batch (W.piv) into R.  Chol/Trsm on one CTA: the pivot row's
// completion flag must have been seen; when it has not, the flags of every pivot of the
// batch not seen yet are read again (one per lane), so rows completed meanwhile cost
// one round trip together.  SPLIT: the values come from the pivot rows' published
// copies and are checked against the sentinel when applied.
template <int MODE, bool SPLIT, typename T>
__device__ __forceinline__ void load_pivot(const DevPlan& P, const T* U, const T* shadow, const WarpBuf<T>& W,
                                           int j, int nq, bool start_at_r, int rbase,
                                           volatile unsigned char* done, unsigned& seen, PivReg<T>& R) {
    const int lane = threadIdx.x & 31;
    const int4 pi = W.piv[j];
    const int len = pi.w;
    R.st = 0;
    R.len = len;
    R.z = pi.z;
    if (len == 0) return;
    if (!SPLIT && MODE != M_UPDATE && !((seen >> j) & 1u)) {
        int dn = 1;
        if (lane < nq && !((seen >> lane) & 1u)) dn = done[W.piv[lane].x - rbase];
        const unsigned now = __ballot_sync(0xffffffffu, dn != 0);
        if (now & ~seen) __threadfence_block();
        seen |= now;
        if (!((seen >> j) & 1u)) {
            R.st = 2;
            return;
        }
    }
    const T* V = SPLIT ? shadow + W.psoff[j] : U;
    R.v = lane < len ? ld_cg(V + pi.z + lane) : T(0);
    R.c = lane < len ? __ldg(P.ucol + pi.z + lane) : 0;
    R.a = start_at_r ? T(0) : ld_cg(U + pi.y);
    R.st = 1;
}

// Apply pivot q (loaded in R) to the target chunk: U_rc -= U_pr * U_pc for the columns
// c of the source segment that lie in the chunk, elements 0..31 from the registers and
// any further ones loaded directly.  False when a wait gave up (timeout or abort).
template <int MODE, bool EXACT, bool SPLIT, typename T>
__device__ __forceinline__ bool apply_pivot(const DevPlan& P, const T* U, const T* shadow, WarpBuf<T>& W, int q,
                                            bool start_at_r, int rbase, volatile unsigned char* done,
                                            unsigned& seen, PivReg<T>& R, int c_0, unsigned span, bool dchunk,
                                            unsigned long long deadline) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const int len = R.len;
    if (len > 0) {
        if (R.st == 2) {  // the pivot row is waited for, then loaded
            const int4 pi = W.piv[q];
            int ok = 1;
            if (lane == 0) ok = wait_row(P, done, pi.x - rbase, deadline);
            if (!__shfl_sync(full, ok, 0)) return false;
            __threadfence_block();
            seen |= 1u << q;
            R.v = lane < len ? ld_cg(U + pi.z + lane) : T(0);
            R.c = lane < len ? __ldg(P.ucol + pi.z + lane) : 0;
            R.a = start_at_r ? T(0) : ld_cg(U + pi.y);
        }
        const T* V = SPLIT ? shadow + W.psoff[q] : U;
        if (SPLIT && lane < len && is_sentinel(R.v)) R.v = await_value(P, V + R.z + lane, deadline);
        const T a = start_at_r ? __shfl_sync(full, R.v, 0) : R.a;
        if (lane < len) {
            const int idx = find_col(W, R.c, c_0, span);
            if (idx >= 0) W.tval[idx] = sub_product<EXACT>(W.tval[idx], a, R.v);
        }
        for (int o = 32 + lane; o < len; o += 32) {
            const T v = SPLIT ? await_value(P, V + R.z + o, deadline) : ld_cg(U + R.z + o);
            apply_one<EXACT>(W, __ldg(P.ucol + R.z + o), c_0, span, a, v);
        }
        if (dchunk && lane == 0) W.abuf[q] = a;  // the diagonal takes the batch's squares at once
    }
    __syncwarp();
    return true;
}

// One target row: r, pivots csc[ca, cb), target segment [tb, te) of row r.
// MODE: Chol (source = pivot row's block-k segment from column r on; wait on pivot
// rows; finalise with sqrt and scaling), Trsm (source = pivot row's block-j segment;
// wait on pivot rows that have one; finalise by dividing by U_rr), Update (Herk/Gemm:
// all inputs final).  start_at_r: the source segment starts at the pivot's entry in
// column r (target block column == block of r).
//
// The target segment is processed in chunks of at most kSegCap entries whose columns
// lie within kMapBits of the chunk's first column, so that a column is found through
// the chunk's bit map and word ranks with no probing.  Pivots are applied one at a
// time in ascending order, lane l taking source elements l, l+32, ... straight from L2
// (ld.cg) into registers.  For Chol and Trsm on one CTA a pivot is loaded
// only once its row's completion flag is seen; a pivot whose row was not complete at
// load time is waited for and loaded when its turn comes.  SPLIT (a Chol/Trsm task
// shared by several CTAs): there are no flags; the values come from the pivot rows'
// published copies (shadow, offsets soffs per row of the block), every value is checked
// against the sentinel on use, and the finished row is published in turn.
template <int MODE, bool EXACT, bool SPLIT, typename T>
__device__ void process_target(const DevPlan& P, T* U, int r, int ca, int cb, int tb, int te,
                               int srcblk, bool start_at_r, int rbase,
                               volatile unsigned char* done, WarpBuf<T>& W,
                               unsigned long long deadline, const int* soffs = nullptr,
                               T* shadow = nullptr) {
    constexpr bool MIXED = std::is_same<T, float>::value;
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    // Trsm: exact mode divides by the pivot itself (the operation of the definition);
    // otherwise the row is multiplied by the pivot's reciprocal, kept by its Chol
    T scale = T(1);
    if (MODE == M_TRSM) {
        if (EXACT) scale = ld_cg(U + __ldg(P.urp + r));
        else scale = T(__ldcg(P.urcp + r));
    }
    int m = 0;
    for (int c0 = tb; c0 < te; c0 += m) {
        // a chunk: at most kSegCap entries whose columns lie within kMapBits of its first
        const int c_0 = __ldg(P.ucol + c0);
        const int mx = min(kSegCap, te - c0);
        m = 0;
        for (int x0 = 0; x0 < mx; x0 += 32) {
            const int x = x0 + lane;
            const int c = x < mx ? __ldg(P.ucol + c0 + x) : INT_MAX;
            const bool in = c - c_0 < kMapBits;  // a prefix: the columns ascend
            if (in) {
                W.tcol[x] = c;
                W.tval[x] = ld_cg(U + c0 + x);
            }
            m += __popc(__ballot_sync(full, in));
        }
        // the FP64 diagonal of a Chol/Herk target row (T = float): first chunk only
        const bool dchunk = MIXED && start_at_r && c0 == tb;
        if (dchunk && lane == 0) W.dacc = __ldcg(P.udiag + r);
        __syncwarp();
        const int nw = ((W.tcol[m - 1] - c_0) >> 5) + 1;
        const unsigned span = unsigned(nw) * 32u;
        for (int w = lane; w < nw; w += 32) W.cmap[w].x = 0u;
        __syncwarp();
        for (int x = lane; x < m; x += 32) {
            const int off = W.tcol[x] - c_0;
            atomicOr(&W.cmap[off >> 5].x, 1u << (off & 31));
            if (x == 0 || ((W.tcol[x - 1] - c_0) >> 5) != (off >> 5)) W.cmap[off >> 5].y = unsigned(x);
        }
        __syncwarp();
        for (int q0 = ca; q0 < cb; q0 += 32) {
            const int nq0 = min(32, cb - q0);
            int dn = 1, len = 0, so = 0;
            int4 pv = make_int4(0, 0, 0, 0);
            if (lane < nq0) {
                const int2 pe = __ldg(P.csc + q0 + lane);
                int sb;
                if (start_at_r) {
                    sb = pe.y;
                    len = __ldg(P.cseg_end + q0 + lane) - pe.y;
                } else {
                    const int2 s = row_segment(P, pe.x, srcblk);
                    sb = s.x;
                    len = s.y - s.x;
                }
                pv = make_int4(pe.x, pe.y, sb, len);
                if (SPLIT) so = len > 0 ? __ldg(soffs + pe.x - rbase) : 0;
                // one CTA's Chol/Trsm: the completion flags of the whole batch, one per lane
                else if (MODE != M_UPDATE && len > 0) dn = done[pe.x - rbase];
            }
            // the batch without the pivots whose source segment is empty (a pivot row
            // with no entry in the source block column contributes nothing; a third of
            // the Trsm pivots, say), in the same ascending order
            const unsigned keep = __ballot_sync(full, len > 0);
            const int pos = __popc(keep & ((1u << lane) - 1u));
            const int nq = __popc(keep);
            if (len > 0) {
                W.piv[pos] = pv;
                if (SPLIT) W.psoff[pos] = so;
            }
            unsigned seen = __reduce_or_sync(full, len > 0 && dn != 0 ? 1u << pos : 0u);
            if (!SPLIT && MODE != M_UPDATE) __threadfence_block();
            __syncwarp();
            // each pivot is loaded when its turn comes (the other warps of the CTA cover
            // the L2 latency; keeping the next pivot in registers meanwhile costs more
            // registers than a 32-warp CTA has)
            PivReg<T> cur;
#pragma unroll 1
            for (int q = 0; q < nq; ++q) {
                load_pivot<MODE, SPLIT>(P, U, shadow, W, q, nq, start_at_r, rbase, done, seen, cur);
                if (!apply_pivot<MODE, EXACT, SPLIT>(P, U, shadow, W, q, start_at_r, rbase, done, seen, cur, c_0,
                                                     span, dchunk, deadline))
                    return;
            }
            __syncwarp();
            if (dchunk) {
                // FP64 diagonal (T = float): d -= sum of the batch's U_pr^2, each square exact
                // in FP64, summed in a fixed tree; a handful of FP64 instructions per batch
                // instead of a dependent multiply-add per pivot on the SM's scarce FP64 unit
                double sq = 0.0;
                if (lane < nq) {
                    const double av = double(W.abuf[lane]);
                    sq = av * av;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(full, sq, o);
                if (lane == 0) W.dacc -= sq;
                __syncwarp();
            }
        }
        if (MODE == M_CHOL) {
            if (c0 == tb) {
                if (lane == 0) {
                    const double d = MIXED ? W.dacc : double(W.tval[0]);
                    if (!(d > 0.0) || !isfinite(d)) note_breakdown(P, r);
                    if (EXACT) {
                        // IEEE square root, then the row divided by the pivot
                        const double piv = sqrt(d);
                        W.tval[0] = T(piv);
                        W.dacc = piv;
                    } else {
                        // the reciprocal pivot first; the row is multiplied by it
                        const double y = rsqrt_newton(d);
                        const double piv = d * y;
                        if (MIXED) __stcg(P.udiag + r, piv);
                        __stcg(P.urcp + r, y);
                        W.tval[0] = T(piv);
                        W.dacc = y;
                    }
                }
                __syncwarp();
                scale = T(W.dacc);
                if (EXACT) for (int x = 1 + lane; x < m; x += 32) W.tval[x] = W.tval[x] / scale;
                else for (int x = 1 + lane; x < m; x += 32) W.tval[x] = W.tval[x] * scale;
            } else {
                if (EXACT) for (int x = lane; x < m; x += 32) W.tval[x] = W.tval[x] / scale;
                else for (int x = lane; x < m; x += 32) W.tval[x] = W.tval[x] * scale;
            }
        } else if (MODE == M_TRSM) {
            if (EXACT) for (int x = lane; x < m; x += 32) W.tval[x] = W.tval[x] / scale;
            else for (int x = lane; x < m; x += 32) W.tval[x] = W.tval[x] * scale;
        } else if (dchunk && lane == 0) {
            __stcg(P.udiag + r, W.dacc);  // Herk: the updated FP64 diagonal
        }
        __syncwarp();
        for (int x = lane; x < m; x += 32) __stcg(U + c0 + x, W.tval[x]);
        if (SPLIT) {
            // publish the finished chunk for the split task's other rows
            T* pub = shadow + __ldg(soffs + r - rbase);
            for (int x = lane; x < m; x += 32) __stcg(pub + c0 + x, W.tval[x]);
        }
        __syncwarp();
    }
}

// Dynamic shared memory of one CTA: scheduler words, per-row flags, per-warp buffers.
constexpr size_t kSmemHead = 32;
template <typename T>
__host__ __device__ constexpr size_t warp_bytes() { return (sizeof(WarpBuf<T>) + 15) / 16 * 16; }
template <typename T>
__host__ __device__ constexpr size_t smem_bytes(int warps) {
    return kSmemHead + kMaxBlockRows + size_t(warps) * warp_bytes<T>();
}
static_assert((kSmemHead + kMaxBlockRows) % 16 == 0, "warp buffers must start 16-byte aligned");

template <int WARPS, bool EXACT, typename T>
__global__ void __launch_bounds__(WARPS * 32)
numeric_persistent(DevPlan P, unsigned long long timeout_ns) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    unsigned char* s_done = smem_raw + kSmemHead;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpBuf<T>& W = *reinterpret_cast<WarpBuf<T>*>(smem_raw + kSmemHead + kMaxBlockRows +
                                                   size_t(warp) * warp_bytes<T>());
    T* U = static_cast<T*>(P.uval);
    const unsigned long long deadline = gtimer() + timeout_ns;
    volatile unsigned char* done = s_done;

    for (;;) {
        if (threadIdx.x == 0) {
            int task = -1, chunk = 0;
            const int slot = atomicAdd(P.counters + 0, 1);
            if (slot < P.total_items) {
                // the claimed item runs once its task's predecessors have all finished
                const int2 it = __ldg(P.claim + slot);
                unsigned spins = 0;
                bool ok = true;
                while (ld_volatile(P.indeg + it.x) != 0) {
                    if ((++spins & 63) == 0) {
                        if (ld_volatile(P.counters + 3)) { ok = false; break; }
                        if (gtimer() > deadline) { set_timeout(P, 1); ok = false; break; }
                    }
                    __nanosleep(64);
                }
                if (ok) {
                    __threadfence();
                    task = it.x;
                    chunk = it.y;
                }
            }
            sm.task = task;
            sm.chunk = chunk;
            sm.slot = slot;
            if (P.trace) sm.t0 = gtimer();
        }
        __syncthreads();
        const int task = sm.task, chunk = sm.chunk;
        if (task < 0) break;
        const int4 Tk = __ldg(P.task + task);
        const int t0 = __ldg(P.tgt_ptr + task), nt = __ldg(P.tgt_ptr + task + 1) - t0;

        if ((Tk.x == T_CHOL || Tk.x == T_TRSM) && __ldg(P.flag_off + task) >= 0) {
            // a split task: every CTA holding one of its items claims rows from the
            // task's counter; finished rows are published in the shadow array
            const int blk = Tk.y;
            const int rbase = __ldg(P.ranges + blk);
            const int* soffs = P.soff + __ldg(P.flag_off + task);
            T* shadow = static_cast<T*>(P.shadow);
            for (;;) {
                int idx = 0;
                if (lane == 0) idx = atomicAdd(P.row_next + task, 1);
                idx = __shfl_sync(0xffffffffu, idx, 0);
                if (idx >= nt) break;
                const int4 g = __ldg(P.tgt + t0 + idx);
                const int gend = __ldg(P.tgt_end + t0 + idx);
                if (Tk.x == T_CHOL)
                    process_target<M_CHOL, EXACT, true, T>(P, U, g.x, g.y, g.z, g.w, gend, blk, true, rbase,
                                                           nullptr, W, deadline, soffs, shadow);
                else
                    process_target<M_TRSM, EXACT, true, T>(P, U, g.x, g.y, g.z, g.w, gend, Tk.w, false,
                                                           rbase, nullptr, W, deadline, soffs, shadow);
            }
        } else if (Tk.x == T_CHOL || Tk.x == T_TRSM) {
            const int blk = Tk.y;
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
                if (Tk.x == T_CHOL)
                    process_target<M_CHOL, EXACT, false, T>(P, U, g.x, g.y, g.z, g.w, gend, blk, true,
                                                            rbase, done, W, deadline);
                else
                    process_target<M_TRSM, EXACT, false, T>(P, U, g.x, g.y, g.z, g.w, gend, Tk.w, false,
                                                            rbase, done, W, deadline);
                __threadfence_block();
                __syncwarp();
                if (lane == 0) done[g.x - rbase] = 1;
            }
        } else {
            const int first = chunk * P.rows_per_item;
            const int last = min(nt, first + P.rows_per_item);
            const bool herk = (Tk.x == T_HERK);
            for (int idx = first + warp; idx < last; idx += WARPS) {
                const int4 g = __ldg(P.tgt + t0 + idx);
                const int gend = __ldg(P.tgt_end + t0 + idx);
                if (herk)
                    process_target<M_UPDATE, EXACT, false, T>(P, U, g.x, g.y, g.z, g.w, gend, Tk.w, true, 0,
                                                              done, W, deadline);
                else
                    process_target<M_UPDATE, EXACT, false, T>(P, U, g.x, g.y, g.z, g.w, gend, Tk.w, false, 0,
                                                              done, W, deadline);
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
                if (P.trace) {
                    unsigned long long* rec = P.trace + 4ull * sm.slot;
                    rec[0] = sm.t0;
                    rec[1] = gtimer();
                    rec[2] = (unsigned long long)(unsigned)task | ((unsigned long long)(unsigned)chunk << 32);
                    rec[3] = smid();
                }
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                const int s0 = __ldg(P.succ_ptr + task), s1 = __ldg(P.succ_ptr + task + 1);
                for (int e = s0 + lane; e < s1; e += 32) atomicSub(P.indeg + __ldg(P.succ + e), 1);
            }
        }
    }
}

// Scatter of B's values onto the pattern S (zero on fill, optional diagonal shift)
// and reset of the scheduler state.  gsrc >= 0: index into A's values; -1: fill;
// <= -2: the diagonal, whose index is -2 - gsrc.  With T = float the off-diagonal
// values are rounded to FP32 and the diagonals go to the FP64 array udiag.
template <typename T>
__global__ void numeric_prepare(DevPlan P, const double* __restrict__ av, double alpha, int nnz_u) {
    constexpr bool MIXED = std::is_same<T, float>::value;
    const int stride = gridDim.x * blockDim.x;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    T* U = static_cast<T*>(P.uval);
    for (int pos = tid; pos < nnz_u; pos += stride) {
        const int s = __ldg(P.gsrc + pos);
        double v = 0.0;
        if (s >= 0) {
            v = __ldg(av + s);
        } else if (s <= -2) {
            v = __ldg(av + (-2 - s));
            if (alpha != 0.0) v = __dadd_rn(v, __dmul_rn(alpha, v));
        }
        U[pos] = T(v);
    }
    if (MIXED)
        for (int i = tid; i < P.n; i += stride) {
            double v = __ldg(av + __ldg(P.diag_src + i));
            if (alpha != 0.0) v = __dadd_rn(v, __dmul_rn(alpha, v));
            P.udiag[i] = v;
        }
    for (int t = tid; t < P.ntasks; t += stride) {
        P.indeg[t] = __ldg(P.indeg0 + t);
        P.items_left[t] = __ldg(P.nitems + t);
        P.row_next[t] = 0;
    }
    if (MIXED) {
        unsigned* sh = static_cast<unsigned*>(P.shadow);
        for (long long i = tid; i < P.nshadow; i += stride) sh[i] = kSentinel32;
    } else {
        unsigned long long* sh = static_cast<unsigned long long*>(P.shadow);
        for (long long i = tid; i < P.nshadow; i += stride) sh[i] = kSentinel64;
    }
    if (tid == 0) {
        P.counters[0] = 0;
        P.counters[1] = 0;
        P.counters[2] = 0;
        P.counters[3] = 0;
        *P.brk_row = 0x7fffffffffffffffLL;
        P.diag[0] = 0;
        P.diag[1] = 0;
    }
}

template <int WARPS, bool EXACT, typename T>
cudaError_t launch_t(const DevPlan& P, int grid, unsigned long long timeout_ns, cudaStream_t s) {
    numeric_persistent<WARPS, EXACT, T><<<grid, WARPS * 32, smem_bytes<T>(WARPS), s>>>(P, timeout_ns);
    return cudaGetLastError();
}

template <int WARPS, bool EXACT, typename T>
cudaError_t occupancy_t(int* blocks) {
    cudaError_t e = cudaFuncSetAttribute(numeric_persistent<WARPS, EXACT, T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem_bytes<T>(WARPS)));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, numeric_persistent<WARPS, EXACT, T>,
                                                         WARPS * 32, smem_bytes<T>(WARPS));
}

}  // namespace

cudaError_t numeric_blocks_per_sm(int warps, bool exact, int dtype, int* blocks) {
    if (dtype == IC_F32)
        return warps == 8 ? occupancy_t<8, false, float>(blocks)
             : warps == 32 ? occupancy_t<32, false, float>(blocks) : occupancy_t<16, false, float>(blocks);
    if (warps == 8) return exact ? occupancy_t<8, true, double>(blocks) : occupancy_t<8, false, double>(blocks);
    if (warps == 32) return exact ? occupancy_t<32, true, double>(blocks) : occupancy_t<32, false, double>(blocks);
    return exact ? occupancy_t<16, true, double>(blocks) : occupancy_t<16, false, double>(blocks);
}

cudaError_t launch_numeric_prepare(const DevPlan& P, const double* avals, double shift_alpha, int dtype,
                                   cudaStream_t s) {
    const int work = P.nnz_u > P.ntasks ? P.nnz_u : P.ntasks;
    int pgrid = (work + 255) / 256;
    pgrid = pgrid < 1 ? 1 : (pgrid > 8192 ? 8192 : pgrid);
    if (dtype == IC_F32)
        numeric_prepare<float><<<pgrid, 256, 0, s>>>(P, avals, shift_alpha, P.nnz_u);
    else
        numeric_prepare<double><<<pgrid, 256, 0, s>>>(P, avals, shift_alpha, P.nnz_u);
    return cudaGetLastError();
}

cudaError_t launch_numeric(const DevPlan& P, int warps, bool exact, int dtype, int grid,
                           unsigned long long timeout_ns, cudaStream_t s) {
    if (dtype == IC_F32)
        return warps == 8 ? launch_t<8, false, float>(P, grid, timeout_ns, s)
             : warps == 32 ? launch_t<32, false, float>(P, grid, timeout_ns, s)
                           : launch_t<16, false, float>(P, grid, timeout_ns, s);
    if (warps == 8)
        return exact ? launch_t<8, true, double>(P, grid, timeout_ns, s)
                     : launch_t<8, false, double>(P, grid, timeout_ns, s);
    if (warps == 32)
        return exact ? launch_t<32, true, double>(P, grid, timeout_ns, s)
                     : launch_t<32, false, double>(P, grid, timeout_ns, s);
    return exact ? launch_t<16, true, double>(P, grid, timeout_ns, s)
                 : launch_t<16, false, double>(P, grid, timeout_ns, s);
}

}  // namespace ick
