// Preconditioner application and PCG on sm_103a (the use of IC(k) named in Section 1;
// the paper does not describe the solves, so they follow the textbook definitions).
//
// ic_apply: z = P (U^T U)^{-1} P^T r.  The forward solve U^T y = P^T r gathers column i
// of U (the column lists built by the symbolic phase); the backward solve U z = y
// gathers row i of U.  Both are synchronisation-free: warps claim rows from an atomic
// counter in an order precomputed by the symbolic phase (rows sorted by their depth in
// the solve's row dependence DAG) and spin, with a bounded wait, on per-row completion
// stamps of the rows they depend on.  A row's inputs have smaller depth and are claimed
// before it, so the earliest unfinished claimed row always has its inputs and no warp
// waits on a row that no running warp owns; rows of equal depth (independent ND
// subtrees, wavefronts inside a part) run concurrently.
#include <cstdint>
#include <mutex>

#include "ick_internal.h"

namespace ick {
namespace {

constexpr int kApplyThreads = 256;

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Ends a solve whose wait gave up: the abort word (stops every other waiting warp of
// this launch; cleared when the next application starts) and, in the word after it, the
// timeout record, which stays set until the host reads it (pcg_solve, ic_apply_status,
// ic_apply_static_status).
__device__ __forceinline__ void raise_abort(int* abort_word) {
    atomicExch(abort_word, 1);
    atomicOr(abort_word + 1, 1);
}

// Spin until flag[i] == want; false on timeout or abort.
__device__ __forceinline__ bool wait_flag(const int* flag, int i, int want, int* abort_word,
                                          unsigned long long deadline) {
    const volatile int* f = flag + i;
    unsigned spins = 0;
    while (*f != want) {
        if ((++spins & 255) == 0) {
            if (*(volatile int*)abort_word) return false;
            if (gtimer() > deadline) { raise_abort(abort_word); return false; }
        }
        __nanosleep(32);
    }
    return true;
}

__global__ void __launch_bounds__(kApplyThreads)
forward_solve(SolvePlan S, const double* __restrict__ r, int stamp, unsigned long long timeout_ns) {
    const int lane = threadIdx.x & 31;
    const unsigned long long deadline = gtimer() + timeout_ns;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(S.counter + 0, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= S.n) break;
        const int i = __ldg(S.fwd_order + t);
        const int a = __ldg(S.cptr + i), b = __ldg(S.cptr + i + 1);
        double acc = 0.0;
        bool ok = true;
        for (int e = a + lane; e < b; e += 32) {
            const int2 pe = __ldg(S.csc + e);
            ok = ok && wait_flag(S.flag, pe.x, stamp, S.counter + 2, deadline);
            acc = fma(__ldg(S.uval + pe.y), __ldcg(S.y + pe.x), acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const double v = (__ldg(r + __ldg(S.perm + i)) - acc) / __ldg(S.uval + __ldg(S.urp + i));
            S.y[i] = v;
            __threadfence();
            *(volatile int*)(S.flag + i) = stamp;
        }
        if (__any_sync(0xffffffffu, !ok)) break;
    }
}

__global__ void __launch_bounds__(kApplyThreads)
backward_solve(SolvePlan S, double* __restrict__ z, int stamp, unsigned long long timeout_ns) {
    const int lane = threadIdx.x & 31;
    const unsigned long long deadline = gtimer() + timeout_ns;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(S.counter + 1, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= S.n) break;
        const int i = __ldg(S.bwd_order + t);
        const long long a = __ldg(S.urp + i), b = __ldg(S.urp + i + 1);
        double acc = 0.0;
        bool ok = true;
        for (long long e = a + 1 + lane; e < b; e += 32) {
            const int c = __ldg(S.ucol + e);
            ok = ok && wait_flag(S.flag, c, stamp, S.counter + 2, deadline);
            acc = fma(__ldg(S.uval + e), __ldcg(S.y + c), acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) {
            const double v = (__ldcg(S.y + i) - acc) / __ldg(S.uval + a);
            S.y[i] = v;
            z[__ldg(S.perm + i)] = v;
            __threadfence();
            *(volatile int*)(S.flag + i) = stamp;
        }
        if (__any_sync(0xffffffffu, !ok)) break;
    }
}

// Solves of ic_apply (and pcg_solve).  Same claim orders and the same per-row sums as
// the kernels above, but a row's value is its own completion flag: the work vectors
// are filled with the bit pattern kUnset (all ones, a NaN that arithmetic does not
// produce) before the launch, a row's value is published with one 8-byte store, and a
// reader polls the value itself.  There is no separate flag store and no fence, so a
// dependence costs one write and one read of L2 instead of two of each.
constexpr long long kUnset = -1LL;

__device__ __forceinline__ double publishable(double v) {
    return __double_as_longlong(v) == kUnset ? __longlong_as_double(0x7fffffffffffffffLL) : v;
}

// Value of x[i] once it is set; false (and 0) on timeout or abort.
__device__ __forceinline__ double await_value(const double* x, int i, int* abort_word,
                                              unsigned long long deadline, bool& ok) {
    const volatile long long* p = reinterpret_cast<const volatile long long*>(x + i);
    long long b = *p;
    unsigned spins = 0;
    while (b == kUnset) {
        if ((++spins & 255) == 0) {
            if (*(volatile int*)abort_word || gtimer() > deadline) {
                raise_abort(abort_word);
                ok = false;
                return 0.0;
            }
        }
        __nanosleep(16);
        b = *p;
    }
    return __longlong_as_double(b);
}

// G lanes per row, 32/G rows per warp: on GB300 an FP64 warp instruction occupies the
// SM's narrow FP64 pipe for the same time however many lanes are active, so packing
// several rows into each FMA and reduction step cuts the FP64 instructions per row.
// Rows of one warp are claimed together (32/G consecutive positions of the padded
// claim order, whose level runs are multiples of 8), so they always belong to one
// dependence level and never wait on each other: a warp-wide reconvergence before a
// row is published can then never block the row's own consumer.  The diagonal is
// applied as a precomputed reciprocal.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
    const int lane = threadIdx.x & 31;
    const unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}

// FP32 counterparts of the value-as-flag helpers (all-ones is a NaN pattern for both).
__device__ __forceinline__ float publishable(float v) {
    return __float_as_int(v) == -1 ? __int_as_float(0x7fffffff) : v;
}
__device__ __forceinline__ float await_value(const float* x, int i, int* abort_word,
                                             unsigned long long deadline, bool& ok) {
    const volatile int* p = reinterpret_cast<const volatile int*>(x + i);
    int b = *p;
    unsigned spins = 0;
    while (b == -1) {
        if ((++spins & 255) == 0) {
            if (*(volatile int*)abort_word || gtimer() > deadline) {
                raise_abort(abort_word);
                ok = false;
                return 0.f;
            }
        }
        __nanosleep(16);
        b = *p;
    }
    return __int_as_float(b);
}

__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ld_cg(const float* p) { return __ldcg(p); }

// T = double: FP64 factor and solves.  T = float: FP32 factor values, work vectors and
// sums; the right-hand side arrives in FP64 and the result leaves in FP64.
template <int G, typename T>
__global__ void __launch_bounds__(kApplyThreads)
forward_solve_v(SolvePlan S, const T* __restrict__ uv, const T* __restrict__ rd_all,
                const double* __restrict__ r, T* yv, unsigned long long timeout_ns) {
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31, sub = lane / G, sl = lane % G;
    const unsigned long long deadline = gtimer() + timeout_ns;
    bool ok = true;
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = atomicAdd(S.counter + 0, R);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= S.nfwd_pad) break;
        const int t = t0 + sub;
        T acc = T(0);
        int i = -1;
        T rhs = T(0), rd = T(0);  // loaded before the waits: off the dependence chain
        if ((i = __ldg(S.fwd_pad + t)) >= 0) {
            if (sl == 0) {
                rhs = T(__ldg(r + __ldg(S.perm + i)));
                rd = __ldg(rd_all + i);
            }
            const int a = __ldg(S.cptr + i), b = __ldg(S.cptr + i + 1);
            for (int e = a + sl; e < b; e += G) {
                const int2 pe = __ldg(S.csc + e);
                const T u = __ldg(uv + pe.y);
                acc = fma(u, ok ? await_value(yv, pe.x, S.counter + 2, deadline, ok) : T(0), acc);
            }
        }
        acc = group_sum<G>(acc);
        if (sl == 0 && i >= 0) {
            const T v = (rhs - acc) * rd;
            *reinterpret_cast<volatile T*>(yv + i) = publishable(v);
        }
        if (__any_sync(0xffffffffu, !ok)) break;
    }
}

template <int G, typename T>
__global__ void __launch_bounds__(kApplyThreads)
backward_solve_v(SolvePlan S, const T* __restrict__ uv, const T* __restrict__ rd_all, const T* yv,
                 T* zv, double* __restrict__ z, unsigned long long timeout_ns) {
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31, sub = lane / G, sl = lane % G;
    const unsigned long long deadline = gtimer() + timeout_ns;
    bool ok = true;
    for (;;) {
        int t0 = 0;
        if (lane == 0) t0 = atomicAdd(S.counter + 1, R);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= S.nbwd_pad) break;
        const int t = t0 + sub;
        T acc = T(0);
        int i = -1;
        T rhs = T(0), rd = T(0);
        int dst = 0;
        if ((i = __ldg(S.bwd_pad + t)) >= 0) {
            if (sl == 0) {
                rhs = ld_cg(yv + i);
                rd = __ldg(rd_all + i);
                dst = __ldg(S.perm + i);
            }
            const long long a = __ldg(S.urp + i), b = __ldg(S.urp + i + 1);
            for (long long e = a + 1 + sl; e < b; e += G) {
                const int c = __ldg(S.ucol + e);
                const T u = __ldg(uv + e);
                acc = fma(u, ok ? await_value(zv, c, S.counter + 2, deadline, ok) : T(0), acc);
            }
        }
        acc = group_sum<G>(acc);
        if (sl == 0 && i >= 0) {
            const T v = (rhs - acc) * rd;
            z[dst] = double(v);
            *reinterpret_cast<volatile T*>(zv + i) = publishable(v);
        }
        if (__any_sync(0xffffffffu, !ok)) break;
    }
}

__global__ void rdiag_kernel(SolvePlan S) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
        if (S.dtype == IC_F32) S.rdiag32[i] = float(1.0 / S.udiag[i]);
        else S.rdiag[i] = 1.0 / S.uval[S.urp[i]];
    }
}

template <typename T>
cudaError_t launch_solves(const SolvePlan& S, const T* uv, const T* rd, const double* r, double* z,
                          T* y, int grid, unsigned long long timeout_ns, cudaStream_t s,
                          cudaEvent_t t0, cudaEvent_t t1) {
    if (t0) cudaEventRecord(t0, s);
    switch (S.lanes_per_row) {
        case 4:
            forward_solve_v<4, T><<<grid, kApplyThreads, 0, s>>>(S, uv, rd, r, y, timeout_ns);
            if (t1) cudaEventRecord(t1, s);
            backward_solve_v<4, T><<<grid, kApplyThreads, 0, s>>>(S, uv, rd, y, y + S.n, z, timeout_ns);
            break;
        case 8:
            forward_solve_v<8, T><<<grid, kApplyThreads, 0, s>>>(S, uv, rd, r, y, timeout_ns);
            if (t1) cudaEventRecord(t1, s);
            backward_solve_v<8, T><<<grid, kApplyThreads, 0, s>>>(S, uv, rd, y, y + S.n, z, timeout_ns);
            break;
        case 16:
            forward_solve_v<16, T><<<grid, kApplyThreads, 0, s>>>(S, uv, rd, r, y, timeout_ns);
            if (t1) cudaEventRecord(t1, s);
            backward_solve_v<16, T><<<grid, kApplyThreads, 0, s>>>(S, uv, rd, y, y + S.n, z, timeout_ns);
            break;
        default:
            forward_solve_v<32, T><<<grid, kApplyThreads, 0, s>>>(S, uv, rd, r, y, timeout_ns);
            if (t1) cudaEventRecord(t1, s);
            backward_solve_v<32, T><<<grid, kApplyThreads, 0, s>>>(S, uv, rd, y, y + S.n, z, timeout_ns);
            break;
    }
    return cudaGetLastError();
}

// y = A x with G threads per row (G in {4, 8, 16, 32}).
template <int G>
__global__ void __launch_bounds__(256)
spmv_kernel(int n, const long long* __restrict__ rp, const int* __restrict__ ci,
            const double* __restrict__ av, const double* __restrict__ x, double* __restrict__ y) {
    // the loop bound is uniform across the warp, so every lane reaches the shuffles
    constexpr int RPW = 32 / G;  // rows per warp and pass
    const int sub = threadIdx.x % G;
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int base = gwarp * RPW; base < n; base += nwarps * RPW) {
        const int i = base + (threadIdx.x & 31) / G;
        double acc = 0.0;
        if (i < n)
            for (long long e = __ldg(rp + i) + sub; e < __ldg(rp + i + 1); e += G)
                acc = fma(__ldg(av + e), __ldg(x + __ldg(ci + e)), acc);
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
        if (sub == 0 && i < n) y[i] = acc;
    }
}

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double s[kRedThreads / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < kRedThreads / 32 ? s[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kRedThreads)
dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int n, double* partial) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        acc = fma(a[i], b[i], acc);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// Deterministic final sum of the partials, then one scalar update.
__global__ void __launch_bounds__(kRedThreads)
finish_kernel(const double* __restrict__ partial, int nparts, PcgScalars* sc, int op) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += partial[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) {
        switch (op) {
            case 0: sc->pq = acc; sc->alpha = sc->rz / acc; break;
            case 1: sc->rr = acc; sc->relres = sqrt(acc) / sc->bnorm; break;
            case 2: sc->rz_new = acc; sc->beta = acc / sc->rz; sc->rz = acc; break;
            case 3: sc->rz = acc; break;
            case 4: sc->bnorm = acc > 0.0 ? sqrt(acc) : 1.0; break;
            default: break;
        }
    }
}

__global__ void __launch_bounds__(kRedThreads)
xr_kernel(int n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
          const double* __restrict__ q, const PcgScalars* sc, double* partial) {
    const double alpha = sc->alpha;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kRedThreads)
p_kernel(int n, double* __restrict__ p, const double* __restrict__ z, const PcgScalars* sc) {
    const double beta = sc->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

__global__ void init_kernel(int n, const double* __restrict__ b, double* __restrict__ x,
                            double* __restrict__ r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = 0.0;
        r[i] = b[i];
    }
}

int vec_grid(int n) {
    int g = (n + kRedThreads - 1) / kRedThreads;
    return g < 1 ? 1 : (g > kMaxParts ? kMaxParts : g);
}

}  // namespace

int pcg_parts(int n) { return vec_grid(n); }

cudaError_t apply_blocks_per_sm(int* blocks) {
    int a = 0, b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, forward_solve, kApplyThreads, 0);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, backward_solve, kApplyThreads, 0);
    *blocks = a < b ? a : b;
    return e;
}

cudaError_t launch_apply(const SolvePlan& S, const double* r, double* z, int epoch,
                         unsigned long long timeout_ns, int grid, cudaStream_t s, cudaEvent_t t0,
                         cudaEvent_t t1) {
    if (S.n == 0) return cudaSuccess;
    (void)epoch;
    if (S.solve_mode == 0) return launch_apply_dag(S, r, z, timeout_ns, grid, s, t0, t1);
    // S.y holds 2n doubles: the forward then the backward result (2n floats for IC_F32)
    const size_t bytes = 2 * size_t(S.n) * (S.dtype == IC_F32 ? sizeof(float) : sizeof(double));
    cudaError_t e = cudaMemsetAsync(S.y, 0xff, bytes, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(S.counter, 0, 3 * sizeof(int), s);  // claims and the abort word
    if (e != cudaSuccess) return e;
    if (S.dtype == IC_F32)
        return launch_solves<float>(S, S.uval32, S.rdiag32, r, z, reinterpret_cast<float*>(S.y), grid,
                                    timeout_ns, s, t0, t1);
    return launch_solves<double>(S, S.uval, S.rdiag, r, z, S.y, grid, timeout_ns, s, t0, t1);
}

cudaError_t launch_solve_prepare(const SolvePlan& S, cudaStream_t s) {
    if (S.n == 0) return cudaSuccess;
    int g = (S.n + 255) / 256;
    rdiag_kernel<<<g > 4096 ? 4096 : g, 256, 0, s>>>(S);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_dag_prepare(S, s);
}

// ---------------------------------------------------------------------------------
// Allocation-free variant of the preconditioner application (ic_apply_static).
//
// Some callers cannot call cudaMalloc where they apply the preconditioner: a plugin
// that runs inside another framework which owns the device's memory budget and hands
// its plugins no allocator, or a loop with a hard latency limit in which a cudaMalloc
// (which may synchronise the device) is not allowed.  For them the solve's scratch --
// the permuted work vector, the per-row completion stamps, the two row-claim counters,
// the abort word and the timeout record -- lives in one file-scope device array, sized
// for at most kStaticApplyRows rows.  Every GPU that loads the library keeps this array
// until the process exits; all calls share it, so calls that overlap on the GPU (on
// different streams, or from different threads) race and must be serialised by the
// caller.  The array keeps the contents of the last call: the claim counters and the
// abort word are cleared at the start of every call, and the completion stamps never
// need clearing because each call on a device uses stamps that no earlier call on that
// device has written (a per-device call counter).  The solves are the row-level
// kernels above (their scratch is one work vector and one stamp per row).
constexpr int kStaticApplyRows = 1 << 20;
constexpr size_t kStaticApplyBytes =
    size_t(kStaticApplyRows) * sizeof(double) + size_t(kStaticApplyRows) * sizeof(int) + 16;

static __device__ __align__(256) unsigned char g_apply_scratch[kStaticApplyBytes];

int static_apply_max_rows() { return kStaticApplyRows; }

namespace {

// Device address of g_apply_scratch on the current device (the symbol's name is only
// a host-side stand-in).  Looked up once per device, with that device current; the
// lookup of each device runs once even when several threads make their first call
// together.
cudaError_t static_apply_scratch(unsigned char** out) {
    static std::once_flag once[kStaticApplyDevices];
    static void* addr[kStaticApplyDevices] = {};
    static cudaError_t err[kStaticApplyDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kStaticApplyDevices) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [dev] {
        void* p = nullptr;
        err[dev] = cudaGetSymbolAddress(&p, g_apply_scratch);
        addr[dev] = p;
    });
    if (err[dev] != cudaSuccess) return err[dev];
    *out = static_cast<unsigned char*>(addr[dev]);
    return cudaSuccess;
}

int* static_counters(unsigned char* base) {
    return reinterpret_cast<int*>(base + size_t(kStaticApplyRows) * (sizeof(double) + sizeof(int)));
}

}  // namespace

cudaError_t launch_apply_static(const SolvePlan& H, const double* r, double* z, int epoch,
                                unsigned long long timeout_ns, int grid, cudaStream_t s,
                                bool clear_stamps) {
    if (H.n == 0) return cudaSuccess;
    if (H.n > kStaticApplyRows) return cudaErrorInvalidValue;
    unsigned char* base = nullptr;
    cudaError_t e = static_apply_scratch(&base);
    if (e != cudaSuccess) return e;
    SolvePlan S = H;
    S.y = reinterpret_cast<double*>(base);
    S.flag = reinterpret_cast<int*>(base + size_t(kStaticApplyRows) * sizeof(double));
    S.counter = static_counters(base);
    if (clear_stamps) {
        e = cudaMemsetAsync(S.flag, 0, size_t(kStaticApplyRows) * sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    e = cudaMemsetAsync(S.counter, 0, 3 * sizeof(int), s);  // claims and the abort word
    if (e != cudaSuccess) return e;
    forward_solve<<<grid, kApplyThreads, 0, s>>>(S, r, 2 * epoch, timeout_ns);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    backward_solve<<<grid, kApplyThreads, 0, s>>>(S, z, 2 * epoch + 1, timeout_ns);
    return cudaGetLastError();
}

cudaError_t static_apply_timeout(int* timed_out, cudaStream_t s) {
    *timed_out = 0;
    unsigned char* base = nullptr;
    cudaError_t e = static_apply_scratch(&base);
    if (e != cudaSuccess) return e;
    int* rec = static_counters(base) + 3;
    int v = 0;
    if ((e = cudaMemcpyAsync(&v, rec, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    if (v) {
        if ((e = cudaMemsetAsync(rec, 0, sizeof(int), s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    }
    *timed_out = v != 0;
    return cudaSuccess;
}

cudaError_t launch_spmv(const SolvePlan& S, const double* av, const double* x, double* y,
                        cudaStream_t s) {
    if (S.n == 0) return cudaSuccess;
    // threads per row from the average row length
    const double avg = double(S.nnz_a) / double(S.n);
    // few lanes per row: fewer FP64 reduction instructions per row (narrow FP64 pipe)
    const int G = avg <= 20 ? 4 : avg <= 48 ? 8 : avg <= 96 ? 16 : 32;
    long long blocks = ((long long)S.n * G + 255) / 256;
    const int grid = int(blocks > 65536 ? 65536 : blocks);
    switch (G) {
        case 4: spmv_kernel<4><<<grid, 256, 0, s>>>(S.n, S.arp, S.acol, av, x, y); break;
        case 8: spmv_kernel<8><<<grid, 256, 0, s>>>(S.n, S.arp, S.acol, av, x, y); break;
        case 16: spmv_kernel<16><<<grid, 256, 0, s>>>(S.n, S.arp, S.acol, av, x, y); break;
        default: spmv_kernel<32><<<grid, 256, 0, s>>>(S.n, S.arp, S.acol, av, x, y); break;
    }
    return cudaGetLastError();
}

cudaError_t pcg_dot(const double* a, const double* b, int n, double* partial, int nparts,
                    cudaStream_t s) {
    dot_kernel<<<nparts, kRedThreads, 0, s>>>(a, b, n, partial);
    return cudaGetLastError();
}

cudaError_t pcg_finish(const double* partial, int nparts, PcgScalars* sc, int op, cudaStream_t s) {
    finish_kernel<<<1, kRedThreads, 0, s>>>(partial, nparts, sc, op);
    return cudaGetLastError();
}

cudaError_t pcg_step_x_r(int n, double* x, double* r, const double* p, const double* q,
                         PcgScalars* sc, double* partial, int nparts, cudaStream_t s) {
    xr_kernel<<<nparts, kRedThreads, 0, s>>>(n, x, r, p, q, sc, partial);
    return cudaGetLastError();
}

cudaError_t pcg_step_p(int n, double* p, const double* z, PcgScalars* sc, cudaStream_t s) {
    p_kernel<<<vec_grid(n), kRedThreads, 0, s>>>(n, p, z, sc);
    return cudaGetLastError();
}

// The loop test of pcg_solve's device-side loop (one thread): the iteration count
// (0 before the first iteration, when the previous r.z is also set to 1 so that the
// first direction update leaves p = z) and the condition of the graph's WHILE node:
// another iteration while relres > tol and fewer than maxit have run.
__global__ void pcg_loop_kernel(PcgScalars* sc, int* it, double tol, int maxit, cudaGraphConditionalHandle cond,
                                int first) {
    const int k = first ? 0 : *it + 1;
    if (first) sc->rz = 1.0;
    *it = k;
    cudaGraphSetConditional(cond, sc->relres > tol && k < maxit ? 1u : 0u);
}

cudaError_t pcg_loop_step(PcgScalars* sc, int* it, double tol, int maxit, cudaGraphConditionalHandle cond,
                          bool first, cudaStream_t s) {
    pcg_loop_kernel<<<1, 1, 0, s>>>(sc, it, tol, maxit, cond, first ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t pcg_init(int n, const double* b, double* x, double* r, cudaStream_t s) {
    init_kernel<<<vec_grid(n), kRedThreads, 0, s>>>(n, b, x, r);
    return cudaGetLastError();
}

}  // namespace ick
