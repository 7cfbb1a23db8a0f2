// C ABI of libick.so (declared in include/ick.h): handle life cycle, device upload of
// the symbolic plan, and the host orchestration of the numeric, apply and PCG kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ick_internal.h"

using namespace ick;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return IC_ERR_CUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

struct ic_handle {
    HostPlan hp;
    ic_opts opts{};
    int device = -1;
    std::vector<void*> allocs;
    DevPlan dp{};
    SolvePlan sp{};
    int grid_numeric = 0;
    int grid_apply = 0;
    int apply_epoch = 0;
    bool factored = false;
    double symbolic_s = 0.0;
    // pinned host mirrors of small device status words
    int* h_counters = nullptr;      // counters[0..3], diag[0..1]
    long long* h_brk = nullptr;
    PcgScalars* h_sc = nullptr;
    // PCG scratch
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *partial = nullptr;
    PcgScalars* sc = nullptr;
    // timing (ic_set_timing)
    bool timing = false;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool apply_pending = false;  // ev[3] (forward) ev[5] (backward) ev[4] (end) of an apply not yet in tm
    ic_timing_t tm{};
    unsigned long long* trace_buf = nullptr;  // ic_set_trace
    unsigned long long* solve_trace_buf = nullptr;
    // systems of a batch (one system for ic_symbolic): row offsets, per-row system id,
    // per-system PCG scalars
    std::vector<int64_t> row_off;
    long long* d_row_off = nullptr;
    int* d_sys = nullptr;
    BatchScalars bs{};
    int* h_nactive = nullptr;      // pinned
    bool numeric_pending = false;  // ic_numeric_async issued, status not read yet
    cudaStream_t cap_stream = nullptr;  // graph capture / replay stream of pcg_solve_batch
    cudaEvent_t cap_ev[2] = {nullptr, nullptr};
    // pcg_solve as one graph: the prologue, then a WHILE node whose body is one
    // iteration and whose condition a kernel sets, so the loop runs on the device.
    // Built for the inputs of the call and kept until they change.
    cudaStream_t body_stream = nullptr;  // captures the WHILE node's body
    cudaGraphExec_t pcg_exec = nullptr;
    const void* pcg_av = nullptr;
    const double* pcg_b = nullptr;
    double* pcg_x = nullptr;
    double pcg_tol = 0.0;
    int pcg_maxit = -1, pcg_grid = 0;
    unsigned long long pcg_tmo = 0;
    int* d_iter = nullptr;  // iterations done (device)

    ~ic_handle() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        for (void* a : allocs) cudaFree(a);
        if (h_counters) cudaFreeHost(h_counters);
        if (h_brk) cudaFreeHost(h_brk);
        if (h_sc) cudaFreeHost(h_sc);
        if (h_nactive) cudaFreeHost(h_nactive);
        for (cudaEvent_t e : cap_ev)
            if (e) cudaEventDestroy(e);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (pcg_exec) cudaGraphExecDestroy(pcg_exec);
        if (body_stream) cudaStreamDestroy(body_stream);
    }

    template <class T>
    int alloc(T** out, size_t count) {
        void* d = nullptr;
        cudaError_t e = cudaMalloc(&d, count ? count * sizeof(T) : 16);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        allocs.push_back(d);
        *out = static_cast<T*>(d);
        return IC_OK;
    }

    template <class T>
    int upload(const T** out, const std::vector<T>& v) {
        T* d = nullptr;
        int st = alloc(&d, v.size());
        if (st) return st;
        if (!v.empty()) {
            cudaError_t e = cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
        }
        *out = d;
        return IC_OK;
    }
};

namespace {

// count: systems in the handle.  One system: a CTA of 32 warps per SM, so the Chol
// tasks of the top separators, which run alone, get a whole SM; a batch of small
// systems: two CTAs of 16 warps per SM, twice the tasks in flight.
// CTAs of the numeric kernel assumed by a host-only handle's claim order (one 32-warp
// CTA per SM of a GB300).
constexpr int kHostOnlyCtas = 152;

ic_opts normalise(const ic_opts* o, int64_t count) {
    ic_opts r{};
    if (o) r = *o;
    if (r.block_rows == 0) r.block_rows = 4096;
    if (r.warps_per_cta == 0) r.warps_per_cta = count > 1 ? 16 : 32;
    if (r.rows_per_item == 0) r.rows_per_item = r.warps_per_cta;
    if (r.timeout_s == 0.0) r.timeout_s = 10.0;
    if (r.solve_lanes == 0) r.solve_lanes = r.solve_mode == 0 ? 8 : 32;
    if (r.solve_ctas_per_sm == 0) r.solve_ctas_per_sm = r.solve_mode == 0 ? 2 : 3;
    return r;
}

int upload_plan(ic_handle* h) {
    HostPlan& P = h->hp;
    DevPlan& D = h->dp;
    int st = 0;
    D.n = int(P.n);
    D.nnz_u = int(P.nnz_u);
    D.nb = int(P.ranges.size()) - 1;
    D.ntasks = int(P.task.size());
    D.total_items = int(P.total_items);
    D.rows_per_item = P.rows_per_item;
    {
        const int64_t* dptr = nullptr;
        if ((st = h->upload(&dptr, P.urp))) return st;
        D.urp = reinterpret_cast<const long long*>(dptr);
    }
    {
        // 16 bytes of padding: the kernels copy whole aligned 16-byte chunks
        int* dcol = nullptr;
        if ((st = h->alloc(&dcol, P.ucol.size() + 4))) return st;
        CK(cudaMemset(dcol + P.ucol.size(), 0xff, 4 * sizeof(int)));
        if (!P.ucol.empty())
            CK(cudaMemcpy(dcol, P.ucol.data(), P.ucol.size() * sizeof(int), cudaMemcpyHostToDevice));
        D.ucol = dcol;
    }
    if ((st = h->upload(&D.gsrc, P.gsrc))) return st;
    if ((st = h->upload(&D.ranges, P.ranges))) return st;
    if ((st = h->upload(&D.rseg_ptr, P.rseg_ptr))) return st;
    if ((st = h->upload(&D.rseg_blk, P.rseg_blk))) return st;
    if ((st = h->upload(&D.rseg_se, P.rseg_se))) return st;
    if ((st = h->upload(&D.cptr, P.cptr))) return st;
    if ((st = h->upload(&D.csc, P.csc))) return st;
    if ((st = h->upload(&D.cseg_end, P.cseg_end))) return st;
    if ((st = h->upload(&D.task, P.task))) return st;
    if ((st = h->upload(&D.tgt_ptr, P.tgt_ptr))) return st;
    if ((st = h->upload(&D.tgt, P.tgt))) return st;
    if ((st = h->upload(&D.tgt_end, P.tgt_end))) return st;
    if ((st = h->upload(&D.nitems, P.nitems))) return st;
    if ((st = h->upload(&D.succ_ptr, P.succ_ptr))) return st;
    if ((st = h->upload(&D.succ, P.succ))) return st;
    if ((st = h->upload(&D.indeg0, P.indeg0))) return st;
    if ((st = h->upload(&D.flag_off, P.flag_off))) return st;
    if ((st = h->upload(&D.soff, P.soff))) return st;
    D.nshadow = P.nshadow;
    if (h->opts.dtype == IC_F32) {
        float* sh = nullptr;
        if ((st = h->alloc(&sh, size_t(P.nshadow)))) return st;
        D.shadow = sh;
    } else {
        double* sh = nullptr;
        if ((st = h->alloc(&sh, size_t(P.nshadow)))) return st;
        D.shadow = sh;
    }
    if ((st = h->alloc(&D.row_next, P.task.size()))) return st;
    // factor values (FP64, or FP32 plus FP64 pivots), padded by 16 bytes
    const bool f32 = h->opts.dtype == IC_F32;
    double* uval = nullptr;
    float* uval32 = nullptr;
    if (f32) {
        if ((st = h->alloc(&uval32, size_t(P.nnz_u) + 4))) return st;
        CK(cudaMemset(uval32, 0, (size_t(P.nnz_u) + 4) * sizeof(float)));
        D.uval = uval32;
        if ((st = h->alloc(&D.udiag, size_t(P.n)))) return st;
        if ((st = h->upload(&D.diag_src, P.udiag_src))) return st;
    } else {
        if ((st = h->alloc(&uval, size_t(P.nnz_u) + 2))) return st;
        CK(cudaMemset(uval, 0, (size_t(P.nnz_u) + 2) * sizeof(double)));
        D.uval = uval;
    }
    if ((st = h->alloc(&D.urcp, size_t(P.n)))) return st;
    if ((st = h->alloc(&D.indeg, P.task.size()))) return st;
    if ((st = h->alloc(&D.items_left, P.task.size()))) return st;
    if ((st = h->alloc(&D.counters, 8))) return st;
    if ((st = h->alloc(&D.brk_row, 1))) return st;
    if ((st = h->alloc(&D.diag, 8))) return st;

    // solve / PCG buffers
    SolvePlan& S = h->sp;
    S.n = int(P.n);
    S.nnz_a = P.nnz_a;
    S.urp = D.urp;
    S.ucol = D.ucol;
    S.cptr = D.cptr;
    S.csc = D.csc;
    S.uval = uval;
    S.uval32 = uval32;
    S.udiag = D.udiag;
    S.dtype = h->opts.dtype;
    if (f32 && (st = h->alloc(&S.rdiag32, size_t(P.n)))) return st;
    S.lanes_per_row = h->opts.solve_lanes;
    if ((st = h->upload(&S.fwd_pad, P.fwd_pad))) return st;
    if ((st = h->upload(&S.bwd_pad, P.bwd_pad))) return st;
    S.nfwd_pad = int(P.fwd_pad.size());
    S.nbwd_pad = int(P.bwd_pad.size());
    if ((st = h->alloc(&S.rdiag, size_t(P.n)))) return st;
    {
        const int32_t* dperm = nullptr;
        if ((st = h->upload(&dperm, P.perm))) return st;
        S.perm = dperm;
        const int64_t* darp = nullptr;
        if ((st = h->upload(&darp, P.arp))) return st;
        S.arp = reinterpret_cast<const long long*>(darp);
        const int32_t* dacol = nullptr;
        if ((st = h->upload(&dacol, P.acol))) return st;
        S.acol = dacol;
        if ((st = h->upload(&S.fwd_order, P.fwd_order))) return st;
        if ((st = h->upload(&S.bwd_order, P.bwd_order))) return st;
    }
    S.solve_mode = h->opts.solve_mode;
    S.nranges = int(P.ranges.size()) - 1;
    S.max_range_rows = P.max_range_rows;
    S.ranges = D.ranges;
    S.nftask = int(P.fs.task.size());
    S.nbtask = int(P.bs.task.size());
    S.noff = int(P.nnz_u - P.n);
    if ((st = h->upload(&S.sf_split, P.sf_split))) return st;
    if ((st = h->upload(&S.sb_nint, P.sb_nint))) return st;
    if ((st = h->upload(&S.lf_ptr, P.lf_ptr))) return st;
    if ((st = h->upload(&S.lf_ord, P.lf_ord))) return st;
    if ((st = h->upload(&S.lb_ptr, P.lb_ptr))) return st;
    if ((st = h->upload(&S.lb_ord, P.lb_ord))) return st;
    if ((st = h->upload(&S.lf_need, P.lf_need))) return st;
    if ((st = h->upload(&S.lb_need, P.lb_need))) return st;
    if ((st = h->upload(&S.xf_ptr, P.xf.ptr))) return st;
    if ((st = h->upload(&S.xf_j, P.xf.j))) return st;
    if ((st = h->upload(&S.xf_pos, P.xf.pos))) return st;
    if ((st = h->upload(&S.xb_ptr, P.xb.ptr))) return st;
    if ((st = h->upload(&S.xb_j, P.xb.j))) return st;
    if ((st = h->upload(&S.xb_pos, P.xb.pos))) return st;
    S.nxf = int(P.xf.j.size());
    S.nxb = int(P.xb.j.size());
    S.uvt = S.xf_val = S.xb_val = nullptr;
    if (S.solve_mode == 0) {
        const size_t cnt[3] = {size_t(P.nnz_u - P.n) + 4, P.xf.j.size() + 4, P.xb.j.size() + 4};
        void** dst[3] = {&S.uvt, &S.xf_val, &S.xb_val};
        for (int q = 0; q < 3; ++q) {
            if (f32) {
                float* t = nullptr;
                if ((st = h->alloc(&t, cnt[q]))) return st;
                *dst[q] = t;
            } else {
                double* t = nullptr;
                if ((st = h->alloc(&t, cnt[q]))) return st;
                *dst[q] = t;
            }
        }
    }
    if ((st = h->upload(&S.ftask, P.fs.task))) return st;
    if ((st = h->upload(&S.btask, P.bs.task))) return st;
    if ((st = h->upload(&S.f_succ_ptr, P.fs.succ_ptr))) return st;
    if ((st = h->upload(&S.f_succ, P.fs.succ))) return st;
    if ((st = h->upload(&S.b_succ_ptr, P.bs.succ_ptr))) return st;
    if ((st = h->upload(&S.b_succ, P.bs.succ))) return st;
    {
        std::vector<int32_t> deg(P.fs.indeg0);
        deg.insert(deg.end(), P.bs.indeg0.begin(), P.bs.indeg0.end());
        if ((st = h->upload(&S.dag_indeg0, deg))) return st;
        if ((st = h->alloc(&S.dag_indeg, deg.size()))) return st;
        if ((st = h->alloc(&S.dag_taken, deg.size()))) return st;
    }
    if ((st = h->upload(&S.f_next, P.fs.next))) return st;
    if ((st = h->upload(&S.b_next, P.bs.next))) return st;
    {
        // forward external sums, then backward ones; a row without external entries in
        // a direction is never written there and keeps the zero set here
        double* w = nullptr;
        if ((st = h->alloc(&w, 2 * size_t(P.n)))) return st;
        CK(cudaMemset(w, 0, 2 * size_t(P.n) * sizeof(double)));
        S.dag_w = w;
    }
    if ((st = h->alloc(&S.y, 2 * size_t(P.n)))) return st;  // forward and backward results
    if ((st = h->alloc(&S.flag, size_t(P.n)))) return st;
    CK(cudaMemset(S.flag, 0, size_t(P.n) * sizeof(int)));
    if ((st = h->alloc(&S.counter, 4))) return st;
    CK(cudaMemset(S.counter, 0, 4 * sizeof(int)));
    if ((st = h->alloc(&h->r, size_t(P.n)))) return st;
    if ((st = h->alloc(&h->z, size_t(P.n)))) return st;
    if ((st = h->alloc(&h->p, size_t(P.n)))) return st;
    if ((st = h->alloc(&h->q, size_t(P.n)))) return st;
    if ((st = h->alloc(&h->partial, size_t(kMaxParts)))) return st;
    if ((st = h->alloc(&h->sc, 1))) return st;
    CK(cudaMallocHost(&h->h_counters, 16 * sizeof(int)));
    CK(cudaMallocHost(&h->h_brk, sizeof(long long)));
    CK(cudaMallocHost(&h->h_sc, sizeof(PcgScalars)));

    int dev = 0, sms = 0, bpsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(numeric_blocks_per_sm(h->opts.warps_per_cta, h->opts.exact != 0, h->opts.dtype, &bpsm));
    if (bpsm < 1) return fail(IC_ERR_CUDA, "numeric kernel cannot be resident");
    h->grid_numeric = sms * bpsm;
    // the order in which the persistent kernel's CTAs claim the work items
    build_claim_order(P, h->grid_numeric);
    if (int64_t(P.claim.size()) != P.total_items) return fail(IC_ERR_ARG, "task graph has a cycle");
    if ((st = h->upload(&D.claim, P.claim))) return st;
    if (S.solve_mode == 0)
        CK(dag_blocks_per_sm(S.lanes_per_row, S.dtype, P.max_range_rows, &bpsm));
    else
        CK(apply_blocks_per_sm(&bpsm));
    if (bpsm < 1) return fail(IC_ERR_CUDA, "solve kernels cannot be resident");
    if (h->opts.solve_ctas_per_sm > 0 && h->opts.solve_ctas_per_sm < bpsm) bpsm = h->opts.solve_ctas_per_sm;
    h->grid_apply = sms * bpsm;
    CK(cudaDeviceSynchronize());
    return IC_OK;
}

// Adds the kernel time of the last apply (waiting for its end event) to the totals.
int fold_apply_time(ic_handle* h) {
    if (!h->apply_pending) return IC_OK;
    CK(cudaEventSynchronize(h->ev[4]));
    float f = 0.f, b = 0.f;
    CK(cudaEventElapsedTime(&f, h->ev[3], h->ev[5]));
    CK(cudaEventElapsedTime(&b, h->ev[5], h->ev[4]));
    h->tm.fwd_ms += f;
    h->tm.bwd_ms += b;
    h->tm.apply_ms += f + b;
    h->apply_pending = false;
    return IC_OK;
}

// Record the systems of the handle (count+1 row offsets into the original ordering)
// and allocate the per-row system ids and per-system PCG scalars.
int attach_batch(ic_handle* h, const int64_t* off, int64_t count) {
    h->row_off.assign(off, off + count + 1);
    const int64_t n = h->hp.n;
    std::vector<int32_t> sys(n);
    for (int64_t s = 0; s < count; ++s)
        for (int64_t i = off[s]; i < off[s + 1]; ++i) sys[i] = int32_t(s);
    int st = 0;
    const int* dsys = nullptr;
    if ((st = h->upload(&dsys, sys))) return st;
    h->d_sys = const_cast<int*>(dsys);
    const int64_t* droff = nullptr;
    if ((st = h->upload(&droff, h->row_off))) return st;
    h->d_row_off = reinterpret_cast<long long*>(const_cast<int64_t*>(droff));
    BatchScalars& B = h->bs;
    double* dbuf = nullptr;
    if ((st = h->alloc(&dbuf, 6 * size_t(count)))) return st;
    B.tmp = dbuf;
    B.rz = dbuf + count;
    B.bnorm = dbuf + 2 * count;
    B.alpha = dbuf + 3 * count;
    B.beta = dbuf + 4 * count;
    B.relres = dbuf + 5 * count;
    int* ibuf = nullptr;
    if ((st = h->alloc(&ibuf, 2 * size_t(count) + 2))) return st;
    B.active = ibuf;
    B.iters = ibuf + count;
    B.nactive = ibuf + 2 * count;
    B.iter = ibuf + 2 * count + 1;
    CK(cudaMallocHost(&h->h_nactive, sizeof(int)));
    return IC_OK;
}

}  // namespace

extern "C" {

const char* ic_strerror(int s) {
    switch (s) {
        case IC_OK: return "ok";
        case IC_ERR_ARG: return "invalid argument";
        case IC_ERR_PATTERN: return "malformed or asymmetric CSR pattern";
        case IC_ERR_BREAKDOWN: return "breakdown: non-positive or non-finite pivot";
        case IC_ERR_TIMEOUT: return "device wait timed out";
        case IC_ERR_CUDA: return "CUDA runtime error";
        case IC_ERR_NOMEM: return "out of memory";
        case IC_ERR_NOCONV: return "PCG did not converge";
        case IC_ERR_STATE: return "call out of order";
        default: return "unknown status";
    }
}

const char* ic_last_error(void) { return g_last_error.c_str(); }

int ic_nd_grid(int nx, int ny, int nz, int dof, int leaf_rows, int sep_colours, int leaf_colours,
               const uint8_t* keep, int32_t* perm_out, int64_t* ranges_out, int64_t* nranges_out,
               int64_t* n_out) {
    try {
        return nd_grid(nx, ny, nz, dof, leaf_rows, sep_colours, leaf_colours, keep, perm_out, ranges_out,
                       nranges_out, n_out);
    } catch (const std::bad_alloc&) {
        return fail(IC_ERR_NOMEM, "host allocation failed");
    }
}

// Shared by ic_symbolic (one system) and ic_symbolic_batch (row_off: count+1 offsets
// of the systems inside the block-diagonal union).
static int symbolic_impl(const ic_csr_pattern* A, int k, const int32_t* perm, const int64_t* ranges,
                         int64_t nranges, const ic_opts* opts, const int64_t* row_off, int64_t count,
                         ic_handle** out) {
    if (!out) return fail(IC_ERR_ARG, "NULL out");
    *out = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    ic_handle* h = nullptr;
    try {
        h = new ic_handle();
        h->opts = normalise(opts, count);
        if (h->opts.warps_per_cta != 8 && h->opts.warps_per_cta != 16 && h->opts.warps_per_cta != 32) {
            delete h;
            return fail(IC_ERR_ARG, "warps_per_cta must be 8, 16 or 32");
        }
        if ((h->opts.dtype != IC_F64 && h->opts.dtype != IC_F32) ||
            (h->opts.dtype == IC_F32 && h->opts.exact)) {
            delete h;
            return fail(IC_ERR_ARG, "dtype must be IC_F64 or IC_F32 (exact=1 needs IC_F64)");
        }
        if (h->opts.rows_per_item < 1 || h->opts.timeout_s < 0 ||
            (h->opts.solve_lanes != 4 && h->opts.solve_lanes != 8 && h->opts.solve_lanes != 16 &&
             h->opts.solve_lanes != 32) || (h->opts.solve_mode != 0 && h->opts.solve_mode != 1)) {
            delete h;
            return fail(IC_ERR_ARG, "rows_per_item / timeout_s / solve_lanes / solve_mode out of range");
        }
        // the solves' grid as upload_plan will size it (SMs of the current device, or
        // kHostOnlyCtas for a host-only handle, times the CTAs per SM asked for)
        int sms = kHostOnlyCtas;
        if (!h->opts.host_only) {
            int dev = 0, cnt = 0;
            if (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&cnt, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && cnt > 0)
                sms = cnt;
        }
        std::string err;
        int st = build_plan(A, k, perm, ranges, nranges, h->opts.block_rows, h->opts.rows_per_item,
                            h->opts.threads, h->opts.exact != 0, sms * std::max(1, h->opts.solve_ctas_per_sm),
                            h->hp, err);
        if (st) {
            delete h;
            return fail(st, err);
        }
        if (h->opts.host_only) {
            build_claim_order(h->hp, kHostOnlyCtas);
            h->row_off.assign(row_off, row_off + count + 1);
            h->symbolic_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            *out = h;
            return IC_OK;
        }
        cudaError_t e = cudaGetDevice(&h->device);
        if (e != cudaSuccess) {
            delete h;
            return cuda_fail(e, "cudaGetDevice");
        }
        st = upload_plan(h);
        if (!st) st = attach_batch(h, row_off, count);
        if (st) {
            delete h;
            return st;
        }
    } catch (const std::bad_alloc&) {
        delete h;
        return fail(IC_ERR_NOMEM, "host allocation failed");
    }
    h->symbolic_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = h;
    return IC_OK;
}

int ic_symbolic(const ic_csr_pattern* A, int k, const int32_t* perm, const int64_t* ranges,
                int64_t nranges, const ic_opts* opts, ic_handle** out) {
    if (!A) return fail(IC_ERR_ARG, "NULL pattern");
    const int64_t off[2] = {0, A->n};
    return symbolic_impl(A, k, perm, ranges, nranges, opts, off, 1, out);
}

int ic_symbolic_batch(int64_t count, const ic_csr_pattern* A, int k, const int32_t* const* perms,
                      const int64_t* const* ranges, const int64_t* nranges, const ic_opts* opts,
                      ic_handle** out) {
    if (!out) return fail(IC_ERR_ARG, "NULL out");
    *out = nullptr;
    if (count < 1 || !A) return fail(IC_ERR_ARG, "count must be >= 1 and A non-NULL");
    try {
        // block-diagonal union: rows and columns of system s shifted by row_off[s]; each
        // system's ordering and ranges are kept and shifted the same way
        std::vector<int64_t> off(count + 1, 0), noff(count + 1, 0);
        for (int64_t s = 0; s < count; ++s) {
            if (A[s].n < 0 || (A[s].n > 0 && (!A[s].rowptr || !A[s].colind)))
                return fail(IC_ERR_ARG, "system " + std::to_string(s) + ": bad pattern");
            off[s + 1] = off[s] + A[s].n;
            noff[s + 1] = noff[s] + (A[s].n ? A[s].rowptr[A[s].n] : 0);
        }
        const int64_t n = off[count];
        if (n > INT32_MAX - 1 || noff[count] > INT32_MAX) return fail(IC_ERR_ARG, "batch too large");
        std::vector<int64_t> rp(n + 1, 0);
        std::vector<int32_t> ci(noff[count]);
        std::vector<int32_t> pm(n);
        std::vector<int64_t> rg(1, 0);
        for (int64_t s = 0; s < count; ++s) {
            const ic_csr_pattern& a = A[s];
            for (int64_t i = 0; i < a.n; ++i) {
                rp[off[s] + i + 1] = noff[s] + a.rowptr[i + 1];
                for (int64_t e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e)
                    ci[noff[s] + e] = int32_t(a.colind[e] + off[s]);
                const int32_t pi = (perms && perms[s]) ? perms[s][i] : int32_t(i);
                if (pi < 0 || pi >= a.n) return fail(IC_ERR_ARG, "system " + std::to_string(s) + ": bad perm");
                pm[off[s] + i] = int32_t(pi + off[s]);
            }
            if (ranges && ranges[s] && nranges) {
                for (int64_t b = 1; b <= nranges[s]; ++b) rg.push_back(ranges[s][b] + off[s]);
                if (nranges[s] < 1 || ranges[s][0] != 0 || ranges[s][nranges[s]] != a.n)
                    return fail(IC_ERR_ARG, "system " + std::to_string(s) + ": ranges must run from 0 to n");
            } else if (a.n > 0) {
                rg.push_back(off[s + 1]);  // the whole system as one range (split by block_rows)
            }
        }
        ic_csr_pattern U{n, rp.data(), ci.data()};
        return symbolic_impl(&U, k, pm.data(), rg.data(), int64_t(rg.size()) - 1, opts, off.data(), count, out);
    } catch (const std::bad_alloc&) {
        return fail(IC_ERR_NOMEM, "host allocation failed");
    }
}

int ic_batch_info(const ic_handle* h, int64_t* count, int64_t* row_off) {
    if (!h || !count) return fail(IC_ERR_ARG, "NULL argument");
    *count = int64_t(h->row_off.size()) - 1;
    if (row_off) std::memcpy(row_off, h->row_off.data(), h->row_off.size() * sizeof(int64_t));
    return IC_OK;
}

// Enqueue the numeric phase and the copies of its status words to pinned host memory.
// With timing on, events bracket the scatter and the task kernel.
static int numeric_enqueue(ic_handle* h, const void* values, cudaStream_t s, bool timing) {
    if (!values && h->hp.nnz_a > 0) return fail(IC_ERR_ARG, "NULL values");
    if (h->opts.host_only) return fail(IC_ERR_STATE, "handle was created with host_only");
    const unsigned long long tmo = (unsigned long long)(h->opts.timeout_s * 1e9);
    if (timing) CK(cudaEventRecord(h->ev[0], s));
    CK(launch_numeric_prepare(h->dp, static_cast<const double*>(values), h->opts.shift_alpha, h->opts.dtype,
                              s));
    ++h->tm.launches;
    if (timing) CK(cudaEventRecord(h->ev[1], s));
    if (h->dp.total_items > 0) {
        CK(launch_numeric(h->dp, h->opts.warps_per_cta, h->opts.exact != 0, h->opts.dtype,
                          h->grid_numeric, tmo, s));
        ++h->tm.launches;
    }
    if (timing) CK(cudaEventRecord(h->ev[2], s));
    CK(launch_solve_prepare(h->sp, s));
    h->tm.launches += 1 + dag_prepare_launches(h->sp);
    CK(cudaMemcpyAsync(h->h_counters, h->dp.counters, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->h_counters + 4, h->dp.diag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->h_brk, h->dp.brk_row, sizeof(long long), cudaMemcpyDeviceToHost, s));
    return IC_OK;
}

// Interpret the status words copied by the last enqueued numeric phase.
static int numeric_status(ic_handle* h, int64_t* breakdown_row) {
    h->numeric_pending = false;
    h->factored = false;
    const int bits = h->h_counters[2];
    if (bits & kStTimeout)
        return fail(IC_ERR_TIMEOUT, "numeric: device wait timed out at site " + std::to_string(h->h_counters[5]));
    if (h->hp.total_items > 0 && h->h_counters[4] != h->hp.total_items)
        return fail(IC_ERR_TIMEOUT, "numeric: " + std::to_string(h->h_counters[4]) + " of " +
                                        std::to_string(h->hp.total_items) + " items completed");
    if (bits & kStBreakdown) {
        if (breakdown_row) *breakdown_row = h->h_brk[0];
        return fail(IC_ERR_BREAKDOWN, "breakdown at row " + std::to_string(h->h_brk[0]));
    }
    h->factored = true;
    return IC_OK;
}

int ic_numeric(ic_handle* h, const void* values, void* stream, int64_t* breakdown_row) {
    if (breakdown_row) *breakdown_row = -1;
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    DeviceGuard g(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    h->factored = false;
    int st = numeric_enqueue(h, values, s, h->timing);
    if (st) return st;
    CK(cudaStreamSynchronize(s));
    if (h->timing) {
        float a = 0.f, b = 0.f;
        CK(cudaEventElapsedTime(&a, h->ev[0], h->ev[1]));
        CK(cudaEventElapsedTime(&b, h->ev[1], h->ev[2]));
        h->tm.prepare_ms = a;
        h->tm.numeric_ms = b;
    }
    return numeric_status(h, breakdown_row);
}

int ic_numeric_async(ic_handle* h, const void* values, void* stream) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    DeviceGuard g(h->device);
    int st = numeric_enqueue(h, values, static_cast<cudaStream_t>(stream), false);
    if (st) return st;
    h->numeric_pending = true;
    h->factored = true;  // provisional until ic_numeric_status reads the status words
    return IC_OK;
}

int ic_numeric_status(ic_handle* h, int64_t* breakdown_row) {
    if (breakdown_row) *breakdown_row = -1;
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    return numeric_status(h, breakdown_row);
}

int ic_apply(ic_handle* h, const void* r, void* z, void* stream) {
    if (!h || ((!r || !z) && h->hp.n > 0)) return fail(IC_ERR_ARG, "NULL argument");
    if (r == z && h->hp.n > 0) return fail(IC_ERR_ARG, "r and z may not alias");
    if (!h->factored) return fail(IC_ERR_STATE, "ic_apply before a successful ic_numeric");
    if (h->hp.n == 0) return IC_OK;
    DeviceGuard g(h->device);
    const int epoch = ++h->apply_epoch;
    const unsigned long long tmo = (unsigned long long)(h->opts.timeout_s * 1e9);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (h->timing) {
        int st = fold_apply_time(h);
        if (st) return st;
    }
    CK(launch_apply(h->sp, static_cast<const double*>(r), static_cast<double*>(z), epoch, tmo,
                    h->grid_apply, s, h->timing ? h->ev[3] : nullptr, h->timing ? h->ev[5] : nullptr));
    h->tm.launches += 2;
    ++h->tm.apply_calls;
    if (h->timing) {
        CK(cudaEventRecord(h->ev[4], s));
        h->apply_pending = true;
    }
    return IC_OK;
}

int ic_apply_status(ic_handle* h, void* stream) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    if (h->opts.host_only || h->hp.n == 0) return IC_OK;
    DeviceGuard g(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rec = 0;
    CK(cudaMemcpyAsync(&rec, h->sp.counter + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!rec) return IC_OK;
    CK(cudaMemsetAsync(h->sp.counter + 3, 0, sizeof(int), s));
    CK(cudaStreamSynchronize(s));
    return fail(IC_ERR_TIMEOUT, "triangular solve wait timed out");
}

int ic_apply_static(ic_handle* h, const void* r, void* z, void* stream) {
    if (!h || ((!r || !z) && h->hp.n > 0)) return fail(IC_ERR_ARG, "NULL argument");
    if (r == z && h->hp.n > 0) return fail(IC_ERR_ARG, "r and z may not alias");
    if (!h->factored) return fail(IC_ERR_STATE, "ic_apply_static before a successful ic_numeric");
    if (h->opts.dtype != IC_F64) return fail(IC_ERR_ARG, "ic_apply_static: IC_F64 factors only");
    if (h->hp.n > static_apply_max_rows())
        return fail(IC_ERR_ARG, "ic_apply_static: n = " + std::to_string(h->hp.n) +
                                    " exceeds the static scratch limit of " +
                                    std::to_string(static_apply_max_rows()) + " rows; use ic_apply");
    if (h->hp.n == 0) return IC_OK;
    DeviceGuard g(h->device);
    // one call counter per device (each device has its own scratch array and stamps):
    // completion stamps 2*epoch and 2*epoch+1 never repeat on that device; the stamps
    // are cleared and its count restarts long before int overflow
    static std::atomic<int> calls[kStaticApplyDevices];
    if (h->device < 0 || h->device >= kStaticApplyDevices)
        return fail(IC_ERR_ARG, "ic_apply_static: device index above the supported range");
    int epoch = ++calls[h->device];
    bool clear = false;
    if (epoch >= (1 << 29)) {
        int expect = epoch;
        calls[h->device].compare_exchange_strong(expect, 1);
        epoch = 1;
        clear = true;
    }
    const unsigned long long tmo = (unsigned long long)(h->opts.timeout_s * 1e9);
    CK(launch_apply_static(h->sp, static_cast<const double*>(r), static_cast<double*>(z), epoch,
                           tmo, h->grid_apply, static_cast<cudaStream_t>(stream), clear));
    h->tm.launches += 2;
    return IC_OK;
}

int ic_apply_static_status(void* stream) {
    int rec = 0;
    CK(static_apply_timeout(&rec, static_cast<cudaStream_t>(stream)));
    return rec ? fail(IC_ERR_TIMEOUT, "ic_apply_static: triangular solve wait timed out") : IC_OK;
}

// pcg_solve's graph: the prologue of the host loop below (r = b, x = 0, |b|, |r|), then
// a WHILE node whose body is one iteration rotated so that the test comes last: the
// preconditioner application, r.z, beta and p of the previous iteration (p starts at
// 0 and the previous r.z at 1, so the first pass gives p = z), then q = A p, alpha, x
// and r, |r| and the loop test.  The arithmetic is the host loop's, operation for
// operation; no iteration is run after the test fails.
static cudaError_t pcg_capture(ic_handle* h, const double* av, const double* b, double* x, double tol, int maxit,
                               unsigned long long tmo) {
    const int n = int(h->hp.n);
    const int parts = pcg_parts(n);
    cudaStream_t s = h->cap_stream;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaStreamCaptureStatus cst;
    cudaGraph_t capg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphConditionalHandle cond = 0;
    cudaGraphNode_t wnode = nullptr;
    cudaGraph_t body = nullptr;
    e = cudaStreamGetCaptureInfo(s, &cst, nullptr, &capg, nullptr, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, capg, 0, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->sp.counter + 3, 0, sizeof(int), s);  // solve timeout record
    if (e == cudaSuccess) e = pcg_init(n, b, x, h->r, s);
    if (e == cudaSuccess) e = pcg_dot(b, b, n, h->partial, parts, s);
    if (e == cudaSuccess) e = pcg_finish(h->partial, parts, h->sc, 4, s);
    if (e == cudaSuccess) e = pcg_dot(h->r, h->r, n, h->partial, parts, s);
    if (e == cudaSuccess) e = pcg_finish(h->partial, parts, h->sc, 1, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->p, 0, size_t(n) * sizeof(double), s);
    if (e == cudaSuccess) e = pcg_loop_step(h->sc, h->d_iter, tol, maxit, cond, true, s);
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(s, &cst, nullptr, &capg, &deps, nullptr, &nd);
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, capg, deps, nullptr, nd, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(s, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    const cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (e == cudaSuccess) e = ee;
    // the body, captured into the node's own graph
    if (e == cudaSuccess) {
        cudaStream_t bs = h->body_stream;
        e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t be = launch_apply(h->sp, h->r, h->z, 0, tmo, h->grid_apply, bs);
            if (be == cudaSuccess) be = pcg_dot(h->r, h->z, n, h->partial, parts, bs);
            if (be == cudaSuccess) be = pcg_finish(h->partial, parts, h->sc, 2, bs);
            if (be == cudaSuccess) be = pcg_step_p(n, h->p, h->z, h->sc, bs);
            if (be == cudaSuccess) be = launch_spmv(h->sp, av, h->p, h->q, bs);
            if (be == cudaSuccess) be = pcg_dot(h->p, h->q, n, h->partial, parts, bs);
            if (be == cudaSuccess) be = pcg_finish(h->partial, parts, h->sc, 0, bs);
            if (be == cudaSuccess) be = pcg_step_x_r(n, x, h->r, h->p, h->q, h->sc, h->partial, parts, bs);
            if (be == cudaSuccess) be = pcg_finish(h->partial, parts, h->sc, 1, bs);
            if (be == cudaSuccess) be = pcg_loop_step(h->sc, h->d_iter, tol, maxit, cond, false, bs);
            cudaGraph_t bg = nullptr;
            const cudaError_t be2 = cudaStreamEndCapture(bs, &bg);
            e = be != cudaSuccess ? be : be2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->pcg_exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    return e;
}

// pcg_solve when no per-kernel timing is asked for: the whole solve is one graph
// launch; the host reads the iteration count, the residual and the solves' timeout
// record once, at the end.
static int pcg_solve_graph(ic_handle* h, const double* av, const double* b, double* x, double tol, int maxit,
                           int* iters, double* relres, cudaStream_t us) {
    const unsigned long long tmo = (unsigned long long)(h->opts.timeout_s * 1e9);
    if (!h->cap_stream) {
        CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->cap_ev[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->cap_ev[1], cudaEventDisableTiming));
    }
    if (!h->body_stream) CK(cudaStreamCreateWithFlags(&h->body_stream, cudaStreamNonBlocking));
    if (!h->d_iter) {
        int st = h->alloc(&h->d_iter, 1);
        if (st) return st;
    }
    if (!h->pcg_exec || h->pcg_av != av || h->pcg_b != b || h->pcg_x != x || h->pcg_tol != tol ||
        h->pcg_maxit != maxit || h->pcg_grid != h->grid_apply || h->pcg_tmo != tmo) {
        if (h->pcg_exec) {
            cudaGraphExecDestroy(h->pcg_exec);
            h->pcg_exec = nullptr;
        }
        const cudaError_t e = pcg_capture(h, av, b, x, tol, maxit, tmo);
        if (e != cudaSuccess) {
            if (h->pcg_exec) cudaGraphExecDestroy(h->pcg_exec);
            h->pcg_exec = nullptr;
            return cuda_fail(e, "pcg_solve: graph capture");
        }
        h->pcg_av = av;
        h->pcg_b = b;
        h->pcg_x = x;
        h->pcg_tol = tol;
        h->pcg_maxit = maxit;
        h->pcg_grid = h->grid_apply;
        h->pcg_tmo = tmo;
    }
    CK(cudaGraphLaunch(h->pcg_exec, us));
    CK(cudaMemcpyAsync(h->h_sc, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, us));
    CK(cudaMemcpyAsync(h->h_counters + 8, h->d_iter, sizeof(int), cudaMemcpyDeviceToHost, us));
    CK(cudaMemcpyAsync(h->h_counters + 9, h->sp.counter + 3, sizeof(int), cudaMemcpyDeviceToHost, us));
    CK(cudaStreamSynchronize(us));
    const int it = h->h_counters[8];
    const double rel = h->h_sc->relres;
    h->tm.launches += 6 + int64_t(it) * 11;  // kernels: prologue 6, each pass 11 (two solves)
    if (h->h_counters[9]) {  // reported here, so the record is cleared
        CK(cudaMemset(h->sp.counter + 3, 0, sizeof(int)));
        return fail(IC_ERR_TIMEOUT, "triangular solve wait timed out");
    }
    if (iters) *iters = it;
    if (relres) *relres = rel;
    if (!(rel <= tol)) return fail(IC_ERR_NOCONV, "PCG reached maxit");
    return IC_OK;
}

int pcg_solve(ic_handle* h, const void* A_vals, const double* b, double* x, double tol, int maxit,
              int* iters, double* relres, void* stream) {
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    const int n = int(h->hp.n);
    if (n > 0 && (!A_vals || !b || !x)) return fail(IC_ERR_ARG, "NULL argument");
    if (!(tol >= 0.0) || maxit < 0) return fail(IC_ERR_ARG, "tol/maxit out of range");
    if (!h->factored) return fail(IC_ERR_STATE, "pcg_solve before a successful ic_numeric");
    if (n == 0) return IC_OK;
    DeviceGuard g(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double* av = static_cast<const double*>(A_vals);
    if (!h->timing) return pcg_solve_graph(h, av, b, x, tol, maxit, iters, relres, s);
    // with per-kernel timing (events around every application, which a graph's loop
    // body cannot hold): the loop on the host, one synchronisation per iteration
    const int parts = pcg_parts(n);
    int st = 0;
    int64_t& nl = h->tm.launches;
    CK(cudaMemsetAsync(h->sp.counter + 3, 0, sizeof(int), s));  // solve timeout record
    ++nl;
    CK(pcg_init(n, b, x, h->r, s));
    ++nl;
    CK(pcg_dot(b, b, n, h->partial, parts, s));
    ++nl;
    CK(pcg_finish(h->partial, parts, h->sc, 4, s));
    if ((st = ic_apply(h, h->r, h->z, s))) return st;
    CK(cudaMemcpyAsync(h->p, h->z, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    ++nl;
    CK(pcg_dot(h->r, h->z, n, h->partial, parts, s));
    ++nl;
    CK(pcg_finish(h->partial, parts, h->sc, 3, s));
    ++nl;
    CK(pcg_dot(h->r, h->r, n, h->partial, parts, s));
    ++nl;
    CK(pcg_finish(h->partial, parts, h->sc, 1, s));
    CK(cudaMemcpyAsync(h->h_sc, h->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double rel = h->h_sc->relres;
    int it = 0;
    while (rel > tol && it < maxit) {
        ++nl;
        CK(launch_spmv(h->sp, av, h->p, h->q, s));
        ++nl;
        CK(pcg_dot(h->p, h->q, n, h->partial, parts, s));
        ++nl;
        CK(pcg_finish(h->partial, parts, h->sc, 0, s));
        ++nl;
        CK(pcg_step_x_r(n, x, h->r, h->p, h->q, h->sc, h->partial, parts, s));
        ++nl;
        CK(pcg_finish(h->partial, parts, h->sc, 1, s));
        CK(cudaMemcpyAsync(&h->h_sc->relres, &h->sc->relres, sizeof(double), cudaMemcpyDeviceToHost, s));
        ++it;
        CK(cudaStreamSynchronize(s));
        rel = h->h_sc->relres;
        if (rel <= tol) break;
        if ((st = ic_apply(h, h->r, h->z, s))) return st;
        ++nl;
        CK(pcg_dot(h->r, h->z, n, h->partial, parts, s));
        ++nl;
        CK(pcg_finish(h->partial, parts, h->sc, 2, s));
        ++nl;
        CK(pcg_step_p(n, h->p, h->z, h->sc, s));
    }
    CK(cudaStreamSynchronize(s));
    {
        int ctr[4];
        CK(cudaMemcpy(ctr, h->sp.counter, sizeof(ctr), cudaMemcpyDeviceToHost));
        if (ctr[3]) {  // reported here, so the record is cleared
            CK(cudaMemset(h->sp.counter + 3, 0, sizeof(int)));
            return fail(IC_ERR_TIMEOUT, "triangular solve wait timed out");
        }
    }
    if (iters) *iters = it;
    if (relres) *relres = rel;
    if (!(rel <= tol)) return fail(IC_ERR_NOCONV, "PCG reached maxit");
    return IC_OK;
}

// One iteration of batched PCG (captured once per solve, replayed as a graph).
static cudaError_t batch_iteration(ic_handle* h, const double* av, double* x, double tol,
                                   unsigned long long tmo, cudaStream_t s) {
    BatchScalars& B = h->bs;
    const int n = int(h->hp.n), count = int(h->row_off.size()) - 1;
    cudaError_t e;
    if ((e = batch_bump(B, s)) != cudaSuccess) return e;
    if ((e = launch_spmv(h->sp, av, h->p, h->q, s)) != cudaSuccess) return e;
    if ((e = batch_dot(h->d_row_off, count, h->p, h->q, B.tmp, s)) != cudaSuccess) return e;
    if ((e = batch_scalars(B, count, 0, tol, s)) != cudaSuccess) return e;
    if ((e = batch_xr(n, h->d_sys, B.alpha, x, h->r, h->p, h->q, s)) != cudaSuccess) return e;
    if ((e = batch_dot(h->d_row_off, count, h->r, h->r, B.tmp, s)) != cudaSuccess) return e;
    if ((e = batch_scalars(B, count, 1, tol, s)) != cudaSuccess) return e;
    if ((e = launch_apply(h->sp, h->r, h->z, 0, tmo, h->grid_apply, s)) != cudaSuccess) return e;
    if ((e = batch_dot(h->d_row_off, count, h->r, h->z, B.tmp, s)) != cudaSuccess) return e;
    if ((e = batch_scalars(B, count, 2, tol, s)) != cudaSuccess) return e;
    return batch_p(n, h->d_sys, B.beta, B.active, h->p, h->z, s);
}

int pcg_solve_batch(ic_handle* h, const void* A_vals, const double* b, double* x, double tol, int maxit,
                    int* iters, double* relres, void* stream) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    const int n = int(h->hp.n), count = int(h->row_off.size()) - 1;
    if (iters)
        for (int s = 0; s < count; ++s) iters[s] = 0;
    if (relres)
        for (int s = 0; s < count; ++s) relres[s] = 0.0;
    if (n > 0 && (!A_vals || !b || !x)) return fail(IC_ERR_ARG, "NULL argument");
    if (!(tol >= 0.0) || maxit < 0) return fail(IC_ERR_ARG, "tol/maxit out of range");
    if (!h->factored) return fail(IC_ERR_STATE, "pcg_solve_batch before a successful ic_numeric");
    if (n == 0 || count < 1) return IC_OK;
    DeviceGuard g(h->device);
    cudaStream_t us = static_cast<cudaStream_t>(stream);
    if (!h->cap_stream) {
        CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->cap_ev[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->cap_ev[1], cudaEventDisableTiming));
    }
    cudaStream_t s = h->cap_stream;  // capturable even when the caller uses the legacy stream
    CK(cudaEventRecord(h->cap_ev[0], us));
    CK(cudaStreamWaitEvent(s, h->cap_ev[0], 0));
    const double* av = static_cast<const double*>(A_vals);
    BatchScalars& B = h->bs;
    const unsigned long long tmo = (unsigned long long)(h->opts.timeout_s * 1e9);
    CK(cudaMemsetAsync(h->sp.counter + 3, 0, sizeof(int), s));  // solve timeout record
    CK(pcg_init(n, b, x, h->r, s));
    CK(batch_dot(h->d_row_off, count, b, b, B.tmp, s));
    CK(batch_scalars(B, count, 4, tol, s));
    CK(launch_apply(h->sp, h->r, h->z, 0, tmo, h->grid_apply, s));
    CK(cudaMemcpyAsync(h->p, h->z, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(batch_dot(h->d_row_off, count, h->r, h->z, B.tmp, s));
    CK(batch_scalars(B, count, 3, tol, s));
    h->tm.launches += 8;
    // capture one iteration and replay it; convergence is read every few iterations
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const cudaError_t ce = batch_iteration(h, av, x, tol, tmo, s);
    const cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (ce != cudaSuccess || ee != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ce != cudaSuccess ? ce : ee, "pcg_solve_batch: graph capture");
    }
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
    int it = 0;
    cudaError_t le = cudaSuccess;
    while (it < maxit) {
        const int burst = std::min(4, maxit - it);
        for (int j = 0; j < burst && le == cudaSuccess; ++j) le = cudaGraphLaunch(exec, s);
        if (le == cudaSuccess) le = cudaMemcpyAsync(h->h_nactive, B.nactive, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (le == cudaSuccess) le = cudaStreamSynchronize(s);
        if (le != cudaSuccess) break;
        it += burst;
        if (*h->h_nactive == 0) break;
    }
    cudaGraphExecDestroy(exec);
    if (le != cudaSuccess) return cuda_fail(le, "pcg_solve_batch: graph launch");
    h->tm.launches += int64_t(it) * 13;
    std::vector<int> its(count);
    std::vector<double> rel(count);
    CK(cudaMemcpy(its.data(), B.iters, count * sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rel.data(), B.relres, count * sizeof(double), cudaMemcpyDeviceToHost));
    int abort_word = 0;
    CK(cudaMemcpy(&abort_word, h->sp.counter + 3, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaEventRecord(h->cap_ev[1], s));
    CK(cudaStreamWaitEvent(us, h->cap_ev[1], 0));
    if (iters) std::memcpy(iters, its.data(), count * sizeof(int));
    if (relres) std::memcpy(relres, rel.data(), count * sizeof(double));
    if (abort_word) {
        CK(cudaMemset(h->sp.counter + 3, 0, sizeof(int)));
        return fail(IC_ERR_TIMEOUT, "triangular solve wait timed out");
    }
    for (int s2 = 0; s2 < count; ++s2)
        if (!(rel[s2] <= tol)) return fail(IC_ERR_NOCONV, "system " + std::to_string(s2) + " reached maxit");
    return IC_OK;
}

int ic_get_factor(ic_handle* h, int64_t* rowptr, int32_t* colind, double* vals, int32_t* levels) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    const HostPlan& P = h->hp;
    const int64_t n = P.n;
    std::vector<double> u;
    if (vals) {
        if (!h->factored) return fail(IC_ERR_STATE, "no successful ic_numeric");
        DeviceGuard g(h->device);
        u.resize(P.nnz_u);
        if (h->opts.dtype == IC_F32) {
            // FP32 off-diagonal values, FP64 pivots
            std::vector<float> u32(P.nnz_u);
            std::vector<double> d(n);
            if (P.nnz_u)
                CK(cudaMemcpy(u32.data(), h->dp.uval, u32.size() * sizeof(float), cudaMemcpyDeviceToHost));
            if (n) CK(cudaMemcpy(d.data(), h->dp.udiag, d.size() * sizeof(double), cudaMemcpyDeviceToHost));
            for (int64_t e = 0; e < P.nnz_u; ++e) u[e] = double(u32[e]);
            for (int64_t i = 0; i < n; ++i) u[P.urp[i]] = d[i];
        } else if (P.nnz_u) {
            CK(cudaMemcpy(u.data(), h->dp.uval, u.size() * sizeof(double), cudaMemcpyDeviceToHost));
        }
    }
    // L row i = U column i: pivots p < i in ascending order, then the diagonal
    int64_t pos = 0;
    if (rowptr) rowptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t e = P.cptr[i]; e < P.cptr[i + 1]; ++e, ++pos) {
            const int2 pe = P.csc[e];
            if (colind) colind[pos] = pe.x;
            if (vals) vals[pos] = u[pe.y];
            if (levels) levels[pos] = P.ulev[pe.y];
        }
        if (colind) colind[pos] = int32_t(i);
        if (vals) vals[pos] = u[P.urp[i]];
        if (levels) levels[pos] = 0;
        ++pos;
        if (rowptr) rowptr[i + 1] = pos;
    }
    return IC_OK;
}

int ic_stats(const ic_handle* h, ic_stats_t* out) {
    if (!h || !out) return fail(IC_ERR_ARG, "NULL argument");
    const HostPlan& P = h->hp;
    std::memset(out, 0, sizeof(*out));
    out->n = P.n;
    out->nnz_a = P.nnz_a;
    out->nnz_l = P.nnz_u;
    out->nranges = int64_t(P.ranges.size()) - 1;
    out->nblocks = int64_t(P.bcol.size());
    out->ntasks = int64_t(P.task.size());
    for (int t = 0; t < 4; ++t) out->ntasks_type[t] = P.ntype[t];
    out->nitems = P.total_items;
    out->critical_path = P.critical_path;
    out->max_level = P.max_level;
    out->flops = P.flops;
    out->bytes = P.bytes;
    out->symbolic_s = h->symbolic_s;
    out->grid_ctas = h->grid_numeric;
    out->solve_depth[0] = P.fwd_depth;
    out->solve_depth[1] = P.bwd_depth;
    out->warps_per_cta = h->opts.warps_per_cta;
    out->rows_per_item = h->opts.rows_per_item;
    out->nsplit = P.nsplit;
    return IC_OK;
}

static int export_dag(const std::vector<int4>& task, const std::vector<int64_t>& pred_ptr,
                      const std::vector<int32_t>& pred, int32_t* type, int32_t* tk, int32_t* ti,
                      int32_t* tj, int64_t* pp, int32_t* pr, int64_t* ntasks, int64_t* npred) {
    if (ntasks) *ntasks = int64_t(task.size());
    if (npred) *npred = int64_t(pred.size());
    for (size_t t = 0; t < task.size(); ++t) {
        if (type) type[t] = task[t].x;
        if (tk) tk[t] = task[t].y;
        if (ti) ti[t] = task[t].z;
        if (tj) tj[t] = task[t].w;
    }
    if (pp) std::memcpy(pp, pred_ptr.data(), pred_ptr.size() * sizeof(int64_t));
    if (pr && !pred.empty()) std::memcpy(pr, pred.data(), pred.size() * sizeof(int32_t));
    return IC_OK;
}

int ic_get_tasks(const ic_handle* h, int32_t* type, int32_t* tk, int32_t* ti, int32_t* tj,
                 int64_t* pred_ptr, int32_t* pred, int64_t* ntasks, int64_t* npred) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    return export_dag(h->hp.task, h->hp.pred_ptr, h->hp.pred, type, tk, ti, tj, pred_ptr, pred,
                      ntasks, npred);
}

int ic_block_dag(int64_t nb, const int64_t* bptr, const int32_t* bcol, int32_t* type, int32_t* tk,
                 int32_t* ti, int32_t* tj, int64_t* pred_ptr, int32_t* pred, int64_t* ntasks,
                 int64_t* npred) {
    std::vector<int4> task;
    std::vector<int64_t> pp;
    std::vector<int32_t> pr;
    try {
        int st = block_dag(nb, bptr, bcol, task, pp, pr);
        if (st) return fail(st, "bad block pattern");
    } catch (const std::bad_alloc&) {
        return fail(IC_ERR_NOMEM, "host allocation failed");
    }
    return export_dag(task, pp, pr, type, tk, ti, tj, pred_ptr, pred, ntasks, npred);
}

int ic_get_task_targets(const ic_handle* h, int64_t t, int32_t* tgt5, int64_t* count) {
    if (!h || !count) return fail(IC_ERR_ARG, "NULL argument");
    const HostPlan& P = h->hp;
    if (t < 0 || t >= int64_t(P.task.size())) return fail(IC_ERR_ARG, "task out of range");
    const int32_t a = P.tgt_ptr[t], b = P.tgt_ptr[t + 1];
    *count = b - a;
    if (tgt5)
        for (int32_t e = a; e < b; ++e) {
            int32_t* o = tgt5 + 5 * (e - a);
            o[0] = P.tgt[e].x;
            o[1] = P.tgt[e].y;
            o[2] = P.tgt[e].z;
            o[3] = P.tgt[e].w;
            o[4] = P.tgt_end[e];
        }
    return IC_OK;
}

int ic_get_upper(const ic_handle* h, int64_t* urp, int32_t* ucol, int64_t* cptr, int32_t* cp,
                 int32_t* cpos) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    const HostPlan& P = h->hp;
    if (urp) std::memcpy(urp, P.urp.data(), P.urp.size() * sizeof(int64_t));
    if (ucol && P.nnz_u) std::memcpy(ucol, P.ucol.data(), P.ucol.size() * sizeof(int32_t));
    if (cptr)
        for (size_t i = 0; i < P.cptr.size(); ++i) cptr[i] = P.cptr[i];
    for (size_t e = 0; e < P.csc.size(); ++e) {
        if (cp) cp[e] = P.csc[e].x;
        if (cpos) cpos[e] = P.csc[e].y;
    }
    return IC_OK;
}

int ic_get_blocks(const ic_handle* h, int64_t* ranges, int64_t* bptr, int32_t* bcol) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    const HostPlan& P = h->hp;
    if (ranges)
        for (size_t b = 0; b < P.ranges.size(); ++b) ranges[b] = P.ranges[b];
    if (bptr) std::memcpy(bptr, P.bptr.data(), P.bptr.size() * sizeof(int64_t));
    if (bcol && !P.bcol.empty()) std::memcpy(bcol, P.bcol.data(), P.bcol.size() * sizeof(int32_t));
    return IC_OK;
}

int ic_get_solve_tasks(const ic_handle* h, int backward, int64_t* ntasks, int32_t* tasks, int32_t* counters,
                       int32_t* succ_ptr, int32_t* succ, int32_t* split, int32_t* order_ptr, int32_t* order,
                       int32_t* need) {
    if (!h || (backward != 0 && backward != 1)) return fail(IC_ERR_ARG, "NULL handle or bad direction");
    const HostPlan& P = h->hp;
    const SolveTasks& ST = backward ? P.bs : P.fs;
    const std::vector<int4>& T = ST.task;
    if (ntasks) *ntasks = int64_t(T.size());
    if (tasks)
        for (size_t t = 0; t < T.size(); ++t) {
            tasks[4 * t] = T[t].x;
            tasks[4 * t + 1] = T[t].y;
            tasks[4 * t + 2] = T[t].z;
            tasks[4 * t + 3] = T[t].w;
        }
    if (counters && !ST.indeg0.empty()) std::memcpy(counters, ST.indeg0.data(), ST.indeg0.size() * sizeof(int32_t));
    const std::vector<int32_t>& sp = ST.succ_ptr;
    const std::vector<int32_t>& sc = ST.succ;
    if (succ_ptr) std::memcpy(succ_ptr, sp.data(), sp.size() * sizeof(int32_t));
    if (succ && !sc.empty()) std::memcpy(succ, sc.data(), sc.size() * sizeof(int32_t));
    const std::vector<int32_t>& spl = backward ? P.sb_nint : P.sf_split;
    if (split && !spl.empty()) std::memcpy(split, spl.data(), spl.size() * sizeof(int32_t));
    const std::vector<int32_t>& op = backward ? P.lb_ptr : P.lf_ptr;
    const std::vector<int32_t>& od = backward ? P.lb_ord : P.lf_ord;
    if (order_ptr) std::memcpy(order_ptr, op.data(), op.size() * sizeof(int32_t));
    if (order && !od.empty()) std::memcpy(order, od.data(), od.size() * sizeof(int32_t));
    const std::vector<int32_t>& nd = backward ? P.lb_need : P.lf_need;
    if (need && !nd.empty()) std::memcpy(need, nd.data(), nd.size() * sizeof(int32_t));
    return IC_OK;
}

int ic_get_solve_entries(const ic_handle* h, int backward, int32_t* ptr, int32_t* j, int32_t* pos) {
    if (!h || (backward != 0 && backward != 1)) return fail(IC_ERR_ARG, "NULL handle or bad direction");
    const HostPlan& P = h->hp;
    const SolveLayout& L = backward ? P.xb : P.xf;
    auto put = [](int32_t* out, const std::vector<int32_t>& v) {
        if (out && !v.empty()) std::memcpy(out, v.data(), v.size() * sizeof(int32_t));
    };
    put(ptr, L.ptr);
    put(j, L.j);
    put(pos, L.pos);
    return IC_OK;
}

int ic_get_claim_order(const ic_handle* h, int32_t* task, int32_t* chunk) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    const std::vector<int2>& c = h->hp.claim;
    for (size_t q = 0; q < c.size(); ++q) {
        if (task) task[q] = c[q].x;
        if (chunk) chunk[q] = c[q].y;
    }
    return IC_OK;
}

int ic_get_split_layout(const ic_handle* h, int32_t* flag_off, int32_t* soff, int64_t* nsoff,
                        int64_t* nshadow) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    const HostPlan& P = h->hp;
    if (nsoff) *nsoff = int64_t(P.soff.size());
    if (nshadow) *nshadow = P.nshadow;
    if (flag_off && !P.flag_off.empty())
        std::memcpy(flag_off, P.flag_off.data(), P.flag_off.size() * sizeof(int32_t));
    if (soff && !P.soff.empty()) std::memcpy(soff, P.soff.data(), P.soff.size() * sizeof(int32_t));
    return IC_OK;
}

int ic_set_timing(ic_handle* h, int on) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    if (h->device < 0) return fail(IC_ERR_STATE, "host-only handle");
    DeviceGuard g(h->device);
    if (on && !h->ev[0])
        for (cudaEvent_t& e : h->ev) CK(cudaEventCreate(&e));
    h->timing = on != 0;
    return IC_OK;
}

int ic_reset_timing(ic_handle* h) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    if (h->timing) {
        int st = fold_apply_time(h);
        if (st) return st;
    }
    h->tm = ic_timing_t{};
    return IC_OK;
}

int ic_get_timing(const ic_handle* hc, ic_timing_t* out) {
    if (!hc || !out) return fail(IC_ERR_ARG, "NULL argument");
    ic_handle* h = const_cast<ic_handle*>(hc);
    if (h->timing) {
        DeviceGuard g(h->device);
        int st = fold_apply_time(h);
        if (st) return st;
    }
    *out = h->tm;
    return IC_OK;
}

int ic_set_trace(ic_handle* h, int on) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    if (h->device < 0) return fail(IC_ERR_STATE, "host-only handle");
    DeviceGuard g(h->device);
    if (on && !h->dp.trace) {
        unsigned long long* t = nullptr;
        int st = h->alloc(&t, 4 * size_t(h->hp.total_items > 0 ? h->hp.total_items : 1));
        if (st) return st;
        CK(cudaMemset(t, 0, 4 * size_t(h->hp.total_items > 0 ? h->hp.total_items : 1) * 8));
        h->trace_buf = t;
        const size_t nt = h->hp.fs.task.size() + h->hp.bs.task.size();
        st = h->alloc(&t, 4 * (nt > 0 ? nt : 1));
        if (st) return st;
        CK(cudaMemset(t, 0, 4 * (nt > 0 ? nt : 1) * 8));
        h->solve_trace_buf = t;
    }
    h->dp.trace = on ? h->trace_buf : nullptr;
    h->sp.trace = on ? h->solve_trace_buf : nullptr;
    return IC_OK;
}

int ic_get_solve_trace(const ic_handle* h, int backward, uint64_t* out) {
    if (!h || !out || (backward != 0 && backward != 1)) return fail(IC_ERR_ARG, "bad argument");
    if (!h->solve_trace_buf) return fail(IC_ERR_STATE, "tracing was never enabled");
    DeviceGuard g(h->device);
    const size_t off = backward ? h->hp.fs.task.size() : 0;
    const size_t cnt = backward ? h->hp.bs.task.size() : h->hp.fs.task.size();
    CK(cudaMemcpy(out, h->solve_trace_buf + 4 * off, 4 * cnt * 8, cudaMemcpyDeviceToHost));
    return IC_OK;
}

int ic_get_trace(const ic_handle* h, uint64_t* out) {
    if (!h || !out) return fail(IC_ERR_ARG, "NULL argument");
    if (!h->trace_buf) return fail(IC_ERR_STATE, "tracing was never enabled");
    DeviceGuard g(h->device);
    CK(cudaMemcpy(out, h->trace_buf, 4 * size_t(h->hp.total_items) * 8, cudaMemcpyDeviceToHost));
    return IC_OK;
}

int ic_fma_peak(int dtype, double* gflops, void* stream) {
    if (!gflops || (dtype != IC_F64 && dtype != IC_F32)) return fail(IC_ERR_ARG, "bad argument");
    *gflops = 0.0;
    CK(measure_fma_peak(dtype, gflops, static_cast<cudaStream_t>(stream)));
    return IC_OK;
}

int ic_test_hold_solve_task(ic_handle* h, int backward, int64_t t, int extra) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    if (h->device < 0) return fail(IC_ERR_STATE, "host-only handle");
    if (h->opts.solve_mode != 0) return fail(IC_ERR_STATE, "the handle's solves are not block-DAG solves");
    const SolveTasks& ST = backward ? h->hp.bs : h->hp.fs;
    if (t < 0 || t >= int64_t(ST.task.size()) || extra < 0) return fail(IC_ERR_ARG, "task out of range");
    DeviceGuard g(h->device);
    const int v = ST.indeg0[t] + extra;
    const size_t off = (backward ? h->hp.fs.task.size() : 0) + size_t(t);
    CK(cudaMemcpy(const_cast<int*>(h->sp.dag_indeg0) + off, &v, sizeof(int), cudaMemcpyHostToDevice));
    return IC_OK;
}

int ic_test_hold_task(ic_handle* h, int64_t t, int extra) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    if (h->device < 0) return fail(IC_ERR_STATE, "host-only handle");
    if (t < 0 || t >= int64_t(h->hp.task.size()) || extra < 0) return fail(IC_ERR_ARG, "task out of range");
    DeviceGuard g(h->device);
    const int v = h->hp.indeg0[t] + extra;
    CK(cudaMemcpy(const_cast<int*>(h->dp.indeg0) + t, &v, sizeof(int), cudaMemcpyHostToDevice));
    return IC_OK;
}

int ic_autotune(int64_t count, const ic_csr_pattern* A, int k, const int32_t* const* perms,
                const int64_t* const* ranges, const int64_t* nranges, const void* values,
                const ic_opts* base, int reps, ic_opts* best, double* times, void* stream) {
    if (!best || !values || reps < 1) return fail(IC_ERR_ARG, "NULL best/values or reps < 1");
    ic_opts cur = normalise(base, count);
    cur.host_only = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // median numeric time of a candidate (rebuilds the plan), or < 0 on error
    auto time_numeric = [&](const ic_opts& o, ic_handle** keep) -> double {
        ic_handle* h = nullptr;
        if (ic_symbolic_batch(count, A, k, perms, ranges, nranges, &o, &h)) return -1.0;
        if (ic_set_timing(h, 1)) { ic_destroy(h); return -1.0; }
        std::vector<double> t;
        for (int r = 0; r <= reps; ++r) {
            if (ic_numeric(h, values, s, nullptr)) { ic_destroy(h); return -1.0; }
            if (r > 0) t.push_back(h->tm.prepare_ms + h->tm.numeric_ms);  // first run warms up
        }
        std::sort(t.begin(), t.end());
        if (keep) *keep = h; else ic_destroy(h);
        return t[t.size() / 2];
    };
    double best_num = -1.0;
    {
        const int cand[] = {1024, 2048, 4096, 8192};
        ic_opts pick = cur;
        for (int br : cand) {
            ic_opts o = cur;
            o.block_rows = br;
            const double t = time_numeric(o, nullptr);
            if (t >= 0 && (best_num < 0 || t < best_num)) { best_num = t; pick = o; }
        }
        if (best_num < 0)
            return fail(IC_ERR_ARG, "autotune: no candidate factored (" + std::string(ic_last_error()) + ")");
        cur = pick;
    }
    for (int w : {8, 16, 32}) {
        if (w == cur.warps_per_cta) continue;
        ic_opts o = cur;
        o.warps_per_cta = w;
        const double t = time_numeric(o, nullptr);
        if (t >= 0 && t < best_num) { best_num = t; cur = o; }
    }
    for (int rpi : {16, 32, 64}) {
        if (rpi == cur.rows_per_item) continue;
        ic_opts o = cur;
        o.rows_per_item = rpi;
        const double t = time_numeric(o, nullptr);
        if (t >= 0 && t < best_num) { best_num = t; cur = o; }
    }
    // solve launch shape on the chosen plan: lanes per row and CTAs per SM
    ic_handle* h = nullptr;
    if (time_numeric(cur, &h) < 0) return fail(IC_ERR_ARG, "autotune: chosen plan failed");
    double best_apply = -1.0;
    {
        DeviceGuard g(h->device);
        int sms = 0, dev = 0, bpsm = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const bool dag = h->sp.solve_mode == 0;
        double* r = nullptr;
        double* z = nullptr;
        CK(cudaMalloc(&r, 2 * size_t(h->hp.n > 0 ? h->hp.n : 1) * sizeof(double)));
        z = r + h->hp.n;
        CK(cudaMemsetAsync(r, 0, 2 * size_t(h->hp.n) * sizeof(double), s));
        std::vector<double> ones(h->hp.n, 1.0);
        CK(cudaMemcpyAsync(r, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        for (int lanes : {8, 16, 32}) {
            if (!dag && lanes == 8) continue;
            if (dag) CK(dag_blocks_per_sm(lanes, h->sp.dtype, h->sp.max_range_rows, &bpsm));
            else CK(apply_blocks_per_sm(&bpsm));
            for (int cps : {2, 3, 4, 6}) {
                if (cps > bpsm) continue;
                h->sp.lanes_per_row = lanes;
                h->grid_apply = sms * cps;
                std::vector<float> t;
                for (int q = 0; q <= reps; ++q) {
                    CK(cudaEventRecord(e0, s));
                    CK(launch_apply(h->sp, r, z, 0, (unsigned long long)(h->opts.timeout_s * 1e9),
                                    h->grid_apply, s));
                    CK(cudaEventRecord(e1, s));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    if (q > 0) t.push_back(ms);
                }
                std::sort(t.begin(), t.end());
                const double med = t[t.size() / 2];
                if (best_apply < 0 || med < best_apply) {
                    best_apply = med;
                    cur.solve_lanes = lanes;
                    cur.solve_ctas_per_sm = cps;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(r);
    }
    ic_destroy(h);
    *best = cur;
    if (times) {
        times[0] = best_num;
        times[1] = best_apply;
    }
    return IC_OK;
}

int ic_shift_features(const ic_handle* h, const void* A_vals, double nu, double* out, void* stream) {
    if (!h || !out || (!A_vals && h->hp.n > 0)) return fail(IC_ERR_ARG, "NULL argument");
    if (h->device < 0) return fail(IC_ERR_STATE, "host-only handle");
    if (h->hp.n == 0) return fail(IC_ERR_ARG, "empty matrix");
    DeviceGuard g(h->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    CK(cudaMallocAsync(&scratch, features_scratch_bytes() + 16 * sizeof(double), s));
    double* dout = reinterpret_cast<double*>(static_cast<char*>(scratch) + features_scratch_bytes());
    cudaError_t e = launch_features(int(h->hp.n), h->sp.arp, h->sp.acol, static_cast<const double*>(A_vals),
                                    h->hp.k, nu, scratch, dout, s);
    double tmp[9] = {0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, dout, 9 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "ic_shift_features");
    if (tmp[8] != 0.0) return fail(IC_ERR_ARG, "a diagonal entry is missing or not positive");
    for (int q = 0; q < 8; ++q) out[q] = tmp[q];
    return IC_OK;
}

int ic_numeric_shifted(ic_handle* h, const void* A_vals, double alpha_first, double alpha0, int max_tries,
                       double* alpha_used, int* attempts, void* stream) {
    if (!h) return fail(IC_ERR_ARG, "NULL handle");
    if (max_tries < 1 || !(alpha_first >= 0.0) || !(alpha0 > 0.0)) return fail(IC_ERR_ARG, "bad retry parameters");
    const double keep = h->opts.shift_alpha;
    double a = alpha_first;
    int st = IC_ERR_BREAKDOWN;
    int t = 0;
    while (t < max_tries) {
        h->opts.shift_alpha = a;
        ++t;
        st = ic_numeric(h, A_vals, stream, nullptr);
        if (st != IC_ERR_BREAKDOWN) break;
        a = a > 0.0 ? 2.0 * a : alpha0;
    }
    h->opts.shift_alpha = keep;
    if (attempts) *attempts = t;
    if (st == IC_OK && alpha_used) *alpha_used = a;  // the loop stops on the first success
    if (st == IC_ERR_BREAKDOWN) return fail(IC_ERR_BREAKDOWN, "every shift attempt broke down");
    return st;
}

}  // extern "C"

struct ic_mlp {
    int device = -1;
    int step = 0;
    MlpDev d{};
    float* X1 = nullptr;    // device scratch for one feature vector and its output
    float* hbuf = nullptr;  // pinned loss
    std::vector<void*> allocs;
    ~ic_mlp() {
        for (void* p : allocs) cudaFree(p);
        if (hbuf) cudaFreeHost(hbuf);
    }
    int alloc(float** out, size_t count) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, count * sizeof(float));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        allocs.push_back(p);
        *out = static_cast<float*>(p);
        return IC_OK;
    }
};

extern "C" {

int ic_mlp_n_params(void) { return kMlpParams; }

int ic_mlp_create(const float* params, ic_mlp** out) {
    if (!out) return fail(IC_ERR_ARG, "NULL argument");
    *out = nullptr;
    ic_mlp* m = new ic_mlp();
    int st = IC_OK;
    CK(cudaGetDevice(&m->device));
    MlpDev& D = m->d;
    float** bufs[] = {&D.theta, &D.m, &D.v, &D.grad};
    for (float** b : bufs)
        if (!st) st = m->alloc(b, kMlpParams);
    if (!st) st = m->alloc(&D.mean, kMlpFeatures);
    if (!st) st = m->alloc(&D.rstd, kMlpFeatures);
    if (!st) st = m->alloc(&D.part, size_t(kMlpMaxBlocks) * kMlpParams);
    if (!st) st = m->alloc(&D.loss_part, kMlpMaxBlocks);
    if (!st) st = m->alloc(&D.loss, 1);
    if (!st) st = m->alloc(&m->X1, 16);
    if (st) {
        delete m;
        return st;
    }
    cudaError_t e = cudaMallocHost(&m->hbuf, 16 * sizeof(float));
    for (float* b : {D.theta, D.m, D.v, D.grad})
        if (e == cudaSuccess) e = cudaMemset(b, 0, kMlpParams * sizeof(float));
    if (e == cudaSuccess && params)
        e = cudaMemcpy(D.theta, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
    const float zero[kMlpFeatures] = {0}, one[kMlpFeatures] = {1, 1, 1, 1, 1, 1, 1, 1};
    if (e == cudaSuccess) e = cudaMemcpy(D.mean, zero, sizeof(zero), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(D.rstd, one, sizeof(one), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "ic_mlp_create");
    }
    *out = m;
    return IC_OK;
}

int ic_mlp_set_params(ic_mlp* m, const float* params) {
    if (!m || !params) return fail(IC_ERR_ARG, "NULL argument");
    DeviceGuard g(m->device);
    CK(cudaMemcpy(m->d.theta, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemset(m->d.m, 0, kMlpParams * sizeof(float)));
    CK(cudaMemset(m->d.v, 0, kMlpParams * sizeof(float)));
    m->step = 0;
    return IC_OK;
}

int ic_mlp_get_params(const ic_mlp* m, float* params) {
    if (!m || !params) return fail(IC_ERR_ARG, "NULL argument");
    DeviceGuard g(m->device);
    CK(cudaMemcpy(params, m->d.theta, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost));
    return IC_OK;
}

int ic_mlp_set_scaling(ic_mlp* m, const float* mean, const float* std) {
    if (!m || !mean || !std) return fail(IC_ERR_ARG, "NULL argument");
    float r[kMlpFeatures];
    for (int f = 0; f < kMlpFeatures; ++f) {
        if (!(std[f] > 0.0f)) return fail(IC_ERR_ARG, "std must be positive");
        r[f] = 1.0f / std[f];
    }
    DeviceGuard g(m->device);
    CK(cudaMemcpy(m->d.mean, mean, sizeof(r), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->d.rstd, r, sizeof(r), cudaMemcpyHostToDevice));
    return IC_OK;
}

int ic_mlp_get_scaling(const ic_mlp* m, float* mean, float* std) {
    if (!m || !mean || !std) return fail(IC_ERR_ARG, "NULL argument");
    DeviceGuard g(m->device);
    float r[kMlpFeatures];
    CK(cudaMemcpy(mean, m->d.mean, sizeof(r), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(r, m->d.rstd, sizeof(r), cudaMemcpyDeviceToHost));
    for (int f = 0; f < kMlpFeatures; ++f) std[f] = 1.0f / r[f];
    return IC_OK;
}

int ic_mlp_forward(ic_mlp* m, const float* X, int64_t n, float* y, void* stream) {
    if (!m || n < 0 || (n > 0 && (!X || !y))) return fail(IC_ERR_ARG, "bad argument");
    DeviceGuard g(m->device);
    CK(launch_mlp_forward(m->d, X, n, y, static_cast<cudaStream_t>(stream)));
    return IC_OK;
}

int ic_mlp_gradient(ic_mlp* m, const float* X, const float* t, int64_t n, float* grad, float* loss, void* stream) {
    if (!m || n < 1 || !X || !t) return fail(IC_ERR_ARG, "bad argument");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(launch_mlp_grad(m->d, X, t, n, s));
    if (grad) CK(cudaMemcpyAsync(grad, m->d.grad, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(m->hbuf, m->d.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (loss) *loss = m->hbuf[0];
    return IC_OK;
}

int ic_mlp_train_step(ic_mlp* m, const float* X, const float* t, int64_t n, float lr, float* loss, void* stream) {
    if (!m || n < 1 || !X || !t || !(lr > 0.0f)) return fail(IC_ERR_ARG, "bad argument");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(launch_mlp_grad(m->d, X, t, n, s));
    CK(launch_mlp_adam(m->d, lr, ++m->step, s));
    if (loss) {
        CK(cudaMemcpyAsync(m->hbuf, m->d.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *loss = m->hbuf[0];
    }
    return IC_OK;
}

int ic_mlp_predict_shift(ic_mlp* m, const double* features, double* alpha, void* stream) {
    if (!m || !features || !alpha) return fail(IC_ERR_ARG, "NULL argument");
    DeviceGuard g(m->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int f = 0; f < kMlpFeatures; ++f) m->hbuf[f] = float(features[f]);
    CK(cudaMemcpyAsync(m->X1, m->hbuf, kMlpFeatures * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(launch_mlp_forward(m->d, m->X1, 1, m->X1 + kMlpFeatures, s));
    CK(cudaMemcpyAsync(m->hbuf + kMlpFeatures, m->X1 + kMlpFeatures, sizeof(float), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *alpha = std::pow(10.0, double(m->hbuf[kMlpFeatures]));
    return IC_OK;
}

void ic_mlp_destroy(ic_mlp* m) {
    if (!m) return;
    DeviceGuard g(m->device);
    delete m;
}

void ic_destroy(ic_handle* h) {
    if (!h) return;
    if (h->device >= 0) {
        DeviceGuard g(h->device);
        delete h;
    } else {
        delete h;
    }
}

}  // extern "C"
