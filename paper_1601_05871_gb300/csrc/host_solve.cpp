// Host side of the block-DAG triangular solves used by ic_apply.
//
// The factor's 2D block structure (Section 3.2) also organises the solves with L and
// L^T: every block row (a range of rows) is a unit of work.  For the forward solve
// L y = r, a row i of range k needs y_p for the entries U_pi of column i of U; the
// entries with p in an earlier range are "external", the others "internal".  Two task
// kinds per range:
//   E(k, c)  sums the external entries of a chunk of k's rows (many CTAs in parallel)
//            once every range k depends on has finished;
//   L(k)     one CTA solves k's rows with the internal entries, rows taken in local
//            dependence-level order, the range's results held in shared memory.
// The backward solve L^T z = y is the mirror image (external = entries of row i in a
// later range).  Nested-dissection leaves have no external entries in the forward
// solve, so they start at once; separators wait for their subdomains.  Tasks are
// claimed in a fixed order: ascending start time of an as-soon-as-possible schedule
// under a simple cost model, which is a topological order of the task DAG.
#include <omp.h>

#include <algorithm>
#include <numeric>

#include "ick_internal.h"

namespace ick {

namespace {

// Cost model of the claim order (microseconds); only the order depends on it.
constexpr double kTaskStartUs = 2.0;    // claim, dependence check, release
constexpr double kLevelUs = 0.25;       // one local dependence level in shared memory
constexpr double kFmaUs = 1.0e-3;       // one FP64 multiply-add of a CTA sharing its SM
constexpr int64_t kChunkEntries = 8192; // external entries per E task, at most
constexpr int kChunkRows = 512;         // rows per E task, at most

// Rows of one range sorted by local level, each level's run padded with -1 to a
// multiple of kClaimPad; appended to out.  need receives, per position, the number of
// the range's rows in lower levels: once that many rows of the range are complete,
// the position's row may run (no row completes before all lower levels have).
void padded_local_order(int32_t s, int32_t e, const std::vector<int32_t>& lev, bool descending,
                        std::vector<int32_t>& out, std::vector<int32_t>& need) {
    const int32_t m = e - s;
    int32_t maxd = 0;
    for (int32_t q = 0; q < m; ++q) maxd = std::max(maxd, lev[s + q]);
    std::vector<int32_t> cnt(size_t(maxd) + 2, 0);
    for (int32_t q = 0; q < m; ++q) ++cnt[lev[s + q] + 1];
    for (int32_t d = 0; d <= maxd; ++d) cnt[d + 1] += cnt[d];
    std::vector<int32_t> ord(m);
    for (int32_t q = 0; q < m; ++q) {
        const int32_t i = descending ? e - 1 - q : s + q;
        ord[cnt[lev[i]]++] = i;
    }
    int32_t before = 0;  // rows of the lower levels
    for (int32_t q = 0; q < m; ++q) {
        out.push_back(ord[q]);
        need.push_back(before);
        if (q + 1 == m || lev[ord[q + 1]] != lev[ord[q]]) {
            while (out.size() % kClaimPad) {
                out.push_back(-1);
                need.push_back(before);
            }
            before = q + 1;
        }
    }
}

// The internal entries of every row, contiguous: entries [ptr[i], ptr[i+1]) with
// src(i, t) = (source row, value position) of the t-th one.
template <class Count, class Src>
void internal_layout(const HostPlan& P, Count count_of_row, Src src_pos, SolveLayout& L) {
    const int64_t n = P.n;
    L.ptr.assign(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) L.ptr[i + 1] = L.ptr[i] + count_of_row(int32_t(i));
    L.j.assign(size_t(L.ptr[n]), 0);
    L.pos.assign(size_t(L.ptr[n]), 0);
    const int32_t nb = int32_t(P.ranges.size()) - 1;
    for (int32_t k = 0; k < nb; ++k)
        for (int32_t i = P.ranges[k]; i < P.ranges[k + 1]; ++i)
            for (int32_t t = 0, q = L.ptr[i]; q < L.ptr[i + 1]; ++t, ++q) {
                const int2 sp = src_pos(i, t);
                L.j[q] = sp.x - P.ranges[k];
                L.pos[q] = sp.y;
            }
}

}  // namespace

void build_solve_dag(HostPlan& P, int nthr) {
    const int64_t n = P.n;
    const int32_t nb = int32_t(P.ranges.size()) - 1;
    P.sf_split.assign(n, 0);
    P.sb_nint.assign(n, 0);
    std::vector<int32_t> lf(n, 0), lb(n, 0);
    std::vector<int64_t> int_f(nb, 0), int_b(nb, 0);
    std::vector<int32_t> dep_f(nb, 0), dep_b(nb, 0);
    P.max_range_rows = 0;
    for (int32_t k = 0; k < nb; ++k)
        P.max_range_rows = std::max(P.max_range_rows, P.ranges[k + 1] - P.ranges[k]);

    // split points and local levels, range by range (ranges are independent here)
#pragma omp parallel for num_threads(nthr) schedule(dynamic, 4)
    for (int32_t k = 0; k < nb; ++k) {
        const int32_t s = P.ranges[k], e = P.ranges[k + 1];
        int64_t fi = 0, bi = 0;
        int32_t df = 0, db = 0;
        for (int32_t i = s; i < e; ++i) {
            // column list of i: pivot rows ascending, so the internal ones are a suffix
            int32_t a = P.cptr[i];
            const int32_t b = P.cptr[i + 1];
            while (a < b && P.csc[a].x < s) ++a;
            P.sf_split[i] = a;
            int32_t d = 0;
            for (int32_t q = a; q < b; ++q) d = std::max(d, lf[P.csc[q].x] + 1);
            lf[i] = d;
            df = std::max(df, d);
            fi += b - a;
        }
        for (int32_t i = e - 1; i >= s; --i) {
            // row i: columns ascending after the diagonal, the internal ones a prefix
            const int64_t a = P.urp[i] + 1, b = P.urp[i + 1];
            int64_t q = a;
            int32_t d = 0;
            while (q < b && P.ucol[q] < e) {
                d = std::max(d, lb[P.ucol[q]] + 1);
                ++q;
            }
            P.sb_nint[i] = int32_t(q - a);
            lb[i] = d;
            db = std::max(db, d);
            bi += q - a;
        }
        int_f[k] = fi;
        int_b[k] = bi;
        dep_f[k] = df + 1;
        dep_b[k] = db + 1;
    }

    P.lf_ptr.assign(nb + 1, 0);
    P.lb_ptr.assign(nb + 1, 0);
    P.lf_ord.clear();
    P.lb_ord.clear();
    P.lf_need.clear();
    P.lb_need.clear();
    for (int32_t k = 0; k < nb; ++k) {
        padded_local_order(P.ranges[k], P.ranges[k + 1], lf, false, P.lf_ord, P.lf_need);
        P.lf_ptr[k + 1] = int32_t(P.lf_ord.size());
        padded_local_order(P.ranges[k], P.ranges[k + 1], lb, true, P.lb_ord, P.lb_need);
        P.lb_ptr[k + 1] = int32_t(P.lb_ord.size());
    }

    // contiguous layouts of the internal entries (forward: column list of i from
    // sf_split; backward: row i after the diagonal, sb_nint entries)
    internal_layout(
        P, [&](int32_t i) { return P.cptr[i + 1] - P.sf_split[i]; },
        [&](int32_t i, int32_t t) { const int2 c = P.csc[P.sf_split[i] + t]; return make_int2(c.x, c.y); }, P.xf);
    internal_layout(
        P, [&](int32_t i) { return P.sb_nint[i]; },
        [&](int32_t i, int32_t t) {
            const int64_t q = P.urp[i] + 1 + t;
            return make_int2(P.ucol[q], int32_t(q));
        },
        P.xb);

    // range dependences from the block pattern (upper, diagonal block first): block
    // (k, j), j > k, means j needs k in the forward solve and k needs j backward
    std::vector<int32_t> bcnt(nb + 1, 0);
    P.fsucc_ptr.assign(nb + 1, 0);
    P.fsucc.clear();
    for (int32_t k = 0; k < nb; ++k) {
        for (int64_t q = P.bptr[k]; q < P.bptr[k + 1]; ++q) {
            const int32_t j = P.bcol[q];
            if (j == k) continue;
            P.fsucc.push_back(j);
            ++bcnt[j + 1];
        }
        P.fsucc_ptr[k + 1] = int32_t(P.fsucc.size());
    }
    P.bsucc_ptr.assign(nb + 1, 0);
    for (int32_t j = 0; j < nb; ++j) P.bsucc_ptr[j + 1] = P.bsucc_ptr[j] + bcnt[j + 1];
    P.bsucc.assign(P.fsucc.size(), 0);
    {
        std::vector<int32_t> fill(P.bsucc_ptr.begin(), P.bsucc_ptr.end() - 1);
        for (int32_t k = 0; k < nb; ++k)
            for (int32_t q = P.fsucc_ptr[k]; q < P.fsucc_ptr[k + 1]; ++q)
                P.bsucc[fill[P.fsucc[q]]++] = k;  // ascending k within each list
    }

    // tasks, counters and the as-soon-as-possible claim order, one direction at a time
    P.dag_cnt0.assign(4 * size_t(nb), 0);
    auto build = [&](bool fwd, std::vector<int4>& out) {
        struct T { double start, cost; int4 t; };
        std::vector<T> tasks;
        std::vector<double> done(nb, 0.0);  // finish time of L(k)
        std::vector<int32_t> order(nb);
        std::iota(order.begin(), order.end(), 0);
        if (!fwd) std::reverse(order.begin(), order.end());
        int32_t* pend = P.dag_cnt0.data() + (fwd ? 0 : 2 * size_t(nb));
        int32_t* epend = pend + nb;
        for (int32_t k : order) {
            const int32_t s = P.ranges[k], e = P.ranges[k + 1];
            // ranges k depends on: all finished earlier in this direction's range order
            double ready = 0.0;
            if (fwd) {
                for (int32_t q = P.bsucc_ptr[k]; q < P.bsucc_ptr[k + 1]; ++q)
                    ready = std::max(ready, done[P.bsucc[q]]);
                pend[k] = P.bsucc_ptr[k + 1] - P.bsucc_ptr[k];
            } else {
                for (int32_t q = P.fsucc_ptr[k]; q < P.fsucc_ptr[k + 1]; ++q)
                    ready = std::max(ready, done[P.fsucc[q]]);
                pend[k] = P.fsucc_ptr[k + 1] - P.fsucc_ptr[k];
            }
            // external entries of each row, cut into chunks
            double lstart = ready;
            int32_t chunks = 0;
            if (pend[k] > 0) {
                int32_t lo = s;
                int64_t acc = 0;
                for (int32_t i = s; i < e; ++i) {
                    const int64_t ext = fwd ? int64_t(P.sf_split[i] - P.cptr[i])
                                            : (P.urp[i + 1] - P.urp[i] - 1) - P.sb_nint[i];
                    acc += ext;
                    if (i + 1 == e || acc >= kChunkEntries || i + 1 - lo >= kChunkRows) {
                        if (acc > 0) {
                            const double c = kTaskStartUs + kFmaUs * double(acc);
                            tasks.push_back({ready, c, make_int4(0, k, lo, i + 1)});
                            lstart = std::max(lstart, ready + c);
                            ++chunks;
                        }
                        lo = i + 1;
                        acc = 0;
                    }
                }
            }
            epend[k] = chunks;
            const double lc = kTaskStartUs + kLevelUs * double(fwd ? dep_f[k] : dep_b[k]) +
                              kFmaUs * double(fwd ? int_f[k] : int_b[k]);
            tasks.push_back({lstart, lc, make_int4(1, k, s, e)});
            done[k] = lstart + lc;
        }
        // ascending start; at equal start, the longer task first; then generation order
        std::vector<size_t> idx(tasks.size());
        std::iota(idx.begin(), idx.end(), size_t(0));
        std::stable_sort(idx.begin(), idx.end(), [&](size_t a, size_t b) {
            if (tasks[a].start != tasks[b].start) return tasks[a].start < tasks[b].start;
            return tasks[a].cost > tasks[b].cost;
        });
        out.resize(tasks.size());
        for (size_t q = 0; q < idx.size(); ++q) out[q] = tasks[idx[q]].t;
    };
    build(true, P.ftask);
    build(false, P.btask);
}

}  // namespace ick
