// Host side of the block-DAG triangular solves used by ic_apply.
//
// The factor's 2D block structure (Section 3.2) also organises the solves with L and
// L^T: every block row (a range of rows) is a unit of work.  For the forward solve
// L y = r, a row i of range k needs y_p for the entries U_pi of column i of U; the
// entries with p in an earlier range are "external", the others "internal".  A
// range's rows are taken in local dependence-level order and cut into parts of a few
// levels; two task kinds per part:
//   E  sums the external entries of a chunk of the part's rows (many CTAs in
//      parallel) once the parts holding their source rows have finished;
//   L  one CTA solves the part's rows with the internal entries, after the range's
//      previous part, the range's results held in shared memory.
// So a separator's first levels run while its subdomains are still finishing their
// last ones.  The backward solve L^T z = y is the mirror image (external = entries of
// row i in a later range).  Nested-dissection leaves have no external entries in the
// forward solve: each is one L task and they start at once.  Tasks are claimed in a
// fixed order: the order in which a list schedule of the task DAG on the solve grid's
// CTAs, under a simple cost model, starts them (a free CTA takes the ready task with
// the longest remaining path), which is a topological order of the task DAG.
#include <omp.h>

#include <algorithm>
#include <numeric>
#include <queue>

#include "ick_internal.h"

namespace ick {

namespace {

// Cost model of the claim order (microseconds); only the order depends on it.
constexpr double kTaskStartUs = 2.0;    // claim, dependence check, release
constexpr double kLevelUs = 1.0;        // one local dependence level in shared memory (measured)
constexpr double kFmaUs = 2.0e-3;       // one external FP64 multiply-add of an E task (measured)
constexpr int64_t kChunkEntries = 8192; // external entries per E task, at most
constexpr int kChunkRows = 512;         // order positions per E task, at most
constexpr int kPartLevels = 24;         // local levels per L task of a range with external entries

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

void build_solve_dag(HostPlan& P, int nthr, int ctas) {
    const int64_t n = P.n;
    const int32_t nb = int32_t(P.ranges.size()) - 1;
    P.sf_split.assign(n, 0);
    P.sb_nint.assign(n, 0);
    std::vector<int32_t> lf(n, 0), lb(n, 0);
    P.max_range_rows = 0;
    for (int32_t k = 0; k < nb; ++k)
        P.max_range_rows = std::max(P.max_range_rows, P.ranges[k + 1] - P.ranges[k]);

    // split points and local levels, range by range (ranges are independent here)
#pragma omp parallel for num_threads(nthr) schedule(dynamic, 4)
    for (int32_t k = 0; k < nb; ++k) {
        const int32_t s = P.ranges[k], e = P.ranges[k + 1];
        for (int32_t i = s; i < e; ++i) {
            // column list of i: pivot rows ascending, so the internal ones are a suffix
            int32_t a = P.cptr[i];
            const int32_t b = P.cptr[i + 1];
            while (a < b && P.csc[a].x < s) ++a;
            P.sf_split[i] = a;
            int32_t d = 0;
            for (int32_t q = a; q < b; ++q) d = std::max(d, lf[P.csc[q].x] + 1);
            lf[i] = d;
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
        }
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

    // tasks, their dependences and the claim order, one direction at a time.  A range
    // whose rows have entries outside it is cut into parts of kPartLevels local levels
    // (one L task each, after the previous part); each part's external sums form E
    // tasks (chunks of at most kChunkEntries entries / kChunkRows order positions) that
    // depend on the L tasks holding their source rows.  A range without external
    // entries is one L task.  Claim order: the start order of a list schedule on ctas
    // CTAs under the cost model (a topological order).
    auto build = [&](bool fwd, SolveTasks& out) {
        struct Tk {
            double start, cost;
            int4 t;
            std::vector<int32_t> preds;
        };
        std::vector<Tk> tk;
        std::vector<int32_t> row_L(n, -1);  // L task holding each row
        const std::vector<int32_t>& lev = fwd ? lf : lb;
        const std::vector<int32_t>& optr = fwd ? P.lf_ptr : P.lb_ptr;
        const std::vector<int32_t>& ord = fwd ? P.lf_ord : P.lb_ord;
        auto ext_of = [&](int32_t i) -> int64_t {
            return fwd ? int64_t(P.sf_split[i] - P.cptr[i]) : (P.urp[i + 1] - P.urp[i] - 1) - P.sb_nint[i];
        };
        auto finish = [&](int32_t t) { return tk[t].start + tk[t].cost; };
        for (int32_t kk = 0; kk < nb; ++kk) {
            const int32_t k = fwd ? kk : nb - 1 - kk;
            const int32_t base = optr[k], end = optr[k + 1];
            bool any_ext = false;
            for (int32_t i = P.ranges[k]; i < P.ranges[k + 1] && !any_ext; ++i) any_ext = ext_of(i) > 0;
            int32_t prevL = -1;
            int32_t lo = base;
            while (lo < end) {
                // the part: whole levels [lev(lo), lev(lo) + kPartLevels) (all levels when
                // the range has no external entries); padding carries its level
                int32_t l0 = -1, hi = lo;
                int32_t lastlev = -1;
                for (; hi < end; ++hi) {
                    const int32_t i = ord[hi];
                    if (i < 0) continue;
                    if (l0 < 0) l0 = lev[i];
                    if (any_ext && lev[i] >= l0 + kPartLevels) break;
                    lastlev = lev[i];
                }
                // E tasks of the part
                std::vector<int32_t> es;
                int32_t c0 = lo;
                int64_t acc = 0;
                std::vector<int32_t> preds;
                auto close_chunk = [&](int32_t c1) {
                    if (acc > 0) {
                        std::sort(preds.begin(), preds.end());
                        preds.erase(std::unique(preds.begin(), preds.end()), preds.end());
                        double st = 0.0;
                        for (int32_t q : preds) st = std::max(st, finish(q));
                        tk.push_back({st, kTaskStartUs + kFmaUs * double(acc), make_int4(0, k, c0, c1), preds});
                        es.push_back(int32_t(tk.size()) - 1);
                    }
                    c0 = c1;
                    acc = 0;
                    preds.clear();
                };
                for (int32_t q = lo; q < hi; ++q) {
                    const int32_t i = ord[q];
                    if (i >= 0 && ext_of(i) > 0) {
                        acc += ext_of(i);
                        if (fwd) {
                            for (int32_t e = P.cptr[i]; e < P.sf_split[i]; ++e) preds.push_back(row_L[P.csc[e].x]);
                        } else {
                            for (int64_t e = P.urp[i] + 1 + P.sb_nint[i]; e < P.urp[i + 1]; ++e)
                                preds.push_back(row_L[P.ucol[e]]);
                        }
                    }
                    if (acc >= kChunkEntries || q + 1 - c0 >= kChunkRows) close_chunk(q + 1);
                }
                close_chunk(hi);
                // the L task
                std::vector<int32_t> lp(es);
                if (prevL >= 0) lp.push_back(prevL);
                double st = 0.0;
                for (int32_t q : lp) st = std::max(st, finish(q));
                const double cost = kTaskStartUs + kLevelUs * double(lastlev - l0 + 1) +
                                    1e-3 * double(lo - base);  // reload of the earlier parts' results
                tk.push_back({st, cost, make_int4(1, k, lo, hi), lp});
                prevL = int32_t(tk.size()) - 1;
                for (int32_t q = lo; q < hi; ++q)
                    if (ord[q] >= 0) row_L[ord[q]] = prevL;
                lo = hi;
            }
        }
        // claim order: a list schedule of the tasks on the grid's CTAs under the cost
        // model.  A free CTA takes the ready task with the longest path to the end of
        // the solve (bottom level); when an L part ends and the range's next part is
        // ready, the same CTA goes on with it, as the kernel does.  The order in which
        // tasks start is the claim order (topological: a task starts only when ready).
        const size_t nt = tk.size();
        std::vector<std::vector<int32_t>> succs(nt);
        std::vector<int32_t> deg(nt, 0), nextg(nt, -1);
        for (size_t q = 0; q < nt; ++q) {
            deg[q] = int32_t(tk[q].preds.size());
            for (int32_t pr : tk[q].preds) {
                succs[pr].push_back(int32_t(q));
                if (tk[q].t.x == 1 && tk[pr].t.x == 1) nextg[pr] = int32_t(q);
            }
        }
        std::vector<double> bottom(nt, 0.0);  // tasks are generated after their predecessors
        for (size_t q = nt; q-- > 0;) {
            double m = 0.0;
            for (int32_t s2 : succs[q]) m = std::max(m, bottom[s2]);
            bottom[q] = tk[q].cost + m;
        }
        using Entry = std::pair<double, int32_t>;
        std::priority_queue<Entry> ready;  // (bottom level, task): largest first
        std::priority_queue<Entry, std::vector<Entry>, std::greater<Entry>> running;  // (finish, task)
        std::vector<uint8_t> started(nt, 0);
        std::vector<int32_t> idx, pos(nt);
        idx.reserve(nt);
        for (size_t q = 0; q < nt; ++q)
            if (deg[q] == 0) ready.push({bottom[q], int32_t(q)});
        int free_ctas = std::max(1, ctas);
        double now = 0.0;
        auto start = [&](int32_t q) {
            started[q] = 1;
            idx.push_back(q);
            running.push({now + tk[q].cost, q});
        };
        while (idx.size() < nt) {
            while (free_ctas > 0 && !ready.empty()) {
                const int32_t q = ready.top().second;
                ready.pop();
                if (started[q]) continue;  // already taken as a continuation
                start(q);
                --free_ctas;
            }
            if (running.empty()) break;  // not reached: the task graph is acyclic
            const Entry ev = running.top();
            running.pop();
            now = ev.first;
            ++free_ctas;
            for (int32_t s2 : succs[ev.second])
                if (--deg[s2] == 0) ready.push({bottom[s2], s2});
            const int32_t nx = nextg[ev.second];
            if (nx >= 0 && deg[nx] == 0 && !started[nx]) {
                start(nx);
                --free_ctas;
            }
        }
        for (size_t q = 0; q < nt; ++q)  // not reached either: every task has started
            if (!started[q]) idx.push_back(int32_t(q));
        for (size_t q = 0; q < nt; ++q) pos[idx[q]] = int32_t(q);
        out.task.resize(nt);
        out.indeg0.assign(nt, 0);
        std::vector<int32_t> cnt(nt + 1, 0);
        for (size_t q = 0; q < nt; ++q) {
            out.task[q] = tk[idx[q]].t;
            out.indeg0[q] = int32_t(tk[idx[q]].preds.size());
            for (int32_t pr : tk[idx[q]].preds) ++cnt[pos[pr] + 1];
        }
        out.succ_ptr.assign(nt + 1, 0);
        for (size_t q = 0; q < nt; ++q) out.succ_ptr[q + 1] = out.succ_ptr[q] + cnt[q + 1];
        out.succ.assign(out.succ_ptr[nt], 0);
        std::vector<int32_t> fill(out.succ_ptr.begin(), out.succ_ptr.end() - 1);
        for (size_t q = 0; q < nt; ++q)
            for (int32_t pr : tk[idx[q]].preds) out.succ[fill[pos[pr]]++] = int32_t(q);
        // next part of the same range (its L task lists the previous part as a predecessor)
        out.next.assign(nt, -1);
        for (size_t q = 0; q < nt; ++q)
            if (tk[idx[q]].t.x == 1)
                for (int32_t pr : tk[idx[q]].preds)
                    if (tk[pr].t.x == 1) out.next[pos[pr]] = int32_t(q);
    };
    build(true, P.fs);
    build(false, P.bs);
}

}  // namespace ick
