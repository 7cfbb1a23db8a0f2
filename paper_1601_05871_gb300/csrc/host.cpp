// Host side of the symbolic phase (Algorithm 1 of Section 3.1, Sections 3.2-3.3):
// geometric nested dissection, the level-k fill pattern by per-row breadth-first
// search, the 2D sparse partitioned-block matrix, the Cholesky-by-blocks task DAG
// and the per-task work lists the persistent numeric kernel consumes.
#include <omp.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <numeric>
#include <queue>

#include "ick_internal.h"

namespace ick {

// --------------------------------------------------------------------------- ND

namespace {

struct NdCtx {
    int nx, ny, nz, dof, leaf_rows;
    int colours;                // separator planes: C x C classes in strips when >= 2
    int leaf_colours;           // boxes: C x C x C classes when >= 2
    const uint8_t* keep;
    const int64_t* kept_index;  // grid dof -> index among kept dofs, -1 if dropped
    int32_t* perm;
    int64_t next;
    int64_t* ranges;
    int64_t nranges;
};

int64_t count_rows(const NdCtx& c, const int lo[3], const int hi[3]) {
    int64_t nodes = int64_t(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    if (!c.keep) return nodes * c.dof;
    int64_t cnt = 0;
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x) {
                int64_t base = (x + int64_t(c.nx) * (y + int64_t(c.ny) * z)) * c.dof;
                for (int d = 0; d < c.dof; ++d) cnt += c.keep[base + d] != 0;
            }
    return cnt;
}

void close_range(NdCtx& c) {
    ++c.nranges;
    if (c.ranges) c.ranges[c.nranges] = c.next;
}

// Numbers one part (cut < 0: a box; else a separator plane cut across axis cut) in
// lexicographic order, x fastest, and closes its range.  With c.colours = C >= 2 a
// plane of R kept rows is instead cut into m = ceil(R / leaf_rows) strips, strip q
// holding rows [q R / m, (q+1) R / m) of the lexicographic order, each a range of its
// own, and a strip is numbered colour class by colour class: the class of a node is
// (u mod C) + C (v mod C), u and v its coordinates along the two other axes (u the
// lower-numbered one), classes ascending, lexicographic inside a class.  The strips
// are the even pieces the block partition would cut the plane into, so the 2D block
// pattern is that of the lexicographic order.  With c.leaf_colours = C >= 2 a box is
// numbered by the classes (x mod C) + C (y mod C) + C^2 (z mod C) the same way, as
// one part.
void number_part(NdCtx& c, const int lo[3], const int hi[3], int cut) {
    const int64_t first = c.next;
    const int want = cut >= 0 ? c.colours : c.leaf_colours;
    const int nc = want > 1 ? want : 1;
    const int a0 = cut == 0 ? 1 : 0;
    const int a1 = cut == 2 ? 1 : 2;
    std::vector<int> key;  // colour class of each row in lexicographic order (nc > 1)
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x) {
                const int q[3] = {x, y, z};
                int64_t base = (x + int64_t(c.nx) * (y + int64_t(c.ny) * z)) * c.dof;
                for (int d = 0; d < c.dof; ++d) {
                    int64_t idx = c.kept_index[base + d];
                    if (idx < 0) continue;
                    c.perm[c.next++] = int32_t(idx);
                    if (nc == 1) continue;
                    key.push_back(cut >= 0 ? q[a0] % nc + nc * (q[a1] % nc)
                                           : x % nc + nc * (y % nc) + nc * nc * (z % nc));
                }
            }
    const int64_t rows = c.next - first;
    if (rows == 0) return;
    if (nc == 1) {
        close_range(c);
        return;
    }
    const int64_t m = cut >= 0 ? (rows + c.leaf_rows - 1) / c.leaf_rows : 1;
    std::vector<int32_t> lex(c.perm + first, c.perm + c.next);
    std::vector<int64_t> ord(rows);
    c.next = first;
    for (int64_t s = 0; s < m; ++s) {
        const int64_t b = rows * s / m, e = rows * (s + 1) / m;
        std::iota(ord.begin() + b, ord.begin() + e, b);
        std::stable_sort(ord.begin() + b, ord.begin() + e,
                         [&](int64_t u, int64_t v) { return key[u] < key[v]; });
        for (int64_t r = b; r < e; ++r) c.perm[c.next++] = lex[ord[r]];
        close_range(c);
    }
}

// Iterative ND over boxes: each stack frame is a box, or a plane to be numbered
// after its two halves (post-order: low, high, separator).
void dissect(NdCtx& c) {
    struct Frame { int lo[3], hi[3]; int cut; };  // cut: the plane's axis, -1 for a box
    std::vector<Frame> st;
    st.push_back({{0, 0, 0}, {c.nx, c.ny, c.nz}, -1});
    while (!st.empty()) {
        Frame f = st.back();
        st.pop_back();
        if (f.hi[0] <= f.lo[0] || f.hi[1] <= f.lo[1] || f.hi[2] <= f.lo[2]) continue;
        if (f.cut >= 0) { number_part(c, f.lo, f.hi, f.cut); continue; }
        int ext[3] = {f.hi[0] - f.lo[0], f.hi[1] - f.lo[1], f.hi[2] - f.lo[2]};
        int ax = 0;
        if (ext[1] > ext[ax]) ax = 1;
        if (ext[2] > ext[ax]) ax = 2;
        if (ext[ax] < 3 || count_rows(c, f.lo, f.hi) <= c.leaf_rows) {
            number_part(c, f.lo, f.hi, -1);
            continue;
        }
        int m = f.lo[ax] + (f.hi[ax] - f.lo[ax]) / 2;
        Frame low = f, high = f, sep = f;
        low.hi[ax] = m;
        high.lo[ax] = m + 1;
        sep.lo[ax] = m;
        sep.hi[ax] = m + 1;
        sep.cut = ax;
        st.push_back(sep);   // popped last
        st.push_back(high);
        st.push_back(low);   // popped first
    }
}

}  // namespace

int nd_grid(int nx, int ny, int nz, int dof, int leaf_rows, int sep_colours, int leaf_colours,
            const uint8_t* keep, int32_t* perm, int64_t* ranges, int64_t* nranges, int64_t* n_out) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || dof <= 0 || leaf_rows <= 0 || !perm) return IC_ERR_ARG;
    if (sep_colours < 0 || sep_colours > 16 || leaf_colours < 0 || leaf_colours > 4) return IC_ERR_ARG;
    const int64_t nfull = int64_t(nx) * ny * nz * dof;
    if (nfull > INT32_MAX) return IC_ERR_ARG;
    std::vector<int64_t> kept(nfull);
    int64_t cnt = 0;
    for (int64_t i = 0; i < nfull; ++i) kept[i] = (!keep || keep[i]) ? cnt++ : -1;
    NdCtx c{nx, ny, nz, dof, leaf_rows, sep_colours, leaf_colours, keep, kept.data(), perm, 0, ranges, 0};
    if (ranges) ranges[0] = 0;
    dissect(c);
    if (nranges) *nranges = c.nranges;
    if (n_out) *n_out = c.next;
    return IC_OK;
}

// --------------------------------------------------------------------------- DAG

// Cholesky-by-blocks task generation (Section 3.3, task generator figure): for each
// block column k, Chol on (k,k), Trsm on every existing (k,j), j > k, and for every
// pair i <= j of those j an update of (i,j) if that block exists (Herk when i == j,
// Gemm otherwise).  Each block records the last task that wrote it (its future); a
// new task depends on the futures of the blocks it reads and writes, so updates to
// one block are serialised in k order.
int block_dag(int64_t nb, const int64_t* bptr, const int32_t* bcol, std::vector<int4>& task,
              std::vector<int64_t>& pred_ptr, std::vector<int32_t>& pred) {
    task.clear();
    pred.clear();
    pred_ptr.assign(1, 0);
    if (nb < 0 || (nb > 0 && (!bptr || !bcol))) return IC_ERR_ARG;
    if (nb == 0) return IC_OK;
    if (bptr[0] != 0) return IC_ERR_PATTERN;
    for (int64_t b = 0; b < nb; ++b) {
        if (bptr[b + 1] <= bptr[b]) return IC_ERR_PATTERN;
        if (bcol[bptr[b]] != b) return IC_ERR_PATTERN;  // diagonal block first
        for (int64_t e = bptr[b] + 1; e < bptr[b + 1]; ++e)
            if (bcol[e] <= bcol[e - 1] || bcol[e] >= nb) return IC_ERR_PATTERN;
    }
    auto find = [&](int64_t i, int64_t j) -> int64_t {
        const int32_t* b = bcol + bptr[i];
        const int32_t* e = bcol + bptr[i + 1];
        const int32_t* p = std::lower_bound(b, e, int32_t(j));
        return (p != e && *p == j) ? int64_t(p - bcol) : -1;
    };
    std::vector<int32_t> last(bptr[nb], -1);
    auto add = [&](int type, int k, int i, int j, std::initializer_list<int64_t> blocks) {
        int32_t t = int32_t(task.size());
        task.push_back(make_int4(type, k, i, j));
        int32_t deps[3];
        int nd = 0;
        for (int64_t b : blocks) {
            int32_t d = last[b];
            if (d < 0) continue;
            bool dup = false;
            for (int q = 0; q < nd; ++q) dup |= deps[q] == d;
            if (!dup) deps[nd++] = d;
        }
        for (int a = 1; a < nd; ++a)  // at most three entries: insertion sort
            for (int b = a; b > 0 && deps[b - 1] > deps[b]; --b) std::swap(deps[b - 1], deps[b]);
        for (int q = 0; q < nd; ++q) pred.push_back(deps[q]);
        pred_ptr.push_back(int64_t(pred.size()));
        return t;
    };
    for (int64_t k = 0; k < nb; ++k) {
        const int64_t bkk = bptr[k];
        last[bkk] = add(T_CHOL, int(k), int(k), int(k), {bkk});
        for (int64_t e = bptr[k] + 1; e < bptr[k + 1]; ++e)
            last[e] = add(T_TRSM, int(k), int(k), bcol[e], {bkk, e});
        for (int64_t ei = bptr[k] + 1; ei < bptr[k + 1]; ++ei) {
            const int64_t i = bcol[ei];
            for (int64_t ej = ei; ej < bptr[k + 1]; ++ej) {
                const int64_t j = bcol[ej];
                const int64_t bij = find(i, j);
                if (bij < 0) continue;
                last[bij] = add(i == j ? T_HERK : T_GEMM, int(k), int(i), int(j), {ei, ej, bij});
            }
        }
    }
    return IC_OK;
}

// ----------------------------------------------------------------------- symbolic

namespace {

int check_pattern(const ic_csr_pattern* A, std::string& err) {
    const int64_t n = A->n;
    if (n < 0 || n > INT32_MAX - 1) { err = "n out of range"; return IC_ERR_ARG; }
    if (n == 0) return IC_OK;
    if (!A->rowptr || !A->colind) { err = "NULL rowptr/colind"; return IC_ERR_ARG; }
    if (A->rowptr[0] != 0) { err = "rowptr[0] != 0"; return IC_ERR_PATTERN; }
    for (int64_t i = 0; i < n; ++i)
        if (A->rowptr[i + 1] < A->rowptr[i]) { err = "rowptr decreases"; return IC_ERR_PATTERN; }
    const int64_t nnz = A->rowptr[n];
    if (nnz > INT32_MAX) { err = "nnz(A) above 2^31-1"; return IC_ERR_ARG; }
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        bool diag = false;
        for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) {
            int32_t c = A->colind[e];
            if (c < 0 || c >= n) { err = "column index out of range"; return IC_ERR_PATTERN; }
            if (e > A->rowptr[i] && c <= A->colind[e - 1]) {
                err = "columns not strictly increasing in row " + std::to_string(i);
                return IC_ERR_PATTERN;
            }
            diag |= c == i;
            ++cnt[c + 1];
        }
        if (!diag) { err = "missing diagonal in row " + std::to_string(i); return IC_ERR_PATTERN; }
    }
    // symmetry: the transpose, built row by row, must equal the pattern itself
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    for (int64_t i = 0; i < n; ++i)
        if (cnt[i + 1] - cnt[i] != A->rowptr[i + 1] - A->rowptr[i]) {
            err = "asymmetric pattern (row/column counts differ at " + std::to_string(i) + ")";
            return IC_ERR_PATTERN;
        }
    std::vector<int32_t> trow(nnz);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) trow[fill[A->colind[e]]++] = int32_t(i);
    for (int64_t e = 0; e < nnz; ++e)
        if (trow[e] != A->colind[e]) { err = "asymmetric pattern"; return IC_ERR_PATTERN; }
    return IC_OK;
}

// Rough duration of every task for the host's ASAP estimates: a fixed cost per task
// plus a cost per pivot application, a Chol/Trsm task's rows spread over one CTA's
// warps, a Herk/Gemm task's rows over CTAs (so its slowest row counts).
std::vector<double> task_costs(const HostPlan& P, const std::vector<std::vector<int4>>& ttgt) {
    constexpr double kTaskCost = 3.0, kPivotCost = 0.7, kRowsInParallel = 32.0;
    const int64_t nt = int64_t(P.task.size());
    std::vector<double> cost(nt);
    for (int64_t t = 0; t < nt; ++t) {
        double sum = 0.0, mx = 0.0;
        for (const int4& g : ttgt[t]) {
            sum += double(g.z - g.y);
            mx = std::max(mx, double(g.z - g.y));
        }
        const int type = P.task[t].x;
        cost[t] = kTaskCost + kPivotCost * ((type == T_CHOL || type == T_TRSM) ? sum / kRowsInParallel : mx);
    }
    return cost;
}

// Order of the updates into each block (FMA mode).  The task generator serialises the
// Herk/Gemm updates of block (i,j) in ascending k, so an update whose inputs are ready
// early waits behind every earlier-k update, however late their inputs come; with a
// geometric ND ordering the updates from one half's top separator hold back those from
// the other half's whole subtree.  Any order of the chain gives a correct factor (the
// same sums, rounded in another order), so the chain is rebuilt in the order of its
// inputs' estimated readiness: an ASAP schedule of the graph under task_costs,
// computed in task generation order, which settles every chain before its consumer
// (the Chol or Trsm of that block) is reached.
// Dependencies otherwise stay those of the task generator: Trsm(k,j) after Chol(k) and
// the last update of (k,j); an update after Trsm(k,i) and Trsm(k,j).
void order_updates(HostPlan& P, const std::vector<std::vector<int4>>& ttgt) {
    const int64_t nt = int64_t(P.task.size());
    auto block_id = [&](int64_t i, int64_t j) -> int64_t {
        auto b = P.bcol.begin() + P.bptr[i], e = P.bcol.begin() + P.bptr[i + 1];
        auto it = std::lower_bound(b, e, int32_t(j));
        return (it != e && *it == j) ? int64_t(it - P.bcol.begin()) : -1;
    };
    const std::vector<double> cost = task_costs(P, ttgt);
    std::vector<double> fin(nt, 0.0);
    const size_t nblk = P.bcol.size();
    std::vector<int32_t> writer(nblk, -1);             // Chol/Trsm task that produced a block
    std::vector<std::vector<int32_t>> upd(nblk);       // updates into a block, generation order
    std::vector<std::vector<int32_t>> pred(nt);
    std::vector<std::pair<double, int32_t>> key;
    for (int64_t t = 0; t < nt; ++t) {
        const int4 T = P.task[t];
        if (T.x == T_HERK || T.x == T_GEMM) {
            upd[block_id(T.z, T.w)].push_back(int32_t(t));
            continue;
        }
        const int64_t b = block_id(T.y, T.x == T_CHOL ? T.y : T.w);
        key.clear();
        for (int32_t u : upd[b]) {
            const int4 Uu = P.task[u];
            const int32_t si = writer[block_id(Uu.y, Uu.z)], sj = writer[block_id(Uu.y, Uu.w)];
            pred[u].assign({si});
            if (sj != si) pred[u].push_back(sj);
            key.emplace_back(std::max(fin[si], fin[sj]), u);
        }
        std::stable_sort(key.begin(), key.end(),
                         [](const std::pair<double, int32_t>& a, const std::pair<double, int32_t>& c) {
                             return a.first < c.first;
                         });
        int32_t prev = -1;
        for (const auto& ku : key) {
            const int32_t u = ku.second;
            double start = ku.first;
            if (prev >= 0) {
                pred[u].push_back(prev);
                start = std::max(start, fin[prev]);
            }
            fin[u] = start + cost[u];
            prev = u;
        }
        double start = 0.0;
        if (T.x == T_TRSM) {
            const int32_t c = writer[block_id(T.y, T.y)];
            pred[t].push_back(c);
            start = fin[c];
        }
        if (prev >= 0) {
            pred[t].push_back(prev);
            start = std::max(start, fin[prev]);
        }
        fin[t] = start + cost[t];
        writer[b] = int32_t(t);
    }
    P.pred_ptr.assign(1, 0);
    P.pred.clear();
    for (int64_t t = 0; t < nt; ++t) {
        std::sort(pred[t].begin(), pred[t].end());
        P.pred.insert(P.pred.end(), pred[t].begin(), pred[t].end());
        P.pred_ptr.push_back(int64_t(P.pred.size()));
    }
}

// Chol and Trsm tasks that would run nearly alone get several CTAs.  Such a task's rows
// form dependence levels inside its block; one CTA works through them with per-row
// flags in shared memory, and at the end of the factorization (the top separators) it
// is the only work on the GPU, bound by one SM's issue rate.  Split into kSplitItems
// items, the task's rows are claimed from a counter in global memory by every CTA that
// holds one of its items, and each finished row is published in a shadow array whose
// entries hold a sentinel until written, so a reader knows every value it uses is
// final without a flag.  The estimate: an ASAP schedule of the final graph under
// task_costs; a Chol/Trsm task of at least kSplitMinRows target rows whose start finds
// fewer than kSplitIdle other work items in flight is split.
void split_tail_tasks(HostPlan& P, const std::vector<std::vector<int4>>& ttgt,
                      const std::vector<std::vector<int32_t>>& tend) {
    constexpr int kSplitItems = 8, kSplitMinRows = 512;
    constexpr int64_t kSplitIdle = 64, kShadowPad = 4;
    const int64_t nt = int64_t(P.task.size());
    P.flag_off.assign(nt, -1);
    P.soff.clear();
    P.nflags = 0;
    P.nsplit = 0;
    P.nshadow = kShadowPad;  // 16-byte copies may reach up to 3 values past either end
    if (nt == 0) return;
    const std::vector<double> cost = task_costs(P, ttgt);
    // ASAP over a topological order of the graph
    std::vector<int32_t> left(nt), order;
    std::vector<std::vector<int32_t>> succ(nt);
    for (int64_t t = 0; t < nt; ++t) {
        left[t] = int32_t(P.pred_ptr[t + 1] - P.pred_ptr[t]);
        for (int64_t e = P.pred_ptr[t]; e < P.pred_ptr[t + 1]; ++e) succ[P.pred[e]].push_back(int32_t(t));
        if (left[t] == 0) order.push_back(int32_t(t));
    }
    std::vector<double> start(nt, 0.0), fin(nt, 0.0);
    for (size_t q = 0; q < order.size(); ++q) {
        const int32_t t = order[q];
        fin[t] = start[t] + cost[t];
        for (int32_t s : succ[t]) {
            start[s] = std::max(start[s], fin[t]);
            if (--left[s] == 0) order.push_back(s);
        }
    }
    if (int64_t(order.size()) != nt) return;  // not a DAG: reported by the caller
    // items in flight at each task's start: sweep over (time, +-items) events
    std::vector<std::pair<double, int64_t>> ev;
    ev.reserve(2 * nt);
    for (int64_t t = 0; t < nt; ++t) {
        ev.emplace_back(fin[t], -int64_t(P.nitems[t]));  // ends sort before starts at equal times
        ev.emplace_back(start[t], int64_t(P.nitems[t]));
    }
    std::sort(ev.begin(), ev.end());
    std::vector<std::pair<double, int32_t>> starts;
    for (int64_t t = 0; t < nt; ++t) {
        const int type = P.task[t].x;
        if ((type == T_CHOL || type == T_TRSM) && int64_t(ttgt[t].size()) >= kSplitMinRows)
            starts.emplace_back(start[t], int32_t(t));
    }
    std::sort(starts.begin(), starts.end());
    int64_t live = 0;
    size_t e = 0;
    for (const auto& st : starts) {
        while (e < ev.size() && ev[e].first <= st.first) live += ev[e++].second;
        const int32_t t = st.second;
        if (live - P.nitems[t] >= kSplitIdle) continue;
        const int32_t blk = P.task[t].y, rbase = P.ranges[blk];
        P.flag_off[t] = int32_t(P.nflags);
        P.nflags += P.ranges[blk + 1] - rbase;
        P.soff.resize(size_t(P.nflags), 0);
        for (size_t i = 0; i < ttgt[t].size(); ++i) {
            const int64_t r = ttgt[t][i].x, tb = ttgt[t][i].w, te = tend[t][i];
            const int64_t pos = P.nshadow + (((tb - P.nshadow) % 4) + 4) % 4;
            P.soff[size_t(P.flag_off[t] + (r - rbase))] = int32_t(pos - tb);
            P.nshadow = pos + (te - tb);
        }
        P.nitems[t] = kSplitItems;
        ++P.nsplit;
    }
    P.nshadow += kShadowPad;
}

}  // namespace

int build_plan(const ic_csr_pattern* A, int k, const int32_t* perm, const int64_t* ranges,
               int64_t nranges, int block_rows, int rows_per_item, int threads, bool k_order,
               int solve_ctas, HostPlan& P, std::string& err) {
    if (!A) { err = "NULL pattern"; return IC_ERR_ARG; }
    if (k < 0) { err = "k < 0"; return IC_ERR_ARG; }
    if (block_rows <= 0 || block_rows > kMaxBlockRows) { err = "block_rows out of range"; return IC_ERR_ARG; }
    int st = check_pattern(A, err);
    if (st) return st;
    const int64_t n = A->n;
    const int nthr = threads > 0 ? threads : omp_get_max_threads();
    P.n = n;
    P.k = k;
    P.rows_per_item = rows_per_item;
    P.nnz_a = n ? A->rowptr[n] : 0;
    P.arp.assign(A->rowptr, A->rowptr + n + 1);
    if (n == 0) P.arp.assign(1, 0);
    P.acol.assign(A->colind, A->colind + P.nnz_a);

    // permutation
    P.perm.resize(n);
    P.iperm.assign(n, -1);
    for (int64_t i = 0; i < n; ++i) {
        int32_t o = perm ? perm[i] : int32_t(i);
        if (o < 0 || o >= n || P.iperm[o] != -1) { err = "perm is not a permutation"; return IC_ERR_ARG; }
        P.perm[i] = o;
        P.iperm[o] = int32_t(i);
    }

    // graph of B = P^T A P without the diagonal, rows sorted; source index per edge
    std::vector<int64_t> gptr(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = P.perm[i];
        gptr[i + 1] = gptr[i] + (A->rowptr[o + 1] - A->rowptr[o] - 1);
    }
    std::vector<int32_t> gadj(gptr[n]);
    std::vector<int32_t> gsrc_e(gptr[n]);
    P.udiag_src.resize(n);
#pragma omp parallel for num_threads(nthr) schedule(static, 4096)
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = P.perm[i], p = gptr[i];
        std::vector<std::pair<int32_t, int32_t>> row;
        row.reserve(A->rowptr[o + 1] - A->rowptr[o]);
        for (int64_t e = A->rowptr[o]; e < A->rowptr[o + 1]; ++e) {
            if (A->colind[e] == o) { P.udiag_src[i] = int32_t(e); continue; }
            row.emplace_back(P.iperm[A->colind[e]], int32_t(e));
        }
        std::sort(row.begin(), row.end());
        for (auto& pr : row) { gadj[p] = pr.first; gsrc_e[p] = pr.second; ++p; }
    }

    // level-k pattern of U row by row: breadth-first search from i through vertices
    // < i; a vertex j > i reached after d+1 edges is fill of level d (<= k).
    const int64_t chunk = 1024;
    const int64_t nchunks = (n + chunk - 1) / chunk;
    std::vector<std::vector<int32_t>> ccol(nchunks), clev(nchunks);
    std::vector<int32_t> rowlen(n);
    int64_t maxlev = 0;
#pragma omp parallel num_threads(nthr) reduction(max : maxlev)
    {
        std::vector<int32_t> mark(n, 0);
        std::vector<int32_t> fr, nx;
        std::vector<std::pair<int32_t, int32_t>> out;
#pragma omp for schedule(dynamic, 1)
        for (int64_t c = 0; c < nchunks; ++c) {
            const int64_t r0 = c * chunk, r1 = std::min(n, r0 + chunk);
            auto& cc = ccol[c];
            auto& cl = clev[c];
            for (int64_t i = r0; i < r1; ++i) {
                const int32_t stamp = int32_t(i + 1);
                out.clear();
                fr.clear();
                fr.push_back(int32_t(i));
                mark[i] = stamp;
                for (int d = 0; d <= k && !fr.empty(); ++d) {
                    nx.clear();
                    for (int32_t v : fr)
                        for (int64_t e = gptr[v]; e < gptr[v + 1]; ++e) {
                            int32_t w = gadj[e];
                            if (mark[w] == stamp) continue;
                            mark[w] = stamp;
                            if (w > i) out.emplace_back(w, d);
                            else if (d + 1 <= k) nx.push_back(w);
                        }
                    std::swap(fr, nx);
                }
                std::sort(out.begin(), out.end());
                cc.push_back(int32_t(i));
                cl.push_back(0);
                for (auto& pr : out) {
                    cc.push_back(pr.first);
                    cl.push_back(pr.second);
                    if (pr.second > maxlev) maxlev = pr.second;
                }
                rowlen[i] = int32_t(out.size() + 1);
            }
        }
    }
    P.max_level = maxlev;
    P.urp.assign(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) P.urp[i + 1] = P.urp[i] + rowlen[i];
    P.nnz_u = P.urp[n];
    if (P.nnz_u > INT32_MAX) { err = "nnz(L) above 2^31-1"; return IC_ERR_ARG; }
    P.ucol.resize(P.nnz_u);
    P.ulev.resize(P.nnz_u);
#pragma omp parallel for num_threads(nthr) schedule(dynamic, 1)
    for (int64_t c = 0; c < nchunks; ++c) {
        const int64_t base = P.urp[c * chunk];
        std::copy(ccol[c].begin(), ccol[c].end(), P.ucol.begin() + base);
        std::copy(clev[c].begin(), clev[c].end(), P.ulev.begin() + base);
        std::vector<int32_t>().swap(ccol[c]);
        std::vector<int32_t>().swap(clev[c]);
    }

    // value gather map: U position -> index of A's value (fill: -1)
    P.gsrc.assign(P.nnz_u, -1);
#pragma omp parallel for num_threads(nthr) schedule(static, 4096)
    for (int64_t i = 0; i < n; ++i) {
        int64_t u = P.urp[i];
        P.gsrc[u] = -2 - P.udiag_src[i];
        ++u;
        for (int64_t e = gptr[i]; e < gptr[i + 1]; ++e) {
            int32_t j = gadj[e];
            if (j < i) continue;
            while (P.ucol[u] < j) ++u;  // every structural entry has level 0, so it is present
            P.gsrc[u] = gsrc_e[e];
        }
    }

    // block ranges: given ranges split into pieces of at most block_rows rows
    P.ranges.assign(1, 0);
    if (ranges) {
        if (nranges < 0 || ranges[0] != 0 || ranges[nranges] != n) { err = "ranges must run from 0 to n"; return IC_ERR_ARG; }
        for (int64_t b = 0; b < nranges; ++b) {
            int64_t lo = ranges[b], hi = ranges[b + 1];
            if (hi <= lo) { err = "ranges must increase"; return IC_ERR_ARG; }
            int64_t len = hi - lo, pieces = (len + block_rows - 1) / block_rows;
            for (int64_t q = 1; q <= pieces; ++q) P.ranges.push_back(int32_t(lo + (len * q) / pieces));
        }
    } else {
        for (int64_t r = block_rows; r < n; r += block_rows) P.ranges.push_back(int32_t(r));
        if (n > 0) P.ranges.push_back(int32_t(n));
    }
    const int64_t nb = int64_t(P.ranges.size()) - 1;
    P.blk_of.resize(n);
    for (int64_t b = 0; b < nb; ++b)
        for (int64_t r = P.ranges[b]; r < P.ranges[b + 1]; ++r) P.blk_of[r] = int32_t(b);

    // per-row block segments of U
    P.rseg_ptr.assign(n + 1, 0);
    for (int64_t p = 0; p < n; ++p) {
        int32_t cnt = 0, prev = -1;
        for (int64_t e = P.urp[p]; e < P.urp[p + 1]; ++e) {
            int32_t b = P.blk_of[P.ucol[e]];
            if (b != prev) { ++cnt; prev = b; }
        }
        P.rseg_ptr[p + 1] = P.rseg_ptr[p] + cnt;
    }
    P.rseg_blk.resize(P.rseg_ptr[n]);
    P.rseg_se.resize(P.rseg_ptr[n]);
    for (int64_t p = 0; p < n; ++p) {
        int32_t s = P.rseg_ptr[p] - 1, prev = -1;
        for (int64_t e = P.urp[p]; e < P.urp[p + 1]; ++e) {
            int32_t b = P.blk_of[P.ucol[e]];
            if (b != prev) {
                ++s;
                P.rseg_blk[s] = b;
                P.rseg_se[s] = make_int2(int(e), int(e));
                prev = b;
            }
            P.rseg_se[s].y = int(e + 1);
        }
    }
    auto seg = [&](int64_t r, int32_t b) -> int2 {
        for (int32_t s = P.rseg_ptr[r]; s < P.rseg_ptr[r + 1]; ++s)
            if (P.rseg_blk[s] == b) return P.rseg_se[s];
        return make_int2(0, 0);
    };

    // column lists of U: entries (p, pos) with p < r for every column r, ascending p
    P.cptr.assign(n + 1, 0);
    for (int64_t p = 0; p < n; ++p)
        for (int64_t e = P.urp[p] + 1; e < P.urp[p + 1]; ++e) ++P.cptr[P.ucol[e] + 1];
    for (int64_t r = 0; r < n; ++r) P.cptr[r + 1] += P.cptr[r];
    P.csc.resize(P.cptr[n]);
    {
        std::vector<int32_t> fill(P.cptr.begin(), P.cptr.end() - 1);
        std::vector<int32_t> send(P.nnz_u);  // end of the block segment holding each position
        for (int64_t p = 0; p < n; ++p)
            for (int32_t s = P.rseg_ptr[p]; s < P.rseg_ptr[p + 1]; ++s)
                for (int32_t e = P.rseg_se[s].x; e < P.rseg_se[s].y; ++e) send[e] = P.rseg_se[s].y;
        P.cseg_end.resize(P.cptr[n]);
        for (int64_t p = 0; p < n; ++p)
            for (int64_t e = P.urp[p] + 1; e < P.urp[p + 1]; ++e) {
                const int32_t at = fill[P.ucol[e]]++;
                P.csc[at] = make_int2(int(p), int(e));
                P.cseg_end[at] = send[e];
            }
    }

    // block pattern: block (bi, bj), bi <= bj, exists iff S has an entry in it
    {
        std::vector<std::vector<int32_t>> brow(nb);
        for (int64_t p = 0; p < n; ++p) {
            auto& v = brow[P.blk_of[p]];
            for (int32_t s = P.rseg_ptr[p]; s < P.rseg_ptr[p + 1]; ++s) v.push_back(P.rseg_blk[s]);
        }
        P.bptr.assign(nb + 1, 0);
        P.bcol.clear();
        for (int64_t b = 0; b < nb; ++b) {
            auto& v = brow[b];
            std::sort(v.begin(), v.end());
            v.erase(std::unique(v.begin(), v.end()), v.end());
            P.bcol.insert(P.bcol.end(), v.begin(), v.end());
            P.bptr[b + 1] = int64_t(P.bcol.size());
        }
    }
    st = block_dag(nb, P.bptr.data(), P.bcol.data(), P.task, P.pred_ptr, P.pred);
    if (st) { err = "block DAG generation failed"; return st; }
    const int64_t nt = int64_t(P.task.size());

    // column groups: for column r, the pivots p of one block k form a contiguous run
    // of its column list.  Diagonal-block runs are kept per row; off-diagonal runs are
    // collected per block (k, blk(r)).
    auto block_id = [&](int64_t i, int64_t j) -> int64_t {
        auto b = P.bcol.begin() + P.bptr[i], e = P.bcol.begin() + P.bptr[i + 1];
        auto it = std::lower_bound(b, e, int32_t(j));
        return (it != e && *it == j) ? int64_t(it - P.bcol.begin()) : -1;
    };
    std::vector<int2> diag_run(n, make_int2(0, 0));
    std::vector<std::vector<int4>> off_runs(P.bcol.size());  // (r, a, b, 0)
    for (int64_t r = 0; r < n; ++r) {
        int32_t a = P.cptr[r];
        const int32_t e = P.cptr[r + 1];
        diag_run[r] = make_int2(P.cptr[r], P.cptr[r]);
        while (a < e) {
            const int32_t kb = P.blk_of[P.csc[a].x];
            int32_t b = a;
            while (b < e && P.blk_of[P.csc[b].x] == kb) ++b;
            if (kb == P.blk_of[r]) diag_run[r] = make_int2(a, b);
            else off_runs[block_id(kb, P.blk_of[r])].push_back(make_int4(int(r), a, b, 0));
            a = b;
        }
    }

    // work lists of every task
    std::vector<std::vector<int4>> ttgt(nt);
    std::vector<std::vector<int32_t>> tend(nt);
#pragma omp parallel for num_threads(nthr) schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; ++t) {
        const int4 T = P.task[t];
        auto& out = ttgt[t];
        auto& oe = tend[t];
        if (T.x == T_CHOL || T.x == T_TRSM) {
            const int32_t blk = T.y, tb = (T.x == T_CHOL) ? T.y : T.w;
            // Rows of a diagonal block depend on earlier rows of the same block (the pivots
            // of their diagonal-block column run that are targets of this task).  Targets
            // are listed in wavefront order -- by dependence level, then row -- so rows
            // claimed one after another are mostly independent and a row's inputs are
            // always listed before it.
            const int32_t rb = P.ranges[blk], nr = P.ranges[blk + 1] - rb;
            std::vector<int32_t> level(nr, -1);
            std::vector<std::pair<int32_t, int32_t>> ord;
            for (int64_t r = rb; r < rb + nr; ++r) {
                int2 s = seg(r, tb);
                if (s.y <= s.x) continue;
                int32_t lv = 0;
                for (int32_t e = diag_run[r].x; e < diag_run[r].y; ++e) {
                    const int32_t lp = level[P.csc[e].x - rb];
                    if (lp >= 0) lv = std::max(lv, lp + 1);
                }
                level[r - rb] = lv;
                ord.emplace_back(lv, int32_t(r));
            }
            std::sort(ord.begin(), ord.end());
            for (const auto& lr : ord) {
                const int64_t r = lr.second;
                int2 s = seg(r, tb);
                out.push_back(make_int4(int(r), diag_run[r].x, diag_run[r].y, s.x));
                oe.push_back(s.y);
            }
        } else {
            const int64_t bki = block_id(T.y, T.z);
            for (const int4& run : off_runs[bki]) {
                int2 s = seg(run.x, T.w);
                if (s.y <= s.x) continue;
                out.push_back(make_int4(run.x, run.y, run.z, s.x));
                oe.push_back(s.y);
            }
        }
    }
    P.tgt_ptr.assign(nt + 1, 0);
    for (int64_t t = 0; t < nt; ++t) P.tgt_ptr[t + 1] = P.tgt_ptr[t] + int32_t(ttgt[t].size());
    P.tgt.resize(P.tgt_ptr[nt]);
    P.tgt_end.resize(P.tgt_ptr[nt]);
    for (int64_t t = 0; t < nt; ++t) {
        std::copy(ttgt[t].begin(), ttgt[t].end(), P.tgt.begin() + P.tgt_ptr[t]);
        std::copy(tend[t].begin(), tend[t].end(), P.tgt_end.begin() + P.tgt_ptr[t]);
    }

    if (!k_order) order_updates(P, ttgt);

    // items, successors, in-degrees, critical path, type counts
    P.nitems.resize(nt);
    P.indeg0.resize(nt);
    P.total_items = 0;
    for (int k2 = 0; k2 < 4; ++k2) P.ntype[k2] = 0;
    for (int64_t t = 0; t < nt; ++t) {
        const int4 T = P.task[t];
        const int32_t cnt = P.tgt_ptr[t + 1] - P.tgt_ptr[t];
        P.nitems[t] = (T.x == T_CHOL || T.x == T_TRSM) ? 1
                      : std::max<int32_t>(1, (cnt + rows_per_item - 1) / rows_per_item);
        P.indeg0[t] = int32_t(P.pred_ptr[t + 1] - P.pred_ptr[t]);
        ++P.ntype[T.x];
    }
    split_tail_tasks(P, ttgt, tend);
    if (P.nflags > INT32_MAX / 2 || P.nshadow > INT32_MAX / 2) { err = "too many split rows"; return IC_ERR_ARG; }
    for (int64_t t = 0; t < nt; ++t) P.total_items += P.nitems[t];
    if (P.total_items > INT32_MAX / 2) { err = "too many work items"; return IC_ERR_ARG; }
    P.succ_ptr.assign(nt + 1, 0);
    for (int32_t d : P.pred) ++P.succ_ptr[d + 1];
    for (int64_t t = 0; t < nt; ++t) P.succ_ptr[t + 1] += P.succ_ptr[t];
    P.succ.resize(P.pred.size());
    {
        std::vector<int32_t> fill(P.succ_ptr.begin(), P.succ_ptr.end() - 1);
        for (int64_t t = 0; t < nt; ++t)
            for (int64_t e = P.pred_ptr[t]; e < P.pred_ptr[t + 1]; ++e) P.succ[fill[P.pred[e]]++] = int32_t(t);
    }
    {
        // longest chain of tasks, over a topological order (in FMA mode an update's
        // predecessor in its block's chain can have a larger index)
        std::vector<int64_t> depth(nt, 1);
        std::vector<int32_t> left(P.indeg0), ready;
        for (int64_t t = 0; t < nt; ++t)
            if (left[t] == 0) ready.push_back(int32_t(t));
        int64_t best = nt ? 1 : 0, seen = 0;
        while (!ready.empty()) {
            const int32_t t = ready.back();
            ready.pop_back();
            ++seen;
            best = std::max(best, depth[t]);
            for (int64_t e = P.succ_ptr[t]; e < P.succ_ptr[t + 1]; ++e) {
                const int32_t s = P.succ[e];
                depth[s] = std::max(depth[s], depth[t] + 1);
                if (--left[s] == 0) ready.push_back(s);
            }
        }
        if (seen != nt) { err = "task graph has a cycle"; return IC_ERR_ARG; }
        P.critical_path = best;
    }

    // claim orders of the triangular solves: rows sorted by their depth in the row
    // dependence DAG (forward: row i needs the rows p of column i of U; backward: row i
    // needs the columns c > i of row i), ties by row index.  A row's inputs always have
    // a smaller depth, so they are claimed before it.
    {
        std::vector<int32_t> lf(n, 0), lb(n, 0);
        int32_t mf = 0, mb = 0;
        for (int64_t i = 0; i < n; ++i) {
            int32_t d = 0;
            for (int32_t e = P.cptr[i]; e < P.cptr[i + 1]; ++e) d = std::max(d, lf[P.csc[e].x] + 1);
            lf[i] = d;
            mf = std::max(mf, d);
        }
        for (int64_t i = n - 1; i >= 0; --i) {
            int32_t d = 0;
            for (int64_t e = P.urp[i] + 1; e < P.urp[i + 1]; ++e) d = std::max(d, lb[P.ucol[e]] + 1);
            lb[i] = d;
            mb = std::max(mb, d);
        }
        auto order_by = [&](const std::vector<int32_t>& lev, int32_t maxd, bool descending_ties,
                            std::vector<int32_t>& out) {
            std::vector<int32_t> cnt(size_t(maxd) + 2, 0);
            for (int64_t i = 0; i < n; ++i) ++cnt[lev[i] + 1];
            for (int32_t d = 0; d <= maxd; ++d) cnt[d + 1] += cnt[d];
            out.resize(n);
            for (int64_t q = 0; q < n; ++q) {
                const int64_t i = descending_ties ? n - 1 - q : q;
                out[cnt[lev[i]]++] = int32_t(i);
            }
        };
        order_by(lf, mf, false, P.fwd_order);
        order_by(lb, mb, true, P.bwd_order);
        // padded copies: every level's run is filled up to a multiple of kClaimPad with
        // -1, so an aligned claim of up to kClaimPad consecutive positions never mixes
        // rows of two levels (rows claimed by one warp are then independent)
        auto pad = [&](const std::vector<int32_t>& order, const std::vector<int32_t>& lev,
                       std::vector<int32_t>& out) {
            out.clear();
            out.reserve(order.size() + order.size() / 2);
            for (size_t q = 0; q < order.size(); ++q) {
                out.push_back(order[q]);
                const bool last = q + 1 == order.size() || lev[order[q + 1]] != lev[order[q]];
                if (last)
                    while (out.size() % kClaimPad) out.push_back(-1);
            }
        };
        pad(P.fwd_order, lf, P.fwd_pad);
        pad(P.bwd_order, lb, P.bwd_pad);
        P.fwd_depth = n ? int64_t(mf) + 1 : 0;
        P.bwd_depth = n ? int64_t(mb) + 1 : 0;
    }

    // algorithmic flops: per pivot p, one sqrt, |S_p|-1 divides, and two flops for each
    // pair (r, c), r <= c, of row p's off-diagonal columns that lands in S
    double upd = 0.0;
#pragma omp parallel for num_threads(nthr) schedule(dynamic, 256) reduction(+ : upd)
    for (int64_t p = 0; p < n; ++p) {
        const int64_t b = P.urp[p] + 1, e = P.urp[p + 1];
        for (int64_t x = b; x < e; ++x) {
            const int32_t r = P.ucol[x];
            // |{c in row p, c >= r} intersect row r|
            int64_t a1 = x, a2 = P.urp[r], cnt = 0;
            const int64_t e2 = P.urp[r + 1];
            while (a1 < e && a2 < e2) {
                if (P.ucol[a1] < P.ucol[a2]) ++a1;
                else if (P.ucol[a1] > P.ucol[a2]) ++a2;
                else { ++cnt; ++a1; ++a2; }
            }
            upd += double(cnt);
        }
    }
    P.flops = double(n) + double(P.nnz_u - n) + 2.0 * upd;
    // compulsory bytes: read the lower triangle of A (values and column indices),
    // write L (values and column indices) and its row pointers
    const double nnz_low = double(P.nnz_a + n) / 2.0;
    P.bytes = nnz_low * (8 + 4) + double(P.nnz_u) * (8 + 4) + double(n + 1) * 8;
    build_solve_dag(P, nthr, solve_ctas);
    return IC_OK;
}

// ---------------------------------------------------------------- claim order

namespace {

// Duration model of a work item (microseconds), fitted on %globaltimer traces of the
// persistent kernel on a GB300 (27-point Laplacian 96^3, IC(2), FP64, 32 warps per CTA:
// median relative error 1-15 % per kind).  A Chol or Trsm task on one CTA runs its
// block's rows in dependence levels (L levels, about 1.3 us each for Chol) plus its
// pivot applications spread over the CTA's warps; an item of a split task advances
// about 2.3 us per level (rows handed between CTAs through L2); a Herk/Gemm item costs
// a fixed part plus about 20 ns per pivot application.  Only the claim order depends on
// these numbers, never the results.
double item_cost(int type, bool split, double levels, double pivots) {
    double d;
    if (split) d = 14.74 + 2.343 * levels + 0.0521 * pivots / 256.0;
    else if (type == T_CHOL) d = -36.83 + 1.298 * levels + 0.774 * pivots / 32.0;
    else if (type == T_TRSM) d = 55.57 + 0.0659 * levels + 0.751 * pivots / 32.0;
    else if (type == T_HERK) d = 6.162 + 0.0213 * pivots;
    else d = 16.41 + 0.0133 * pivots;
    return std::max(d, 0.5);
}

}  // namespace

// Claim order of the persistent numeric kernel's work items (Section 2.2's scheduler
// duty of running ready tasks, with an order chosen on the host): a list schedule of
// the task DAG on nctas CTAs under item_cost, in which a free CTA takes the ready item
// whose task has the longest remaining path to the end of the DAG; the order in which
// items start is the order in which the kernel's CTAs claim them.  An item is listed
// only after every item of its task's predecessors, so a CTA that waits for an item's
// predecessors waits only for items claimed before it, held by running CTAs.
void build_claim_order(HostPlan& P, int nctas) {
    const int64_t nt = int64_t(P.task.size()), n = P.n;
    P.claim.clear();
    if (nt == 0) return;
    nctas = std::max(nctas, 1);
    // dependence levels of every block's rows (the Chol/Trsm chain of that block)
    std::vector<int32_t> lev(size_t(n), 0);
    std::vector<int32_t> blev(P.ranges.size(), 0);
    for (int64_t r = 0; r < n; ++r) {
        const int32_t b = P.blk_of[r];
        int32_t d = 0;
        for (int32_t e = P.cptr[r]; e < P.cptr[r + 1]; ++e) {
            const int32_t p = P.csc[e].x;
            if (P.blk_of[p] == b) d = std::max(d, lev[p] + 1);
        }
        lev[r] = d;
        blev[b] = std::max(blev[b], d + 1);
    }
    // item costs and task durations
    std::vector<int64_t> first(nt + 1, 0);
    for (int64_t t = 0; t < nt; ++t) first[t + 1] = first[t] + P.nitems[t];
    std::vector<double> cost(static_cast<size_t>(first[nt])), tdur(static_cast<size_t>(nt));
    const int rpi = std::max(P.rows_per_item, 1);
    for (int64_t t = 0; t < nt; ++t) {
        const int type = P.task[t].x;
        const int32_t a = P.tgt_ptr[t], b = P.tgt_ptr[t + 1];
        if (type == T_CHOL || type == T_TRSM) {
            double piv = 0.0;
            for (int32_t q = a; q < b; ++q) piv += double(P.tgt[q].z - P.tgt[q].y);
            const double c = item_cost(type, P.nitems[t] > 1, double(blev[P.task[t].y]), piv);
            for (int64_t it = first[t]; it < first[t + 1]; ++it) cost[it] = c;
            tdur[t] = c;
        } else {
            double sum = 0.0;
            for (int32_t c = 0; c < P.nitems[t]; ++c) {
                double piv = 0.0;
                for (int32_t q = a + c * rpi; q < std::min(b, a + (c + 1) * rpi); ++q)
                    piv += double(P.tgt[q].z - P.tgt[q].y);
                cost[first[t] + c] = item_cost(type, false, 0.0, piv);
                sum += cost[first[t] + c];
            }
            tdur[t] = sum / double(std::min<int64_t>(P.nitems[t], nctas));
        }
    }
    // longest remaining path of every task, over a topological order
    std::vector<int32_t> left(P.indeg0), topo;
    topo.reserve(nt);
    for (int64_t t = 0; t < nt; ++t)
        if (left[t] == 0) topo.push_back(int32_t(t));
    for (size_t q = 0; q < topo.size(); ++q)
        for (int32_t e = P.succ_ptr[topo[q]]; e < P.succ_ptr[topo[q] + 1]; ++e)
            if (--left[P.succ[e]] == 0) topo.push_back(P.succ[e]);
    if (int64_t(topo.size()) != nt) return;  // not a DAG: reported by the caller
    std::vector<double> rem(nt, 0.0);
    for (int64_t q = nt - 1; q >= 0; --q) {
        const int32_t t = topo[q];
        double m = 0.0;
        for (int32_t e = P.succ_ptr[t]; e < P.succ_ptr[t + 1]; ++e) m = std::max(m, rem[P.succ[e]]);
        rem[t] = tdur[t] + m;
    }
    // the list schedule (1 us per claim)
    struct Ready {
        double rem;
        int32_t task, chunk;
        bool operator<(const Ready& o) const {  // max-heap: longest remaining path first
            if (rem != o.rem) return rem < o.rem;
            if (task != o.task) return task > o.task;
            return chunk > o.chunk;
        }
    };
    std::priority_queue<Ready> ready;
    using Ev = std::pair<double, int32_t>;  // (finish time, task)
    std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> running;
    std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
    for (int c = 0; c < nctas; ++c) free_at.push(0.0);
    std::vector<int32_t> deg(P.indeg0), items_left(P.nitems);
    for (int64_t t = 0; t < nt; ++t)
        if (deg[t] == 0)
            for (int32_t c = 0; c < P.nitems[t]; ++c) ready.push({rem[t], int32_t(t), c});
    P.claim.reserve(size_t(first[nt]));
    while (int64_t(P.claim.size()) < first[nt]) {
        const double tf = free_at.top();
        free_at.pop();
        while (!running.empty() && running.top().first <= tf) {
            const int32_t t = running.top().second;
            running.pop();
            if (--items_left[t] == 0)
                for (int32_t e = P.succ_ptr[t]; e < P.succ_ptr[t + 1]; ++e) {
                    const int32_t u = P.succ[e];
                    if (--deg[u] == 0)
                        for (int32_t c = 0; c < P.nitems[u]; ++c) ready.push({rem[u], u, c});
                }
        }
        if (!ready.empty()) {
            const Ready r = ready.top();
            ready.pop();
            P.claim.push_back(make_int2(r.task, r.chunk));
            const double fin = tf + 1.0 + cost[first[r.task] + r.chunk];
            running.push({fin, r.task});
            free_at.push(fin);
        } else if (!running.empty()) {
            free_at.push(running.top().first);
        } else {
            break;  // cannot happen in a DAG
        }
    }
}

}  // namespace ick
