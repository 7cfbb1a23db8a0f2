/*
 * CPU oracle for level-of-fill incomplete Cholesky IC(k) -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this file.
 * It shares no code, header or table with the CUDA library; it is plain, single
 * threaded, FP64 C, written to be checked against the paper by eye:
 *
 *   orc_nd_grid   geometric nested dissection (Algorithm 1, step 1; Section 3.1):
 *                 the longest box axis is cut by a one-node plane at lo+(hi-lo)/2,
 *                 low half, high half, then the plane; stop at <= leaf_rows rows or
 *                 an extent below 3; lexicographic (x fastest) inside a part.  With
 *                 colours C >= 2 a plane of R rows cut across axis a becomes m =
 *                 ceil(R / leaf_rows) even strips of its lexicographic order, each a
 *                 part, each reordered by a stable sort on the key (u mod C) +
 *                 C (v mod C), u < v the other two axes' coordinates (the paper
 *                 leaves the order inside a separator to Scotch).  With
 *                 leaf_colours C >= 2 a leaf box is sorted the same way by the key
 *                 (x mod C) + C (y mod C) + C^2 (z mod C).
 *   orc_ic_create symmetric reordering B = P^T A P (Algorithm 1, step 2) and the
 *                 level-k fill pattern (Algorithm 1, step 4).  Levels follow the
 *                 definition in the Section 1 footnote: original entries have level
 *                 0, and eliminating pivot j gives entry (i,m) the level
 *                 lev(i,j) + lev(m,j) + 1; entries above k are never created.  This is
 *                 the classic row-by-row (IKJ) symbolic pass, a different algorithm
 *                 from the per-row breadth-first search the library uses.
 *   orc_ic_numeric
 *                 the numeric phase (Section 3.3): the unique L with the pattern S,
 *                 positive diagonal and (L L^T)_ij = B_ij on S, computed row by row
 *                 (up-looking IKJ).  Updates that fall outside S are discarded.  Each
 *                 entry receives its updates in ascending pivot order, one multiply
 *                 and one subtract at a time (compile with -ffp-contract=off).
 *                 A pivot that is <= 0 or not finite is a breakdown at that row.
 *   orc_ic_apply  z = (L L^T)^{-1} r by forward and backward substitution.
 *   orc_pcg       textbook preconditioned conjugate gradients (x0 = 0, stop when
 *                 ||r||_2 / ||b||_2 <= tol); the paper uses IC(k) as the PCG
 *                 preconditioner (Section 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_BREAKDOWN 3
#define ORC_ERR_NOMEM 6
#define ORC_ERR_NOCONV 7

/* ------------------------------------------------------------------ ND */

typedef struct {
    int nx, ny, nz, dof, leaf_rows;
    int colours;      /* separator planes sorted by C x C colour key when >= 2 */
    int leaf_colours; /* leaf boxes sorted by C x C x C colour key when >= 2 */
    const uint8_t* keep;
    const int64_t* full_of; /* kept index -> grid dof index (colours >= 2 only) */
    int failed;             /* an allocation failed */
    int32_t* perm;
    int64_t next;    /* next new index */
    int64_t* ranges; /* boundaries of the ordered parts, may be NULL */
    int64_t nranges;
} nd_state;

static int64_t box_rows(const nd_state* s, const int lo[3], const int hi[3]) {
    if (!s->keep)
        return (int64_t)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]) * s->dof;
    int64_t c = 0;
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x) {
                int64_t node = x + (int64_t)s->nx * (y + (int64_t)s->ny * z);
                for (int d = 0; d < s->dof; ++d) c += s->keep[node * s->dof + d] ? 1 : 0;
            }
    return c;
}

/* Number the kept dofs of a box lexicographically (x fastest), node-major. */
static void emit_box(nd_state* s, const int lo[3], const int hi[3], int64_t* old2new) {
    int64_t start = s->next;
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x) {
                int64_t node = x + (int64_t)s->nx * (y + (int64_t)s->ny * z);
                for (int d = 0; d < s->dof; ++d) {
                    int64_t full = node * s->dof + d;
                    if (s->keep && !s->keep[full]) continue;
                    s->perm[s->next++] = (int32_t)old2new[full];
                }
            }
    if (s->next > start && s->ranges) s->ranges[++s->nranges] = s->next;
}

/* Stable counting sort of the rows perm[first..last) by the colour key of their grid
 * node: for a separator plane cut across axis ax, (u mod C) + C (v mod C) with u < v the
 * other two axes and C = colours; for a leaf box (ax < 0), (x mod C) + C (y mod C) +
 * C^2 (z mod C) with C = leaf_colours. */
static void colour_sort(nd_state* s, int64_t first, int64_t last, int ax) {
    const int C = ax >= 0 ? s->colours : s->leaf_colours;
    const int nkeys = ax >= 0 ? C * C : C * C * C;
    const int u_ax = ax == 0 ? 1 : 0, v_ax = ax == 2 ? 1 : 2;
    const int64_t m = last - first;
    if (m <= 1) return;
    int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * m);
    int* key = (int*)malloc(sizeof(int) * m);
    int64_t* count = (int64_t*)calloc((size_t)nkeys + 1, sizeof(int64_t));
    if (!tmp || !key || !count) {
        s->failed = 1;
    } else {
        for (int64_t r = 0; r < m; ++r) {
            int64_t node = s->full_of[s->perm[first + r]] / s->dof;
            int q[3];
            q[0] = (int)(node % s->nx);
            q[1] = (int)((node / s->nx) % s->ny);
            q[2] = (int)(node / ((int64_t)s->nx * s->ny));
            if (ax >= 0)
                key[r] = q[u_ax] % C + C * (q[v_ax] % C);
            else
                key[r] = q[0] % C + C * (q[1] % C) + C * C * (q[2] % C);
            count[key[r] + 1]++;
        }
        for (int k = 0; k < nkeys; ++k) count[k + 1] += count[k];
        for (int64_t r = 0; r < m; ++r) tmp[count[key[r]]++] = s->perm[first + r];
        memcpy(s->perm + first, tmp, sizeof(int32_t) * m);
    }
    free(count);
    free(key);
    free(tmp);
}

static void nd_rec(nd_state* s, const int lo[3], const int hi[3], int64_t* old2new) {
    int ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
    if (ext[0] <= 0 || ext[1] <= 0 || ext[2] <= 0) return;
    int ax = 0;
    if (ext[1] > ext[ax]) ax = 1;
    if (ext[2] > ext[ax]) ax = 2;
    if (box_rows(s, lo, hi) <= s->leaf_rows || ext[ax] < 3) {
        int64_t first = s->next;
        emit_box(s, lo, hi, old2new);
        if (s->leaf_colours >= 2) colour_sort(s, first, s->next, -1);
        return;
    }
    int m = lo[ax] + (hi[ax] - lo[ax]) / 2;
    int lo1[3] = {lo[0], lo[1], lo[2]}, hi1[3] = {hi[0], hi[1], hi[2]};
    int lo2[3] = {lo[0], lo[1], lo[2]}, hi2[3] = {hi[0], hi[1], hi[2]};
    int los[3] = {lo[0], lo[1], lo[2]}, his[3] = {hi[0], hi[1], hi[2]};
    hi1[ax] = m;
    lo2[ax] = m + 1;
    los[ax] = m;
    his[ax] = m + 1;
    nd_rec(s, lo1, hi1, old2new);
    nd_rec(s, lo2, hi2, old2new);
    int64_t first = s->next;
    emit_box(s, los, his, old2new);
    if (s->colours >= 2 && s->next > first) {
        /* the plane's one range becomes m even strips, each sorted by colour key */
        int64_t rows = s->next - first;
        int64_t m = (rows + s->leaf_rows - 1) / s->leaf_rows;
        s->nranges--;
        for (int64_t q = 0; q < m; ++q) {
            int64_t lo_q = first + rows * q / m, hi_q = first + rows * (q + 1) / m;
            colour_sort(s, lo_q, hi_q, ax);
            if (s->ranges) s->ranges[++s->nranges] = hi_q;
        }
    }
}

/* perm[new] = old (index into the kept dofs, in grid order).  ranges (optional, size
 * >= n+1) receives 0 followed by the end of every ordered part.  Returns n. */
int64_t orc_nd_grid(int nx, int ny, int nz, int dof, int leaf_rows, int colours, int leaf_colours,
                    const uint8_t* keep, int32_t* perm, int64_t* ranges, int64_t* nranges) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || dof <= 0 || leaf_rows <= 0 || colours < 0 || leaf_colours < 0)
        return -1;
    int64_t nfull = (int64_t)nx * ny * nz * dof;
    int64_t* old2new = (int64_t*)malloc(sizeof(int64_t) * nfull);
    if (!old2new) return -1;
    const int any_colours = colours >= 2 || leaf_colours >= 2;
    int64_t* full_of = any_colours ? (int64_t*)malloc(sizeof(int64_t) * nfull) : NULL;
    if (any_colours && !full_of) {
        free(old2new);
        return -1;
    }
    int64_t c = 0;
    for (int64_t i = 0; i < nfull; ++i) {
        old2new[i] = (!keep || keep[i]) ? c : -1;
        if (!keep || keep[i]) {
            if (full_of) full_of[c] = i;
            ++c;
        }
    }
    nd_state s = {nx, ny, nz, dof, leaf_rows, colours, leaf_colours, keep, full_of, 0, perm, 0, ranges, 0};
    if (ranges) ranges[0] = 0;
    int lo[3] = {0, 0, 0}, hi[3] = {nx, ny, nz};
    nd_rec(&s, lo, hi, old2new);
    free(full_of);
    free(old2new);
    if (s.failed) return -1;
    if (nranges) *nranges = s.nranges;
    return s.next;
}

/* ------------------------------------------------------------ IC(k) */

typedef struct {
    int64_t n;
    int k;
    int32_t* perm;
    int32_t* iperm;
    /* lower triangle of B = P^T A P, rows sorted, diagonal included */
    int64_t* bptr;
    int32_t* bcol;
    int64_t* bsrc; /* index of the value in A's CSR */
    /* L in row form: entries of row i sorted, diagonal last */
    int64_t* lptr;
    int32_t* lcol;
    int32_t* llev;
    double* lval;
    /* column lists of L: for entry e (row i, col j), next entry of column j */
    int64_t* colhead;
    int64_t* colnext;
    int64_t* erow;
    int64_t nnz;
    double flops;
} orc_ic;

static void* xmalloc(size_t b) { return malloc(b ? b : 1); }

void orc_ic_free(orc_ic* h) {
    if (!h) return;
    free(h->perm); free(h->iperm); free(h->bptr); free(h->bcol); free(h->bsrc);
    free(h->lptr); free(h->lcol); free(h->llev); free(h->lval);
    free(h->colhead); free(h->colnext); free(h->erow);
    free(h);
}

/* Build the permuted lower triangle of B. */
static int build_b(orc_ic* h, const int64_t* rowptr, const int32_t* colind) {
    int64_t n = h->n;
    h->bptr = (int64_t*)xmalloc(sizeof(int64_t) * (n + 1));
    if (!h->bptr) return ORC_ERR_NOMEM;
    h->bptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = h->perm[i], c = 0;
        for (int64_t e = rowptr[o]; e < rowptr[o + 1]; ++e) {
            int32_t oc = colind[e];
            if (oc < 0 || oc >= n) return ORC_ERR_ARG;
            if (h->iperm[oc] <= i) ++c;
        }
        h->bptr[i + 1] = h->bptr[i] + c;
    }
    int64_t nb = h->bptr[n];
    h->bcol = (int32_t*)xmalloc(sizeof(int32_t) * nb);
    h->bsrc = (int64_t*)xmalloc(sizeof(int64_t) * nb);
    if (!h->bcol || !h->bsrc) return ORC_ERR_NOMEM;
    for (int64_t i = 0; i < n; ++i) {
        int64_t o = h->perm[i], p = h->bptr[i];
        for (int64_t e = rowptr[o]; e < rowptr[o + 1]; ++e) {
            int32_t j = h->iperm[colind[e]];
            if (j <= i) { h->bcol[p] = j; h->bsrc[p] = e; ++p; }
        }
        /* insertion sort of the row by column (rows are short) */
        for (int64_t a = h->bptr[i] + 1; a < h->bptr[i + 1]; ++a) {
            int32_t cj = h->bcol[a];
            int64_t cs = h->bsrc[a], b = a - 1;
            while (b >= h->bptr[i] && h->bcol[b] > cj) {
                h->bcol[b + 1] = h->bcol[b]; h->bsrc[b + 1] = h->bsrc[b]; --b;
            }
            h->bcol[b + 1] = cj; h->bsrc[b + 1] = cs;
        }
        for (int64_t a = h->bptr[i] + 1; a < h->bptr[i + 1]; ++a)
            if (h->bcol[a] == h->bcol[a - 1]) return ORC_ERR_ARG; /* duplicate entry */
    }
    return ORC_OK;
}

static int grow(void** p, int64_t* cap, int64_t need, size_t elt) {
    if (need <= *cap) return 0;
    int64_t c = *cap ? *cap : 1024;
    while (c < need) c *= 2;
    void* q = realloc(*p, c * elt);
    if (!q) return -1;
    *p = q;
    *cap = c;
    return 0;
}

/* Level-k symbolic pass, row by row.  For row i the candidate columns j < i are
 * visited in ascending order through a sorted linked list that may grow ahead of
 * the cursor; every entry (m, j) already in column j of L (rows j < m < i) offers
 * lev(i,m) = lev(i,j) + lev(m,j) + 1, kept when it is <= k. */
static int symbolic(orc_ic* h) {
    int64_t n = h->n;
    int k = h->k;
    int32_t* lev = (int32_t*)xmalloc(sizeof(int32_t) * n);
    int64_t* nxt = (int64_t*)xmalloc(sizeof(int64_t) * (n + 1));
    h->lptr = (int64_t*)xmalloc(sizeof(int64_t) * (n + 1));
    h->colhead = (int64_t*)xmalloc(sizeof(int64_t) * n);
    int64_t* coltail = (int64_t*)xmalloc(sizeof(int64_t) * n);
    if (!lev || !nxt || !h->lptr || !h->colhead || !coltail) return ORC_ERR_NOMEM;
    for (int64_t i = 0; i < n; ++i) { lev[i] = INT32_MAX; h->colhead[i] = -1; coltail[i] = -1; }
    int64_t cap = 0, nnz = 0;
    h->lcol = NULL; h->llev = NULL; h->colnext = NULL; h->erow = NULL;
    int64_t cap1 = 0, cap2 = 0, cap3 = 0;
    const int64_t END = n; /* list terminator */
    h->lptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        /* seed the sorted list with the structural entries j < i of row i */
        int64_t head = END, tail = END;
        int has_diag = 0;
        for (int64_t e = h->bptr[i]; e < h->bptr[i + 1]; ++e) {
            int32_t j = h->bcol[e];
            if (j == i) { has_diag = 1; continue; }
            lev[j] = 0;
            if (head == END) head = j; else nxt[tail] = j;
            tail = j;
            nxt[j] = END;
        }
        (void)has_diag; /* the diagonal is always part of the pattern */
        for (int64_t j = head; j != END; j = nxt[j]) {
            int32_t lij = lev[j];
            int64_t ins = j; /* insertion cursor: every new m is > j */
            for (int64_t e = h->colhead[j]; e != -1; e = h->colnext[e]) {
                int64_t m = h->erow[e];
                int32_t nl = lij + h->llev[e] + 1;
                if (nl > k) continue;
                if (lev[m] == INT32_MAX) {
                    while (nxt[ins] != END && nxt[ins] < m) ins = nxt[ins];
                    nxt[m] = nxt[ins];
                    nxt[ins] = m;
                    lev[m] = nl;
                    ins = m;
                } else if (nl < lev[m]) {
                    lev[m] = nl;
                }
            }
        }
        /* write row i: list entries, then the diagonal */
        int64_t cnt = 1;
        for (int64_t j = head; j != END; j = nxt[j]) ++cnt;
        if (grow((void**)&h->lcol, &cap, nnz + cnt, sizeof(int32_t)) ||
            grow((void**)&h->llev, &cap1, nnz + cnt, sizeof(int32_t)) ||
            grow((void**)&h->colnext, &cap2, nnz + cnt, sizeof(int64_t)) ||
            grow((void**)&h->erow, &cap3, nnz + cnt, sizeof(int64_t)))
            return ORC_ERR_NOMEM;
        for (int64_t j = head; j != END;) {
            int64_t nj = nxt[j];
            h->lcol[nnz] = (int32_t)j;
            h->llev[nnz] = lev[j];
            h->erow[nnz] = i;
            h->colnext[nnz] = -1;
            if (coltail[j] == -1) h->colhead[j] = nnz; else h->colnext[coltail[j]] = nnz;
            coltail[j] = nnz;
            lev[j] = INT32_MAX;
            ++nnz;
            j = nj;
        }
        h->lcol[nnz] = (int32_t)i;
        h->llev[nnz] = 0;
        h->erow[nnz] = i;
        h->colnext[nnz] = -1; /* the diagonal is not part of any column list */
        ++nnz;
        h->lptr[i + 1] = nnz;
    }
    h->nnz = nnz;
    free(lev); free(nxt); free(coltail);
    h->lval = (double*)xmalloc(sizeof(double) * (nnz ? nnz : 1));
    return h->lval ? ORC_OK : ORC_ERR_NOMEM;
}

/* Returns a handle for the permuted matrix and its IC(k) pattern, or NULL. */
orc_ic* orc_ic_create(int64_t n, const int64_t* rowptr, const int32_t* colind, const int32_t* perm,
                      int k, int* status) {
    int st = ORC_ERR_ARG;
    orc_ic* h = NULL;
    if (n < 0 || k < 0 || (n > 0 && (!rowptr || !colind))) goto fail;
    h = (orc_ic*)calloc(1, sizeof(orc_ic));
    if (!h) { st = ORC_ERR_NOMEM; goto fail; }
    h->n = n;
    h->k = k;
    h->perm = (int32_t*)xmalloc(sizeof(int32_t) * n);
    h->iperm = (int32_t*)xmalloc(sizeof(int32_t) * n);
    if (!h->perm || !h->iperm) { st = ORC_ERR_NOMEM; goto fail; }
    for (int64_t i = 0; i < n; ++i) h->iperm[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int32_t o = perm ? perm[i] : (int32_t)i;
        if (o < 0 || o >= n || h->iperm[o] != -1) goto fail;
        h->perm[i] = o;
        h->iperm[o] = (int32_t)i;
    }
    st = build_b(h, rowptr, colind);
    if (st) goto fail;
    st = symbolic(h);
    if (st) goto fail;
    if (status) *status = ORC_OK;
    return h;
fail:
    orc_ic_free(h);
    if (status) *status = st;
    return NULL;
}

int64_t orc_ic_nnz(const orc_ic* h) { return h->nnz; }
double orc_ic_flops(const orc_ic* h) { return h->flops; }

/* Pattern of L (lower, rows sorted, diagonal last) and the level of each entry. */
void orc_ic_pattern(const orc_ic* h, int64_t* lptr, int32_t* lcol, int32_t* llev) {
    memcpy(lptr, h->lptr, sizeof(int64_t) * (h->n + 1));
    memcpy(lcol, h->lcol, sizeof(int32_t) * h->nnz);
    if (llev) memcpy(llev, h->llev, sizeof(int32_t) * h->nnz);
}

void orc_ic_values(const orc_ic* h, double* lval) { memcpy(lval, h->lval, sizeof(double) * h->nnz); }

/* Up-looking numeric IC(k): vals are A's values in A's CSR order.  On breakdown
 * returns ORC_ERR_BREAKDOWN with *brk_row = first failing row (permuted order). */
int orc_ic_numeric(orc_ic* h, const double* vals, double shift_alpha, int64_t* brk_row) {
    int64_t n = h->n;
    double* w = (double*)xmalloc(sizeof(double) * n);
    int64_t* mark = (int64_t*)xmalloc(sizeof(int64_t) * n);
    if (!w || !mark) { free(w); free(mark); return ORC_ERR_NOMEM; }
    for (int64_t i = 0; i < n; ++i) mark[i] = -1;
    double flops = 0.0;
    int st = ORC_OK;
    if (brk_row) *brk_row = -1;
    for (int64_t i = 0; i < n; ++i) {
        /* w := row i of B on S_i, zero on fill */
        for (int64_t e = h->lptr[i]; e < h->lptr[i + 1]; ++e) {
            w[h->lcol[e]] = 0.0;
            mark[h->lcol[e]] = i;
        }
        for (int64_t e = h->bptr[i]; e < h->bptr[i + 1]; ++e) w[h->bcol[e]] = vals[h->bsrc[e]];
        if (shift_alpha != 0.0) w[i] = w[i] + shift_alpha * w[i];
        int64_t dpos = h->lptr[i + 1] - 1;
        for (int64_t e = h->lptr[i]; e < dpos; ++e) {
            int32_t j = h->lcol[e];
            double lij = w[j] / h->lval[h->lptr[j + 1] - 1];
            h->lval[e] = lij;
            flops += 1.0;
            for (int64_t f = h->colhead[j]; f != -1; f = h->colnext[f]) {
                int64_t m = h->erow[f];
                if (m >= i) break; /* column lists are in ascending row order */
                if (mark[m] == i) {
                    double prod = lij * h->lval[f];
                    w[m] = w[m] - prod;
                    flops += 2.0;
                }
            }
            double sq = lij * lij;
            w[i] = w[i] - sq;
            flops += 2.0;
        }
        double d = w[i];
        flops += 1.0;
        if (!(d > 0.0) || !isfinite(d)) {
            if (brk_row) *brk_row = i;
            st = ORC_ERR_BREAKDOWN;
            h->lval[dpos] = NAN;
            break;
        }
        h->lval[dpos] = sqrt(d);
    }
    h->flops = flops;
    free(w);
    free(mark);
    return st;
}

/* z = (L L^T)^{-1} r in the original ordering (r, z of length n; may not alias). */
int orc_ic_apply(const orc_ic* h, const double* r, double* z) {
    int64_t n = h->n;
    double* y = (double*)xmalloc(sizeof(double) * n);
    if (!y) return ORC_ERR_NOMEM;
    for (int64_t i = 0; i < n; ++i) {
        double s = r[h->perm[i]];
        int64_t dpos = h->lptr[i + 1] - 1;
        for (int64_t e = h->lptr[i]; e < dpos; ++e) s = s - h->lval[e] * y[h->lcol[e]];
        y[i] = s / h->lval[dpos];
    }
    /* backward with L^T: column i of L holds L_mi for m > i */
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int64_t f = h->colhead[i]; f != -1; f = h->colnext[f])
            s = s - h->lval[f] * y[h->erow[f]];
        y[i] = s / h->lval[h->lptr[i + 1] - 1];
    }
    for (int64_t i = 0; i < n; ++i) z[h->perm[i]] = y[i];
    free(y);
    return ORC_OK;
}

static void spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* x,
                 double* y) {
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s = s + v[e] * x[ci[e]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
}

/* Preconditioned CG on A x = b with M = L L^T (h may be NULL: M = I).  x0 = 0. */
int orc_pcg(const orc_ic* h, int64_t n, const int64_t* rp, const int32_t* ci, const double* av,
            const double* b, double* x, double tol, int maxit, int* iters, double* relres) {
    double* r = (double*)xmalloc(sizeof(double) * n);
    double* z = (double*)xmalloc(sizeof(double) * n);
    double* p = (double*)xmalloc(sizeof(double) * n);
    double* q = (double*)xmalloc(sizeof(double) * n);
    if (!r || !z || !p || !q) { free(r); free(z); free(p); free(q); return ORC_ERR_NOMEM; }
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
    double bn = sqrt(dot(n, b, b));
    if (bn == 0.0) bn = 1.0;
    if (h) orc_ic_apply(h, r, z); else memcpy(z, r, sizeof(double) * n);
    memcpy(p, z, sizeof(double) * n);
    double rz = dot(n, r, z);
    double rel = sqrt(dot(n, r, r)) / bn;
    int it = 0, st = ORC_ERR_NOCONV;
    if (rel <= tol) st = ORC_OK;
    while (st != ORC_OK && it < maxit) {
        spmv(n, rp, ci, av, p, q);
        double alpha = rz / dot(n, p, q);
        for (int64_t i = 0; i < n; ++i) { x[i] = x[i] + alpha * p[i]; r[i] = r[i] - alpha * q[i]; }
        ++it;
        rel = sqrt(dot(n, r, r)) / bn;
        if (rel <= tol) { st = ORC_OK; break; }
        if (h) orc_ic_apply(h, r, z); else memcpy(z, r, sizeof(double) * n);
        double rz2 = dot(n, r, z);
        double beta = rz2 / rz;
        rz = rz2;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (iters) *iters = it;
    if (relres) *relres = rel;
    free(r); free(z); free(p); free(q);
    return st;
}
