/*
 * oracle.c -- plain CPU oracle for the node-aware parallel SpMV (NAPSpMV).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the
 * benchmark's CPU-baseline leg are the only code that may load this file's
 * library.  The CUDA library never links, includes or calls it, and the two
 * share no code, header, table or helper.
 *
 * Source: A. Bienz, W. D. Gropp, L. N. Olson, "Node aware sparse
 * matrix-vector multiplication" (arXiv 1612.08060).  Every function below
 * follows a definition of the paper, evaluated by plain enumeration:
 *
 *   orc_row_start / orc_owner   Sec. 2, Eqs. R and R_pn (row partition)
 *   strided partition           Sec. 5 (SuiteSparse runs): row i on rank
 *                               i mod n_p (flag ORC_STRIDED)
 *   classification              Sec. 2, Eqs. on_proc, off_proc, on_node,
 *                               off_node
 *   STD list                    Sec. 2.1, Eqs. P and D
 *   NODE list, T/U              Sec. 4.1, Eqs. N, E, T, U and the mapping
 *                               rule stated after Eq. U
 *   INTER list                  Sec. 4.1, Eqs. G and IGset_send (I)
 *   J0 / J1 / J2 lists          Sec. 4.2, Eqs. L0/IL0, L1_send/IL1, L2/IL2
 *   orc_napspmv                 Algorithm "NAPSpMV" with "local_comm",
 *                               every message executed as a copy
 *   orc_spmv                    Sec. 1: w <- A v, plain FP64 row loop
 *   orc_spmv_f32                FP32-stored values, FP32 products summed in
 *                               FP64 (the precision variant of the build)
 *   orc_cg                      plain FP64 conjugate gradients
 *
 * Readings of points the paper leaves open (each is also listed, with its
 * justification, in the design notes of the repository):
 *   - D(r,t) and E(n,m) hold the COLUMN index j owned by the sender (the
 *     equations print the row index i; the paper's tables list j).
 *   - When n_p does not divide N, rank r starts at r*q + min(r, N mod n_p)
 *     with q = floor(N/n_p): the first N mod n_p ranks hold q+1 rows.
 *   - Rank r is (r mod ppn, floor(r/ppn)); the last node may hold fewer
 *     than ppn ranks when ppn does not divide n_p.
 *   - Mapping of node pairs to processes (default, matches the paper's
 *     tables T, U, G): on the sending node n, sort N(n) by |E(n,m)|
 *     descending, ties by m ascending, and give the k-th to local process
 *     k mod P(n); on the receiving node m, sort the senders by |E(n,m)|
 *     ASCENDING, ties by n ascending, and give the k-th to local process
 *     P(m)-1-(k mod P(m)), where P(x) is the number of ranks on node x.
 *     Flag ORC_MAP_TEXT sorts the receiving side by |E| descending, as the
 *     prose states.  Without ORC_MAP_SPLIT a node is never split over several
 *     processes (the tables do not split).
 *   - Flag ORC_MAP_SPLIT (the text after Eq. U: when N(n) holds fewer nodes
 *     than n has processes, a node is mapped to several processes so that
 *     all of them communicate).  On a node x with P(x) processes and K < P(x)
 *     partner nodes (sorted as above), partner k gets a contiguous group of
 *     floor(P/K) + (k < P mod K) processes: on the sending side counted from
 *     process 0 upwards, on the receiving side from process P-1 downwards
 *     (the first partner gets the highest group).  With K >= P(x) each group
 *     is the single process of the default rule.  For the pair (n,m) with
 *     sending group S and receiving group R (ascending), E(n,m) in ascending
 *     j is cut into c = max(|S|,|R|) contiguous pieces, piece i holding
 *     positions floor(i e / c) .. floor((i+1) e / c) - 1 (e = |E(n,m)|);
 *     piece i is sent by S[i mod |S|] to R[i mod |R|]; empty pieces send
 *     nothing.  G and I follow from these messages; T/U report the first
 *     process of each group.  Excludes ORC_MAP_MAJORITY.
 *   - Flag ORC_MAP_MAJORITY (the alternative the text names after Eq. U):
 *     node pair (n,m) is sent by the process of n that owns the most values
 *     of E(n,m), and received by the process of m whose rows use the most
 *     of them; ties go to the lowest local process.
 *   - J(on_node -> off_node) from (p,n) to (s,n) is the set of j owned by
 *     (p,n) that appear in some I((s,n),(q,m)); s != p.
 *   - J(off_node -> on_node) from (q,m) to (s,m) is the set of j received
 *     by (q,m) through any inter-node message that rank s uses; s != q.
 *   - The off_node -> on_node local_comm forwards g_recv (the algorithm
 *     prints v|R there).
 *   - "A_ij != 0" is structural: every stored entry counts.
 *   - A process never sends to itself.
 *   - Ordering: within a message ascending j; messages by (src, dst).
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared (see build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_PLAN (-7) /* a value the algorithm needs was never delivered */

#define ORC_MAP_TEXT 2 /* same bit as the library's flag, chosen independently */
#define ORC_STRIDED 4  /* row i belongs to rank i mod n_p (Sec. 5's strided partition) */
#define ORC_MAP_MAJORITY 8 /* the majority mapping named after Eq. U (see orc_plan_build) */
#define ORC_MAP_SPLIT 16   /* node splitting when a node has fewer partners than processes */

enum { L_STD = 0, L_NODE, L_INTER, L_J0, L_J1, L_J2, L_BLL, L_BNL, L_LBUF, L_COUNT };

typedef struct {
    int64_t m;     /* number of messages (or non-empty per-rank lists)    */
    int64_t total; /* number of indices over all messages                 */
    int64_t *src;  /* [m] sending rank (node id for the NODE list)        */
    int64_t *dst;  /* [m] receiving rank (node id for the NODE list)      */
    int64_t *ptr;  /* [m+1] offsets into idx                              */
    int64_t *idx;  /* [total] global column indices, ascending per message */
} orc_list;

typedef struct {
    int64_t n, np, ppn, nn, flags;
    orc_list l[L_COUNT];
    int64_t *send_proc; /* [NODE.m] local process on the sending node (T)   */
    int64_t *recv_proc; /* [NODE.m] local process on the receiving node (U) */
    int64_t *split;     /* [3n] per row: on_process, on_node, off_node nnz */
} orc_plan;

/* ---------------------------------------------------------------- partition */

/* Eq. R generalised to any n_p <= N (first N mod n_p ranks get one more). */
int64_t orc_row_start(int64_t n, int64_t np, int64_t r)
{
    int64_t q = n / np, rem = n % np;
    return r * q + (r < rem ? r : rem);
}

/* The rank r with row_start(r) <= j < row_start(r+1), by bisection. */
int64_t orc_owner(int64_t n, int64_t np, int64_t j)
{
    int64_t lo = 0, hi = np - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (orc_row_start(n, np, mid) <= j)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

/* The owner of row / column j under the plan's partition. */
static int64_t own(const orc_plan *P, int64_t j)
{
    if (P->flags & ORC_STRIDED) return j % P->np;
    return orc_owner(P->n, P->np, j);
}

static int64_t procs_on_node(const orc_plan *P, int64_t node)
{
    int64_t left = P->np - node * P->ppn;
    return left < P->ppn ? left : P->ppn;
}

/* ------------------------------------------------------------ triple sets */

typedef struct { int64_t a, b, c; } trip;
typedef struct { trip *v; int64_t n, cap; } tvec;

static int tpush(tvec *t, int64_t a, int64_t b, int64_t c)
{
    if (t->n == t->cap) {
        int64_t cap = t->cap ? 2 * t->cap : 1024;
        trip *nv = (trip *)realloc(t->v, (size_t)cap * sizeof(trip));
        if (!nv) return ORC_ERR_OOM;
        t->v = nv;
        t->cap = cap;
    }
    t->v[t->n].a = a;
    t->v[t->n].b = b;
    t->v[t->n].c = c;
    t->n++;
    return ORC_OK;
}

static int tcmp(const void *x, const void *y)
{
    const trip *p = (const trip *)x, *q = (const trip *)y;
    if (p->a != q->a) return p->a < q->a ? -1 : 1;
    if (p->b != q->b) return p->b < q->b ? -1 : 1;
    if (p->c != q->c) return p->c < q->c ? -1 : 1;
    return 0;
}

/* Sort and drop repeats: the triples become a set. */
static void tset(tvec *t)
{
    if (t->n == 0) return;
    qsort(t->v, (size_t)t->n, sizeof(trip), tcmp);
    int64_t w = 1;
    for (int64_t i = 1; i < t->n; i++)
        if (tcmp(&t->v[i], &t->v[w - 1]) != 0) t->v[w++] = t->v[i];
    t->n = w;
}

/* A sorted set of (src, dst, j) triples becomes a message list. */
static int tlist(const tvec *t, orc_list *L)
{
    int64_t m = 0;
    for (int64_t i = 0; i < t->n; i++)
        if (i == 0 || t->v[i].a != t->v[i - 1].a || t->v[i].b != t->v[i - 1].b) m++;
    L->m = m;
    L->total = t->n;
    L->src = (int64_t *)calloc((size_t)(m ? m : 1), sizeof(int64_t));
    L->dst = (int64_t *)calloc((size_t)(m ? m : 1), sizeof(int64_t));
    L->ptr = (int64_t *)calloc((size_t)(m + 1), sizeof(int64_t));
    L->idx = (int64_t *)calloc((size_t)(t->n ? t->n : 1), sizeof(int64_t));
    if (!L->src || !L->dst || !L->ptr || !L->idx) return ORC_ERR_OOM;
    int64_t k = -1;
    for (int64_t i = 0; i < t->n; i++) {
        if (i == 0 || t->v[i].a != t->v[i - 1].a || t->v[i].b != t->v[i - 1].b) {
            k++;
            L->src[k] = t->v[i].a;
            L->dst[k] = t->v[i].b;
            L->ptr[k] = i;
        }
        L->idx[i] = t->v[i].c;
    }
    L->ptr[m] = t->n;
    return ORC_OK;
}

static void lfree(orc_list *L)
{
    free(L->src);
    free(L->dst);
    free(L->ptr);
    free(L->idx);
    memset(L, 0, sizeof(*L));
}

/* Position of j inside message k of L (ascending idx), or -1. */
static int64_t lfind(const orc_list *L, int64_t k, int64_t j)
{
    int64_t lo = L->ptr[k], hi = L->ptr[k + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (L->idx[mid] == j) return mid;
        if (L->idx[mid] < j)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

/* Message of a per-rank list (BLL, BNL, LBUF) that belongs to rank r, or -1. */
static int64_t lrank(const orc_list *L, int64_t r)
{
    int64_t lo = 0, hi = L->m - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (L->src[mid] == r) return mid;
        if (L->src[mid] < r)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

/* ---------------------------------------------------------- plan building */

typedef struct { int64_t len, other, msg; } tu_entry;
static int tu_desc(const void *x, const void *y)
{
    const tu_entry *p = (const tu_entry *)x, *q = (const tu_entry *)y;
    if (p->len != q->len) return p->len > q->len ? -1 : 1;
    return p->other < q->other ? -1 : (p->other > q->other);
}
static int tu_asc(const void *x, const void *y)
{
    const tu_entry *p = (const tu_entry *)x, *q = (const tu_entry *)y;
    if (p->len != q->len) return p->len < q->len ? -1 : 1;
    return p->other < q->other ? -1 : (p->other > q->other);
}

void orc_plan_free(orc_plan *P)
{
    if (!P) return;
    for (int i = 0; i < L_COUNT; i++) lfree(&P->l[i]);
    free(P->send_proc);
    free(P->recv_proc);
    free(P->split);
    free(P);
}

/* Checks of the CSR input: row_ptr starts at 0, never decreases and ends at
 * nnz; every column lies in [0, n); no (i, j) is stored twice. */
static int check_csr(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col)
{
    if (n < 1 || nnz < 0 || !rp || (nnz > 0 && !col)) return ORC_ERR_ARG;
    if (rp[0] != 0 || rp[n] != nnz) return ORC_ERR_ARG;
    for (int64_t i = 0; i < n; i++) {
        if (rp[i + 1] < rp[i]) return ORC_ERR_ARG;
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
            if (col[k] < 0 || col[k] >= n) return ORC_ERR_ARG;
            for (int64_t q = rp[i]; q < k; q++)
                if (col[q] == col[k]) return ORC_ERR_ARG;
        }
    }
    return ORC_OK;
}

int orc_plan_build(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                   int64_t np, int64_t ppn, int64_t flags, orc_plan **out)
{
    int rc = ORC_OK;
    *out = NULL;
    if (np < 1 || np > n || ppn < 1) return ORC_ERR_ARG;
    /* unknown bits are refused, not ignored: a caller's flag from another
     * numbering must not silently select the default mapping */
    if (flags & ~(int64_t)(ORC_MAP_TEXT | ORC_STRIDED | ORC_MAP_MAJORITY | ORC_MAP_SPLIT))
        return ORC_ERR_ARG;
    if ((flags & ORC_MAP_MAJORITY) && (flags & (ORC_MAP_TEXT | ORC_MAP_SPLIT))) return ORC_ERR_ARG;
    rc = check_csr(n, nnz, row_ptr, col);
    if (rc) return rc;

    orc_plan *P = (orc_plan *)calloc(1, sizeof(orc_plan));
    if (!P) return ORC_ERR_OOM;
    P->n = n;
    P->np = np;
    P->ppn = ppn;
    P->nn = (np + ppn - 1) / ppn;
    P->flags = flags;
    P->split = (int64_t *)calloc((size_t)(3 * n), sizeof(int64_t));
    tvec std_ = {0}, node = {0}, j2 = {0}, bll = {0}, bnl = {0}, inter = {0}, j0 = {0},
         lbuf = {0}, j1 = {0};
    if (!P->split) { rc = ORC_ERR_OOM; goto done; }

    /* Eqs. on_proc / on_node / off_node: every stored A_ij of row i in R(t)
     * with column j in R(r).  Off-process entries define P and D (Eqs. P,
     * D); on-node ones define L2/J2 (Eqs. L2, IL2) and the on-node receive
     * set of t; off-node ones define N and E (Eqs. N, E) and the off-node
     * receive set of t. */
    for (int64_t i = 0; i < n; i++) {
        int64_t t = own(P, i);
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
            int64_t j = col[k];
            int64_t r = own(P, j);
            if (r == t) {
                P->split[3 * i + 0]++;
            } else if (r / ppn == t / ppn) {
                P->split[3 * i + 1]++;
                if (tpush(&std_, r, t, j) || tpush(&j2, r, t, j) || tpush(&bll, t, t, j)) {
                    rc = ORC_ERR_OOM;
                    goto done;
                }
            } else {
                P->split[3 * i + 2]++;
                if (tpush(&std_, r, t, j) || tpush(&node, r / ppn, t / ppn, j) ||
                    tpush(&bnl, t, t, j)) {
                    rc = ORC_ERR_OOM;
                    goto done;
                }
            }
        }
    }
    tset(&std_);
    tset(&node);
    tset(&j2);
    tset(&bll);
    tset(&bnl);
    if ((rc = tlist(&std_, &P->l[L_STD])) || (rc = tlist(&node, &P->l[L_NODE])) ||
        (rc = tlist(&j2, &P->l[L_J2])) || (rc = tlist(&bll, &P->l[L_BLL])) ||
        (rc = tlist(&bnl, &P->l[L_BNL])))
        goto done;

    /* T and U (Eqs. T, U and the mapping rule after them). */
    {
        orc_list *N = &P->l[L_NODE];
        int64_t m = N->m;
        P->send_proc = (int64_t *)calloc((size_t)(m ? m : 1), sizeof(int64_t));
        P->recv_proc = (int64_t *)calloc((size_t)(m ? m : 1), sizeof(int64_t));
        /* group sizes (1 unless the pair's node is split, ORC_MAP_SPLIT) */
        int64_t *send_cnt = (int64_t *)calloc((size_t)(m ? m : 1), sizeof(int64_t));
        int64_t *recv_cnt = (int64_t *)calloc((size_t)(m ? m : 1), sizeof(int64_t));
        tu_entry *e = (tu_entry *)calloc((size_t)(m ? m : 1), sizeof(tu_entry));
        if (!P->send_proc || !P->recv_proc || !send_cnt || !recv_cnt || !e) {
            free(e);
            free(send_cnt);
            free(recv_cnt);
            rc = ORC_ERR_OOM;
            goto done;
        }
        for (int64_t k = 0; k < m; k++) send_cnt[k] = recv_cnt[k] = 1;
        if (flags & ORC_MAP_MAJORITY) {
            /* per node pair, count the values of E(n,m) each process of n owns
             * and the values each process of m uses, and take the largest */
            const orc_list *BN = &P->l[L_BNL];
            for (int64_t k = 0; k < m; k++) {
                int64_t sn = N->src[k], dn = N->dst[k];
                int64_t best = -1, arg = 0;
                for (int64_t p = 0; p < procs_on_node(P, sn); p++) {
                    int64_t c = 0;
                    for (int64_t q = N->ptr[k]; q < N->ptr[k + 1]; q++)
                        if (own(P, N->idx[q]) == sn * ppn + p) c++;
                    if (c > best) { best = c; arg = p; }
                }
                P->send_proc[k] = arg;
                best = -1;
                arg = 0;
                for (int64_t p = 0; p < procs_on_node(P, dn); p++) {
                    int64_t c = 0, bs = lrank(BN, dn * ppn + p);
                    if (bs >= 0)
                        for (int64_t q = N->ptr[k]; q < N->ptr[k + 1]; q++)
                            if (lfind(BN, bs, N->idx[q]) >= 0) c++;
                    if (c > best) { best = c; arg = p; }
                }
                P->recv_proc[k] = arg;
            }
        } else {
            for (int64_t nd = 0; nd < P->nn; nd++) {
                /* sending side: the nodes of N(nd) */
                int64_t c = 0;
                for (int64_t k = 0; k < m; k++)
                    if (N->src[k] == nd) {
                        e[c].len = N->ptr[k + 1] - N->ptr[k];
                        e[c].other = N->dst[k];
                        e[c].msg = k;
                        c++;
                    }
                qsort(e, (size_t)c, sizeof(tu_entry), tu_desc);
                int64_t pn = procs_on_node(P, nd);
                if ((flags & ORC_MAP_SPLIT) && c < pn) {
                    /* partner k: processes first .. first + size - 1, upwards */
                    int64_t first = 0;
                    for (int64_t k = 0; k < c; k++) {
                        int64_t size = pn / c + (k < pn % c ? 1 : 0);
                        P->send_proc[e[k].msg] = first;
                        send_cnt[e[k].msg] = size;
                        first += size;
                    }
                } else {
                    for (int64_t k = 0; k < c; k++) P->send_proc[e[k].msg] = k % pn;
                }
                /* receiving side: the nodes that have nd in their N(.) */
                c = 0;
                for (int64_t k = 0; k < m; k++)
                    if (N->dst[k] == nd) {
                        e[c].len = N->ptr[k + 1] - N->ptr[k];
                        e[c].other = N->src[k];
                        e[c].msg = k;
                        c++;
                    }
                qsort(e, (size_t)c, sizeof(tu_entry), (flags & ORC_MAP_TEXT) ? tu_desc : tu_asc);
                if ((flags & ORC_MAP_SPLIT) && c < pn) {
                    /* partner k: the group below the earlier partners' groups,
                     * counted down from process pn - 1 */
                    int64_t top = pn;
                    for (int64_t k = 0; k < c; k++) {
                        int64_t size = pn / c + (k < pn % c ? 1 : 0);
                        P->recv_proc[e[k].msg] = top - size;
                        recv_cnt[e[k].msg] = size;
                        top -= size;
                    }
                } else {
                    for (int64_t k = 0; k < c; k++) P->recv_proc[e[k].msg] = pn - 1 - (k % pn);
                }
            }
        }
        free(e);

        /* G and I (Eqs. G, IGset_send): one message per node pair, from the
         * process T assigns on n to the process U assigns on m, carrying
         * E(n,m); with ORC_MAP_SPLIT, piece i of E(n,m) from the i-th process
         * of the sending group to the i-th of the receiving group (cyclic). */
        for (int64_t k = 0; k < m; k++) {
            int64_t ns = send_cnt[k], nr = recv_cnt[k];
            int64_t c = ns > nr ? ns : nr, len = N->ptr[k + 1] - N->ptr[k];
            for (int64_t i = 0; i < c; i++) {
                int64_t s = N->src[k] * ppn + P->send_proc[k] + i % ns;
                int64_t d = N->dst[k] * ppn + P->recv_proc[k] + i % nr;
                int64_t lo = i * len / c, hi = (i + 1) * len / c;
                for (int64_t q = N->ptr[k] + lo; q < N->ptr[k] + hi; q++)
                    if (tpush(&inter, s, d, N->idx[q])) {
                        free(send_cnt);
                        free(recv_cnt);
                        rc = ORC_ERR_OOM;
                        goto done;
                    }
            }
        }
        free(send_cnt);
        free(recv_cnt);
        tset(&inter);
        if ((rc = tlist(&inter, &P->l[L_INTER]))) goto done;
    }

    /* J(on_node -> off_node) (Eqs. L0, IL0): every j the aggregator s sends
     * off-node but does not own comes from its owner p on the same node. */
    {
        orc_list *I = &P->l[L_INTER];
        for (int64_t k = 0; k < I->m; k++) {
            int64_t s = I->src[k];
            for (int64_t q = I->ptr[k]; q < I->ptr[k + 1]; q++) {
                int64_t j = I->idx[q];
                int64_t p = own(P, j);
                if (p != s && (tpush(&j0, p, s, j) || tpush(&lbuf, s, s, j))) {
                    rc = ORC_ERR_OOM;
                    goto done;
                }
            }
        }
        tset(&j0);
        tset(&lbuf);
        if ((rc = tlist(&j0, &P->l[L_J0])) || (rc = tlist(&lbuf, &P->l[L_LBUF]))) goto done;

        /* J(off_node -> on_node) (Eqs. L1_send, IL1): the receiver q forwards
         * each received j to every other rank s of its node whose rows use
         * j.  "Rows of s use j" is membership of j in the off-node receive
         * set of s (j lies on another node, so it is off-node for s). */
        orc_list *B = &P->l[L_BNL];
        for (int64_t k = 0; k < I->m; k++) {
            int64_t q = I->dst[k], m = q / ppn;
            for (int64_t s = m * ppn; s < m * ppn + procs_on_node(P, m); s++) {
                if (s == q) continue;
                int64_t bs = lrank(B, s);
                if (bs < 0) continue;
                for (int64_t x = I->ptr[k]; x < I->ptr[k + 1]; x++)
                    if (lfind(B, bs, I->idx[x]) >= 0 && tpush(&j1, q, s, I->idx[x])) {
                        rc = ORC_ERR_OOM;
                        goto done;
                    }
            }
        }
        tset(&j1);
        if ((rc = tlist(&j1, &P->l[L_J1]))) goto done;
    }

done:
    free(std_.v);
    free(node.v);
    free(j2.v);
    free(bll.v);
    free(bnl.v);
    free(inter.v);
    free(j0.v);
    free(lbuf.v);
    free(j1.v);
    if (rc) {
        orc_plan_free(P);
        return rc;
    }
    *out = P;
    return ORC_OK;
}

/* --------------------------------------------------------------- accessors */

const orc_list *orc_plan_list(const orc_plan *P, int which)
{
    if (!P || which < 0 || which >= L_COUNT) return NULL;
    return &P->l[which];
}
const int64_t *orc_plan_send_proc(const orc_plan *P) { return P->send_proc; }
const int64_t *orc_plan_recv_proc(const orc_plan *P) { return P->recv_proc; }
const int64_t *orc_plan_split(const orc_plan *P) { return P->split; }

/* ------------------------------------------------------------------ stats */

/* Totals and per-process maxima (over sending processes) of message counts
 * and sizes in values, for the standard plan (P, D) and for the node-aware
 * plan (inter-node: I; intra-node: J0 + J1 + J2).  Layout of out[33]:
 *  0 std_msgs  1 std_vals  2 std_intra_msgs  3 std_intra_vals
 *  4 std_inter_msgs  5 std_inter_vals  6 std_max_inter_msgs_proc
 *  7 std_max_inter_vals_proc  8 std_max_intra_msgs_proc
 *  9 std_max_intra_vals_proc  10 std_max_msg_vals
 * 11 nap_inter_msgs  12 nap_inter_vals  13 j0_msgs  14 j0_vals
 * 15 j1_msgs  16 j1_vals  17 j2_msgs  18 j2_vals  19 nap_intra_msgs
 * 20 nap_intra_vals  21 nap_max_inter_msgs_proc  22 nap_max_inter_vals_proc
 * 23 nap_max_intra_msgs_proc  24 nap_max_intra_vals_proc
 * 25 nap_max_inter_msg_vals  26 node_pairs  27 bll_total  28 bnl_total
 * 29 lbuf_total  30 nnz_on_process  31 nnz_on_node  32 nnz_off_node */
void orc_plan_stats(const orc_plan *P, int64_t *out)
{
    memset(out, 0, 33 * sizeof(int64_t));
    int64_t np = P->np, ppn = P->ppn;
    int64_t *a = (int64_t *)calloc((size_t)(4 * np), sizeof(int64_t));
    int64_t *b = (int64_t *)calloc((size_t)(4 * np), sizeof(int64_t));
    const orc_list *S = &P->l[L_STD];
    for (int64_t k = 0; k < S->m; k++) {
        int64_t len = S->ptr[k + 1] - S->ptr[k];
        int inter = (S->src[k] / ppn) != (S->dst[k] / ppn);
        out[0]++;
        out[1] += len;
        out[inter ? 4 : 2]++;
        out[inter ? 5 : 3] += len;
        if (len > out[10]) out[10] = len;
        a[4 * S->src[k] + (inter ? 0 : 2)]++;
        a[4 * S->src[k] + (inter ? 1 : 3)] += len;
    }
    const orc_list *I = &P->l[L_INTER];
    for (int64_t k = 0; k < I->m; k++) {
        int64_t len = I->ptr[k + 1] - I->ptr[k];
        out[11]++;
        out[12] += len;
        if (len > out[25]) out[25] = len;
        b[4 * I->src[k] + 0]++;
        b[4 * I->src[k] + 1] += len;
    }
    const int lj[3] = {L_J0, L_J1, L_J2};
    for (int q = 0; q < 3; q++) {
        const orc_list *J = &P->l[lj[q]];
        for (int64_t k = 0; k < J->m; k++) {
            int64_t len = J->ptr[k + 1] - J->ptr[k];
            out[13 + 2 * q]++;
            out[14 + 2 * q] += len;
            b[4 * J->src[k] + 2]++;
            b[4 * J->src[k] + 3] += len;
        }
    }
    out[19] = out[13] + out[15] + out[17];
    out[20] = out[14] + out[16] + out[18];
    for (int64_t r = 0; r < np; r++) {
        for (int q = 0; q < 4; q++) {
            if (a[4 * r + q] > out[6 + q]) out[6 + q] = a[4 * r + q];
            if (b[4 * r + q] > out[21 + q]) out[21 + q] = b[4 * r + q];
        }
    }
    out[26] = P->l[L_NODE].m;
    out[27] = P->l[L_BLL].total;
    out[28] = P->l[L_BNL].total;
    out[29] = P->l[L_LBUF].total;
    for (int64_t i = 0; i < P->n; i++) {
        out[30] += P->split[3 * i];
        out[31] += P->split[3 * i + 1];
        out[32] += P->split[3 * i + 2];
    }
    free(a);
    free(b);
}

/* --------------------------------------------------------------- products */

/* Sec. 1: w_i = sum_j A_ij v_j, rows in order, stored column order, FP64. */
void orc_spmv(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
              const double *v, double *w)
{
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) s += val[k] * v[col[k]];
        w[i] = s;
    }
}

/* FP32-stored values: each product is rounded to FP32 (value and v_j both
 * in FP32), and the products are summed in FP64, in stored order. */
void orc_spmv_f32(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *val,
                  const double *v, double *w)
{
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
            float x = (float)v[col[k]];
            float p = val[k] * x;
            s += (double)p;
        }
        w[i] = s;
    }
}

/* Algorithm NAPSpMV for every rank, each message a copy between per-rank
 * buffers: on->on and on->off local_comm, the inter-node exchange of g_send
 * into g_recv, the off->on local_comm from g_recv, then local_spmv over the
 * on_process, on_node and off_node blocks, accumulated into w in that
 * order.  Every received value starts as NaN; a value that is used but was
 * never delivered makes the call fail with ORC_ERR_PLAN. */
int orc_napspmv(const orc_plan *P, const int64_t *row_ptr, const int32_t *col,
                const double *val, const double *v, double *w)
{
    int64_t n = P->n, np = P->np;
    const orc_list *BL = &P->l[L_BLL], *BN = &P->l[L_BNL], *LB = &P->l[L_LBUF];
    const orc_list *I = &P->l[L_INTER];
    double *bll = (double *)malloc((size_t)(BL->total + 1) * sizeof(double));
    double *bnl = (double *)malloc((size_t)(BN->total + 1) * sizeof(double));
    double *lbf = (double *)malloc((size_t)(LB->total + 1) * sizeof(double));
    double *grecv = (double *)malloc((size_t)(I->total + 1) * sizeof(double));
    int rc = ORC_OK;
    if (!bll || !bnl || !lbf || !grecv) { rc = ORC_ERR_OOM; goto out; }
    for (int64_t k = 0; k < BL->total; k++) bll[k] = NAN;
    for (int64_t k = 0; k < BN->total; k++) bnl[k] = NAN;
    for (int64_t k = 0; k < LB->total; k++) lbf[k] = NAN;
    for (int64_t k = 0; k < I->total; k++) grecv[k] = NAN;

    /* local_comm(on_node -> on_node): b_{l->l} of s receives v_j from p. */
    const orc_list *J2 = &P->l[L_J2];
    for (int64_t k = 0; k < J2->m; k++) {
        int64_t p = J2->src[k], s = J2->dst[k], bs = lrank(BL, s);
        for (int64_t x = J2->ptr[k]; x < J2->ptr[k + 1]; x++) {
            int64_t j = J2->idx[x];
            int64_t pos = bs < 0 ? -1 : lfind(BL, bs, j);
            if (pos < 0 || own(P, j) != p) { rc = ORC_ERR_PLAN; goto out; }
            bll[pos] = v[j];
        }
    }
    /* local_comm(on_node -> off_node): b_{l->nl} of aggregator s. */
    const orc_list *J0 = &P->l[L_J0];
    for (int64_t k = 0; k < J0->m; k++) {
        int64_t p = J0->src[k], s = J0->dst[k], bs = lrank(LB, s);
        for (int64_t x = J0->ptr[k]; x < J0->ptr[k + 1]; x++) {
            int64_t j = J0->idx[x];
            int64_t pos = bs < 0 ? -1 : lfind(LB, bs, j);
            if (pos < 0 || own(P, j) != p) { rc = ORC_ERR_PLAN; goto out; }
            lbf[pos] = v[j];
        }
    }
    /* Inter-node step: g_send packed from v (own values) or b_{l->nl},
     * delivered into g_recv of the destination. */
    for (int64_t k = 0; k < I->m; k++) {
        int64_t p = I->src[k], bs = lrank(LB, p);
        for (int64_t x = I->ptr[k]; x < I->ptr[k + 1]; x++) {
            int64_t j = I->idx[x];
            double val_j;
            if (own(P, j) == p) {
                val_j = v[j];
            } else {
                int64_t pos = bs < 0 ? -1 : lfind(LB, bs, j);
                if (pos < 0 || isnan(lbf[pos])) { rc = ORC_ERR_PLAN; goto out; }
                val_j = lbf[pos];
            }
            grecv[x] = val_j;
        }
    }
    /* local_comm(off_node -> on_node), forwarding g_recv; the receiver keeps
     * what its own rows use. */
    for (int64_t s = 0; s < np; s++) {
        int64_t bs = lrank(BN, s);
        if (bs < 0) continue;
        for (int64_t x = BN->ptr[bs]; x < BN->ptr[bs + 1]; x++) {
            int64_t j = BN->idx[x];
            /* the inter-node message into a rank of s's node carrying j */
            int64_t found = -1, via = -1;
            for (int64_t k = 0; k < I->m && found < 0; k++) {
                if (I->dst[k] / P->ppn != s / P->ppn) continue;
                int64_t pos = lfind(I, k, j);
                if (pos >= 0) { found = pos; via = I->dst[k]; }
            }
            if (found < 0) { rc = ORC_ERR_PLAN; goto out; }
            if (via != s) {
                /* must travel in a J1 message via -> s */
                int64_t ok = 0;
                const orc_list *J1 = &P->l[L_J1];
                for (int64_t k = 0; k < J1->m && !ok; k++)
                    if (J1->src[k] == via && J1->dst[k] == s && lfind(J1, k, j) >= 0) ok = 1;
                if (!ok) { rc = ORC_ERR_PLAN; goto out; }
            }
            bnl[x] = grecv[found];
        }
    }
    /* local_spmv over the three blocks, accumulated into w. */
    for (int64_t i = 0; i < n; i++) {
        int64_t t = own(P, i);
        int64_t bl = lrank(BL, t), bn = lrank(BN, t);
        double s = 0.0;
        for (int blk = 0; blk < 3; blk++) {
            for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; k++) {
                int64_t j = col[k], r = own(P, j);
                int b = (r == t) ? 0 : (r / P->ppn == t / P->ppn ? 1 : 2);
                if (b != blk) continue;
                double x;
                if (b == 0) {
                    x = v[j];
                } else {
                    const orc_list *L = b == 1 ? BL : BN;
                    int64_t q = b == 1 ? bl : bn;
                    int64_t pos = q < 0 ? -1 : lfind(L, q, j);
                    if (pos < 0) { rc = ORC_ERR_PLAN; goto out; }
                    x = b == 1 ? bll[pos] : bnl[pos];
                    if (isnan(x)) { rc = ORC_ERR_PLAN; goto out; }
                }
                s += val[k] * x;
            }
        }
        w[i] = s;
    }
out:
    free(bll);
    free(bnl);
    free(lbf);
    free(grecv);
    return rc;
}

/* ----------------------------------------------------------------------- CG */

static double dot(int64_t n, const double *x, const double *y)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += x[i] * y[i];
    return s;
}

/* Conjugate gradients in FP64 from the initial guess in x; stops when
 * ||r_k|| / ||b|| <= rtol for the recursively updated residual, or after
 * max_it iterations.  On return *relres is ||b - A x|| / ||b|| recomputed
 * from x. */
int orc_cg(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *val,
           const double *b, double *x, double rtol, int64_t max_it, int64_t *iters,
           double *relres)
{
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *ap = (double *)malloc((size_t)n * sizeof(double));
    if (!r || !p || !ap) {
        free(r);
        free(p);
        free(ap);
        return ORC_ERR_OOM;
    }
    orc_spmv(n, row_ptr, col, val, x, ap);
    for (int64_t i = 0; i < n; i++) {
        r[i] = b[i] - ap[i];
        p[i] = r[i];
    }
    double bn = sqrt(dot(n, b, b));
    if (bn == 0.0) bn = 1.0;
    double rr = dot(n, r, r);
    int64_t it = 0;
    while (it < max_it && sqrt(rr) / bn > rtol) {
        orc_spmv(n, row_ptr, col, val, p, ap);
        double alpha = rr / dot(n, p, ap);
        for (int64_t i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * ap[i];
        }
        double rr2 = dot(n, r, r);
        double beta = rr2 / rr;
        rr = rr2;
        for (int64_t i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        it++;
    }
    orc_spmv(n, row_ptr, col, val, x, ap);
    for (int64_t i = 0; i < n; i++) r[i] = b[i] - ap[i];
    *relres = sqrt(dot(n, r, r)) / bn;
    *iters = it;
    free(r);
    free(p);
    free(ap);
    return ORC_OK;
}
