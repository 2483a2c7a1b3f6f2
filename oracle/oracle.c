/*
 * CPU ORACLE — test infrastructure only.
 *
 * A plain, slow, single-threaded FP64 implementation of what the solver
 * computes, written so that it can be checked against the paper by eye.  It
 * shares no code with the CUDA path.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it; the product never does.
 *
 *  - or_analyze   : geometric nested-dissection ordering (Section 4, the block
 *                   form of P A P^T with V1, V2 before the separator S; with
 *                   patch ids, e.g. the six faces of a cubed sphere, the
 *                   patch sets are dissected first: the lowest two patches
 *                   against the rest, two patches one against the other),
 *                   then
 *                   the structure of L by explicit set unions over the
 *                   elimination tree (the fill characterisation of the
 *                   Lemma in Section 4), the elimination tree parent and
 *                   column counts read off that structure, fundamental
 *                   supernodes and relaxed amalgamation.
 *  - or_factor    : left-looking Cholesky  P A P^T = L L^T  (Section 4),
 *                   column by column, with correctly rounded sqrt.
 *  - or_solve     : x = P^T L^-T L^-1 P b  (the exact inverse of the
 *                   compressed matrix applied to right-hand sides; Sections
 *                   1 and 5.1/5.2).
 *  - or_logdet    : 2 sum log L_jj with Neumaier compensated summation.
 *  - or_apply_L   : s = P^T L z (Gaussian random field samples, Eq.
 *                   CholFastField of Section 5.3, with G = I).
 *  - or_selinv    : entries of A^-1 on the pattern of L by the scalar
 *                   Takahashi recurrences, processed from the last column to
 *                   the first.
 *
 * Compile with -O2 -ffp-contract=off so no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct or_ctx {
    int64_t n;
    /* ordering */
    int32_t *perm, *iperm;
    /* P A P^T lower CSC with the index of the source value */
    int64_t *pcolptr;
    int32_t *prow;
    int64_t *psrc;
    /* structure of L (diagonal first, then rows ascending) */
    int64_t *Lp;
    int32_t *Li;
    double *Lx;
    int32_t *parent;
    int64_t *colcount;
    /* supernodes */
    int32_t nsuper;
    int32_t *sfirst;      /* nsuper + 1 */
    int64_t *srowptr;     /* nsuper + 1 */
    int32_t *srows;
    int factored;
    /* orientation of every permuted lower entry: 1 when (row, col) of
       P A P^T is the transposed position (col, row) of its source entry */
    int8_t *pswap;
    /* LU without pivoting (or_factor_lu): L with unit diagonal in Lux, U
       transposed (column j holds row j of U) in Uux, both on L's pattern */
    double *Lux, *Uux;
    int lu_factored;
    /* LDL^T without pivoting (or_factor_ldlt): L with unit diagonal on L's
       pattern, d_j stored in place of L's diagonal entry */
    double *Ldx;
    int ldlt_factored;
} or_ctx;

or_ctx *or_create(void) { return (or_ctx *)calloc(1, sizeof(or_ctx)); }

static void free_numeric(or_ctx *c) {
    free(c->Lx);
    c->Lx = NULL;
    c->factored = 0;
}

static void free_lu(or_ctx *c) {
    free(c->Lux);
    free(c->Uux);
    c->Lux = c->Uux = NULL;
    c->lu_factored = 0;
}

static void free_ldlt(or_ctx *c) {
    free(c->Ldx);
    c->Ldx = NULL;
    c->ldlt_factored = 0;
}

static void free_all(or_ctx *c) {
    free_lu(c);
    free_ldlt(c);
    free(c->pswap);
    free(c->perm); free(c->iperm); free(c->pcolptr); free(c->prow); free(c->psrc);
    free(c->Lp); free(c->Li); free(c->parent); free(c->colcount);
    free(c->sfirst); free(c->srowptr); free(c->srows);
    free_numeric(c);
    memset(c, 0, sizeof(*c));
}

void or_destroy(or_ctx *c) {
    if (!c) return;
    free_all(c);
    free(c);
}

/* ------------------------------------------------------------------ */
/* nested dissection                                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    int dim;
    const int64_t *adjp; /* full adjacency without the diagonal */
    const int32_t *adj;
    const int32_t *level, *lo, *side;
    const int32_t *patch; /* optional patch id per vertex (NULL: one patch) */
    int32_t leaf;
    int32_t *stamp;  /* membership stamp per vertex */
    int32_t *inS;
    int32_t *sd;     /* side per vertex */
    int32_t cur;
    int32_t *out;
    int64_t pos;
    int64_t *tree;     /* optional: 4 positions per dissection node */
    int64_t ntree, tree_cap;
} nd_state;

static int cmp_int32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static const int32_t *g_level_for_sort;
/* separator order: finer level first (level descending), then index ascending */
static int cmp_sep(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    int32_t lx = g_level_for_sort[x], ly = g_level_for_sort[y];
    if (lx != ly) return (lx < ly) ? 1 : -1;
    return (x > y) - (x < y);
}

/* Split of a set of patches (bit mask, more than one bit): the lowest two
   patches against the rest, or the lower against the higher of two. */
static uint32_t patch_split(uint32_t mask) {
    uint32_t first = mask & (~mask + 1u);
    uint32_t rest = mask & ~first;
    if ((rest & (rest - 1u)) == 0u) return first; /* two patches: {p0} | {p1} */
    return first | (rest & (~rest + 1u));         /* {p0, p1} | rest */
}

static void nd_rec(nd_state *st, int32_t *V, int64_t nv, const int64_t *rlo, const int64_t *rhi,
                   uint32_t pmask) {
    int dim = st->dim;
    int one_cell = 1;
    for (int a = 0; a < dim; ++a)
        if (rhi[a] - rlo[a] > 1) one_cell = 0;
    int multi = st->patch && (pmask & (pmask - 1u)) != 0u;
    if (nv <= st->leaf || (one_cell && !multi)) {
        qsort(V, (size_t)nv, sizeof(int32_t), cmp_int32);
        for (int64_t i = 0; i < nv; ++i) st->out[st->pos++] = V[i];
        return;
    }
    if (multi) {
        /* the patches first: side 0 = the patches of the first group */
        uint32_t ma = patch_split(pmask), mb = pmask & ~ma;
        int32_t stamp = ++st->cur;
        for (int64_t i = 0; i < nv; ++i) {
            int32_t v = V[i];
            st->stamp[v] = stamp;
            st->inS[v] = 0;
            st->sd[v] = ((ma >> st->patch[v]) & 1u) ? 0 : 1;
        }
        for (int64_t i = 0; i < nv; ++i) {
            int32_t u = V[i];
            for (int64_t q = st->adjp[u]; q < st->adjp[u + 1]; ++q) {
                int32_t w = st->adj[q];
                if (st->stamp[w] != stamp || st->sd[w] == st->sd[u]) continue;
                int32_t pick;
                if (st->level[u] != st->level[w])
                    pick = (st->level[u] < st->level[w]) ? u : w;
                else if (st->side[u] != st->side[w])
                    pick = (st->side[u] > st->side[w]) ? u : w;
                else
                    pick = (st->sd[u] == 0) ? u : w;
                st->inS[pick] = 1;
            }
        }
        int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
        int64_t n0 = 0, n1 = 0, ns = 0;
        for (int64_t i = 0; i < nv; ++i)
            if (!st->inS[V[i]] && st->sd[V[i]] == 0) buf[n0++] = V[i];
        for (int64_t i = 0; i < nv; ++i)
            if (!st->inS[V[i]] && st->sd[V[i]] == 1) buf[n0 + n1++] = V[i];
        for (int64_t i = 0; i < nv; ++i)
            if (st->inS[V[i]]) buf[n0 + n1 + ns++] = V[i];
        int32_t *S = buf + n0 + n1;
        int64_t p0 = st->pos;
        nd_rec(st, buf, n0, rlo, rhi, ma);
        int64_t p1 = st->pos;
        nd_rec(st, buf + n0, n1, rlo, rhi, mb);
        int64_t p2 = st->pos;
        if (st->tree && st->ntree < st->tree_cap) {
            int64_t *t = st->tree + 4 * st->ntree++;
            t[0] = p0; t[1] = p1; t[2] = p2; t[3] = p2 + ns;
        }
        g_level_for_sort = st->level;
        qsort(S, (size_t)ns, sizeof(int32_t), cmp_sep);
        for (int64_t i = 0; i < ns; ++i) st->out[st->pos++] = S[i];
        free(buf);
        return;
    }
    int axis = 0;
    for (int a = 1; a < dim; ++a)
        if (rhi[a] - rlo[a] > rhi[axis] - rlo[axis]) axis = a;
    int64_t cut = rlo[axis] + (rhi[axis] - rlo[axis]) / 2;
    int32_t stamp = ++st->cur;
    for (int64_t i = 0; i < nv; ++i) {
        int32_t v = V[i];
        st->stamp[v] = stamp;
        st->inS[v] = 0;
        int64_t twice_center = 2 * (int64_t)st->lo[(int64_t)v * dim + axis] + st->side[v];
        st->sd[v] = (twice_center < 2 * cut) ? 0 : 1;
    }
    for (int64_t i = 0; i < nv; ++i) {
        int32_t u = V[i];
        for (int64_t q = st->adjp[u]; q < st->adjp[u + 1]; ++q) {
            int32_t w = st->adj[q];
            if (st->stamp[w] != stamp || st->sd[w] == st->sd[u]) continue;
            int32_t pick;
            if (st->level[u] != st->level[w])
                pick = (st->level[u] < st->level[w]) ? u : w;
            else if (st->side[u] != st->side[w])
                pick = (st->side[u] > st->side[w]) ? u : w;
            else
                pick = (st->sd[u] == 0) ? u : w;
            st->inS[pick] = 1;
        }
    }
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nv > 0 ? nv : 1));
    int64_t n0 = 0, n1 = 0, ns = 0;
    for (int64_t i = 0; i < nv; ++i)
        if (!st->inS[V[i]] && st->sd[V[i]] == 0) buf[n0++] = V[i];
    for (int64_t i = 0; i < nv; ++i)
        if (!st->inS[V[i]] && st->sd[V[i]] == 1) buf[n0 + n1++] = V[i];
    for (int64_t i = 0; i < nv; ++i)
        if (st->inS[V[i]]) buf[n0 + n1 + ns++] = V[i];
    int64_t llo[3], lhi[3], hlo[3], hhi[3];
    for (int a = 0; a < dim; ++a) {
        llo[a] = hlo[a] = rlo[a];
        lhi[a] = hhi[a] = rhi[a];
    }
    lhi[axis] = cut;
    hlo[axis] = cut;
    /* copy the separator out before recursion reuses the stamps */
    int32_t *S = buf + n0 + n1;
    int64_t p0 = st->pos;
    nd_rec(st, buf, n0, llo, lhi, pmask);
    int64_t p1 = st->pos;
    nd_rec(st, buf + n0, n1, hlo, hhi, pmask);
    int64_t p2 = st->pos;
    if (st->tree && st->ntree < st->tree_cap) {
        int64_t *t = st->tree + 4 * st->ntree++;
        t[0] = p0; t[1] = p1; t[2] = p2; t[3] = p2 + ns;
    }
    g_level_for_sort = st->level;
    qsort(S, (size_t)ns, sizeof(int32_t), cmp_sep);
    for (int64_t i = 0; i < ns; ++i) st->out[st->pos++] = S[i];
    free(buf);
}

/* full symmetric adjacency (no diagonal) from a lower CSC */
static void full_adjacency(int64_t n, const int64_t *cp, const int32_t *ri, int64_t **adjp_out,
                           int32_t **adj_out) {
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = cp[j]; q < cp[j + 1]; ++q) {
            int32_t i = ri[q];
            if (i == j) continue;
            deg[i]++;
            deg[j]++;
        }
    int64_t *adjp = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    adjp[0] = 0;
    for (int64_t v = 0; v < n; ++v) adjp[v + 1] = adjp[v] + deg[v];
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(adjp[n] > 0 ? adjp[n] : 1));
    for (int64_t v = 0; v < n; ++v) deg[v] = adjp[v];
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = cp[j]; q < cp[j + 1]; ++q) {
            int32_t i = ri[q];
            if (i == j) continue;
            adj[deg[i]++] = (int32_t)j;
            adj[deg[j]++] = i;
        }
    free(deg);
    *adjp_out = adjp;
    *adj_out = adj;
}

/* geometric ND; perm[new] = old.  If tree != NULL, up to tree_cap dissection
   nodes are recorded as 4 positions (V1 start, V2 start, S start, S end) and
   their number is stored in *ntree. */
int or_nd_order_tree(int64_t n, const int64_t *cp, const int32_t *ri, int dim,
                     const int32_t *level, const int32_t *lo, const int32_t *side,
                     const int32_t *patch, int32_t leaf, int32_t *perm, int64_t *tree,
                     int64_t tree_cap, int64_t *ntree) {
    if (n <= 0 || dim < 1 || dim > 3) return -1;
    uint32_t pmask = 1u; /* one patch unless patch ids are given */
    if (patch) {
        pmask = 0u;
        for (int64_t v = 0; v < n; ++v) {
            if (patch[v] < 0 || patch[v] > 31) return -1;
            pmask |= 1u << patch[v];
        }
    }
    int64_t *adjp;
    int32_t *adj;
    full_adjacency(n, cp, ri, &adjp, &adj);
    nd_state st;
    memset(&st, 0, sizeof(st));
    st.n = n; st.dim = dim; st.adjp = adjp; st.adj = adj;
    st.level = level; st.lo = lo; st.side = side; st.patch = patch; st.leaf = leaf;
    st.stamp = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    st.inS = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    st.sd = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    st.out = perm;
    st.tree = tree;
    st.tree_cap = tree ? tree_cap : 0;
    int64_t rlo[3] = {0, 0, 0}, rhi[3] = {0, 0, 0};
    for (int64_t v = 0; v < n; ++v)
        for (int a = 0; a < dim; ++a) {
            int64_t e = (int64_t)lo[v * dim + a] + side[v];
            if (e > rhi[a]) rhi[a] = e;
        }
    int32_t *V = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t v = 0; v < n; ++v) V[v] = (int32_t)v;
    nd_rec(&st, V, n, rlo, rhi, pmask);
    free(V);
    free(st.stamp); free(st.inS); free(st.sd); free(adjp); free(adj);
    if (ntree) *ntree = st.ntree;
    return st.pos == n ? 0 : -2;
}

int or_nd_order(int64_t n, const int64_t *cp, const int32_t *ri, int dim, const int32_t *level,
                const int32_t *lo, const int32_t *side, const int32_t *patch, int32_t leaf,
                int32_t *perm) {
    return or_nd_order_tree(n, cp, ri, dim, level, lo, side, patch, leaf, perm, NULL, 0, NULL);
}

/* ------------------------------------------------------------------ */
/* symbolic analysis by explicit set unions                            */
/* ------------------------------------------------------------------ */

/* P A P^T lower CSC; rows sorted; psrc maps each entry to the input value */
static void permute_lower(or_ctx *c, const int64_t *cp, const int32_t *ri) {
    int64_t n = c->n, nnz = cp[n];
    c->pcolptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    c->prow = (int32_t *)malloc(sizeof(int32_t) * (size_t)nnz);
    c->psrc = (int64_t *)malloc(sizeof(int64_t) * (size_t)nnz);
    c->pswap = (int8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = cp[j]; q < cp[j + 1]; ++q) {
            int32_t a = c->iperm[ri[q]], b = c->iperm[j];
            c->pcolptr[(a < b ? a : b) + 1]++;
        }
    for (int64_t j = 0; j < n; ++j) c->pcolptr[j + 1] += c->pcolptr[j];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    memcpy(fill, c->pcolptr, sizeof(int64_t) * (size_t)n);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = cp[j]; q < cp[j + 1]; ++q) {
            int32_t a = c->iperm[ri[q]], b = c->iperm[j];
            int32_t col = a < b ? a : b, row = a < b ? b : a;
            int64_t d = fill[col]++;
            c->prow[d] = row;
            c->psrc[d] = q;
            c->pswap[d] = (int8_t)(a < b);
        }
    free(fill);
    /* insertion sort each column by row (columns are short) */
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t q = c->pcolptr[j] + 1; q < c->pcolptr[j + 1]; ++q) {
            int32_t r = c->prow[q];
            int64_t s = c->psrc[q];
            int8_t w = c->pswap[q];
            int64_t t = q - 1;
            while (t >= c->pcolptr[j] && c->prow[t] > r) {
                c->prow[t + 1] = c->prow[t];
                c->psrc[t + 1] = c->psrc[t];
                c->pswap[t + 1] = c->pswap[t];
                --t;
            }
            c->prow[t + 1] = r;
            c->psrc[t + 1] = s;
            c->pswap[t + 1] = w;
        }
    }
}

/*
 * struct(L_j) = {i > j : a_ij != 0}  U  (union over etree children k of
 * struct(L_k) minus {j}).  parent[j] = min struct(L_j), c_j = |struct|+1.
 * Columns are processed in order, so all children are done before j.
 */
static int symbolic_unions(or_ctx *c) {
    int64_t n = c->n;
    int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) mark[i] = -1;
    /* children lists, built as columns finish */
    int32_t *chead = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *cnext = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) chead[i] = -1;
    c->parent = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    c->colcount = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t cap = c->pcolptr[n] * 2 + n + 16, used = 0;
    int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    c->Lp = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) {
        int64_t t = 0;
        mark[j] = (int32_t)j;
        for (int64_t q = c->pcolptr[j]; q < c->pcolptr[j + 1]; ++q) {
            int32_t i = c->prow[q];
            if (mark[i] != j) { mark[i] = (int32_t)j; tmp[t++] = i; }
        }
        for (int32_t k = chead[j]; k != -1; k = cnext[k]) {
            for (int64_t q = c->Lp[k] + 1; q < c->Lp[k + 1]; ++q) {
                int32_t i = rows[q];
                if (mark[i] != j) { mark[i] = (int32_t)j; tmp[t++] = i; }
            }
        }
        qsort(tmp, (size_t)t, sizeof(int32_t), cmp_int32);
        if (used + t + 1 > cap) {
            cap = (used + t + 1) * 2;
            rows = (int32_t *)realloc(rows, sizeof(int32_t) * (size_t)cap);
        }
        c->Lp[j] = used;
        rows[used++] = (int32_t)j;   /* diagonal first */
        for (int64_t s = 0; s < t; ++s) rows[used++] = tmp[s];
        c->Lp[j + 1] = used;
        c->colcount[j] = t + 1;
        int32_t p = (t > 0) ? tmp[0] : -1;
        c->parent[j] = p;
        if (p >= 0) { cnext[j] = chead[p]; chead[p] = (int32_t)j; }
    }
    c->Li = (int32_t *)realloc(rows, sizeof(int32_t) * (size_t)(used > 0 ? used : 1));
    free(mark); free(chead); free(cnext); free(tmp);
    return 0;
}

static int64_t trap(int64_t k, int64_t m) { return k * m - k * (k - 1) / 2; }

/* fundamental supernodes, then the relaxed merge scan over consecutive ones */
static void supernodes(or_ctx *c, int32_t relax_k, int32_t relax_pct) {
    int64_t n = c->n;
    int32_t *nchild = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    for (int64_t j = 0; j < n; ++j)
        if (c->parent[j] >= 0) nchild[c->parent[j]]++;
    /* fundamental: j+1 joins j's supernode iff parent[j]==j+1,
       c_j == c_{j+1}+1 and j+1 has exactly one child */
    int32_t *ffirst = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t nf = 0;
    for (int64_t j = 0; j < n; ++j) {
        int join = (j > 0) && c->parent[j - 1] == j && c->colcount[j - 1] == c->colcount[j] + 1 &&
                   nchild[j] == 1;
        if (!join) ffirst[nf++] = (int32_t)j;
    }
    ffirst[nf] = (int32_t)n;
    /* merge scan */
    int32_t *gfirst = (int32_t *)malloc(sizeof(int32_t) * ((size_t)nf + 1));
    int32_t ng = 0;
    int64_t gk = 0, gsum = 0;
    int32_t glast = -1;
    for (int32_t t = 0; t < nf; ++t) {
        int64_t f = ffirst[t], l = ffirst[t + 1] - 1;
        int64_t kt = l - f + 1;
        int64_t below = c->colcount[f] - kt;
        int64_t sumt = 0;
        for (int64_t j = f; j <= l; ++j) sumt += c->colcount[j];
        if (ng > 0 && c->parent[glast] == f) {
            int64_t k2 = gk + kt, m2 = k2 + below, s2 = gsum + sumt;
            int64_t tr = trap(k2, m2), z = tr - s2;
            if (k2 <= relax_k || 100 * z <= (int64_t)relax_pct * tr) {
                gk = k2;
                gsum = s2;
                glast = (int32_t)l;
                continue;
            }
        }
        gfirst[ng++] = (int32_t)f;
        gk = kt;
        gsum = sumt;
        glast = (int32_t)l;
    }
    gfirst[ng] = (int32_t)n;
    c->nsuper = ng;
    c->sfirst = gfirst;
    /* rows of supernode s: its own columns, then struct of its last column
       below the supernode (all of which lie beyond the last column) */
    c->srowptr = (int64_t *)malloc(sizeof(int64_t) * ((size_t)ng + 1));
    int64_t tot = 0;
    for (int32_t s = 0; s < ng; ++s) {
        int64_t f = gfirst[s], l = gfirst[s + 1] - 1;
        tot += (l - f + 1) + (c->Lp[l + 1] - c->Lp[l] - 1);
    }
    c->srows = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot > 0 ? tot : 1));
    int64_t u = 0;
    for (int32_t s = 0; s < ng; ++s) {
        int64_t f = gfirst[s], l = gfirst[s + 1] - 1;
        c->srowptr[s] = u;
        for (int64_t j = f; j <= l; ++j) c->srows[u++] = (int32_t)j;
        for (int64_t q = c->Lp[l] + 1; q < c->Lp[l + 1]; ++q) c->srows[u++] = c->Li[q];
    }
    c->srowptr[ng] = u;
    free(nchild);
    free(ffirst);
}

/*
 * perm_in: optional ordering to use instead of ND (perm[new] = old).
 * dim == 0 or level == NULL: no geometry; the identity order is used unless
 * perm_in is given.
 */
int or_analyze(or_ctx *c, int64_t n, const int64_t *cp, const int32_t *ri, int dim,
               const int32_t *level, const int32_t *lo, const int32_t *side, const int32_t *patch,
               int32_t leaf, int32_t relax_k, int32_t relax_pct, const int32_t *perm_in) {
    free_all(c);
    if (n <= 0) return -1;
    /* validation: sorted, in range, diagonal first */
    for (int64_t j = 0; j < n; ++j) {
        if (cp[j + 1] <= cp[j] || ri[cp[j]] != j) return -3;
        for (int64_t q = cp[j] + 1; q < cp[j + 1]; ++q)
            if (ri[q] <= ri[q - 1] || ri[q] >= n) return -3;
    }
    c->n = n;
    c->perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    c->iperm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (perm_in) {
        memcpy(c->perm, perm_in, sizeof(int32_t) * (size_t)n);
    } else if (dim > 0 && level) {
        int rc = or_nd_order(n, cp, ri, dim, level, lo, side, patch, leaf, c->perm);
        if (rc) return rc;
    } else {
        for (int64_t i = 0; i < n; ++i) c->perm[i] = (int32_t)i;
    }
    for (int64_t i = 0; i < n; ++i) c->iperm[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int32_t o = c->perm[i];
        if (o < 0 || o >= n || c->iperm[o] != -1) return -4;
        c->iperm[o] = (int32_t)i;
    }
    permute_lower(c, cp, ri);
    symbolic_unions(c);
    supernodes(c, relax_k, relax_pct);
    return 0;
}

int64_t or_n(const or_ctx *c) { return c->n; }
int64_t or_nnzL(const or_ctx *c) { return c->Lp ? c->Lp[c->n] : 0; }
int32_t or_nsuper(const or_ctx *c) { return c->nsuper; }
int64_t or_nsuper_rows(const or_ctx *c) { return c->srowptr ? c->srowptr[c->nsuper] : 0; }

void or_get_symbolic(const or_ctx *c, int32_t *perm, int32_t *parent, int64_t *colcount,
                     int32_t *sfirst, int64_t *srowptr, int32_t *srows) {
    int64_t n = c->n;
    if (perm) memcpy(perm, c->perm, sizeof(int32_t) * (size_t)n);
    if (parent) memcpy(parent, c->parent, sizeof(int32_t) * (size_t)n);
    if (colcount) memcpy(colcount, c->colcount, sizeof(int64_t) * (size_t)n);
    if (sfirst) memcpy(sfirst, c->sfirst, sizeof(int32_t) * ((size_t)c->nsuper + 1));
    if (srowptr) memcpy(srowptr, c->srowptr, sizeof(int64_t) * ((size_t)c->nsuper + 1));
    if (srows) memcpy(srows, c->srows, sizeof(int32_t) * (size_t)c->srowptr[c->nsuper]);
}

void or_get_Lpattern(const or_ctx *c, int64_t *Lp, int32_t *Li) {
    memcpy(Lp, c->Lp, sizeof(int64_t) * ((size_t)c->n + 1));
    memcpy(Li, c->Li, sizeof(int32_t) * (size_t)c->Lp[c->n]);
}

/* ------------------------------------------------------------------ */
/* numeric                                                             */
/* ------------------------------------------------------------------ */

/* left-looking Cholesky of the first ncols columns of P A P^T (all of them
   if ncols < 0 or ncols > n).  Returns 0, or -(j+1) if the pivot of column j
   is not positive (j = the first such column).  Only a full factorization
   leaves the context factored. */
int64_t or_factor_cols(or_ctx *c, const double *values, int64_t ncols) {
    int64_t n = c->n;
    int64_t stop = (ncols < 0 || ncols > n) ? n : ncols;
    free_numeric(c);
    c->Lx = (double *)malloc(sizeof(double) * (size_t)c->Lp[n]);
    double *w = (double *)calloc((size_t)n, sizeof(double));
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *head = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *link = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *ks = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) head[j] = -1;
    int64_t status = 0;
    for (int64_t j = 0; j < stop; ++j) {
        for (int64_t q = c->pcolptr[j]; q < c->pcolptr[j + 1]; ++q)
            w[c->prow[q]] = values[c->psrc[q]];
        /* columns k < j with L_jk != 0, ascending */
        int64_t nk = 0;
        for (int32_t k = head[j]; k != -1; k = link[k]) ks[nk++] = k;
        qsort(ks, (size_t)nk, sizeof(int32_t), cmp_int32);
        for (int64_t t = 0; t < nk; ++t) {
            int32_t k = ks[t];
            int64_t p = next[k];
            double ljk = c->Lx[p];
            for (int64_t q = p; q < c->Lp[k + 1]; ++q) w[c->Li[q]] -= c->Lx[q] * ljk;
            next[k] = p + 1;
            if (p + 1 < c->Lp[k + 1]) {
                int32_t r = c->Li[p + 1];
                link[k] = head[r];
                head[r] = k;
            }
        }
        double d = w[j];
        if (!(d > 0.0)) { status = -(j + 1); break; }
        double ljj = sqrt(d);
        c->Lx[c->Lp[j]] = ljj;
        w[j] = 0.0;
        for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) {
            int32_t i = c->Li[q];
            c->Lx[q] = w[i] / ljj;
            w[i] = 0.0;
        }
        next[j] = c->Lp[j] + 1;
        if (next[j] < c->Lp[j + 1]) {
            int32_t r = c->Li[next[j]];
            link[j] = head[r];
            head[r] = (int32_t)j;
        }
    }
    free(w); free(next); free(head); free(link); free(ks);
    if (status) { free_numeric(c); return status; }
    c->factored = (stop == n);
    return 0;
}

int64_t or_factor(or_ctx *c, const double *values) { return or_factor_cols(c, values, -1); }

void or_get_L(const or_ctx *c, double *Lx) {
    memcpy(Lx, c->Lx, sizeof(double) * (size_t)c->Lp[c->n]);
}

/* B (n x nrhs, column-major, leading dim ldb, original order) := A^-1 B */
int or_solve(const or_ctx *c, double *B, int64_t nrhs, int64_t ldb) {
    if (!c->factored) return -1;
    int64_t n = c->n;
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t r = 0; r < nrhs; ++r) {
        double *b = B + r * ldb;
        for (int64_t i = 0; i < n; ++i) y[i] = b[c->perm[i]];
        /* forward, column oriented: y := L^-1 y */
        for (int64_t j = 0; j < n; ++j) {
            y[j] /= c->Lx[c->Lp[j]];
            double yj = y[j];
            for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) y[c->Li[q]] -= c->Lx[q] * yj;
        }
        /* backward, row oriented on L^T: y := L^-T y */
        for (int64_t j = n - 1; j >= 0; --j) {
            double s = y[j];
            for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) s -= c->Lx[q] * y[c->Li[q]];
            y[j] = s / c->Lx[c->Lp[j]];
        }
        for (int64_t i = 0; i < n; ++i) b[c->perm[i]] = y[i];
    }
    free(y);
    return 0;
}

/* The two substitutions of or_solve restricted to the columns j < ncols of
   L (final after or_factor_cols(ncols)), on B in factor order.  Not a solve:
   a bounded share of the solve's work, the same loops over fewer columns,
   for timing the oracle on large factorizations. */
int or_solve_prefix(const or_ctx *c, double *B, int64_t nrhs, int64_t ldb, int64_t ncols) {
    if (!c->Lx || ncols < 0 || ncols > c->n) return -1;
    for (int64_t r = 0; r < nrhs; ++r) {
        double *y = B + r * ldb;
        for (int64_t j = 0; j < ncols; ++j) {
            y[j] /= c->Lx[c->Lp[j]];
            double yj = y[j];
            for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) y[c->Li[q]] -= c->Lx[q] * yj;
        }
        for (int64_t j = ncols - 1; j >= 0; --j) {
            double s = y[j];
            for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) s -= c->Lx[q] * y[c->Li[q]];
            y[j] = s / c->Lx[c->Lp[j]];
        }
    }
    return 0;
}

/* LU factorization without pivoting of a matrix with the analyzed
   (symmetric) pattern, P A P^T = L U with L unit lower triangular (Section 4:
   Cholesky and LU share the nested dissection ordering; the pattern of U is
   that of L transposed).  Input: for every stored lower entry e = (r, c),
   r >= c, of the analyzed lower CSC, lower[e] = A[r][c] and upper[e] =
   A[c][r] (the diagonal taken from lower).  Left-looking, column j of L and
   row j of U together (the Doolittle recurrences):
     U[j][j] = A[j][j] - sum_{k<j} L[j][k] U[k][j]
     L[i][j] = (A[i][j] - sum_{k<j} L[i][k] U[k][j]) / U[j][j],   i > j
     U[j][i] =  A[j][i] - sum_{k<j} L[j][k] U[k][i],               i > j
   the sums running over the k with L[j][k] != 0 (equivalently U[k][j] != 0),
   in ascending order.  Returns 0, or -(j+1) for the first zero pivot. */
int64_t or_factor_lu(or_ctx *c, const double *lower, const double *upper) {
    int64_t n = c->n;
    free_lu(c);
    int64_t nnzl = c->Lp[n];
    c->Lux = (double *)malloc(sizeof(double) * (size_t)(nnzl > 0 ? nnzl : 1));
    c->Uux = (double *)malloc(sizeof(double) * (size_t)(nnzl > 0 ? nnzl : 1));
    double *wl = (double *)calloc((size_t)n, sizeof(double));
    double *wu = (double *)calloc((size_t)n, sizeof(double));
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *head = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *link = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *ks = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) head[j] = -1;
    int64_t status = 0;
    for (int64_t j = 0; j < n; ++j) {
        /* column j of P A P^T from the diagonal down into wl, row j to the
           right of the diagonal into wu */
        for (int64_t q = c->pcolptr[j]; q < c->pcolptr[j + 1]; ++q) {
            int32_t i = c->prow[q];
            int64_t e = c->psrc[q];
            if (i == j) {
                wl[i] = lower[e];
            } else {
                wl[i] = c->pswap[q] ? upper[e] : lower[e];
                wu[i] = c->pswap[q] ? lower[e] : upper[e];
            }
        }
        int64_t nk = 0;
        for (int32_t k = head[j]; k != -1; k = link[k]) ks[nk++] = k;
        qsort(ks, (size_t)nk, sizeof(int32_t), cmp_int32);
        for (int64_t t = 0; t < nk; ++t) {
            int32_t k = ks[t];
            int64_t p = next[k];            /* entry (j, k) of L's pattern */
            double ljk = c->Lux[p], ukj = c->Uux[p];
            for (int64_t q = p; q < c->Lp[k + 1]; ++q) {
                int32_t i = c->Li[q];
                wl[i] -= c->Lux[q] * ukj;
                if (i > j) wu[i] -= ljk * c->Uux[q];
            }
            next[k] = p + 1;
            if (p + 1 < c->Lp[k + 1]) {
                int32_t r = c->Li[p + 1];
                link[k] = head[r];
                head[r] = k;
            }
        }
        double ujj = wl[j];
        if (!(ujj != 0.0) || isnan(ujj)) { status = -(j + 1); break; }
        c->Lux[c->Lp[j]] = 1.0;
        c->Uux[c->Lp[j]] = ujj;
        wl[j] = 0.0;
        for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) {
            int32_t i = c->Li[q];
            c->Lux[q] = wl[i] / ujj;
            c->Uux[q] = wu[i];
            wl[i] = 0.0;
            wu[i] = 0.0;
        }
        next[j] = c->Lp[j] + 1;
        if (c->Lp[j] + 1 < c->Lp[j + 1]) {
            int32_t r = c->Li[c->Lp[j] + 1];
            link[j] = head[r];
            head[r] = (int32_t)j;
        }
    }
    free(wl); free(wu); free(next); free(head); free(link); free(ks);
    c->lu_factored = status == 0;
    return status;
}

void or_get_lu(const or_ctx *c, double *Lx, double *Ut) {
    memcpy(Lx, c->Lux, sizeof(double) * (size_t)c->Lp[c->n]);
    memcpy(Ut, c->Uux, sizeof(double) * (size_t)c->Lp[c->n]);
}

/* B (n x nrhs, column-major, original order) := A^-1 B with the LU factors:
   y = L^-1 P b column-oriented (unit diagonal), x = P^T U^-1 y row-oriented */
int or_solve_lu(const or_ctx *c, double *B, int64_t nrhs, int64_t ldb) {
    if (!c->lu_factored) return -1;
    int64_t n = c->n;
    double *y = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t r = 0; r < nrhs; ++r) {
        double *b = B + r * ldb;
        for (int64_t i = 0; i < n; ++i) y[i] = b[c->perm[i]];
        for (int64_t j = 0; j < n; ++j) {
            double yj = y[j];
            for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) y[c->Li[q]] -= c->Lux[q] * yj;
        }
        for (int64_t j = n - 1; j >= 0; --j) {
            double s = y[j];
            for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) s -= c->Uux[q] * y[c->Li[q]];
            y[j] = s / c->Uux[c->Lp[j]];
        }
        for (int64_t i = 0; i < n; ++i) b[c->perm[i]] = y[i];
    }
    free(y);
    return 0;
}

/* log |det A| = sum_j log |U[j][j]| (Neumaier compensated); *sign = the sign
   of det A (det P = det P^T cancel) */
double or_logdet_lu(const or_ctx *c, int32_t *sign) {
    double s = 0.0, comp = 0.0;
    int32_t sg = 1;
    for (int64_t j = 0; j < c->n; ++j) {
        double u = c->Uux[c->Lp[j]];
        if (u < 0) sg = -sg;
        double v = log(fabs(u));
        double t = s + v;
        if (fabs(s) >= fabs(v)) comp += (s - t) + v;
        else comp += (v - t) + s;
        s = t;
    }
    *sign = sg;
    return s + comp;
}

/* LDL^T without pivoting of a symmetric (possibly indefinite) matrix, the
   symmetric case of the LU decomposition (Section 4: "a Cholesky
   decomposition or an LU decomposition" on the same ordering):
   P A P^T = L D L^T, L unit lower triangular on L's pattern, D diagonal.
   Left-looking, column by column, as or_factor_cols but with the pivot kept
   as d_j instead of its square root:
     w = column j of P A P^T (rows >= j);
     for each k < j with L_jk != 0, ascending: w_i -= L_ik d_k L_jk (i >= j);
     d_j = w_j (zero or NaN: the first such column is reported);
     L_ij = w_i / d_j.
   Returns 0, or -(j+1) for the first zero pivot (permuted order). */
int64_t or_factor_ldlt(or_ctx *c, const double *values) {
    int64_t n = c->n;
    free_ldlt(c);
    int64_t nnzl = c->Lp[n];
    c->Ldx = (double *)malloc(sizeof(double) * (size_t)(nnzl > 0 ? nnzl : 1));
    double *w = (double *)calloc((size_t)n, sizeof(double));
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *head = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *link = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *ks = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) head[j] = -1;
    int64_t status = 0;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t q = c->pcolptr[j]; q < c->pcolptr[j + 1]; ++q) w[c->prow[q]] = values[c->psrc[q]];
        int64_t nk = 0;
        for (int32_t k = head[j]; k != -1; k = link[k]) ks[nk++] = k;
        qsort(ks, (size_t)nk, sizeof(int32_t), cmp_int32);
        for (int64_t t = 0; t < nk; ++t) {
            int32_t k = ks[t];
            int64_t p = next[k];                            /* entry (j, k) */
            double s = c->Ldx[c->Lp[k]] * c->Ldx[p];        /* d_k L_jk */
            for (int64_t q = p; q < c->Lp[k + 1]; ++q) w[c->Li[q]] -= c->Ldx[q] * s;
            next[k] = p + 1;
            if (p + 1 < c->Lp[k + 1]) {
                int32_t r = c->Li[p + 1];
                link[k] = head[r];
                head[r] = k;
            }
        }
        double d = w[j];
        if (!(d != 0.0) || isnan(d)) { status = -(j + 1); break; }
        c->Ldx[c->Lp[j]] = d;
        w[j] = 0.0;
        for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) {
            int32_t i = c->Li[q];
            c->Ldx[q] = w[i] / d;
            w[i] = 0.0;
        }
        next[j] = c->Lp[j] + 1;
        if (next[j] < c->Lp[j + 1]) {
            int32_t r = c->Li[next[j]];
            link[j] = head[r];
            head[r] = (int32_t)j;
        }
    }
    free(w); free(next); free(head); free(link); free(ks);
    if (status) { free_ldlt(c); return status; }
    c->ldlt_factored = 1;
    return 0;
}

/* L (unit diagonal stored as 1) and d on L's pattern */
void or_get_ldlt(const or_ctx *c, double *Lx, double *d) {
    for (int64_t j = 0; j < c->n; ++j) {
        d[j] = c->Ldx[c->Lp[j]];
        Lx[c->Lp[j]] = 1.0;
        for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) Lx[q] = c->Ldx[q];
    }
}

/* B := A^-1 B with the LDL^T factors: y = L^-1 P b (column-oriented), y /= d,
   x = P^T L^-T y (row-oriented) */
int or_solve_ldlt(const or_ctx *c, double *B, int64_t nrhs, int64_t ldb) {
    if (!c->ldlt_factored) return -1;
    int64_t n = c->n;
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t r = 0; r < nrhs; ++r) {
        double *b = B + r * ldb;
        for (int64_t i = 0; i < n; ++i) y[i] = b[c->perm[i]];
        for (int64_t j = 0; j < n; ++j) {
            double yj = y[j];
            for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) y[c->Li[q]] -= c->Ldx[q] * yj;
        }
        for (int64_t j = 0; j < n; ++j) y[j] /= c->Ldx[c->Lp[j]];
        for (int64_t j = n - 1; j >= 0; --j) {
            double s = y[j];
            for (int64_t q = c->Lp[j] + 1; q < c->Lp[j + 1]; ++q) s -= c->Ldx[q] * y[c->Li[q]];
            y[j] = s;
        }
        for (int64_t i = 0; i < n; ++i) b[c->perm[i]] = y[i];
    }
    free(y);
    return 0;
}

/* log |det A| = sum_j log |d_j| (Neumaier compensated); *sign = sign of
   det A; *nneg = number of negative d_j, which by Sylvester's law of inertia
   is the number of negative eigenvalues of A */
double or_logdet_ldlt(const or_ctx *c, int32_t *sign, int64_t *nneg) {
    double s = 0.0, comp = 0.0;
    int32_t sg = 1;
    int64_t neg = 0;
    for (int64_t j = 0; j < c->n; ++j) {
        double d = c->Ldx[c->Lp[j]];
        if (d < 0) { sg = -sg; ++neg; }
        double v = log(fabs(d));
        double t = s + v;
        if (fabs(s) >= fabs(v)) comp += (s - t) + v;
        else comp += (v - t) + s;
        s = t;
    }
    *sign = sg;
    *nneg = neg;
    return s + comp;
}

/* 2 sum_j log L_jj, Neumaier compensated */
double or_logdet(const or_ctx *c) {
    double s = 0.0, comp = 0.0;
    for (int64_t j = 0; j < c->n; ++j) {
        double v = 2.0 * log(c->Lx[c->Lp[j]]);
        double t = s + v;
        if (fabs(s) >= fabs(v)) comp += (s - t) + v;
        else comp += (v - t) + s;
        s = t;
    }
    return s + comp;
}

/* S = P^T L Z (Z in factor order, S in original order), both n x nrhs */
int or_apply_L(const or_ctx *c, const double *Z, double *S, int64_t nrhs, int64_t ld) {
    if (!c->factored) return -1;
    int64_t n = c->n;
    double *t = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t r = 0; r < nrhs; ++r) {
        const double *z = Z + r * ld;
        for (int64_t i = 0; i < n; ++i) t[i] = 0.0;
        for (int64_t j = 0; j < n; ++j)
            for (int64_t q = c->Lp[j]; q < c->Lp[j + 1]; ++q) t[c->Li[q]] += c->Lx[q] * z[j];
        for (int64_t i = 0; i < n; ++i) S[r * ld + c->perm[i]] = t[i];
    }
    free(t);
    return 0;
}

static int64_t find_entry(const or_ctx *c, int32_t col, int32_t row) {
    int64_t lo = c->Lp[col], hi = c->Lp[col + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (c->Li[mid] == row) return mid;
        if (c->Li[mid] < row) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* Z := (P A P^T)^-1 on the pattern of L (same layout as L).  Takahashi:
     Z_ij = -(1/L_jj) sum_{k in struct(j), k>j} L_kj Z_ik   (i in struct(j), i>j)
     Z_jj = (1/L_jj) (1/L_jj - sum_{i in struct(j), i>j} L_ij Z_ij)
   for j = n-1 down to 0. */
int or_selinv(const or_ctx *c, double *Z) {
    if (!c->factored) return -1;
    for (int64_t j = c->n - 1; j >= 0; --j) {
        int64_t d = c->Lp[j], e = c->Lp[j + 1];
        double ljj = c->Lx[d];
        for (int64_t a = d + 1; a < e; ++a) {
            int32_t i = c->Li[a];
            double s = 0.0;
            for (int64_t b = d + 1; b < e; ++b) {
                int32_t k = c->Li[b];
                int32_t col = i < k ? i : k, row = i < k ? k : i;
                int64_t pos = find_entry(c, col, row);
                if (pos < 0) return -2;
                s += c->Lx[b] * Z[pos];
            }
            Z[a] = -s / ljj;
        }
        double s = 0.0;
        for (int64_t a = d + 1; a < e; ++a) s += c->Lx[a] * Z[a];
        Z[d] = (1.0 / ljj - s) / ljj;
    }
    return 0;
}

/* P A P^T values on its lower pattern in the layout of L (zeros where A has
   no entry); used to compute residuals on the pattern of L. */
void or_get_permuted_lower(const or_ctx *c, int64_t *pcolptr, int32_t *prow, int64_t *psrc) {
    int64_t n = c->n;
    memcpy(pcolptr, c->pcolptr, sizeof(int64_t) * ((size_t)n + 1));
    memcpy(prow, c->prow, sizeof(int32_t) * (size_t)c->pcolptr[n]);
    memcpy(psrc, c->psrc, sizeof(int64_t) * (size_t)c->pcolptr[n]);
}
