// Host-side symbolic analysis (Section 4 of the paper): nested-dissection
// ordering, elimination tree, column counts, supernodes and the index maps of
// the multifrontal engine.  Deterministic and exact (integer work only).
#include "symbolic.h"

#include <algorithm>
#include <cstring>
#include <numeric>

namespace wd {

enum { OK = 0, ERR_INVALID_ARG = 1, ERR_PATTERN = 2 };

namespace {

// Full adjacency (no diagonal) of the symmetric pattern given by its lower CSC.
void build_graph(int64_t n, const int64_t *cp, const int32_t *ri, std::vector<int64_t> &xadj,
                 std::vector<int32_t> &adj) {
    xadj.assign(n + 1, 0);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = cp[j] + 1; q < cp[j + 1]; ++q) {
            ++xadj[ri[q] + 1];
            ++xadj[j + 1];
        }
    for (int64_t v = 0; v < n; ++v) xadj[v + 1] += xadj[v];
    adj.resize(xadj[n]);
    std::vector<int64_t> fill(xadj.begin(), xadj.end() - 1);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = cp[j] + 1; q < cp[j + 1]; ++q) {
            adj[fill[ri[q]]++] = (int32_t)j;
            adj[fill[j]++] = ri[q];
        }
}

// Geometric nested dissection.  A region R (integer box) and its vertex set
// V are split at the midpoint of R's longest axis; every vertex goes to the
// side of its support centre (strictly left of the cut -> side 0).  For every
// edge that crosses the cut one endpoint joins the separator S: the coarser
// level, then the larger support, then the side-0 vertex.  Order: V1, V2
// (recursively), then S with finer levels first and the coarsest functions
// last.  Regions of one cell or sets of <= leaf vertices are emitted in index
// order.  With patch ids (several parameter domains, e.g. the faces of a
// cubed sphere) a set spanning more than one patch is first cut along patch
// boundaries: its lowest two patches against the others, or, for two patches,
// one against the other; the side of a vertex is its patch's group and the
// separator rule is the same.  Implemented with an explicit task stack.
struct NDTask {
    int kind;                 // 0 = dissect, 1 = emit separator
    std::vector<int32_t> V;
    int64_t lo[3], hi[3];
    uint32_t pmask;           // patches of V (bit p)
};

// patch group of the first side: {p0} of {p0, p1}, else {p0, p1} of more
uint32_t first_patch_group(uint32_t mask) {
    const uint32_t low = mask & (~mask + 1u);
    const uint32_t others = mask & ~low;
    if ((others & (others - 1u)) == 0u) return low;
    return low | (others & (~others + 1u));
}

void nested_dissection(int64_t n, int dim, const std::vector<int64_t> &xadj,
                       const std::vector<int32_t> &adj, const int32_t *level, const int32_t *blo,
                       const int32_t *bside, const int32_t *patch, int leaf,
                       std::vector<int32_t> &perm) {
    perm.clear();
    perm.reserve(n);
    std::vector<int64_t> tag(n, -1);
    std::vector<uint8_t> side(n, 0), sep(n, 0);
    std::vector<NDTask> stack;
    NDTask root;
    root.kind = 0;
    root.V.resize(n);
    std::iota(root.V.begin(), root.V.end(), 0);
    for (int a = 0; a < 3; ++a) root.lo[a] = root.hi[a] = 0;
    for (int64_t v = 0; v < n; ++v)
        for (int a = 0; a < dim; ++a)
            root.hi[a] = std::max<int64_t>(root.hi[a], (int64_t)blo[v * dim + a] + bside[v]);
    root.pmask = 1u;
    if (patch) {
        root.pmask = 0u;
        for (int64_t v = 0; v < n; ++v) root.pmask |= 1u << patch[v];
    }
    stack.push_back(std::move(root));
    int64_t next_tag = 0;
    while (!stack.empty()) {
        NDTask t = std::move(stack.back());
        stack.pop_back();
        if (t.kind == 1) {
            std::sort(t.V.begin(), t.V.end(), [&](int32_t a, int32_t b) {
                if (level[a] != level[b]) return level[a] > level[b];
                return a < b;
            });
            perm.insert(perm.end(), t.V.begin(), t.V.end());
            continue;
        }
        bool single = true;
        int axis = 0;
        for (int a = 0; a < dim; ++a) {
            if (t.hi[a] - t.lo[a] > 1) single = false;
            if (t.hi[a] - t.lo[a] > t.hi[axis] - t.lo[axis]) axis = a;
        }
        const bool multi = patch && (t.pmask & (t.pmask - 1u)) != 0u;
        if ((int64_t)t.V.size() <= leaf || (single && !multi)) {
            std::sort(t.V.begin(), t.V.end());
            perm.insert(perm.end(), t.V.begin(), t.V.end());
            continue;
        }
        const int64_t cut = t.lo[axis] + (t.hi[axis] - t.lo[axis]) / 2;
        const uint32_t group0 = multi ? first_patch_group(t.pmask) : 0u;
        const int64_t id = next_tag++;
        for (int32_t v : t.V) {
            tag[v] = id;
            sep[v] = 0;
            if (multi)
                side[v] = ((group0 >> patch[v]) & 1u) ? 0 : 1;
            else
                side[v] = (2 * (int64_t)blo[(int64_t)v * dim + axis] + bside[v] < 2 * cut) ? 0 : 1;
        }
        for (int32_t u : t.V) {
            for (int64_t q = xadj[u]; q < xadj[u + 1]; ++q) {
                const int32_t w = adj[q];
                if (tag[w] != id || side[w] == side[u] || w < u) continue;  // each edge once
                int32_t pick;
                if (level[u] != level[w]) pick = level[u] < level[w] ? u : w;
                else if (bside[u] != bside[w]) pick = bside[u] > bside[w] ? u : w;
                else pick = side[u] == 0 ? u : w;
                sep[pick] = 1;
            }
        }
        NDTask a, b, s;
        a.kind = b.kind = 0;
        s.kind = 1;
        for (int32_t v : t.V) {
            if (sep[v]) s.V.push_back(v);
            else if (side[v] == 0) a.V.push_back(v);
            else b.V.push_back(v);
        }
        for (int d = 0; d < 3; ++d) {
            a.lo[d] = b.lo[d] = t.lo[d];
            a.hi[d] = b.hi[d] = t.hi[d];
        }
        if (multi) {
            a.pmask = group0;
            b.pmask = t.pmask & ~group0;
        } else {
            a.pmask = b.pmask = t.pmask;
            a.hi[axis] = cut;
            b.lo[axis] = cut;
        }
        stack.push_back(std::move(s));
        stack.push_back(std::move(b));
        stack.push_back(std::move(a));
    }
}

}  // namespace

int analyze(Symbolic &S, int64_t n, const int64_t *cp, const int32_t *ri, int dim,
            const int32_t *level, const int32_t *blo, const int32_t *bside, const int32_t *patch,
            int leaf, int relax_k, int relax_pct, std::string &msg) {
    S = Symbolic();
    if (n <= 0 || n > INT32_MAX - 1 || !cp || !ri) {
        msg = "invalid size or null pattern";
        return ERR_INVALID_ARG;
    }
    if (cp[0] != 0) {
        msg = "colptr[0] != 0";
        return ERR_PATTERN;
    }
    for (int64_t j = 0; j < n; ++j) {
        if (cp[j + 1] <= cp[j]) {
            msg = "empty column " + std::to_string(j) + " (diagonal missing)";
            return ERR_PATTERN;
        }
        if (ri[cp[j]] != j) {
            msg = "column " + std::to_string(j) + ": diagonal is not the first entry";
            return ERR_PATTERN;
        }
        for (int64_t q = cp[j] + 1; q < cp[j + 1]; ++q)
            if (ri[q] <= ri[q - 1] || ri[q] >= n) {
                msg = "column " + std::to_string(j) + ": rows unsorted, duplicated or out of range";
                return ERR_PATTERN;
            }
    }
    const int64_t nnz = cp[n];
    // the full symmetric CSR (2 nnz - n entries) is indexed with 32-bit positions
    if (nnz > INT32_MAX || 2 * nnz - n > INT32_MAX) {
        msg = "more than 2^31-1 entries in the full symmetric matrix";
        return ERR_INVALID_ARG;
    }
    S.n = n;

    // ---- ordering -------------------------------------------------------
    if (dim > 0 && level && blo && bside) {
        if (dim > 3) {
            msg = "geometry dim must be 1..3";
            return ERR_INVALID_ARG;
        }
        if (patch)
            for (int64_t v = 0; v < n; ++v)
                if (patch[v] < 0 || patch[v] > 31) {
                    msg = "patch ids must be 0..31";
                    return ERR_INVALID_ARG;
                }
        std::vector<int64_t> xadj;
        std::vector<int32_t> adj;
        build_graph(n, cp, ri, xadj, adj);
        nested_dissection(n, dim, xadj, adj, level, blo, bside, patch, std::max(leaf, 1), S.perm);
    } else {
        S.perm.resize(n);
        std::iota(S.perm.begin(), S.perm.end(), 0);
    }
    S.iperm.assign(n, -1);
    for (int64_t i = 0; i < n; ++i) S.iperm[S.perm[i]] = (int32_t)i;

    // ---- lower triangle of P A P^T, columns sorted ------------------------
    S.pcp.assign(n + 1, 0);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t q = cp[j]; q < cp[j + 1]; ++q)
            ++S.pcp[std::min(S.iperm[ri[q]], S.iperm[j]) + 1];
    for (int64_t j = 0; j < n; ++j) S.pcp[j + 1] += S.pcp[j];
    {
        std::vector<std::pair<int32_t, int32_t>> ent(nnz);
        std::vector<int64_t> fill(S.pcp.begin(), S.pcp.end() - 1);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t q = cp[j]; q < cp[j + 1]; ++q) {
                int32_t a = S.iperm[ri[q]], b = S.iperm[j];
                ent[fill[std::min(a, b)]++] = {std::max(a, b), (int32_t)q};
            }
        for (int64_t j = 0; j < n; ++j) std::sort(ent.begin() + S.pcp[j], ent.begin() + S.pcp[j + 1]);
        S.prow.resize(nnz);
        S.psrc.resize(nnz);
        S.pswap.resize(nnz);
        for (int64_t e = 0; e < nnz; ++e) {
            S.prow[e] = ent[e].first;
            S.psrc[e] = ent[e].second;
            S.pswap[e] = (int8_t)(S.iperm[ri[ent[e].second]] != ent[e].first);
        }
    }

    // row lists of the strictly lower part: for row i, the columns j < i
    std::vector<int64_t> rp(n + 1, 0);
    for (int64_t j = 0; j < n; ++j)
        for (int64_t e = S.pcp[j] + 1; e < S.pcp[j + 1]; ++e) ++rp[S.prow[e] + 1];
    for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
    std::vector<int32_t> rc(rp[n] > 0 ? rp[n] : 1);
    {
        std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
        for (int64_t j = 0; j < n; ++j)
            for (int64_t e = S.pcp[j] + 1; e < S.pcp[j + 1]; ++e) rc[fill[S.prow[e]]++] = (int32_t)j;
    }

    // ---- elimination tree (Liu, with path compression) --------------------
    S.parent.assign(n, -1);
    {
        std::vector<int32_t> anc(n, -1);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t q = rp[i]; q < rp[i + 1]; ++q) {
                int32_t r = rc[q];
                while (anc[r] != -1 && anc[r] != i) {
                    int32_t nx = anc[r];
                    anc[r] = (int32_t)i;
                    r = nx;
                }
                if (anc[r] == -1) {
                    anc[r] = (int32_t)i;
                    S.parent[r] = (int32_t)i;
                }
            }
    }
    // ---- column counts by row subtrees ------------------------------------
    S.colcount.assign(n, 1);
    {
        std::vector<int32_t> mark(n, -1);
        for (int64_t i = 0; i < n; ++i) {
            mark[i] = (int32_t)i;
            for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
                for (int32_t k = rc[q]; mark[k] != i; k = S.parent[k]) {
                    ++S.colcount[k];
                    mark[k] = (int32_t)i;
                }
        }
    }
    S.flops = 0.0;
    S.nnzL = 0;
    for (int64_t j = 0; j < n; ++j) {
        S.flops += (double)S.colcount[j] * (double)S.colcount[j];
        S.nnzL += S.colcount[j];
    }

    // ---- fundamental supernodes, relaxed amalgamation ---------------------
    std::vector<int32_t> nchild(n, 0);
    for (int64_t j = 0; j < n; ++j)
        if (S.parent[j] >= 0) ++nchild[S.parent[j]];
    std::vector<int32_t> fstart;
    for (int64_t j = 0; j < n; ++j) {
        bool cont = j > 0 && S.parent[j - 1] == j && S.colcount[j - 1] == S.colcount[j] + 1 &&
                    nchild[j] == 1;
        if (!cont) fstart.push_back((int32_t)j);
    }
    fstart.push_back((int32_t)n);
    auto trap = [](int64_t k, int64_t m) { return k * m - k * (k - 1) / 2; };
    S.sfirst.clear();
    {
        int64_t width = 0, sum = 0, last = -1;
        for (size_t t = 0; t + 1 < fstart.size(); ++t) {
            const int64_t f = fstart[t], l = fstart[t + 1] - 1, kt = l - f + 1;
            const int64_t below = S.colcount[f] - kt;
            int64_t st = 0;
            for (int64_t j = f; j <= l; ++j) st += S.colcount[j];
            if (!S.sfirst.empty() && S.parent[last] == f) {
                const int64_t k2 = width + kt, m2 = k2 + below, s2 = sum + st;
                const int64_t tr = trap(k2, m2);
                if (k2 <= relax_k || 100 * (tr - s2) <= (int64_t)relax_pct * tr) {
                    width = k2;
                    sum = s2;
                    last = l;
                    continue;
                }
            }
            S.sfirst.push_back((int32_t)f);
            width = kt;
            sum = st;
            last = l;
        }
        S.sfirst.push_back((int32_t)n);
    }
    const int32_t ns = (int32_t)S.sfirst.size() - 1;
    S.ns = ns;
    std::vector<int32_t> col2s(n);
    for (int32_t s = 0; s < ns; ++s)
        for (int32_t j = S.sfirst[s]; j < S.sfirst[s + 1]; ++j) col2s[j] = s;
    S.sparent.assign(ns, -1);
    for (int32_t s = 0; s < ns; ++s) {
        int32_t p = S.parent[S.sfirst[s + 1] - 1];
        S.sparent[s] = p < 0 ? -1 : col2s[p];
    }
    S.child_ptr.assign(ns + 1, 0);
    for (int32_t s = 0; s < ns; ++s)
        if (S.sparent[s] >= 0) ++S.child_ptr[S.sparent[s] + 1];
    for (int32_t s = 0; s < ns; ++s) S.child_ptr[s + 1] += S.child_ptr[s];
    S.children.resize(S.child_ptr[ns]);
    {
        std::vector<int32_t> fill(S.child_ptr.begin(), S.child_ptr.end() - 1);
        for (int32_t s = 0; s < ns; ++s)
            if (S.sparent[s] >= 0) S.children[fill[S.sparent[s]]++] = s;
    }

    // ---- front rows: own columns, A's rows below, children's update rows --
    S.srowptr.assign(ns + 1, 0);
    S.srows.clear();
    {
        std::vector<int32_t> mark(n, -1), tmp;
        for (int32_t s = 0; s < ns; ++s) {
            const int32_t f = S.sfirst[s], l = S.sfirst[s + 1] - 1;
            tmp.clear();
            for (int32_t j = f; j <= l; ++j)
                for (int64_t e = S.pcp[j]; e < S.pcp[j + 1]; ++e) {
                    int32_t i = S.prow[e];
                    if (i > l && mark[i] != s) {
                        mark[i] = s;
                        tmp.push_back(i);
                    }
                }
            for (int32_t c = S.child_ptr[s]; c < S.child_ptr[s + 1]; ++c) {
                const int32_t ch = S.children[c];
                for (int64_t q = S.srowptr[ch] + S.k(ch); q < S.srowptr[ch + 1]; ++q) {
                    int32_t i = S.srows[q];
                    if (i > l && mark[i] != s) {
                        mark[i] = s;
                        tmp.push_back(i);
                    }
                }
            }
            std::sort(tmp.begin(), tmp.end());
            for (int32_t j = f; j <= l; ++j) S.srows.push_back(j);
            S.srows.insert(S.srows.end(), tmp.begin(), tmp.end());
            S.srowptr[s + 1] = (int64_t)S.srows.size();
            if ((int64_t)tmp.size() != S.colcount[l] - 1) {
                msg = "internal: supernode row count disagrees with column count";
                return ERR_INVALID_ARG;
            }
        }
    }
    S.nnzL_stored = 0;
    for (int32_t s = 0; s < ns; ++s) S.nnzL_stored += trap(S.k(s), S.m(s));

    // ---- levels (height in the supernodal tree) ---------------------------
    S.slevel.assign(ns, 0);
    for (int32_t s = 0; s < ns; ++s)
        if (S.sparent[s] >= 0) S.slevel[S.sparent[s]] = std::max(S.slevel[S.sparent[s]], S.slevel[s] + 1);
    S.nlevels = 0;
    for (int32_t s = 0; s < ns; ++s) S.nlevels = std::max(S.nlevels, S.slevel[s] + 1);
    S.level_ptr.assign(S.nlevels + 1, 0);
    for (int32_t s = 0; s < ns; ++s) ++S.level_ptr[S.slevel[s] + 1];
    for (int32_t l = 0; l < S.nlevels; ++l) S.level_ptr[l + 1] += S.level_ptr[l];
    S.level_nodes.resize(ns);
    {
        std::vector<int32_t> fill(S.level_ptr.begin(), S.level_ptr.end() - 1);
        for (int32_t s = 0; s < ns; ++s) S.level_nodes[fill[S.slevel[s]]++] = s;
    }

    // ---- extend-add gather maps ------------------------------------------
    S.mapoff.assign(ns, -1);
    {
        int64_t tot = 0;
        for (int32_t s = 0; s < ns; ++s)
            if (S.sparent[s] >= 0) {
                S.mapoff[s] = tot;
                tot += S.m(S.sparent[s]);
            }
        S.relmap.assign(tot, -1);
        std::vector<int32_t> pos(n, -1);
        for (int32_t c = 0; c < ns; ++c) {
            const int32_t p = S.sparent[c];
            if (p < 0) continue;
            const int32_t kc = S.k(c);
            for (int64_t q = S.srowptr[c] + kc; q < S.srowptr[c + 1]; ++q)
                pos[S.srows[q]] = (int32_t)(q - S.srowptr[c] - kc);
            for (int64_t r = 0; r < S.m(p); ++r)
                S.relmap[S.mapoff[c] + r] = pos[S.srows[S.srowptr[p] + r]];
            for (int64_t q = S.srowptr[c] + kc; q < S.srowptr[c + 1]; ++q) pos[S.srows[q]] = -1;
        }
    }
    // ---- assembly: local row of each lower entry in its front -------------
    S.alrow.assign(nnz, -1);
    {
        std::vector<int32_t> loc(n, -1);
        for (int32_t s = 0; s < ns; ++s) {
            for (int64_t q = S.srowptr[s]; q < S.srowptr[s + 1]; ++q)
                loc[S.srows[q]] = (int32_t)(q - S.srowptr[s]);
            for (int32_t j = S.sfirst[s]; j < S.sfirst[s + 1]; ++j)
                for (int64_t e = S.pcp[j]; e < S.pcp[j + 1]; ++e) S.alrow[e] = loc[S.prow[e]];
            for (int64_t q = S.srowptr[s]; q < S.srowptr[s + 1]; ++q) loc[S.srows[q]] = -1;
        }
    }
    return OK;
}

// Block-diagonal union of independent analyses: instance i occupies columns
// [coff_i, coff_i + n_i), its supernodes, rows, stored values and maps are
// shifted by the running totals; levels (tree heights) merge, so one launch
// per level covers every instance.
int merge(Symbolic &S, const std::vector<const Symbolic *> &parts, std::string &msg) {
    S = Symbolic();
    int64_t n = 0, nnz = 0, nrows = 0, nmap = 0;
    int64_t ns = 0;
    int32_t nlev = 0;
    for (const Symbolic *P : parts) {
        n += P->n;
        nnz += P->pcp[P->n];
        nrows += (int64_t)P->srows.size();
        nmap += (int64_t)P->relmap.size();
        ns += P->ns;
        nlev = std::max(nlev, P->nlevels);
    }
    if (n > INT32_MAX || nnz > INT32_MAX || 2 * nnz - n > INT32_MAX || ns > INT32_MAX ||
        nrows > INT64_MAX / 2) {
        msg = "batch too large for 32-bit column / value indices";
        return ERR_INVALID_ARG;
    }
    S.n = n;
    S.perm.reserve(n);
    S.iperm.reserve(n);
    S.parent.reserve(n);
    S.colcount.reserve(n);
    S.pcp.assign(1, 0);
    S.pcp.reserve(n + 1);
    S.prow.reserve(nnz);
    S.psrc.reserve(nnz);
    S.pswap.reserve(nnz);
    S.alrow.reserve(nnz);
    S.sfirst.reserve(ns + 1);
    S.srowptr.assign(1, 0);
    S.srowptr.reserve(ns + 1);
    S.srows.reserve(nrows);
    S.sparent.reserve(ns);
    S.slevel.reserve(ns);
    S.mapoff.reserve(ns);
    S.relmap.reserve(nmap);
    int32_t coff = 0, soff = 0;
    int64_t voff = 0, roff = 0, moff = 0;
    for (const Symbolic *P : parts) {
        for (int64_t j = 0; j < P->n; ++j) {
            S.perm.push_back(P->perm[j] + coff);
            S.iperm.push_back(P->iperm[j] + coff);
            S.parent.push_back(P->parent[j] < 0 ? -1 : P->parent[j] + coff);
            S.colcount.push_back(P->colcount[j]);
            S.pcp.push_back(P->pcp[j + 1] + voff);
        }
        for (size_t e = 0; e < P->prow.size(); ++e) {
            S.prow.push_back(P->prow[e] + coff);
            S.psrc.push_back((int32_t)(P->psrc[e] + voff));
            S.pswap.push_back(P->pswap[e]);
            S.alrow.push_back(P->alrow[e]);
        }
        for (int32_t t = 0; t < P->ns; ++t) {
            S.sfirst.push_back(P->sfirst[t] + coff);
            S.srowptr.push_back(P->srowptr[t + 1] + roff);
            S.sparent.push_back(P->sparent[t] < 0 ? -1 : P->sparent[t] + soff);
            S.slevel.push_back(P->slevel[t]);
            S.mapoff.push_back(P->mapoff[t] < 0 ? -1 : P->mapoff[t] + moff);
        }
        for (int32_t r : P->srows) S.srows.push_back(r + coff);
        S.relmap.insert(S.relmap.end(), P->relmap.begin(), P->relmap.end());
        S.flops += P->flops;
        S.nnzL += P->nnzL;
        S.nnzL_stored += P->nnzL_stored;
        coff += (int32_t)P->n;
        soff += P->ns;
        voff += P->pcp[P->n];
        roff += (int64_t)P->srows.size();
        moff += (int64_t)P->relmap.size();
    }
    S.sfirst.push_back((int32_t)n);
    S.ns = (int32_t)ns;
    S.child_ptr.assign(ns + 1, 0);
    for (int32_t t = 0; t < S.ns; ++t)
        if (S.sparent[t] >= 0) ++S.child_ptr[S.sparent[t] + 1];
    for (int32_t t = 0; t < S.ns; ++t) S.child_ptr[t + 1] += S.child_ptr[t];
    S.children.resize(S.child_ptr[ns]);
    {
        std::vector<int32_t> fill(S.child_ptr.begin(), S.child_ptr.end() - 1);
        for (int32_t t = 0; t < S.ns; ++t)
            if (S.sparent[t] >= 0) S.children[fill[S.sparent[t]]++] = t;
    }
    S.nlevels = nlev;
    S.level_ptr.assign(nlev + 1, 0);
    for (int32_t t = 0; t < S.ns; ++t) ++S.level_ptr[S.slevel[t] + 1];
    for (int32_t l = 0; l < nlev; ++l) S.level_ptr[l + 1] += S.level_ptr[l];
    S.level_nodes.resize(ns);
    {
        std::vector<int32_t> fill(S.level_ptr.begin(), S.level_ptr.end() - 1);
        for (int32_t t = 0; t < S.ns; ++t) S.level_nodes[fill[S.slevel[t]]++] = t;
    }
    return OK;
}

}  // namespace wd
