// Host-side symbolic analysis of P A P^T for the multifrontal Cholesky engine.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace wd {

struct Symbolic {
    int64_t n = 0;
    std::vector<int32_t> perm, iperm;        // perm[new] = old
    std::vector<int32_t> parent;             // elimination tree of P A P^T
    std::vector<int64_t> colcount;           // nonzeros of L(:, j) incl. diagonal

    // lower triangle of P A P^T by columns: row and index of the source value
    std::vector<int64_t> pcp;
    std::vector<int32_t> prow;
    std::vector<int32_t> psrc;
    // 1 where the entry (row, col) of P A P^T is the transposed position of
    // its source entry (the caller's row maps to the column), for
    // nonsymmetric values given as both triangles
    std::vector<int8_t> pswap;

    // supernodes (contiguous column ranges)
    int32_t ns = 0;
    std::vector<int32_t> sfirst;             // ns + 1
    std::vector<int64_t> srowptr;            // ns + 1
    std::vector<int32_t> srows;              // front rows, own columns first
    std::vector<int32_t> sparent;            // supernodal tree, -1 for roots
    std::vector<int32_t> slevel;             // height: leaves 0
    std::vector<int32_t> child_ptr, children;
    int32_t nlevels = 0;
    std::vector<int32_t> level_ptr, level_nodes;  // supernodes by level

    // extend-add gather map of child c: for each row r of its parent's front,
    // the index of that row among c's update rows, or -1 (length m_parent)
    std::vector<int64_t> mapoff;
    std::vector<int32_t> relmap;
    // local row (within its supernode's front) of every lower entry of P A P^T
    std::vector<int32_t> alrow;

    double flops = 0.0;                      // sum_j c_j^2
    int64_t nnzL = 0, nnzL_stored = 0;

    int32_t k(int32_t s) const { return sfirst[s + 1] - sfirst[s]; }
    int32_t m(int32_t s) const { return (int32_t)(srowptr[s + 1] - srowptr[s]); }
};

// Returns 0 or a wd_status code, with msg describing the failure.
// patch: optional patch id (0..31) per vertex, NULL for a single domain.
int analyze(Symbolic &S, int64_t n, const int64_t *colptr, const int32_t *rowidx, int dim,
            const int32_t *level, const int32_t *box_lo, const int32_t *box_side,
            const int32_t *patch, int leaf, int relax_k, int relax_pct, std::string &msg);

// Block-diagonal union of independent analyses (instances in order).
int merge(Symbolic &S, const std::vector<const Symbolic *> &parts, std::string &msg);

}  // namespace wd
