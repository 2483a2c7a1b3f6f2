// Device-side data of the multifrontal engine and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace wd {

// status word of a factorization: smallest failing column (UINT64_MAX = none)
using status_t = unsigned long long;

constexpr int NB = 64;        // pivot block width and Schur tile size
constexpr int RB = 64;        // rows per panel (TRSM) block

// Device pointers of the analysis (all arrays are owned by the handle).
struct DevSym {
    int64_t n;
    int32_t ns;
    const int32_t *sfirst;      // ns+1: first column of each supernode
    const int32_t *sk;          // ns: width k_s
    const int32_t *sm;          // ns: number of front rows m_s
    const int32_t *skp;         // ns: k_s rounded up to 32 (first row of R in the front)
    const int32_t *sld;         // ns: leading dimension of the front (multiple of 32)
    const int64_t *foff;        // ns: offset of front s in the front pool
    const int64_t *rowptr;      // ns+1: offset of the rows of s
    const int32_t *rows;        // front rows (global permuted indices)
    const int32_t *child_ptr;   // ns+1
    const int32_t *children;
    const int64_t *mapoff;      // ns: offset of child's gather map (length m_parent)
    const int32_t *relmap;
    const int64_t *pcp;         // n+1: lower CSC of P A P^T
    const int32_t *alrow;       // front row of each lower entry in its supernode's front
    const int64_t *csr_ptr;     // n+1: full CSR of P A P^T
    const int32_t *csr_col;
    const int64_t *csr_diag;    // n: position of the diagonal in each CSR row
    const double *csr_val;      // FP64 values of P A P^T (full)
    const int64_t *woff;        // ns: prefix sum of (m_s - k_s) (solve workspace)
    const int64_t *dinvoff;     // ns: offset of the supernode's inverse diagonal blocks
    const int64_t *pkoff;       // ns: byte offset of the supernode's packed tf32 panel lines
    const int32_t *perm;        // n
};

// Set the dynamic shared-memory limits of all kernels (once per process,
// before any stream capture).
void init_front_attributes();
void init_solve_attributes();
void init_tc_attributes();
void init_blocked_attributes();
void init_tc_solve_attributes();
void init_lu_attributes();
void init_oz_attributes();
void init_chain_attributes();
inline void init_kernel_attributes() {
    init_front_attributes();
    init_solve_attributes();
    init_tc_attributes();
    init_blocked_attributes();
    init_tc_solve_attributes();
    init_lu_attributes();
    init_oz_attributes();
    init_chain_attributes();
}


// ---- factorization (front_kernels.cu) ------------------------------------
template <class T>
void launch_front_init(const DevSym &d, T *front, const int4 *items, int count, cudaStream_t st);
// diagonal block (s, kb) of each item: L11 into the front, L11^-1 into dinv
// at dinvoff + (kb / NB) NB^2; FP32 fronts of width >= diag64_min_k (> 0)
// factor the block in FP64
template <class T>
void launch_diag_factor(const DevSym &d, T *front, T *dinv, const int4 *items, int count, int diag64_min_k,
                        status_t *status, cudaStream_t st);
// panel of pivot block kb (L11^-1 in dinv): L21 = F21 L11^-T for the items'
// 64-row blocks; pk != nullptr (FP32 only): also write the packed tf32 lines
template <class T>
void launch_panel(const DevSym &d, T *front, const T *dinv, unsigned char *pk, const int4 *items, int count,
                  int kb, cudaStream_t st);
// mode 0: pivot-column update of step kb, then the CTA of tile (0, 0) factors
// diagonal block kb + NB (into the front and dinv); mode 1: final update
// matrix (syrk)
template <class T>
void launch_schur(const DevSym &d, T *front, T *dinv, const int4 *items, int count, int kb,
                  int mode, status_t *status, cudaStream_t st);
constexpr int SCHUR_BM = 128, SCHUR_BN = 64;

// Packed tf32 operand lines of a supernode's L panel (FP32 fronts, tensor-core
// Schur updates): for each chunk kc of 32 pivot columns and plane p (0 = hi,
// 1 = lo part of the split), one 128-byte line per front row holding the 32
// tf32 values, its 16-byte groups XOR-swizzled by (row & 7) -- the 128-byte
// swizzled K-major image of the MMA operand, so rows [r, r + 128) of a chunk
// (r a multiple of 8) form one contiguous 16 KB tile.  Rows are padded by 128
// so that every window starting below mp stays inside the allocation.
__host__ __device__ inline int pack_rows(int mp) { return ((mp + 7) / 8) * 8 + 128; }
__host__ __device__ inline int pack_chunks(int k) { return 2 * ((k + 63) / 64); }
__host__ __device__ inline int64_t pack_offset(int kc, int p, int row, int prow) {
    return ((int64_t)(kc * 2 + p) * prow + row) * 128;
}
__host__ __device__ inline int64_t pack_bytes(int k, int mp) {
    return (int64_t)pack_chunks(k) * 2 * pack_rows(mp) * 128;
}

// tensor-core Schur update of FP32 fronts (tc_schur.cu); 128 x 128 tiles;
// mode 0 also factors the next diagonal block in the CTA of tile (0, 0) (in
// FP64 for fronts of width >= diag64_min_k > 0).  Bounded waits: wait_limit
// polls (0: the default); gate != nullptr: every CTA also waits, after its
// products, for *gate != 0 (a test of the timeout path).  tstatus != 0 after
// the launch means a bounded wait expired.
constexpr int TC_BM = 128, TC_BN = 128;
struct TcArgs {
    float *dinv;
    status_t *status;
    status_t *tstatus;
    int diag64_min_k;
    uint32_t wait_limit;
    const unsigned *gate;
    int ctas;               // mode 1: > 0 runs the persistent kernel on this many CTAs (one per SM)
};
void launch_tc_schur(const DevSym &d, float *front, const unsigned char *pk, const int4 *items,
                     int count, int kb, int mode, const TcArgs &a, cudaStream_t st);
void init_tc_attributes();

// Pivot columns of the FP32 fronts of one level in one launch (tc_chain.cu):
// items (s, c, ti) in dependency order (column block c, then row tile ti of
// 128 rows from row 64c, then front); each task forms its tile of the pivot
// columns with a tensor-core product over all earlier column blocks, the
// ti = 0 task factors the diagonal block (L11, L11^-1 into dinv) and every
// task writes its panel rows (front and packed tf32 lines).  Dependency
// words: flags + flagoff[s], ready[j * nrb + rb] for row block rb of column
// block j (nrb = ceil(mp / 64) + 1), then diag[j]; counter[level] hands out
// the tasks; all of them zero before the launch.  Bounded waits as in the
// Schur kernel; *gabort != 0 after a timeout in any CTA.
struct ChainArgs {
    float *dinv;
    unsigned char *lpack;   // L11^-1 of every diagonal block as a tf32 hi / lo operand (32 KB each,
                            // block c of supernode s at (dinvoff[s] / NB^2 + c) x 32 KB)
    status_t *status;
    status_t *tstatus;
    uint32_t wait_limit;
    const unsigned *gate;
    unsigned *flags;
    const int64_t *flagoff;
    unsigned *counter;
    unsigned *gabort;
};
__host__ __device__ inline int64_t chain_flag_words(int k, int mp) {
    const int64_t ncb = (k + NB - 1) / NB, nrb = (mp + NB - 1) / NB + 1;
    return ncb * nrb + ncb;
}
void launch_tc_chain(const DevSym &d, float *front, unsigned char *pk, const int4 *items, int count, int level,
                     const ChainArgs &a, cudaStream_t st);

// FP64 Schur updates through bf16 slices on the tensor cores (oz_schur.cu):
// per supernode s and 64-column pivot block b, eight planes of 128-byte lines
// (one per front row, pack_rows(mp) rows) at sl + soff[s] + ((b * 8 + q) *
// pack_rows(mp) + row) * 128, and the row scales' exponents at ex + eoff[s] +
// b * pack_rows(mp) + row
struct OzArgs {
    unsigned char *sl;
    int16_t *ex;
    const int64_t *soff;
    const int64_t *eoff;
    double *dinv;
    status_t *status;
    status_t *tstatus;
    uint32_t wait_limit;
};
void launch_oz_slice(const DevSym &d, const double *front, const OzArgs &a, const int4 *items, int count, int kb,
                     cudaStream_t st);
void launch_oz_schur(const DevSym &d, double *front, const int4 *items, int count, int kb, int mode,
                     const OzArgs &a, cudaStream_t st);
void init_oz_attributes();

// ---- values, solves and reductions (solve_kernels.cu) ---------------------
// csr_val = values in CSR order; hi / lo (nullable): its double-float split
void launch_gather_values(const int32_t *csr_src, const double *values, double *csr_val, float *hi,
                          float *lo, int64_t nnz, cudaStream_t st);
template <class T>
void launch_permute_in(const double *B, int64_t ldb, T *Y, const int32_t *perm, int64_t n,
                       int64_t nrhs, cudaStream_t st);
template <class T>
void launch_permute_out(const T *Y, double *B, int64_t ldb, const int32_t *perm, int64_t n,
                        int64_t nrhs, cudaStream_t st);
template <class T>
void launch_apply_L(const DevSym &d, const T *front, const T *Z, T *Out, T *W,
                    const int4 *items, int count, int nrhs, cudaStream_t st);
// Y += alpha G X, G given by its values on the full CSR of P A P^T (FP64,
// row-major n x nrhs vectors, factor order)
void launch_spmv_axpy(const DevSym &d, const double *vals, const double *X, double alpha, double *Y,
                      int64_t nrhs, cudaStream_t st);
// refinement vectors are row-major (n x nrhs, right-hand sides contiguous)
void launch_permute_in_rm(const double *B, int64_t ldb, double *Bp, const int32_t *perm, int64_t n,
                          int64_t nrhs, cudaStream_t st);
// theta-scheme staging: Bp = a U + g F (F nullable), X = x U, both in factor
// order, row-major; U, F column-major n x nrhs (ld) in the original order
void launch_theta_stage(const double *U, const double *F, int64_t ld, const int32_t *perm, int64_t n,
                        int64_t nrhs, double a, double x, double g, double *Bp, double *X, cudaStream_t st);
void launch_permute_out_rm(const double *X, double *B, int64_t ldb, const int32_t *perm, int64_t n,
                           int64_t nrhs, cudaStream_t st);
// dir 0: C (column-major) = Rm; dir 1: Rm (=, or += if accumulate) C
template <class Tc>
void launch_transpose(Tc *C, double *Rm, int64_t n, int64_t nrhs, int dir, int accumulate,
                      cudaStream_t st);
// chunks: (row, first entry, end, slot or -1); fin: (row, first slot, slots);
// bad: smallest CSR position whose column index is outside [0, n) (atomic
// minimum; the caller sets it to UINT64_MAX first; used for nrhs <= 8)
constexpr int SPMV_CHUNK = 512;
void launch_spmv_residual(const DevSym &d, const int4 *chunks, int nchunks, const int4 *fin,
                          int nfin, const double *X, const double *Bp, double *R, double *P,
                          int64_t nrhs, unsigned long long *bad, cudaStream_t st);
// the same residual in double-float arithmetic (vh + vl = the CSR values;
// Xp: n x nrhs scratch for the split of X as (hi, lo) pairs)
void launch_spmv_residual_df(const DevSym &d, const int4 *chunks, int nchunks, const int4 *fin, int nfin,
                             const float *vh, const float *vl, const double *X, float2 *Xp,
                             const double *Bp, double *R, double *P, int64_t nrhs, cudaStream_t st);
// R = S - A x in double-float arithmetic for x exactly FP32 (Xf, row-major
// n x nrhs): the refinement's first residual (S = b) and its recurrence
// r <- r - A d (S = R, in place)
void launch_spmv_residual_df32(const DevSym &d, const int4 *chunks, int nchunks, const int4 *fin, int nfin,
                               const float *vh, const float *vl, const float *Xf, const double *S, double *R,
                               double *P, int64_t nrhs, cudaStream_t st);
// Y (FP32, column-major) into X (FP64 row-major; = or +=) and Xf (FP32 row-major)
void launch_xupdate(const float *Y, double *X, float *Xf, int64_t n, int64_t nrhs, int accumulate,
                    cudaStream_t st);
void launch_norm_inf_rows(const DevSym &d, const int4 *chunks, int nchunks, const int4 *fin,
                          int nfin, double *partial, double *out, cudaStream_t st);
void launch_colmax3(const double *R, const double *X, const double *Bp, int64_t n,
                    int64_t nrhs, double *out3, cudaStream_t st);
template <class T>
void launch_axpy_into(double *X, const T *D, int64_t count, int accumulate, cudaStream_t st);
template <class T>
void launch_cast(const double *src, T *dst, int64_t count, cudaStream_t st);
template <class T>
void launch_logdet_partial(const DevSym &d, const T *front, double *partial, int nblocks,
                           cudaStream_t st);
void launch_sum_final(const double *partial, int count, double *out, cudaStream_t st);
template <class T>
void launch_export_panels(const DevSym &d, const T *front, double *panels,
                          const int64_t *poff, cudaStream_t st);

// ---- selected inverse (selinv.cu), FP64 --------------------------------------
// C(i, j) (+)= alpha sum_{p in [p0, p1)} A(i, p) B(j, p) on the 64 x 64 tile at
// (i0, j0) of an M x N matrix C; element (r, c) of X at X[r * x_rs + c * x_cs]
enum { GEMM_A_SYM_LOWER = 1, GEMM_C_LOWER = 2, GEMM_ACCUMULATE = 4 };
struct GemmItem {
    const double *A;
    const double *B;
    double *C;
    int64_t a_rs, a_cs, b_rs, b_cs, c_rs, c_cs;
    int M, N, p0, p1, i0, j0, flags, pad;
    double alpha;
};
void launch_gemm_items(const GemmItem *items, int count, cudaStream_t st);
void launch_trinv(const DevSym &d, const double *front, const double *dinv, double *xpool,
                  const int64_t *xoff, const int4 *items, int count, cudaStream_t st);
void launch_zgather(const DevSym &d, double *zpool, const int32_t *upmap, const int64_t *upoff,
                    const int4 *items, int count, cudaStream_t st);
void launch_zextract(const DevSym &d, const double *zpool, const int32_t *col2s, const int32_t *psrc,
                     double *out, cudaStream_t st);
// out[src] = alpha * (pattern part of U V^T + V U^T) + zscale * w * Zsel[src] (Zsel nullable)
void launch_sym_outer(const DevSym &d, const int32_t *prow, const int32_t *psrc, const double *U,
                      const double *V, int64_t ncols, int64_t ld, double alpha, const double *Zsel,
                      double zscale, double *out, cudaStream_t st);

// ---- solves by super-blocks (solve_blocked.cu) ----------------------------
// A supernode's pivot columns are cut into super-blocks of SB columns; the
// explicit inverse of every super-block's diagonal block is stored (X, and
// its transpose XT) at xsoff[s] + sb * SB * SB, column-major with leading
// dimension wp = roundup(width, NB).
constexpr int SB = 512;
template <class T>
void launch_sbinv_diag(const DevSym &d, const T *dinv, T *xpool, const int64_t *xsoff, const int4 *items,
                       int count, cudaStream_t st);
template <class T>
void launch_sbinv_stage(const DevSym &d, const T *front, const T *dinv, T *xpool, const int64_t *xsoff,
                        const int4 *items, int count, int t, cudaStream_t st);
template <class T>
void launch_sbinv_transpose(const DevSym &d, const T *xpool, T *xtpool, const int64_t *xsoff,
                            const int4 *items, int count, cudaStream_t st);
// rgt: right-hand sides per CTA tile (64 or 16)
template <class T>
void launch_bfwd_gather(const DevSym &d, const T *Y, T *Tt, T *W, const int4 *items, int count, int rgt,
                        int nrhs, cudaStream_t st);
// xapply / bupdate / breduce modes ("large"): 0 -> tiles of 64 rows x 32
// right-hand sides per CTA; 1 -> FP32 on the tensor cores, tiles of 128 rows
// x 64 right-hand sides (tc_solve.cu); 2 -> up to 8 right-hand sides, matrix-vector
// shaped (32 rows per xapply / bupdate CTA, lanes over rows; breduce keeps the
// 64-column items and the 64 x 32 partial layout of mode 0); the partial-sum
// tile sizes (the same for both modes):
int solve_tile_rows(int large);
int solve_tile_rhs(int large);
// rows per CTA of the xapply / bupdate items (mode 0: 64, mode 2: 32)
int solve_update_rows(int large);
template <class T>
void launch_xapply(const DevSym &d, const T *xp, const int64_t *xsoff, const T *in, T *out,
                   const int4 *items, int count, int upper, int large, int nrhs, cudaStream_t st);
template <class T>
void launch_bupdate(const DevSym &d, const T *front, const T *Y, T *Tt, T *W, const int4 *items, int count,
                    int large, int nrhs, cudaStream_t st);
// split reduction of the backward pass: partial sums of KSR-row splits into
// P (rows x rhs of the tile per slot), then Tt = y - sum over the splits in order
constexpr int SOLVE_KSR = 128;
template <class T>
void launch_breduce(const DevSym &d, const T *front, const T *Y, T *P, const int4 *items, int count,
                    int large, int nrhs, cudaStream_t st);
template <class T>
void launch_breduce_finish(const DevSym &d, const T *Y, T *Tt, const T *P, const int4 *items, int count,
                           int large, int nrhs, cudaStream_t st);

// ---- tensor-core products of the solves (tc_solve.cu; FP32 fronts, mode 1) --
// Tiles of 128 rows (xapply, bupdate) or 128 pivot columns (breduce) x 64
// right-hand sides; items as in mode 0 with these tile sizes; breduce splits
// the rows below a super-block into SOLVE_KSR_TC storage rows of the front,
// counted from the first 32-row boundary at or above the super-block's end.
constexpr int SOLVE_KSR_TC = 256;
struct TcSolveArgs {
    const float *front;           // FP32 fronts
    const unsigned char *pk;      // packed tf32 lines of L (bupdate's A)
    const float *xp;              // xapply: forward X^T, backward X (super-block inverses)
    const int64_t *xsoff;
    const float *in;              // xapply: t; bupdate: y; breduce: x
    float *out;                   // xapply: y / x; bupdate: the pending right-hand side; breduce: partials
    float *W;                     // bupdate: update vectors
    status_t *tstatus;            // nonzero after the launch: a bounded wait expired
    int nrhs;
    int upper;                    // xapply: 0 forward (lower X), 1 backward (X^T)
    uint32_t wait_limit;          // 0: the default
    float *ksw;                   // split inner dimension: one partial tile per CTA
    int *kcnt;                    // split inner dimension: arrivals per output tile (zero between launches)
    int sms;                      // the device's SMs: a bupdate launch of more CTAs than SMs runs two per SM
};
constexpr int TC_SOLVE_TILE = 128 * 64;   // entries of one output tile of the tensor-core solve products
void launch_tc_xapply(const DevSym &d, const TcSolveArgs &a, const int4 *items, int count, cudaStream_t st);
void launch_tc_bupdate(const DevSym &d, const TcSolveArgs &a, const int4 *items, int count, cudaStream_t st);
void launch_tc_breduce(const DevSym &d, const TcSolveArgs &a, const int4 *items, int count, cudaStream_t st);

// ---- per-instance reductions of a block-diagonal batch (batch.cu) ----------
// out[i] = ||A_i||_inf from the residual product's chunk items (partial:
// scratch of one double per slot)
void launch_seg_norm_inf(const DevSym &d, const int4 *chunks, int nchunks, const int4 *fin, int nfin,
                         double *partial, const int64_t *coff, int count, double *out, cudaStream_t st);
void launch_seg_colmax3(const double *R, const double *X, const double *B, const int64_t *coff, int count,
                        int nrhs, double *out, cudaStream_t st);
// out[i] = log det A_i (sdl: scratch of one double per supernode)
template <class T>
void launch_seg_logdet(const DevSym &d, const T *front, const int32_t *soff, int count, double *sdl,
                       double *out, cudaStream_t st);

// ---- LU without pivoting, FP64 (lu.cu) --------------------------------------
// code[e] of a full-CSR position: 0 -> (entry, transposed) = (lower, upper)
// of its source, 1 -> (upper, lower), 2 -> (lower, lower) (the diagonal)
void launch_lu_gather(const int32_t *src, const int8_t *code, const double *lower, const double *upper,
                      double *vrow, double *vcol, int64_t nnz, cudaStream_t st);
void launch_lu_init(const DevSym &d, double *front, const double *vrow, const double *vcol, const int4 *items,
                    int count, cudaStream_t st);
void launch_lu_diag(const DevSym &d, double *front, double *linv, double *uinv, const int4 *items, int count,
                    int kb, status_t *status, cudaStream_t st);
// items (s, block, side): side 0 rows below the pivot block, side 1 columns right of it
void launch_lu_panel(const DevSym &d, double *front, const double *linv, const double *uinv, const int4 *items,
                     int count, int kb, cudaStream_t st);
// items (s, ti, tj): 64 x 64 tiles of the trailing square of step kb
void launch_lu_update(const DevSym &d, double *front, const int4 *items, int count, int kb, cudaStream_t st);
// substitutions on Y (n x nrhs, nrhs <= 64, column-major, factor order):
// forward items (s, block) (block 0: y of the pivot block; >= 1: 64 later rows),
// backward items (s, 0, 0, 0)
void launch_lu_fwd(const DevSym &d, const double *front, const double *linv, double *Y, double *Tt, double *W,
                   const int4 *items, int count, int kb, int nrhs, cudaStream_t st);
void launch_lu_bwd(const DevSym &d, const double *front, const double *uinv, double *Y, const int4 *items,
                   int count, int kb, int nrhs, cudaStream_t st);
// partial[b] = sum of log |U_jj| over a grid-stride share of the supernodes,
// partial[nblocks + b] = the number of negative pivots there
void launch_lu_logdet(const DevSym &d, const double *front, double *partial, int nblocks, cudaStream_t st);
// factor panels for export: L with its unit diagonal, and U^T, each m_s x k_s per supernode
void launch_lu_export(const DevSym &d, const double *front, double *lpan, double *upan, const int64_t *poff,
                      cudaStream_t st);

// ---- allocation-free export of the factor (noalloc.cu) ---------------------
// the panel offsets sit in a static device array of NOALLOC_MAX_SUPERNODES + 1
// entries; *addr = its address on `device` (looked up once per device)
constexpr int NOALLOC_MAX_SUPERNODES = 65536;
cudaError_t noalloc_panel_offsets(int device, int64_t **addr);
// writes the offsets of all d.ns panels (d.ns <= NOALLOC_MAX_SUPERNODES)
void launch_panel_offsets_noalloc(const DevSym &d, cudaStream_t st);

}  // namespace wd
