// Selected inverse: Z = (P A P^T)^-1 on the pattern of L (Takahashi's
// recurrences in supernodal form), FP64, top-down over the supernodal tree.
//
// From Z L = L^-T (L^-T is upper triangular, so its (R, J) block is zero),
// for a supernode with pivot columns J and rows R below it:
//   W    = L_RJ L_JJ^-1
//   Z_RJ = -Z_RR W
//   Z_JJ = L_JJ^-T L_JJ^-1 - W^T Z_RJ
// Z_RR (the rows of R are a clique of L's graph, all owned by ancestors) is
// gathered from the parent's Z front through the extend-add row maps.  Every
// supernode stores its whole Z front (rows x rows, lower), laid out like its
// factor front.  L_JJ^-1 is built by blocked inversion from the stored
// inverses of the 64 x 64 diagonal blocks:
//   X(bi, bj) = -D(bi)^-1 sum_{p in blocks bj .. bi-1} L(bi, p) X(p, bj).
#include "dev_common.cuh"
#include "engine.h"

namespace wd {
namespace {

constexpr int THREADS = 256;
constexpr int TM = 64, TN = 64, TK = 16;

// C(i, j) (+)= alpha sum_p A(i, p) B(j, p) on one 64 x 64 tile.  a_pfast /
// b_pfast: the operand is contiguous along p (load p-fastest for coalescing).
template <class FA, class FB>
__device__ __forceinline__ void tile_acc(FA a_at, FB b_at, bool a_pfast, bool b_pfast, int M, int N,
                                         int p0, int p1, int i0, int j0, double (&acc)[4][4],
                                         double *smem) {
    double(*As)[TM + 1] = reinterpret_cast<double(*)[TM + 1]>(smem);
    double(*Bs)[TN + 1] = reinterpret_cast<double(*)[TN + 1]>(smem + TK * (TM + 1));
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    for (int k0 = p0; k0 < p1; k0 += TK) {
        for (int idx = tid; idx < TK * TM; idx += THREADS) {
            const int kk = a_pfast ? idx % TK : idx / TM, r = a_pfast ? idx / TK : idx % TM;
            const int p = k0 + kk;
            As[kk][r] = (p < p1 && i0 + r < M) ? a_at(i0 + r, p) : 0.0;
        }
        for (int idx = tid; idx < TK * TN; idx += THREADS) {
            const int kk = b_pfast ? idx % TK : idx / TN, r = b_pfast ? idx / TK : idx % TN;
            const int p = k0 + kk;
            Bs[kk][r] = (p < p1 && j0 + r < N) ? b_at(j0 + r, p) : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < TK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(THREADS) gemm_items_kernel(const GemmItem *__restrict__ items) {
    __shared__ double smem[TK * (TM + 1) + TK * (TN + 1)];
    const GemmItem g = items[blockIdx.x];
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    const bool asym = g.flags & GEMM_A_SYM_LOWER;
    auto a_at = [&](int i, int p) -> double {
        if (asym) {
            const int hi = i > p ? i : p, lo = i > p ? p : i;
            return g.A[(int64_t)hi * g.a_rs + (int64_t)lo * g.a_cs];
        }
        return g.A[(int64_t)i * g.a_rs + (int64_t)p * g.a_cs];
    };
    auto b_at = [&](int j, int p) -> double { return g.B[(int64_t)j * g.b_rs + (int64_t)p * g.b_cs]; };
    tile_acc(a_at, b_at, !asym && g.a_cs == 1, g.b_cs == 1, g.M, g.N, g.p0, g.p1, g.i0, g.j0, acc,
             smem);
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = g.j0 + ty + 16 * j;
        if (c >= g.N) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = g.i0 + tx + 16 * i;
            if (r >= g.M) continue;
            if ((g.flags & GEMM_C_LOWER) && r < c) continue;
            double *cp = g.C + (int64_t)r * g.c_rs + (int64_t)c * g.c_cs;
            const double v = g.alpha * acc[i][j];
            *cp = (g.flags & GEMM_ACCUMULATE) ? *cp + v : v;
        }
    }
}

// X(bi, bj) = -D(bi)^-1 T with T = sum_{p in [bj*64, bi*64)} L(bi*64 + r, p) X(p, bj*64 + c),
// or X(bi, bi) = D(bi)^-1 when bj == bi.  item = (supernode, bi, bj)
__global__ void __launch_bounds__(THREADS) trinv_kernel(DevSym d, const double *__restrict__ front,
                                                        const double *__restrict__ dinv,
                                                        double *__restrict__ xpool,
                                                        const int64_t *__restrict__ xoff,
                                                        const int4 *__restrict__ items) {
    // the tile product's staging buffers, then (after it) the 64 x 64 result
    __shared__ double smem[NB * (NB + 1)];
    static_assert(TK * (TM + 1) + TK * (TN + 1) <= NB * (NB + 1), "staging fits");
    double(*Ts)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(smem);
    const int4 it = items[blockIdx.x];
    const int s = it.x, bi = it.y, bj = it.z;
    const int k = d.sk[s], ld = d.sld[s];
    const double *L = front + d.foff[s];
    double *X = xpool + xoff[s];  // k x k, ld k
    const double *Db = dinv + d.dinvoff[s] + (int64_t)bi * NB * NB;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int r0 = bi * NB, c0 = bj * NB;
    if (bi == bj) {
        for (int idx = tid; idx < NB * NB; idx += THREADS) {
            const int r = idx % NB, c = idx / NB;
            if (r0 + r < k && c0 + c < k) X[(int64_t)(c0 + c) * k + r0 + r] = Db[idx];
        }
        return;
    }
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    auto a_at = [&](int i, int p) -> double { return L[(int64_t)p * ld + i]; };
    auto b_at = [&](int j, int p) -> double { return X[(int64_t)j * k + p]; };
    tile_acc(a_at, b_at, false, true, k, k, c0, r0, r0, c0, acc, smem);
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) Ts[tx + 16 * i][ty + 16 * j] = acc[i][j];
    __syncthreads();
    // X(bi, bj) = -Db Ts  (Db lower triangular, column-major NB x NB; rows of a
    // partial last block beyond k are not used)
    const int kv = min(NB, k - r0);
    for (int idx = tid; idx < NB * NB; idx += THREADS) {
        const int r = idx % NB, c = idx / NB;
        double v = 0.0;
        if (r < kv)
            for (int p = 0; p <= r; ++p) v += Db[(int64_t)p * NB + r] * Ts[p][c];
        if (r0 + r < k && c0 + c < k) X[(int64_t)(c0 + c) * k + r0 + r] = -v;
    }
}

// Z front of s, rows/cols in R (front rows >= kp): Z_s(fr_i, fr_j) =
// Z_parent(fr_p(i), fr_p(j)), lower part; one warp per column of R
__global__ void __launch_bounds__(THREADS) zgather_kernel(DevSym d, double *__restrict__ zpool,
                                                          const int32_t *__restrict__ upmap,
                                                          const int64_t *__restrict__ upoff,
                                                          const int4 *__restrict__ items, int count) {
    const int w = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= count) return;
    const int4 it = items[w];
    const int s = it.x, j = it.y;  // column j of R
    const int k = d.sk[s], m = d.sm[s], kp = d.skp[s], ld = d.sld[s];
    const int p = it.z;
    const int ldp = d.sld[p];
    const int32_t *map = upmap + upoff[s];  // R row -> parent front row
    const double *Zp = zpool + d.foff[p];
    double *Zs = zpool + d.foff[s] + (int64_t)(kp + j) * ld + kp;
    const int pj = map[j];
    for (int i = j + lane; i < m - k; i += 32) {
        const int pi = map[i];
        const int hi = pi > pj ? pi : pj, lo = pi > pj ? pj : pi;
        Zs[i] = Zp[(int64_t)lo * ldp + hi];
    }
}

// out[src[e]] = Z at the lower entries of P A P^T (original lower CSC order)
__global__ void zextract_kernel(DevSym d, const double *__restrict__ zpool,
                                const int32_t *__restrict__ col2s, const int32_t *__restrict__ psrc,
                                double *__restrict__ out) {
    const int64_t n = d.n;
    const int64_t j = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const int s = col2s[j];
    const double *Z = zpool + d.foff[s] + (int64_t)(j - d.sfirst[s]) * d.sld[s];
    for (int64_t e = d.pcp[j] + lane; e < d.pcp[j + 1]; e += 32) out[psrc[e]] = Z[d.alrow[e]];
}

// out[src[e]] = alpha o_e + zscale w_e Zsel[src[e]] for every stored lower entry
// e = (i, j) of A, where o_e = sum_c U(i, c) V(j, c) + U(j, c) V(i, c) and
// w_e = 2 off the diagonal, o_e = sum_c U(i, c) V(i, c) and w_e = 1 on it
// (Zsel may be null: no second term); walks the lower CSC of P A P^T
// (i = perm[row], j = perm[column]), one warp per column
__global__ void sym_outer_kernel(DevSym d, const int32_t *__restrict__ prow,
                                 const int32_t *__restrict__ psrc, const double *__restrict__ U,
                                 const double *__restrict__ V, int64_t ncols, int64_t ld, double alpha,
                                 const double *__restrict__ Zsel, double zscale,
                                 double *__restrict__ out) {
    const int64_t jp = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (jp >= d.n) return;
    const int64_t j = d.perm[jp];
    for (int64_t e = d.pcp[jp] + lane; e < d.pcp[jp + 1]; e += 32) {
        const int64_t i = d.perm[prow[e]];
        double acc = 0.0;
        if (i == j) {
            for (int64_t c = 0; c < ncols; ++c) acc += U[i + c * ld] * V[i + c * ld];
        } else {
            for (int64_t c = 0; c < ncols; ++c)
                acc += U[i + c * ld] * V[j + c * ld] + U[j + c * ld] * V[i + c * ld];
        }
        const int64_t o = psrc[e];
        double v = alpha * acc;
        if (Zsel) v += zscale * (i == j ? 1.0 : 2.0) * Zsel[o];
        out[o] = v;
    }
}

}  // namespace

void launch_gemm_items(const GemmItem *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    gemm_items_kernel<<<count, THREADS, 0, st>>>(items);
}

void launch_trinv(const DevSym &d, const double *front, const double *dinv, double *xpool,
                  const int64_t *xoff, const int4 *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    trinv_kernel<<<count, THREADS, 0, st>>>(d, front, dinv, xpool, xoff, items);
}

void launch_zgather(const DevSym &d, double *zpool, const int32_t *upmap, const int64_t *upoff,
                    const int4 *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    zgather_kernel<<<(count + 7) / 8, THREADS, 0, st>>>(d, zpool, upmap, upoff, items, count);
}

void launch_zextract(const DevSym &d, const double *zpool, const int32_t *col2s, const int32_t *psrc,
                     double *out, cudaStream_t st) {
    zextract_kernel<<<(int)((d.n + 7) / 8), THREADS, 0, st>>>(d, zpool, col2s, psrc, out);
}

void launch_sym_outer(const DevSym &d, const int32_t *prow, const int32_t *psrc, const double *U,
                      const double *V, int64_t ncols, int64_t ld, double alpha, const double *Zsel,
                      double zscale, double *out, cudaStream_t st) {
    sym_outer_kernel<<<(int)((d.n + 7) / 8), THREADS, 0, st>>>(d, prow, psrc, U, V, ncols, ld, alpha, Zsel,
                                                               zscale, out);
}

}  // namespace wd
