// LU factorization without pivoting of a nonsymmetric matrix with a symmetric
// pattern, P A P^T = L U (L unit lower triangular), on the nested-dissection
// ordering and the supernodal analysis of the Cholesky path (Section 4: both
// factorizations share the ordering; U has the pattern of L transposed), and
// its substitutions.  FP64, multifrontal: the front of supernode s is the
// full square F_s (column-major, leading dimension ld_s, rows and columns as
// in the Cholesky fronts); after its k_s pivot steps it holds L (strict lower
// part of the pivot columns), U (upper part of the pivot rows, diagonal
// included) and the update matrix S = F22 - L21 U12 that the parent gathers.
//
// Phases for the fronts of one level:
//   lu_init      A's entries (both triangles) plus the children's update
//                matrices, gathered through the relative row maps (every
//                front entry written by one thread, no atomics)
//   per pivot block kb:
//     lu_diag    F11 = L11 U11 (one CTA per front) and the inverses L11^-1,
//                U11^-1 (kept for the panels and the substitutions)
//     lu_panel   L21 = F21 U11^-1 (rows below), U12 = L11^-1 F12 (columns
//                to the right)
//     lu_update  F22 -= L21 U12 on the whole trailing square (64 x 64 tiles)
#include "dev_common.cuh"
#include "engine.h"

namespace wd {
namespace {

constexpr int THREADS = 256;
constexpr int TL = 64;            // tile of the update and the panels
constexpr int INIT_ROWS = 128;
constexpr int INIT_MAXCH = 16;

struct Dims {
    int k, m, kp, mp, ld, f;
};
__device__ __forceinline__ Dims dims(const DevSym &d, int s) {
    Dims z;
    z.k = d.sk[s];
    z.m = d.sm[s];
    z.kp = d.skp[s];
    z.mp = z.kp + z.m - z.k;
    z.ld = d.sld[s];
    z.f = d.sfirst[s];
    return z;
}
// local index (0 .. m-1, pivot rows first) of front row fr, or -1 for padding
__device__ __forceinline__ int local_of(const Dims &z, int fr) {
    return fr < z.k ? fr : (fr < z.kp ? -1 : fr - (z.kp - z.k));
}

// ---------------------------------------------------------------------------
// assembly + extend-add of the full square: a CTA = 8 consecutive columns of
// one front (one warp each; padding items have q < 0), rows in slices of 128
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS) lu_init_kernel(DevSym d, double *__restrict__ front,
                                                          const double *__restrict__ vrow,
                                                          const double *__restrict__ vcol,
                                                          const int4 *__restrict__ items, int count) {
    __shared__ int32_t smap[INIT_MAXCH][INIT_ROWS];
    __shared__ int32_t sch[INIT_MAXCH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * (THREADS / 32) + warp;
    const int4 it = items[min(w, count - 1)];
    const int s = items[blockIdx.x * (THREADS / 32)].x;
    const int q = (w < count && it.x == s) ? it.y : -1;
    const Dims z = dims(d, s);
    const int qc = q < 0 ? -1 : local_of(z, q);
    double *F = front + d.foff[s] + (int64_t)max(q, 0) * z.ld;
    const int cb = d.child_ptr[s], ce = d.child_ptr[s + 1];
    for (int r0 = 0; r0 < z.mp; r0 += INIT_ROWS) {
        double acc[INIT_ROWS / 32];
#pragma unroll
        for (int u = 0; u < INIT_ROWS / 32; ++u) acc[u] = 0.0;
        for (int g0 = cb; g0 < ce; g0 += INIT_MAXCH) {
            const int ng = min(INIT_MAXCH, ce - g0);
            __syncthreads();
            if (threadIdx.x < ng) sch[threadIdx.x] = d.children[g0 + threadIdx.x];
            __syncthreads();
            for (int idx = threadIdx.x; idx < ng * INIT_ROWS; idx += THREADS) {
                const int gi = idx / INIT_ROWS, rr = idx % INIT_ROWS;
                const int fr = r0 + rr;
                const int r = fr < z.mp ? local_of(z, fr) : -1;
                smap[gi][rr] = r >= 0 ? d.relmap[d.mapoff[sch[gi]] + r] : -1;
            }
            __syncthreads();
            if (qc >= 0) {
                for (int gi = 0; gi < ng; ++gi) {
                    const int c = sch[gi];
                    const int ic = d.relmap[d.mapoff[c] + qc];
                    if (ic < 0) continue;
                    const int kpc = d.skp[c], ldc = d.sld[c];
                    // column ic of the child's update matrix (rows kpc + ir)
                    const double *U = front + d.foff[c] + (int64_t)(kpc + ic) * ldc + kpc;
#pragma unroll
                    for (int u = 0; u < INIT_ROWS / 32; ++u) {
                        const int ir = smap[gi][u * 32 + lane];
                        if (ir >= 0) acc[u] += U[ir];
                    }
                }
            }
        }
        if (q >= 0) {
#pragma unroll
            for (int u = 0; u < INIT_ROWS / 32; ++u) {
                const int fr = r0 + u * 32 + lane;
                if (fr < z.mp) F[fr] = acc[u];
            }
        }
    }
    __syncwarp();
    if (q >= 0 && qc >= 0) {
        // A's entries of this column (each written by its column's warp only):
        // a pivot column q takes (i, j) of P A P^T for i >= j (j = f + q) from
        // CSR row j's suffix; every column (global index g) takes the rows of
        // U above it, (j, g) for the pivots j < g, from CSR row g's entries in
        // the pivot range (stored there as the transposed value)
        double *Fq = front + d.foff[s] + (int64_t)q * z.ld;
        const int64_t g = d.rows[d.rowptr[s] + qc];
        if (q < z.k) {
            const int64_t e0 = d.csr_diag[g], e1 = d.csr_ptr[g + 1], l0 = d.pcp[g];
            for (int64_t e = e0 + lane; e < e1; e += 32) Fq[d.alrow[l0 + (e - e0)]] += vcol[e];
        }
        // pivot range of row g: columns in [f, min(f + k, g)), before the diagonal
        const int64_t jlo = z.f, jhi = min((int64_t)z.f + z.k, g);
        int64_t a = d.csr_ptr[g], b = d.csr_diag[g];   // first column >= jlo
        while (a < b) {
            const int64_t mid = (a + b) / 2;
            if (d.csr_col[mid] < jlo) a = mid + 1;
            else b = mid;
        }
        for (int64_t e = a + lane; e < d.csr_diag[g]; e += 32) {
            const int64_t j = d.csr_col[e];
            if (j >= jhi) break;
            Fq[j - z.f] += vcol[e];
        }
    }
}

// ---------------------------------------------------------------------------
// F11 = L11 U11 without pivoting and the inverses L11^-1 (unit lower), U11^-1
// (upper), one CTA per (s, kb); L11 / U11 back into the front, the inverses
// (zero-padded NB x NB, column-major) into linv / uinv at dinvoff + (kb/NB) NB^2
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS) lu_diag_kernel(DevSym d, double *__restrict__ front,
                                                          double *__restrict__ linv, double *__restrict__ uinv,
                                                          const int4 *__restrict__ items, int kb,
                                                          status_t *status) {
    __shared__ double A[NB][NB + 1];
    const int s = items[blockIdx.x].x;
    const Dims z = dims(d, s);
    const int nb = min(NB, z.k - kb);
    double *F = front + d.foff[s] + (int64_t)kb * z.ld + kb;
    for (int idx = threadIdx.x; idx < NB * NB; idx += THREADS) {
        const int r = idx % NB, c = idx / NB;
        A[r][c] = (r < nb && c < nb) ? F[(int64_t)c * z.ld + r] : (r == c ? 1.0 : 0.0);
    }
    __syncthreads();
    // right-looking, one pivot at a time (a zero pivot is reported and taken
    // as 1 so that the arithmetic stays finite)
    for (int p = 0; p < nb; ++p) {
        double piv = A[p][p];
        if (!(piv != 0.0)) {
            if (threadIdx.x == 0) {
                atomicMin(status, (status_t)(z.f + kb + p));
                A[p][p] = 1.0;
            }
            piv = 1.0;
        }
        __syncthreads();
        for (int i = p + 1 + threadIdx.x; i < nb; i += THREADS) A[i][p] /= piv;
        __syncthreads();
        const int rem = nb - p - 1;
        for (int idx = threadIdx.x; idx < rem * rem; idx += THREADS) {
            const int i = p + 1 + idx % rem, c = p + 1 + idx / rem;
            A[i][c] -= A[i][p] * A[p][c];
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < nb * nb; idx += THREADS) {
        const int r = idx % nb, c = idx / nb;
        F[(int64_t)c * z.ld + r] = A[r][c];
    }
    // inverses: thread c < NB: column c of L11^-1 (forward, unit diagonal);
    // thread NB + c: column c of U11^-1 (backward)
    double *Li = linv + d.dinvoff[s] + (int64_t)(kb / NB) * NB * NB;
    double *Ui = uinv + d.dinvoff[s] + (int64_t)(kb / NB) * NB * NB;
    const int t = threadIdx.x;
    if (t < NB) {
        const int c = t;
        for (int r = 0; r < NB; ++r) {
            double x = 0.0;
            if (r >= c && r < nb && c < nb) {
                x = r == c ? 1.0 : 0.0;
                for (int p = c; p < r; ++p) x -= A[r][p] * Li[(int64_t)c * NB + p];
            }
            Li[(int64_t)c * NB + r] = x;
        }
    } else if (t < 2 * NB) {
        const int c = t - NB;
        for (int r = NB - 1; r >= 0; --r) {
            double x = 0.0;
            if (r <= c && c < nb) {
                x = r == c ? 1.0 : 0.0;
                for (int p = r + 1; p <= c; ++p) x -= A[r][p] * Ui[(int64_t)c * NB + p];
                x /= A[r][r];
            }
            Ui[(int64_t)c * NB + r] = x;
        }
    }
}

// ---------------------------------------------------------------------------
// panels of step kb: item (s, blk, side): side 0 -> rows [r0, r0+64) below the
// pivot block, L21 := F21 U11^-1; side 1 -> columns [c0, c0+64) right of it,
// U12 := L11^-1 F12.  r0 / c0 start at kb + nb, or at kp for the last block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS) lu_panel_kernel(DevSym d, double *__restrict__ front,
                                                           const double *__restrict__ linv,
                                                           const double *__restrict__ uinv,
                                                           const int4 *__restrict__ items, int kb) {
    extern __shared__ double lu_smem[];
    double(*X)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(lu_smem);                // the panel block
    double(*V)[NB + 1] = reinterpret_cast<double(*)[NB + 1]>(lu_smem + TL * (NB + 1));  // the inverse
    const int4 it = items[blockIdx.x];
    const int s = it.x, blk = it.y, side = it.z;
    const Dims z = dims(d, s);
    const int nb = min(NB, z.k - kb);
    const int t0 = kb + nb;
    const int start = (t0 == z.k ? z.kp : t0) + blk * TL;
    double *F = front + d.foff[s];
    const double *Inv = (side == 0 ? uinv : linv) + d.dinvoff[s] + (int64_t)(kb / NB) * NB * NB;
    for (int idx = threadIdx.x; idx < NB * NB; idx += THREADS) {
        const int r = idx % NB, c = idx / NB;
        V[r][c] = Inv[idx];
        const int g = start + r;   // side 0: front row; side 1: front column
        double v = 0.0;
        if (g < z.mp && c < nb) v = side == 0 ? F[(int64_t)(kb + c) * z.ld + g] : F[(int64_t)g * z.ld + kb + c];
        X[r][c] = v;   // side 0: X[row][pivot col]; side 1: X[col][pivot row] (F12 transposed)
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TL * NB; idx += THREADS) {
        const int r = idx % TL, c = idx / TL;
        const int g = start + r;
        if (g >= z.mp || c >= nb) continue;
        double acc = 0.0;
        if (side == 0) {
            // L21[r][c] = sum_{p <= c} F21[r][p] Uinv[p][c]
            for (int p = 0; p <= c; ++p) acc += X[r][p] * V[p][c];
            F[(int64_t)(kb + c) * z.ld + g] = acc;
        } else {
            // U12[c][g] = sum_{p <= c} Linv[c][p] F12[p][g]
            for (int p = 0; p <= c; ++p) acc += V[c][p] * X[r][p];
            F[(int64_t)g * z.ld + kb + c] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// trailing update of step kb: tile (ti, tj) of the square from kb + nb:
// F[i][j] -= sum_p L[i][kb + p] U[kb + p][j]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS) lu_update_kernel(DevSym d, double *__restrict__ front,
                                                            const int4 *__restrict__ items, int kb) {
    extern __shared__ double lu_smem[];
    double(*Ls)[TL + 1] = reinterpret_cast<double(*)[TL + 1]>(lu_smem);                // [p][row]
    double(*Us)[TL + 1] = reinterpret_cast<double(*)[TL + 1]>(lu_smem + NB * (TL + 1));  // [p][col]
    const int4 it = items[blockIdx.x];
    const int s = it.x, ti = it.y, tj = it.z;
    const Dims z = dims(d, s);
    const int nb = min(NB, z.k - kb);
    const int base = kb + nb;
    const int r0 = base + ti * TL, c0 = base + tj * TL;
    double *F = front + d.foff[s];
    for (int idx = threadIdx.x; idx < NB * TL; idx += THREADS) {
        const int rr = idx % TL, p = idx / TL;
        const bool vp = p < nb;
        Ls[p][rr] = (vp && r0 + rr < z.mp) ? F[(int64_t)(kb + p) * z.ld + r0 + rr] : 0.0;
        Us[p][rr] = (vp && c0 + rr < z.mp) ? F[(int64_t)(c0 + rr) * z.ld + kb + p] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int p = 0; p < nb; ++p) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = Ls[p][tx + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Us[p][ty + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = c0 + ty + 16 * j;
        if (c >= z.mp) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = r0 + tx + 16 * i;
            if (r < z.mp) F[(int64_t)c * z.ld + r] -= acc[i][j];
        }
    }
}

// ---------------------------------------------------------------------------
// substitutions (FP64, Y: n x nrhs column-major in factor order)
// forward block step kb: item (s, blk): y_kb = L11^-1 t_kb (each CTA computes
// it); blk 0 writes y_kb to Y, blk >= 1 covers 64 later rows (pivot rows of
// the front in Tt, then rows of R in the update vector W_s):
// target -= L(rows, kb block) y_kb
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS) lu_fwd_kernel(DevSym d, const double *__restrict__ front,
                                                         const double *__restrict__ linv,
                                                         double *__restrict__ Y, double *__restrict__ Tt,
                                                         double *__restrict__ W, const int4 *__restrict__ items,
                                                         int kb, int nrhs) {
    extern __shared__ double ys[];          // [nb][nrhs] y_kb
    const int4 it = items[blockIdx.x];
    const int s = it.x, blk = it.y;
    const Dims z = dims(d, s);
    const int nb = min(NB, z.k - kb);
    const int64_t n = d.n;
    const double *Li = linv + d.dinvoff[s] + (int64_t)(kb / NB) * NB * NB;
    for (int idx = threadIdx.x; idx < nb * nrhs; idx += THREADS) {
        const int r = idx % nb, c = idx / nb;
        double acc = 0.0;
        for (int p = 0; p <= r; ++p) acc += Li[(int64_t)p * NB + r] * Tt[z.f + kb + p + (int64_t)c * n];
        ys[c * nb + r] = acc;
    }
    __syncthreads();
    if (blk == 0) {
        for (int idx = threadIdx.x; idx < nb * nrhs; idx += THREADS) {
            const int r = idx % nb, c = idx / nb;
            Y[z.f + kb + r + (int64_t)c * n] = ys[c * nb + r];
        }
        return;
    }
    const double *F = front + d.foff[s];
    const int t0 = kb + nb;
    for (int idx = threadIdx.x; idx < TL * nrhs; idx += THREADS) {
        const int rr = idx % TL, c = idx / TL;
        const int li = t0 + (blk - 1) * TL + rr;     // local row index (pivot rows, then R)
        if (li >= z.m) continue;
        const int fr = li < z.k ? li : li + (z.kp - z.k);
        double acc = 0.0;
        for (int p = 0; p < nb; ++p) acc += F[(int64_t)(kb + p) * z.ld + fr] * ys[c * nb + p];
        if (li < z.k) Tt[z.f + li + (int64_t)c * n] -= acc;
        else W[d.woff[s] * nrhs + (li - z.k) + (int64_t)c * (z.m - z.k)] -= acc;
    }
}

// backward block step kb: item (s): x_kb = U11^-1 (y_kb - U(kb block, later
// columns) x(later)), later = pivot columns after the block and the rows of R
// (their x is final: higher levels and later blocks are done)
__global__ void __launch_bounds__(THREADS) lu_bwd_kernel(DevSym d, const double *__restrict__ front,
                                                         const double *__restrict__ uinv,
                                                         double *__restrict__ Y, const int4 *__restrict__ items,
                                                         int kb, int nrhs) {
    extern __shared__ double ts[];          // [nrhs][nb] the reduced right-hand side
    const int s = items[blockIdx.x].x;
    const Dims z = dims(d, s);
    const int nb = min(NB, z.k - kb);
    const int64_t n = d.n;
    const double *F = front + d.foff[s];
    const int32_t *rows = d.rows + d.rowptr[s];
    for (int idx = threadIdx.x; idx < nb * nrhs; idx += THREADS) {
        const int r = idx % nb, c = idx / nb;
        double acc = Y[z.f + kb + r + (int64_t)c * n];
        for (int li = kb + nb; li < z.m; ++li) {
            const int fc = li < z.k ? li : li + (z.kp - z.k);
            acc -= F[(int64_t)fc * z.ld + kb + r] * Y[rows[li] + (int64_t)c * n];
        }
        ts[c * nb + r] = acc;
    }
    __syncthreads();
    const double *Ui = uinv + d.dinvoff[s] + (int64_t)(kb / NB) * NB * NB;
    for (int idx = threadIdx.x; idx < nb * nrhs; idx += THREADS) {
        const int r = idx % nb, c = idx / nb;
        double acc = 0.0;
        for (int p = r; p < nb; ++p) acc += Ui[(int64_t)p * NB + r] * ts[c * nb + p];
        Y[z.f + kb + r + (int64_t)c * n] = acc;
    }
}

// log |U_jj| of every pivot, summed per block of the grid into partial[],
// negative pivots counted in partial[gridDim.x + block]
__global__ void lu_logdet_kernel(DevSym d, const double *__restrict__ front, double *__restrict__ partial) {
    __shared__ double sh[THREADS];
    __shared__ double sg[THREADS];
    double acc = 0.0, neg = 0.0;
    for (int s = blockIdx.x; s < d.ns; s += gridDim.x) {
        const int k = d.sk[s], ld = d.sld[s];
        const double *F = front + d.foff[s];
        for (int q = threadIdx.x; q < k; q += THREADS) {
            const double u = F[(int64_t)q * ld + q];
            acc += log(fabs(u));
            neg += u < 0.0 ? 1.0 : 0.0;
        }
    }
    sh[threadIdx.x] = acc;
    sg[threadIdx.x] = neg;
    __syncthreads();
    for (int o = THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[threadIdx.x] += sh[threadIdx.x + o];
            sg[threadIdx.x] += sg[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = sh[0];
        partial[gridDim.x + blockIdx.x] = sg[0];
    }
}

// P A P^T values on the full CSR for a nonsymmetric A: vrow[e] = entry (i, j)
// (row i, column j of the CSR position), vcol[e] = entry (j, i); code[e]: 0 ->
// (lower, upper) of the source entry, 1 -> (upper, lower), 2 -> the diagonal
__global__ void lu_gather_kernel(const int32_t *__restrict__ src, const int8_t *__restrict__ code,
                                 const double *__restrict__ lower, const double *__restrict__ upper,
                                 double *__restrict__ vrow, double *__restrict__ vcol, int64_t nnz) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = src[e];
        const double a = lower[q], b = upper[q];
        const int c = code[e];
        vrow[e] = c == 1 ? b : a;
        vcol[e] = c == 0 ? b : a;
    }
}

// export: supernode s (one CTA), entry (r, c) of its m x k panels (r local
// row, c local pivot column): L with unit diagonal, and U^T (U[c][row r])
__global__ void lu_export_kernel(DevSym d, const double *__restrict__ front, double *__restrict__ lpan,
                                 double *__restrict__ upan, const int64_t *__restrict__ poff) {
    const int s = blockIdx.x;
    const Dims z = dims(d, s);
    const double *F = front + d.foff[s];
    double *Lp = lpan + poff[s], *Up = upan + poff[s];
    for (int64_t idx = threadIdx.x; idx < (int64_t)z.m * z.k; idx += THREADS) {
        const int r = (int)(idx % z.m), c = (int)(idx / z.m);
        const int fr = r < z.k ? r : r + z.kp - z.k;
        Lp[idx] = r > c ? F[(int64_t)c * z.ld + fr] : (r == c ? 1.0 : 0.0);
        Up[idx] = r >= c ? F[(int64_t)fr * z.ld + c] : 0.0;
    }
}

constexpr size_t PANEL_SMEM = (size_t)(TL + NB) * (NB + 1) * sizeof(double);
constexpr size_t UPDATE_SMEM = (size_t)2 * NB * (TL + 1) * sizeof(double);

inline int grid_of(int64_t work) {
    int64_t g = (work + THREADS - 1) / THREADS;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

void init_lu_attributes() {
    cudaFuncSetAttribute(lu_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PANEL_SMEM);
    cudaFuncSetAttribute(lu_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UPDATE_SMEM);
}

void launch_lu_gather(const int32_t *src, const int8_t *code, const double *lower, const double *upper,
                      double *vrow, double *vcol, int64_t nnz, cudaStream_t st) {
    if (nnz > 0) lu_gather_kernel<<<grid_of(nnz), THREADS, 0, st>>>(src, code, lower, upper, vrow, vcol, nnz);
}
void launch_lu_init(const DevSym &d, double *front, const double *vrow, const double *vcol, const int4 *items,
                    int count, cudaStream_t st) {
    if (count <= 0) return;
    const int warps = THREADS / 32;
    lu_init_kernel<<<(count + warps - 1) / warps, THREADS, 0, st>>>(d, front, vrow, vcol, items, count);
}
void launch_lu_diag(const DevSym &d, double *front, double *linv, double *uinv, const int4 *items, int count,
                    int kb, status_t *status, cudaStream_t st) {
    if (count > 0) lu_diag_kernel<<<count, THREADS, 0, st>>>(d, front, linv, uinv, items, kb, status);
}
void launch_lu_panel(const DevSym &d, double *front, const double *linv, const double *uinv, const int4 *items,
                     int count, int kb, cudaStream_t st) {
    if (count > 0) lu_panel_kernel<<<count, THREADS, PANEL_SMEM, st>>>(d, front, linv, uinv, items, kb);
}
void launch_lu_update(const DevSym &d, double *front, const int4 *items, int count, int kb, cudaStream_t st) {
    if (count > 0) lu_update_kernel<<<count, THREADS, UPDATE_SMEM, st>>>(d, front, items, kb);
}
void launch_lu_fwd(const DevSym &d, const double *front, const double *linv, double *Y, double *Tt, double *W,
                   const int4 *items, int count, int kb, int nrhs, cudaStream_t st) {
    if (count > 0)
        lu_fwd_kernel<<<count, THREADS, (size_t)NB * nrhs * sizeof(double), st>>>(d, front, linv, Y, Tt, W, items,
                                                                                kb, nrhs);
}
void launch_lu_bwd(const DevSym &d, const double *front, const double *uinv, double *Y, const int4 *items,
                   int count, int kb, int nrhs, cudaStream_t st) {
    if (count > 0)
        lu_bwd_kernel<<<count, THREADS, (size_t)NB * nrhs * sizeof(double), st>>>(d, front, uinv, Y, items, kb,
                                                                                nrhs);
}
void launch_lu_logdet(const DevSym &d, const double *front, double *partial, int nblocks, cudaStream_t st) {
    lu_logdet_kernel<<<nblocks, THREADS, 0, st>>>(d, front, partial);
}
void launch_lu_export(const DevSym &d, const double *front, double *lpan, double *upan, const int64_t *poff,
                      cudaStream_t st) {
    lu_export_kernel<<<d.ns, THREADS, 0, st>>>(d, front, lpan, upan, poff);
}

}  // namespace wd
