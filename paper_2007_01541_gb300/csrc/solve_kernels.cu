// Supernodal triangular solves, P^T L z, FP64 residuals and reductions.
//
// The solve applies the exact inverse of the compressed matrix (Sections 1
// and 5):  x = P^T L^-T L^-1 P b.  Both substitutions walk the supernodal
// tree level by level; inside a supernode they proceed by pivot blocks of NB
// columns.  Forward: every supernode produces an update vector u_s for the
// rows below its diagonal block, which its parent gathers through the same
// relative row maps as the factorization (no atomics).  Backward: every
// supernode reads the already final x of its front rows.
#include "dev_common.cuh"
#include "engine.h"

namespace wd {
namespace {

constexpr int THREADS = 256;
constexpr int RG = 16;  // right-hand sides per block

// ---------------------------------------------------------------------------
template <class T>
__global__ void permute_in_kernel(const double *__restrict__ B, int64_t ldb, T *__restrict__ Y,
                                  const int32_t *__restrict__ perm, int64_t n, int64_t nrhs) {
    const int64_t tot = n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % n, c = t / n;
        Y[t] = (T)B[perm[i] + c * ldb];
    }
}

template <class T>
__global__ void permute_out_kernel(const T *__restrict__ Y, double *__restrict__ B, int64_t ldb,
                                   const int32_t *__restrict__ perm, int64_t n, int64_t nrhs) {
    const int64_t tot = n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % n, c = t / n;
        B[perm[i] + c * ldb] = (double)Y[t];
    }
}

__global__ void gather_values_kernel(const int32_t *__restrict__ src, const double *__restrict__ v,
                                     double *__restrict__ out, int64_t nnz) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = v[src[e]];
}

// ---------------------------------------------------------------------------
// forward: t = [b_J; 0] + sum over children of their update vectors
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(THREADS) fwd_gather_kernel(DevSym d, T *__restrict__ Y,
                                                             T *__restrict__ W,
                                                             const int4 *__restrict__ items,
                                                             int nrhs) {
    const int4 it = items[blockIdx.x];
    const int s = it.x;
    const int r = it.y * THREADS + threadIdx.x;
    const int m = d.sm[s], k = d.sk[s];
    if (r >= m) return;
    const int64_t n = d.n;
    const int f = d.sfirst[s];
    const int cb = d.child_ptr[s], ce = d.child_ptr[s + 1];
    T *Ws = W + d.woff[s] * nrhs;
    for (int col = 0; col < nrhs; ++col) {
        T t = (r < k) ? Y[f + r + col * n] : T(0);
        for (int ci = cb; ci < ce; ++ci) {
            const int c = d.children[ci];
            const int ic = d.relmap[d.mapoff[c] + r];
            if (ic >= 0) {
                const int ldc = d.sm[c] - d.sk[c];
                t += W[d.woff[c] * nrhs + (int64_t)col * ldc + ic];
            }
        }
        if (r < k) Y[f + r + col * n] = t;
        else Ws[(int64_t)col * (m - k) + (r - k)] = t;
    }
}

// Y rows [rowbase + j0, +nb), rhs [c0, c0+nc) := Dinv Y (trans = 0) or Dinv^T Y
// (trans = 1), Dinv the stored NB x NB inverse of the diagonal block (zero
// beyond nb).  Must be called by all THREADS threads.
template <class T>
__device__ void diag_apply(const T *Dv, int trans, int nb, T *Y, int64_t n, int64_t rowbase,
                           int j0, int c0, int nc, T *smem) {
    T *Ds = smem;  // Ds[p * NB + r] = (trans ? Dinv(p, r) : Dinv(r, p))
    T(*Ts)[RG] = reinterpret_cast<T(*)[RG]>(smem + NB * NB);
    const int tid = threadIdx.x;
    if (!trans) {
        stage_tile<T, THREADS>(Ds, NB, Dv, NB, NB, NB, NB, NB);
    } else {
        for (int idx = tid; idx < NB * NB; idx += THREADS) {
            const int p = idx % NB, r = idx / NB;  // Dv[idx] = Dinv(p, r)
            cp_async_elem(Ds + p * NB + r, Dv + idx, true);
        }
    }
    for (int idx = tid; idx < NB * RG; idx += THREADS) {
        const int r = idx % NB, c = idx / NB;
        cp_async_elem(&Ts[r][c], Y + rowbase + j0 + r + (int64_t)(c0 + c) * n, r < nb && c < nc);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int r = tid % NB, cg = tid / NB;
    T acc[RG / 4];
#pragma unroll
    for (int u = 0; u < RG / 4; ++u) acc[u] = T(0);
    for (int p = 0; p < nb; ++p) {
        const T dv = Ds[p * NB + r];
#pragma unroll
        for (int u = 0; u < RG / 4; ++u) acc[u] += dv * Ts[p][cg + 4 * u];
    }
    __syncthreads();
    if (r < nb) {
#pragma unroll
        for (int u = 0; u < RG / 4; ++u) {
            const int c = cg + 4 * u;
            if (c < nc) Y[rowbase + j0 + r + (int64_t)(c0 + c) * n] = acc[u];
        }
    }
    __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(THREADS) fwd_diag_first_kernel(DevSym d, const T *__restrict__ dinv,
                                                                 T *__restrict__ Y,
                                                                 const int4 *__restrict__ items,
                                                                 int nrhs) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int4 it = items[blockIdx.x];
    const int s = it.x, c0 = it.y * RG;
    const int k = d.sk[s];
    diag_apply<T>(dinv + d.dinvoff[s], 0, min(NB, k), Y, d.n, d.sfirst[s], 0, c0,
                  min(RG, nrhs - c0), reinterpret_cast<T *>(smem_raw));
}

// pivot rows [t0 + rb*SOLVE_RB, k) -= L(rows, kb:kb+NB) y(kb:kb+NB); the block
// holding the next diagonal block then applies its inverse.
template <class T>
__global__ void __launch_bounds__(THREADS) fwd_update_kernel(DevSym d, const T *__restrict__ front,
                                                             const T *__restrict__ dinv,
                                                             T *__restrict__ Y,
                                                             const int4 *__restrict__ items,
                                                             int kb, int nrhs) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *Ls = sm;                                                  // [p][r], ld SOLVE_RB
    T(*Ys)[RG] = reinterpret_cast<T(*)[RG]>(sm + NB * SOLVE_RB);  // [p][c]
    const int4 it = items[blockIdx.x];
    const int s = it.x, rb = it.y, c0 = it.z * RG;
    const int k = d.sk[s], ld = d.sld[s];
    const int t0 = kb + NB;  // only blocks followed by another pivot block
    const int nc = min(RG, nrhs - c0);
    const int64_t n = d.n;
    const int f = d.sfirst[s];
    const T *F = front + d.foff[s];
    const int r0 = t0 + rb * SOLVE_RB;
    const int tid = threadIdx.x;
    stage_tile<T, THREADS>(Ls, SOLVE_RB, F + (int64_t)kb * ld + r0, ld, SOLVE_RB, NB, k - r0, NB);
    for (int idx = tid; idx < NB * RG; idx += THREADS) {
        const int p = idx % NB, c = idx / NB;
        cp_async_elem(&Ys[p][c], Y + f + kb + p + (int64_t)(c0 + c) * n, c < nc);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int rl = tid % SOLVE_RB, cg = tid / SOLVE_RB;  // 4 column groups
    const int r = r0 + rl;
    T acc[RG / 4];
#pragma unroll
    for (int u = 0; u < RG / 4; ++u) acc[u] = T(0);
#pragma unroll 8
    for (int p = 0; p < NB; ++p) {
        const T l = Ls[p * SOLVE_RB + rl];
#pragma unroll
        for (int u = 0; u < RG / 4; ++u) acc[u] += l * Ys[p][cg + 4 * u];
    }
    if (r < k) {
#pragma unroll
        for (int u = 0; u < RG / 4; ++u) {
            const int c = cg + 4 * u;
            if (c < nc) Y[f + r + (int64_t)(c0 + c) * n] -= acc[u];
        }
    }
    if (rb == 0) {
        __syncthreads();
        diag_apply<T>(dinv + d.dinvoff[s] + (int64_t)(t0 / NB) * NB * NB, 0, min(NB, k - t0), Y, n,
                      f, t0, c0, nc, sm);
    }
}

// rows of R: W_s -= L(R, 0:k) y(0:k), once the whole pivot block is solved;
// the pivot columns are streamed in chunks of NB, double buffered.
template <class T>
__global__ void __launch_bounds__(THREADS) fwd_rgemm_kernel(DevSym d, const T *__restrict__ front,
                                                            const T *__restrict__ Y,
                                                            T *__restrict__ W,
                                                            const int4 *__restrict__ items,
                                                            int nrhs) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *Ls[2] = {sm, sm + NB * SOLVE_RB};
    T *Ys[2] = {sm + 2 * NB * SOLVE_RB, sm + 2 * NB * SOLVE_RB + NB * RG};
    const int4 it = items[blockIdx.x];
    const int s = it.x, rb = it.y, c0 = it.z * RG;
    const int m = d.sm[s], k = d.sk[s], kp = d.skp[s], ld = d.sld[s];
    const int nc = min(RG, nrhs - c0);
    const int64_t n = d.n;
    const int f = d.sfirst[s];
    const int i0 = rb * SOLVE_RB;  // first local row of R
    const T *F = front + d.foff[s] + kp + i0;
    T *Ws = W + d.woff[s] * nrhs;
    const int tid = threadIdx.x;
    const int rl = tid % SOLVE_RB, cg = tid / SOLVE_RB;
    auto stage = [&](int buf, int p0) {
        stage_tile<T, THREADS>(Ls[buf], SOLVE_RB, F + (int64_t)p0 * ld, ld, SOLVE_RB, NB,
                               (m - k) - i0, k - p0);
        for (int idx = tid; idx < NB * RG; idx += THREADS) {
            const int p = idx % NB, c = idx / NB;
            cp_async_elem(Ys[buf] + p * RG + c, Y + f + p0 + p + (int64_t)(c0 + c) * n,
                          p0 + p < k && c < nc);
        }
        cp_async_commit();
    };
    T acc[RG / 4];
#pragma unroll
    for (int u = 0; u < RG / 4; ++u) acc[u] = T(0);
    const int nchunk = (k + NB - 1) / NB;
    stage(0, 0);
    for (int ch = 0; ch < nchunk; ++ch) {
        const int cur = ch & 1;
        if (ch + 1 < nchunk) {
            stage(cur ^ 1, (ch + 1) * NB);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const T *L = Ls[cur];
        const T *Yc = Ys[cur];
#pragma unroll 8
        for (int p = 0; p < NB; ++p) {
            const T l = L[p * SOLVE_RB + rl];
#pragma unroll
            for (int u = 0; u < RG / 4; ++u) acc[u] += l * Yc[p * RG + cg + 4 * u];
        }
        __syncthreads();
    }
    const int i = i0 + rl;
    if (i < m - k) {
#pragma unroll
        for (int u = 0; u < RG / 4; ++u) {
            const int c = cg + 4 * u;
            if (c < nc) Ws[(int64_t)(c0 + c) * (m - k) + i] -= acc[u];
        }
    }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
// y(J block jb) -= L(R, jb)^T x(R) with x(R) read at the front rows beyond the
// supernode (64-row chunks, double buffered); the last block of J then
// applies its inverse.
template <class T>
__global__ void __launch_bounds__(THREADS) bwd_init_kernel(DevSym d, const T *__restrict__ front,
                                                           const T *__restrict__ dinv,
                                                           T *__restrict__ Y,
                                                           const int4 *__restrict__ items,
                                                           int nrhs) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    constexpr int LST = 64 * (NB + 1), XST = 64 * RG;
    T *Ls[2] = {sm, sm + LST + XST};     // [rr][c], ld NB + 1
    T *Xs[2] = {sm + LST, sm + 2 * LST + XST};  // [rr][c], ld RG
    const int4 it = items[blockIdx.x];
    const int s = it.x, jblk = it.y, c0 = it.z * RG;
    const int m = d.sm[s], k = d.sk[s], kp = d.skp[s], ld = d.sld[s];
    const int j0 = jblk * NB, nb = min(NB, k - j0);
    const int nc = min(RG, nrhs - c0);
    const int64_t n = d.n;
    const int f = d.sfirst[s];
    const T *F = front + d.foff[s] + (int64_t)j0 * ld + kp;
    const int32_t *rows = d.rows + d.rowptr[s] + k;
    const int tid = threadIdx.x;
    const int cl = tid % NB, cg = tid / NB;  // column of the block, rhs group of 4
    const int nR = m - k;
    auto stage = [&](int buf, int i0) {
        const int nr = min(64, nR - i0);
        for (int idx = tid; idx < 64 * NB; idx += THREADS) {
            const int rr = idx % 64, c = idx / 64;
            cp_async_elem(Ls[buf] + rr * (NB + 1) + c, F + (int64_t)c * ld + i0 + rr, rr < nr && c < nb);
        }
        for (int idx = tid; idx < 64 * RG; idx += THREADS) {
            const int rr = idx % 64, c = idx / 64;
            const bool v = rr < nr && c < nc;
            cp_async_elem(Xs[buf] + rr * RG + c, v ? Y + rows[i0 + rr] + (int64_t)(c0 + c) * n : Y, v);
        }
        cp_async_commit();
    };
    T acc[RG / 4];
#pragma unroll
    for (int u = 0; u < RG / 4; ++u) acc[u] = T(0);
    const int nchunk = (nR + 63) / 64;
    if (nchunk > 0) stage(0, 0);
    for (int ch = 0; ch < nchunk; ++ch) {
        const int cur = ch & 1;
        if (ch + 1 < nchunk) {
            stage(cur ^ 1, (ch + 1) * 64);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const T *L = Ls[cur];
        const T *X = Xs[cur];
#pragma unroll 8
        for (int rr = 0; rr < 64; ++rr) {
            const T l = L[rr * (NB + 1) + cl];
#pragma unroll
            for (int u = 0; u < RG / 4; ++u) acc[u] += l * X[rr * RG + cg + 4 * u];
        }
        __syncthreads();
    }
    if (cl < nb) {
#pragma unroll
        for (int u = 0; u < RG / 4; ++u) {
            const int c = cg + 4 * u;
            if (c < nc) Y[f + j0 + cl + (int64_t)(c0 + c) * n] -= acc[u];
        }
    }
    if (j0 + nb == k) {
        __syncthreads();
        diag_apply<T>(dinv + d.dinvoff[s] + (int64_t)jblk * NB * NB, 1, nb, Y, n, f, j0, c0, nc, sm);
    }
}

// y(block jb) -= L(block ib+1, jb)^T x(block ib+1); block ib then applies
// its inverse
template <class T>
__global__ void __launch_bounds__(THREADS) bwd_step_kernel(DevSym d, const T *__restrict__ front,
                                                           const T *__restrict__ dinv,
                                                           T *__restrict__ Y,
                                                           const int4 *__restrict__ items,
                                                           int ib, int nrhs) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *Ls = sm;                        // [rr][c], ld NB + 1
    T *Xs = sm + NB * (NB + 1);        // [rr][c], ld RG
    const int4 it = items[blockIdx.x];
    const int s = it.x, jblk = it.y, c0 = it.z * RG;
    const int k = d.sk[s], ld = d.sld[s];
    const int j0 = jblk * NB, nbj = min(NB, k - j0);
    const int r0 = (ib + 1) * NB, nr = min(NB, k - r0);
    const int nc = min(RG, nrhs - c0);
    const int64_t n = d.n;
    const int f = d.sfirst[s];
    const T *F = front + d.foff[s];
    const int tid = threadIdx.x;
    for (int idx = tid; idx < NB * NB; idx += THREADS) {
        const int rr = idx % NB, c = idx / NB;
        cp_async_elem(Ls + rr * (NB + 1) + c, F + (int64_t)(j0 + c) * ld + r0 + rr, rr < nr && c < nbj);
    }
    for (int idx = tid; idx < NB * RG; idx += THREADS) {
        const int rr = idx % NB, c = idx / NB;
        cp_async_elem(Xs + rr * RG + c, Y + f + r0 + rr + (int64_t)(c0 + c) * n, rr < nr && c < nc);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int cl = tid % NB, cg = tid / NB;
    T acc[RG / 4];
#pragma unroll
    for (int u = 0; u < RG / 4; ++u) acc[u] = T(0);
#pragma unroll 8
    for (int rr = 0; rr < NB; ++rr) {
        const T l = Ls[rr * (NB + 1) + cl];
#pragma unroll
        for (int u = 0; u < RG / 4; ++u) acc[u] += l * Xs[rr * RG + cg + 4 * u];
    }
    if (cl < nbj) {
#pragma unroll
        for (int u = 0; u < RG / 4; ++u) {
            const int c = cg + 4 * u;
            if (c < nc) Y[f + j0 + cl + (int64_t)(c0 + c) * n] -= acc[u];
        }
    }
    if (jblk == ib) {
        __syncthreads();
        diag_apply<T>(dinv + d.dinvoff[s] + (int64_t)jblk * NB * NB, 1, nbj, Y, n, f, j0, c0, nc, sm);
    }
}

// ---------------------------------------------------------------------------
// out = L z, multifrontal: rows of J go to Out, rows of R to the update
// vector gathered by the parent.  One thread per front row.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(THREADS) apply_L_kernel(DevSym d, const T *__restrict__ front,
                                                          const T *__restrict__ Z,
                                                          T *__restrict__ Out, T *__restrict__ W,
                                                          const int4 *__restrict__ items,
                                                          int nrhs) {
    const int4 it = items[blockIdx.x];
    const int s = it.x;
    const int r = it.y * THREADS + threadIdx.x;
    const int m = d.sm[s], k = d.sk[s], kp = d.skp[s], ld = d.sld[s];
    if (r >= m) return;
    const int64_t n = d.n;
    const int f = d.sfirst[s];
    const T *F = front + d.foff[s] + (r < k ? r : r + kp - k);
    const int cb = d.child_ptr[s], ce = d.child_ptr[s + 1];
    const int pmax = min(r + 1, k);
    for (int col = 0; col < nrhs; ++col) {
        T t = T(0);
        for (int ci = cb; ci < ce; ++ci) {
            const int c = d.children[ci];
            const int ic = d.relmap[d.mapoff[c] + r];
            if (ic >= 0) t += W[d.woff[c] * nrhs + (int64_t)col * (d.sm[c] - d.sk[c]) + ic];
        }
        const T *z = Z + f + (int64_t)col * n;
        for (int p = 0; p < pmax; ++p) t += F[(int64_t)p * ld] * z[p];
        if (r < k) Out[f + r + (int64_t)col * n] = t;
        else W[d.woff[s] * nrhs + (int64_t)col * (m - k) + (r - k)] = t;
    }
}

// ---------------------------------------------------------------------------
// Refinement vectors live in row-major (right-hand sides contiguous) FP64
// arrays, so that the sparse product reads x coalesced across lanes.
// ---------------------------------------------------------------------------
// Bp[i*nrhs + c] = B[perm[i] + c*ldb]
__global__ void permute_in_rm_kernel(const double *__restrict__ B, int64_t ldb,
                                     double *__restrict__ Bp, const int32_t *__restrict__ perm,
                                     int64_t n, int64_t nrhs) {
    const int64_t tot = n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / nrhs, c = t % nrhs;
        Bp[t] = B[perm[i] + c * ldb];
    }
}

// B[perm[i] + c*ldb] = X[i*nrhs + c]
__global__ void permute_out_rm_kernel(const double *__restrict__ X, double *__restrict__ B,
                                      int64_t ldb, const int32_t *__restrict__ perm, int64_t n,
                                      int64_t nrhs) {
    const int64_t tot = n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / nrhs, c = t % nrhs;
        B[perm[i] + c * ldb] = X[t];
    }
}

// tiled transposes between column-major C (ld n) and row-major Rm (ld nrhs)
//   dir 0: C[i + c n] = (Tc) Rm[i nrhs + c]
//   dir 1: Rm[i nrhs + c] (= or +=) (double) C[i + c n]
template <class Tc>
__global__ void transpose_kernel(Tc *__restrict__ C, double *__restrict__ Rm, int64_t n,
                                 int64_t nrhs, int dir, int accumulate) {
    __shared__ double tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    if (dir == 0) {
        for (int j = ty; j < 32; j += 8) {
            const int64_t i = i0 + j, c = c0 + tx;
            tile[j][tx] = (i < n && c < nrhs) ? Rm[i * nrhs + c] : 0.0;
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const int64_t i = i0 + tx, c = c0 + j;
            if (i < n && c < nrhs) C[i + c * n] = (Tc)tile[tx][j];
        }
    } else {
        for (int j = ty; j < 32; j += 8) {
            const int64_t i = i0 + tx, c = c0 + j;
            tile[j][tx] = (i < n && c < nrhs) ? (double)C[i + c * n] : 0.0;
        }
        __syncthreads();
        for (int j = ty; j < 32; j += 8) {
            const int64_t i = i0 + j, c = c0 + tx;
            if (i < n && c < nrhs) {
                const double v = tile[tx][j];
                Rm[i * nrhs + c] = accumulate ? Rm[i * nrhs + c] + v : v;
            }
        }
    }
}

// R = Bp - A_p X in FP64 on the full CSR of P A P^T (row-major vectors).
// The rows of the coarsest wavelets are dense, so rows are cut into chunks
// of at most SPMV_CHUNK entries: a chunk item is (row, first entry, end,
// slot); slot < 0 means the whole row, written to R directly; otherwise the
// partial sums go to P[slot] and a second pass adds a row's slots in order.
// Many right-hand sides: one warp per chunk, lanes over right-hand sides.
__global__ void __launch_bounds__(THREADS) spmv_wide_kernel(DevSym d, const int4 *__restrict__ items,
                                                            int count, const double *__restrict__ X,
                                                            const double *__restrict__ Bp,
                                                            double *__restrict__ R,
                                                            double *__restrict__ P, int nrhs) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= count) return;
    const int4 it = items[w];
    const int64_t row = it.x;
    const int e0 = it.y, e1 = it.z, slot = it.w;
    for (int c0 = 0; c0 < nrhs; c0 += 64) {
        const int ca = c0 + lane, cb = c0 + 32 + lane;
        double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
        int e = e0;
        for (; e + 1 < e1; e += 2) {
            const double v0 = d.csr_val[e], v1 = d.csr_val[e + 1];
            const double *x0 = X + (int64_t)d.csr_col[e] * nrhs;
            const double *x1 = X + (int64_t)d.csr_col[e + 1] * nrhs;
            if (ca < nrhs) {
                a0 += v0 * x0[ca];
                a1 += v1 * x1[ca];
            }
            if (cb < nrhs) {
                b0 += v0 * x0[cb];
                b1 += v1 * x1[cb];
            }
        }
        if (e < e1) {
            const double v0 = d.csr_val[e];
            const double *x0 = X + (int64_t)d.csr_col[e] * nrhs;
            if (ca < nrhs) a0 += v0 * x0[ca];
            if (cb < nrhs) b0 += v0 * x0[cb];
        }
        if (slot < 0) {
            if (ca < nrhs) R[row * nrhs + ca] = Bp[row * nrhs + ca] - (a0 + a1);
            if (cb < nrhs) R[row * nrhs + cb] = Bp[row * nrhs + cb] - (b0 + b1);
        } else {
            if (ca < nrhs) P[(int64_t)slot * nrhs + ca] = a0 + a1;
            if (cb < nrhs) P[(int64_t)slot * nrhs + cb] = b0 + b1;
        }
    }
}

// Few right-hand sides (<= 8): lanes over the entries of the chunk.
__global__ void __launch_bounds__(THREADS) spmv_narrow_kernel(DevSym d, const int4 *__restrict__ items,
                                                              int count, const double *__restrict__ X,
                                                              const double *__restrict__ Bp,
                                                              double *__restrict__ R,
                                                              double *__restrict__ P, int nrhs) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= count) return;
    const int4 it = items[w];
    const int64_t row = it.x;
    const int slot = it.w;
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.0;
    for (int e = it.y + lane; e < it.z; e += 32) {
        const double v = d.csr_val[e];
        const double *x = X + (int64_t)d.csr_col[e] * nrhs;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c < nrhs) acc[c] += v * x[c];
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        double a = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0 && c < nrhs) {
            if (slot < 0) R[row * nrhs + c] = Bp[row * nrhs + c] - a;
            else P[(int64_t)slot * nrhs + c] = a;
        }
    }
}

// rows cut into several chunks: item = (row, first slot, number of slots)
__global__ void spmv_finish_kernel(const int4 *__restrict__ items, int count,
                                   const double *__restrict__ Bp, double *__restrict__ R,
                                   const double *__restrict__ P, int nrhs) {
    const int i = blockIdx.x;
    if (i >= count) return;
    const int4 it = items[i];
    const int64_t row = it.x;
    for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
        double acc = 0.0;
        for (int q = 0; q < it.z; ++q) acc += P[(int64_t)(it.y + q) * nrhs + c];
        R[row * nrhs + c] = Bp[row * nrhs + c] - acc;
    }
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// ||A||_inf: row sums of |a| over the chunk items of the residual product
// (single-chunk rows go straight to the maximum, cut rows through partial[])
__global__ void norm_inf_chunks_kernel(DevSym d, const int4 *__restrict__ items, int count,
                                       double *__restrict__ partial, double *out) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= count) return;
    const int4 it = items[w];
    double acc = 0.0;
    for (int e = it.y + lane; e < it.z; e += 32) acc += fabs(d.csr_val[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        if (it.w < 0) atomic_max_nonneg(out, acc);
        else partial[it.w] = acc;
    }
}

__global__ void norm_inf_finish_kernel(const int4 *__restrict__ fin, int nfin,
                                       const double *__restrict__ partial, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nfin) return;
    double acc = 0.0;
    for (int q = 0; q < fin[i].z; ++q) acc += partial[fin[i].y + q];
    atomic_max_nonneg(out, acc);
}

// per column c: out[3c] = max|R|, out[3c+1] = max|X|, out[3c+2] = max|B|
// (row-major arrays; out must be zeroed; blocks take chunks of rows)
__global__ void colmax3_rm_kernel(const double *__restrict__ R, const double *__restrict__ X,
                                  const double *__restrict__ B, int64_t n, int nrhs,
                                  int64_t rows_per_block, double *out) {
    const int64_t r0 = blockIdx.x * rows_per_block;
    const int64_t r1 = min(n, r0 + rows_per_block);
    for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
        double a = 0, b = 0, e = 0;
        for (int64_t i = r0; i < r1; ++i) {
            a = fmax(a, fabs(R[i * nrhs + c]));
            b = fmax(b, fabs(X[i * nrhs + c]));
            e = fmax(e, fabs(B[i * nrhs + c]));
        }
        atomic_max_nonneg(out + 3 * c, a);
        atomic_max_nonneg(out + 3 * c + 1, b);
        atomic_max_nonneg(out + 3 * c + 2, e);
    }
}

template <class T>
__global__ void axpy_into_kernel(double *__restrict__ X, const T *__restrict__ D, int64_t cnt,
                                 int acc) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt;
         t += (int64_t)gridDim.x * blockDim.x)
        X[t] = acc ? X[t] + (double)D[t] : (double)D[t];
}

template <class T>
__global__ void cast_kernel(const double *__restrict__ src, T *__restrict__ dst, int64_t cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt;
         t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = (T)src[t];
}

// block-wise pairwise sums of 2 log L_jj (fixed order, deterministic)
template <class T>
__global__ void logdet_partial_kernel(DevSym d, const T *__restrict__ front, double *partial) {
    __shared__ double red[THREADS];
    double acc = 0.0;
    for (int s = blockIdx.x; s < d.ns; s += gridDim.x) {
        const int k = d.sk[s], ld = d.sld[s];
        const T *F = front + d.foff[s];
        for (int j = threadIdx.x; j < k; j += THREADS) acc += 2.0 * log((double)F[(int64_t)j * ld + j]);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void sum_final_kernel(const double *partial, int cnt, double *out) {
    __shared__ double red[THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < cnt; i += THREADS) acc += partial[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = THREADS / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

template <class T>
__global__ void export_panels_kernel(DevSym d, const T *__restrict__ front,
                                     double *__restrict__ out, const int64_t *__restrict__ poff) {
    const int s = blockIdx.x;
    const int m = d.sm[s], k = d.sk[s], kp = d.skp[s], ld = d.sld[s];
    const T *F = front + d.foff[s];
    double *P = out + poff[s];
    for (int64_t idx = threadIdx.x; idx < (int64_t)m * k; idx += THREADS) {
        const int r = (int)(idx % m), c = (int)(idx / m);
        const int fr = r < k ? r : r + kp - k;
        P[idx] = (r >= c) ? (double)F[(int64_t)c * ld + fr] : 0.0;
    }
}

inline int grid_for(int64_t work) {
    int64_t g = (work + THREADS - 1) / THREADS;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

template <class T>
constexpr size_t diag_smem() { return sizeof(T) * (NB * (NB + 1) + NB * RG); }
template <class T>
constexpr size_t bwd_init_smem() { return 2 * sizeof(T) * (64 * (NB + 1) + 64 * RG); }
template <class T>
constexpr size_t rgemm_smem() { return 2 * sizeof(T) * (NB * SOLVE_RB + NB * RG); }

template <class T>
void set_attrs() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(fwd_diag_first_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)diag_smem<T>());
    cudaFuncSetAttribute(fwd_update_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)diag_smem<T>());
    cudaFuncSetAttribute(bwd_init_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bwd_init_smem<T>());
    cudaFuncSetAttribute(bwd_step_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)diag_smem<T>());
    cudaFuncSetAttribute(fwd_rgemm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rgemm_smem<T>());
    done = true;
}

}  // namespace

void init_solve_attributes() {
    set_attrs<double>();
    set_attrs<float>();
}

void launch_gather_values(const int32_t *src, const double *values, double *out, int64_t nnz,
                          cudaStream_t st) {
    if (nnz <= 0) return;
    gather_values_kernel<<<grid_for(nnz), THREADS, 0, st>>>(src, values, out, nnz);
}

template <class T>
void launch_permute_in(const double *B, int64_t ldb, T *Y, const int32_t *perm, int64_t n,
                       int64_t nrhs, cudaStream_t st) {
    permute_in_kernel<T><<<grid_for(n * nrhs), THREADS, 0, st>>>(B, ldb, Y, perm, n, nrhs);
}

template <class T>
void launch_permute_out(const T *Y, double *B, int64_t ldb, const int32_t *perm, int64_t n,
                        int64_t nrhs, cudaStream_t st) {
    permute_out_kernel<T><<<grid_for(n * nrhs), THREADS, 0, st>>>(Y, B, ldb, perm, n, nrhs);
}

template <class T>
void launch_fwd_gather(const DevSym &d, const T *, T *Y, T *W, const int4 *items, int count,
                       int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    fwd_gather_kernel<T><<<count, THREADS, 0, st>>>(d, Y, W, items, nrhs);
}

template <class T>
void launch_fwd_diag_first(const DevSym &d, const T *dinv, T *Y, const int4 *items, int count,
                           int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    set_attrs<T>();
    fwd_diag_first_kernel<T><<<count, THREADS, diag_smem<T>(), st>>>(d, dinv, Y, items, nrhs);
}

template <class T>
void launch_fwd_update(const DevSym &d, const T *front, const T *dinv, T *Y, const int4 *items,
                       int count, int kb, int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    set_attrs<T>();
    fwd_update_kernel<T><<<count, THREADS, diag_smem<T>(), st>>>(d, front, dinv, Y, items, kb, nrhs);
}

template <class T>
void launch_fwd_rgemm(const DevSym &d, const T *front, const T *Y, T *W, const int4 *items,
                      int count, int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    set_attrs<T>();
    fwd_rgemm_kernel<T><<<count, THREADS, rgemm_smem<T>(), st>>>(d, front, Y, W, items, nrhs);
}

template <class T>
void launch_bwd_init(const DevSym &d, const T *front, const T *dinv, T *Y, const int4 *items,
                     int count, int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    set_attrs<T>();
    bwd_init_kernel<T><<<count, THREADS, bwd_init_smem<T>(), st>>>(d, front, dinv, Y, items, nrhs);
}

template <class T>
void launch_bwd_step(const DevSym &d, const T *front, const T *dinv, T *Y, const int4 *items,
                     int count, int ib, int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    set_attrs<T>();
    bwd_step_kernel<T><<<count, THREADS, diag_smem<T>(), st>>>(d, front, dinv, Y, items, ib, nrhs);
}

template <class T>
void launch_apply_L(const DevSym &d, const T *front, const T *Z, T *Out, T *W,
                    const int4 *items, int count, int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    apply_L_kernel<T><<<count, THREADS, 0, st>>>(d, front, Z, Out, W, items, nrhs);
}

void launch_permute_in_rm(const double *B, int64_t ldb, double *Bp, const int32_t *perm, int64_t n,
                          int64_t nrhs, cudaStream_t st) {
    permute_in_rm_kernel<<<grid_for(n * nrhs), THREADS, 0, st>>>(B, ldb, Bp, perm, n, nrhs);
}

void launch_permute_out_rm(const double *X, double *B, int64_t ldb, const int32_t *perm, int64_t n,
                           int64_t nrhs, cudaStream_t st) {
    permute_out_rm_kernel<<<grid_for(n * nrhs), THREADS, 0, st>>>(X, B, ldb, perm, n, nrhs);
}

template <class Tc>
void launch_transpose(Tc *C, double *Rm, int64_t n, int64_t nrhs, int dir, int accumulate,
                      cudaStream_t st) {
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((nrhs + 31) / 32));
    transpose_kernel<Tc><<<grid, dim3(32, 8), 0, st>>>(C, Rm, n, nrhs, dir, accumulate);
}

void launch_spmv_residual(const DevSym &d, const int4 *chunks, int nchunks, const int4 *fin,
                          int nfin, const double *X, const double *Bp, double *R, double *P,
                          int64_t nrhs, cudaStream_t st) {
    const int blocks = (int)(((int64_t)nchunks * 32 + THREADS - 1) / THREADS);
    if (nrhs <= 8)
        spmv_narrow_kernel<<<blocks, THREADS, 0, st>>>(d, chunks, nchunks, X, Bp, R, P, (int)nrhs);
    else
        spmv_wide_kernel<<<blocks, THREADS, 0, st>>>(d, chunks, nchunks, X, Bp, R, P, (int)nrhs);
    if (nfin > 0) spmv_finish_kernel<<<nfin, 64, 0, st>>>(fin, nfin, Bp, R, P, (int)nrhs);
}

void launch_norm_inf_rows(const DevSym &d, const int4 *chunks, int nchunks, const int4 *fin,
                          int nfin, double *partial, double *out, cudaStream_t st) {
    cudaMemsetAsync(out, 0, sizeof(double), st);
    norm_inf_chunks_kernel<<<(int)(((int64_t)nchunks * 32 + THREADS - 1) / THREADS), THREADS, 0, st>>>(
        d, chunks, nchunks, partial, out);
    if (nfin > 0) norm_inf_finish_kernel<<<(nfin + 127) / 128, 128, 0, st>>>(fin, nfin, partial, out);
}

void launch_colmax3(const double *R, const double *X, const double *Bp, int64_t n, int64_t nrhs,
                    double *out3, cudaStream_t st) {
    cudaMemsetAsync(out3, 0, 3 * nrhs * sizeof(double), st);
    const int64_t rpb = 32;
    colmax3_rm_kernel<<<(int)((n + rpb - 1) / rpb), 64, 0, st>>>(R, X, Bp, n, (int)nrhs, rpb, out3);
}

template <class T>
void launch_axpy_into(double *X, const T *D, int64_t cnt, int acc, cudaStream_t st) {
    axpy_into_kernel<T><<<grid_for(cnt), THREADS, 0, st>>>(X, D, cnt, acc);
}

template <class T>
void launch_cast(const double *src, T *dst, int64_t cnt, cudaStream_t st) {
    cast_kernel<T><<<grid_for(cnt), THREADS, 0, st>>>(src, dst, cnt);
}

template <class T>
void launch_logdet_partial(const DevSym &d, const T *front, double *partial, int nblocks,
                           cudaStream_t st) {
    logdet_partial_kernel<T><<<nblocks, THREADS, 0, st>>>(d, front, partial);
}

void launch_sum_final(const double *partial, int cnt, double *out, cudaStream_t st) {
    sum_final_kernel<<<1, THREADS, 0, st>>>(partial, cnt, out);
}

template <class T>
void launch_export_panels(const DevSym &d, const T *front, double *panels, const int64_t *poff,
                          cudaStream_t st) {
    export_panels_kernel<T><<<d.ns, THREADS, 0, st>>>(d, front, panels, poff);
}

#define WD_INST(T)                                                                               \
    template void launch_permute_in<T>(const double *, int64_t, T *, const int32_t *, int64_t,   \
                                       int64_t, cudaStream_t);                                   \
    template void launch_permute_out<T>(const T *, double *, int64_t, const int32_t *, int64_t,  \
                                        int64_t, cudaStream_t);                                  \
    template void launch_fwd_gather<T>(const DevSym &, const T *, T *, T *, const int4 *, int,   \
                                       int, cudaStream_t);                                       \
    template void launch_fwd_diag_first<T>(const DevSym &, const T *, T *, const int4 *, int,    \
                                           int, cudaStream_t);                                   \
    template void launch_fwd_update<T>(const DevSym &, const T *, const T *, T *, const int4 *,  \
                                       int, int, int, cudaStream_t);                             \
    template void launch_fwd_rgemm<T>(const DevSym &, const T *, const T *, T *, const int4 *,   \
                                      int, int, cudaStream_t);                                   \
    template void launch_bwd_init<T>(const DevSym &, const T *, const T *, T *, const int4 *,    \
                                     int, int, cudaStream_t);                                    \
    template void launch_bwd_step<T>(const DevSym &, const T *, const T *, T *, const int4 *,    \
                                     int, int, int, cudaStream_t);                               \
    template void launch_apply_L<T>(const DevSym &, const T *, const T *, T *, T *,              \
                                    const int4 *, int, int, cudaStream_t);                       \
    template void launch_axpy_into<T>(double *, const T *, int64_t, int, cudaStream_t);          \
    template void launch_transpose<T>(T *, double *, int64_t, int64_t, int, int, cudaStream_t);  \
    template void launch_cast<T>(const double *, T *, int64_t, cudaStream_t);                    \
    template void launch_logdet_partial<T>(const DevSym &, const T *, double *, int,             \
                                           cudaStream_t);                                        \
    template void launch_export_panels<T>(const DevSym &, const T *, double *, const int64_t *,  \
                                          cudaStream_t);
WD_INST(double)
WD_INST(float)
#undef WD_INST

}  // namespace wd
