// Factorization of one NB x NB diagonal block of a front, L11 = chol(F11),
// and the inverse of its factor, by one CTA of NT >= 256 threads (the
// pivot block step P A P^T = L L^T of Section 4, restated for a dense block).
//
// The block is read from the front (type TF), factored in the compute type TC
// (TF, or double for an FP32 front whose diagonal blocks are kept in FP64),
// and written back: L11 into the front, L11^-1 (zero-padded to NB x NB,
// column-major) into the inverse store.  Right-looking by sub-blocks of 16:
//   1. one warp factors the 16 x 16 diagonal sub-block, one row per lane in
//      registers (shuffles, no block barrier);
//   2. the rows below are solved against it, one row per thread;
//   3. the trailing lower part is updated with register tiles of 2 x 4.
// The inverse, by 16 x 16 blocks X(i, j) of L11^-1: the diagonal inverses
// X(i, i) (one warp each, one column per lane); then W(i, k) = X(i, i) L(i, k)
// for all i > k at once; then one barrier step per block row i = 1, 2, 3:
// X(i, j) = -sum_{k=j}^{i-1} W(i, k) X(k, j), which only reads block rows
// finished before.  A pivot that is not positive records its global column in
// *status (smallest wins) and is replaced by 1 so that the arithmetic stays
// finite.
#pragma once
#include "engine.h"

namespace wd {
namespace blk {

constexpr int SB = 16;

// pivot d > 0 -> (sqrt(d), 1/sqrt(d)).  FP64: correctly rounded square root
// and division.  FP32 (the refined mixed-precision path): the hardware's
// approximate reciprocal square root (rsqrt.approx, pivots are never
// subnormal here), which keeps the serial pivot chain short; its few ulps of
// error are far below what iterative refinement removes.
__device__ __forceinline__ void pivot_root(double d, double &s, double &is) {
    s = sqrt(d);
    is = 1.0 / s;
}
__device__ __forceinline__ void pivot_root(float d, float &s, float &is) {
    asm("rsqrt.approx.ftz.f32 %0, %1;\n" : "=f"(is) : "f"(d));
    s = d * is;
}

// four consecutive shared-memory elements (16-byte aligned for float, two
// 16-byte halves for double)
__device__ __forceinline__ void load4(float (&v)[4], const float *p) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
__device__ __forceinline__ void load4(double (&v)[4], const double *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}

// Pivot C of a 16 x 16 Cholesky held by one warp, one row per lane (v),
// then pivots C+1, ...: compile-time recursion, so every register index is a
// constant.  dc is pivot C's value, broadcast.  The first pivot that is not
// positive is kept in `bad` (the caller reports it) and replaced by 1, so the
// unrolled chain has no branch.  The next pivot is updated and broadcast
// before the rest of the column (lane C+1 holds both of its factors), and the
// column itself goes to every lane through shared memory (col, 16 elements,
// 16-byte aligned, private to the warp): one store and four vector loads
// instead of fifteen shuffles.
template <class T, int C>
struct WarpChol {
    static __device__ __forceinline__ void step(T (&v)[SB], T &myinv, int lane, int w, int &bad, T dc, T *col) {
        bad = (C < w && !(dc > T(0)) && bad < 0) ? C : bad;
        dc = (C < w && dc > T(0)) ? dc : T(1);
        T sc, ic;
        pivot_root(dc, sc, ic);
        v[C] = lane == C ? sc : (lane > C ? v[C] * ic : v[C]);
        myinv = lane == C ? ic : myinv;
        T dn = T(0);
        if (C + 1 < SB) dn = __shfl_sync(0xffffffffu, v[C + 1 < SB ? C + 1 : C] - v[C] * v[C], C + 1 < SB ? C + 1 : C);
        if (lane < SB) col[lane] = v[C];
        __syncwarp();
#pragma unroll
        for (int q = (C + 1) / 4 * 4; q < SB; q += 4) {
            T t[4];
            load4(t, col + q);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (q + u > C && lane >= q + u) v[q + u] -= v[C] * t[u];
        }
        __syncwarp();
        WarpChol<T, C + 1>::step(v, myinv, lane, w, bad, dn, col);
    }
};
template <class T>
struct WarpChol<T, SB> {
    static __device__ __forceinline__ void step(T (&)[SB], T &, int, int, int &, T, T *) {}
};

// Shared memory of the block factorization (element offsets, in TC): the
// factor A[NB][NB + 1]; the inverse stored transposed, XT[c * XLD + r] =
// Linv(r, c), with 16-byte aligned rows (XLD = NB + 4) so that four
// consecutive entries are one vector load; the reciprocal pivots; the warp
// Cholesky's column buffer.  The strictly lower 16 x 16 blocks of XT (Linv's
// zero upper part) hold the products W(i, k).
constexpr int XLD = NB + 4;
constexpr int BP_XT = NB * (NB + 1);
constexpr int BP_INVD = BP_XT + NB * XLD;
constexpr int BP_COL = BP_INVD + NB;      // the pivot column broadcast of the warp Cholesky
constexpr int BP_ELEMS = BP_COL + SB;
template <class TC>
constexpr size_t block_smem_bytes() { return sizeof(TC) * BP_ELEMS; }

// Loads the lower part of the nb x nb block at F (column-major, ld) into A
// (converted to TC, zero outside the block) and zeroes XT.  All of a thread's
// loads are issued before the first store, so their latencies overlap.  Ends
// with a block barrier.
template <class TC, class TF, int NT>
__device__ void block_load(const TF *F, int ld, int nb, TC *smem) {
    TC(*A)[NB + 1] = reinterpret_cast<TC(*)[NB + 1]>(smem);
    TC *XT = smem + BP_XT;
    constexpr int PER = (NB * NB + NT - 1) / NT;
    TF v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        const int r = idx % NB, c = idx / NB;
        v[u] = (idx < NB * NB && r >= c && r < nb && c < nb) ? F[(int64_t)c * ld + r] : TF(0);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int idx = threadIdx.x + u * NT;
        if (idx < NB * NB) {
            const int r = idx % NB, c = idx / NB;
            A[r][c] = (TC)v[u];
            XT[c * XLD + r] = TC(0);
        }
    }
    __syncthreads();
}

template <class TC, int NT>
__device__ void block_inverse(int nb, const TC (*A)[NB + 1], TC *XT, const TC *invd);

// Factors the block that block_load brought in, leaving L in A and Linv in
// XT (visible to the whole block when it returns).  Threads beyond the first
// 256 take part in the barriers and the strided loops only.
template <class TC, int NT>
__device__ void block_potrf_inv(int nb, int64_t gcol0, status_t *status, TC *smem) {
    static_assert(NT >= 256, "the 16 x 16 block products use 256 threads");
    TC(*A)[NB + 1] = reinterpret_cast<TC(*)[NB + 1]>(smem);
    TC *XT = smem + BP_XT;
    TC *invd = smem + BP_INVD;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
#pragma unroll 1
    for (int jb = 0; jb < nb; jb += SB) {
        const int w = min(SB, nb - jb);
        if (warp == 0) {
            TC v[SB], myinv = TC(1);
#pragma unroll 16
            for (int c = 0; c < SB; ++c) v[c] = (lane < w && c <= lane) ? A[jb + lane][jb + c] : TC(0);
            int bad = -1;
            WarpChol<TC, 0>::step(v, myinv, lane, w, bad, __shfl_sync(0xffffffffu, v[0], 0), smem + BP_COL);
            if (bad >= 0 && lane == 0) atomicMin(status, (status_t)(gcol0 + jb + bad));
            if (lane < w) {
#pragma unroll 16
                for (int c = 0; c < SB; ++c)
                    if (c <= lane) A[jb + lane][jb + c] = v[c];
                invd[jb + lane] = myinv;
            }
        }
        __syncthreads();
        const int rem = nb - jb - w;
        if (tid < rem) {
            const int i = jb + w + tid;
            TC x[SB];
#pragma unroll 16
            for (int c = 0; c < SB; ++c) x[c] = A[i][jb + c];
#pragma unroll 16
            for (int c = 0; c < SB; ++c) {
                TC acc0 = x[c], acc1 = TC(0);
#pragma unroll 8
                for (int p = 0; p + 1 < c; p += 2) {
                    acc0 -= x[p] * A[jb + c][jb + p];
                    acc1 -= x[p + 1] * A[jb + c][jb + p + 1];
                }
                if (c & 1) acc0 -= x[c - 1] * A[jb + c][jb + c - 1];
                x[c] = (acc0 + acc1) * invd[jb + c];
            }
#pragma unroll 16
            for (int c = 0; c < SB; ++c) A[i][jb + c] = x[c];
        }
        __syncthreads();
        // trailing lower part, 2 x 4 register tiles
        const int t0 = jb + w, ntr = (rem + 1) / 2, ntc = (rem + 3) / 4;
        for (int q = tid; q < ntr * ntc; q += NT) {
            const int bi = q % ntr, bj = q / ntr;
            const int r0 = t0 + 2 * bi, c0 = t0 + 4 * bj;
            if (r0 + 1 < c0) continue;
            TC acc[2][4];
#pragma unroll 2
            for (int i = 0; i < 2; ++i)
#pragma unroll 4
                for (int j = 0; j < 4; ++j) acc[i][j] = TC(0);
#pragma unroll 4
            for (int p = 0; p < SB; ++p) {
                TC ar[2], ac[4];
#pragma unroll 2
                for (int i = 0; i < 2; ++i) ar[i] = A[min(r0 + i, NB - 1)][jb + p];
#pragma unroll 4
                for (int j = 0; j < 4; ++j) ac[j] = A[min(c0 + j, NB - 1)][jb + p];
#pragma unroll 2
                for (int i = 0; i < 2; ++i)
#pragma unroll 4
                    for (int j = 0; j < 4; ++j) acc[i][j] += ar[i] * ac[j];
            }
#pragma unroll 2
            for (int i = 0; i < 2; ++i)
#pragma unroll 4
                for (int j = 0; j < 4; ++j) {
                    const int r = r0 + i, c = c0 + j;
                    if (r < nb && c <= r) A[r][c] -= acc[i][j];
                }
        }
        __syncthreads();
    }
    block_inverse<TC, NT>(nb, A, XT, invd);
}

// L11^-1 of the factor in A (rows and columns [0, nb)) into XT (XT[c * XLD +
// r] = Linv(r, c); XT zero on entry), from the reciprocal pivots invd.  All
// NT >= 256 threads take part; the result is visible to the whole block on
// return.
template <class TC, int NT>
__device__ void block_inverse(int nb, const TC (*A)[NB + 1], TC *XT, const TC *invd) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // X(i, i): the diagonal 16 x 16 inverses, one warp each, one column per lane
    const int nsb = (nb + SB - 1) / SB;
    if (warp < nsb && lane < SB) {
        const int b0 = warp * SB, wv = min(SB, nb - b0), c = lane;
        TC x[SB];
#pragma unroll 16
        for (int r = 0; r < SB; ++r) {
            TC acc0 = (r == c) ? TC(1) : TC(0), acc1 = TC(0);
#pragma unroll 8
            for (int p = 0; p + 1 < r; p += 2) {
                acc0 -= A[b0 + r][b0 + p] * x[p];
                acc1 -= A[b0 + r][b0 + p + 1] * x[p + 1];
            }
            if (r & 1) acc0 -= A[b0 + r][b0 + r - 1] * x[r - 1];
            x[r] = (r < wv && c < wv) ? (acc0 + acc1) * invd[min(b0 + r, NB - 1)] : TC(0);
        }
#pragma unroll 16
        for (int r = 0; r < SB; ++r)
            if (r >= c) XT[(b0 + c) * XLD + b0 + r] = x[r];
    }
    __syncthreads();
    // W(i, k) = X(i, i) L(i, k), i > k, into XT's block (i, k); X(i, i)(r, t) is
    // zero for t > r, so the sum runs over the whole sub-block
    if (tid < SB * SB) {
        const int r = tid % SB, q = tid / SB;
        for (int i = 1; i < nsb; ++i)
            for (int k = 0; k < i; ++k) {
                TC acc0 = TC(0), acc1 = TC(0);
#pragma unroll
                for (int t = 0; t < SB; t += 2) {
                    acc0 += XT[(SB * i + t) * XLD + SB * i + r] * A[SB * i + t][SB * k + q];
                    acc1 += XT[(SB * i + t + 1) * XLD + SB * i + r] * A[SB * i + t + 1][SB * k + q];
                }
                XT[(SB * i + r) * XLD + SB * k + q] = acc0 + acc1;
            }
    }
    __syncthreads();
    // X(i, j)(r, c) = -sum_k sum_q W(i, k)(r, q) X(k, j)(q, c); both operands
    // are rows of XT, read four entries at a time
    {
        const int r = tid % SB, c = tid / SB;
#pragma unroll 1
        for (int i = 1; i < nsb; ++i) {
            if (tid < SB * SB) {
                for (int j = 0; j < i; ++j) {
                    TC acc[4] = {TC(0), TC(0), TC(0), TC(0)};
                    for (int k = j; k < i; ++k) {
                        const TC *wp = XT + (SB * i + r) * XLD + SB * k;
                        const TC *xp = XT + (SB * j + c) * XLD + SB * k;
#pragma unroll
                        for (int q = 0; q < SB; q += 4) {
                            TC wv[4], xv[4];
                            load4(wv, wp + q);
                            load4(xv, xp + q);
#pragma unroll
                            for (int u = 0; u < 4; ++u) acc[u] += wv[u] * xv[u];
                        }
                    }
                    XT[(SB * j + c) * XLD + SB * i + r] = -((acc[0] + acc[1]) + (acc[2] + acc[3]));
                }
            }
            __syncthreads();
        }
    }
}

// Factor diagonal block kb of front s (nb = min(NB, k - kb) columns) in TC:
// L11 back into the front, L11^-1 into Dinv at dinvoff[s] + (kb / NB) NB^2.
// Called by all NT threads of the CTA; `smem` holds block_smem_bytes<TC>().
// Must follow a barrier after which the block's final values are visible.
template <class TC, class TF, int NT>
__device__ void factor_diag_block(const DevSym &d, TF *front, TF *dinv, int s, int kb, status_t *status,
                                  void *smem) {
    TC *Psm = reinterpret_cast<TC *>(smem);
    const int k = d.sk[s], ld = d.sld[s];
    const int nb = min(NB, k - kb);
    TF *F = front + d.foff[s] + (int64_t)kb * ld + kb;
    block_load<TC, TF, NT>(F, ld, nb, Psm);
    block_potrf_inv<TC, NT>(nb, d.sfirst[s] + kb, status, Psm);
    const TC(*A)[NB + 1] = reinterpret_cast<const TC(*)[NB + 1]>(Psm);
    const TC *XT = Psm + BP_XT;
    TF *Dv = dinv + d.dinvoff[s] + (int64_t)(kb / NB) * NB * NB;
    for (int idx = threadIdx.x; idx < NB * NB; idx += NT) {
        const int r = idx % NB, c = idx / NB;
        if (r >= c && r < nb) F[(int64_t)c * ld + r] = (TF)A[r][c];
        Dv[idx] = (r >= c) ? (TF)XT[c * XLD + r] : TF(0);
    }
}

}  // namespace blk
}  // namespace wd
