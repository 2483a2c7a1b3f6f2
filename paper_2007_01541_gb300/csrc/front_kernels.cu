// Multifrontal numeric factorization kernels (FP64 and FP32 fronts).
//
// Each supernode s owns a dense front F_s (column-major, lower triangle used)
// whose rows are: its k_s pivot rows, zero padding up to kp_s = k_s rounded
// up to 32, then the m_s - k_s rows below the supernode.  Its leading
// dimension ld_s is a multiple of 32 elements, so every column and every tile
// starting at a multiple of 32 rows is 128-byte aligned.  The first k_s
// columns become the supernode's columns of L; the trailing block from
// (kp_s, kp_s) on becomes the update matrix U_s = F22 - L21 L21^T that the
// parent gathers (extend-add).  This is the block form of P A P^T under
// nested dissection (Section 4): fronts of disjoint subtrees are
// independent, so every level of the supernodal tree is processed by one
// launch per phase.
//
// Phases for the fronts of one level:
//   front_init   assemble A's entries and gather the children's update
//                matrices through relative row maps (no atomics: every front
//                entry is written by exactly one thread)
//   per pivot block kb = 0, NB, 2NB, ... < k_s:
//     potrf      Cholesky of the NB x NB diagonal block and the inverse of
//                that block (kept for the panel and the solves)
//     panel      L21 := F21 L11^-T  as a product with the stored inverse
//     update     pivot columns [kb+NB, k) of the trailing rows -= L21 L21^T
//   syrk         U = F22 - L(R, 0:k) L(R, 0:k)^T, one product with the whole
//                pivot width as inner dimension
// Tiles are staged into shared memory with cp.async (many loads in flight
// per thread) and double buffered along the inner dimension.
#include "dev_common.cuh"
#include "engine.h"

namespace wd {
namespace {

constexpr int THREADS = 256;
constexpr int BM = SCHUR_BM;   // rows of a Schur tile
constexpr int BN = SCHUR_BN;   // columns of a Schur tile
constexpr int BK = 32;         // inner-dimension chunk

// pivot d > 0 -> (sqrt(d), 1/sqrt(d)).  FP64: correctly rounded square root
// and division.  FP32 (the refined mixed-precision path): the hardware
// reciprocal square root, which keeps the serial pivot chain short; its few
// ulps of error are far below what iterative refinement removes.
__device__ __forceinline__ void pivot_root(double d, double &s, double &is) {
    s = sqrt(d);
    is = 1.0 / s;
}
__device__ __forceinline__ void pivot_root(float d, float &s, float &is) {
    is = rsqrtf(d);
    s = d * is;
}

// four consecutive shared-memory elements (16-byte aligned for float,
// two 16-byte halves for double)
__device__ __forceinline__ void load4(float (&v)[4], const float *p) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
__device__ __forceinline__ void load4(double (&v)[4], const double *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ __forceinline__ void store4(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// x = hi + lo, hi = x rounded to tf32 (cvt.rna), lo = (x - hi) rounded to tf32
__device__ __forceinline__ void split_tf32_bits(float x, uint32_t &hi, uint32_t &lo) {
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(hi) : "f"(x));
    const float rem = x - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(lo) : "f"(rem));
}

struct Dims {
    int k, m, kp, mp, ld;
};
__device__ __forceinline__ Dims dims(const DevSym &d, int s) {
    Dims z;
    z.k = d.sk[s];
    z.m = d.sm[s];
    z.kp = d.skp[s];
    z.mp = z.kp + z.m - z.k;
    z.ld = d.sld[s];
    return z;
}

// ---------------------------------------------------------------------------
// assemble + extend-add: a CTA = 8 consecutive columns of one front (one warp
// each; the plan pads every front's column list to a multiple of 8, padding
// items have q < 0).  Rows go in slices of 128: the children's relative maps
// of the slice are staged in shared memory once for the 8 columns, so a front
// entry costs one independent global load per child.
// ---------------------------------------------------------------------------
constexpr int INIT_ROWS = 128;
constexpr int INIT_MAXCH = 16;   // children staged at once (more are taken in groups)

template <class T>
__global__ void __launch_bounds__(THREADS) front_init_kernel(DevSym d, T *__restrict__ front,
                                                             const int4 *__restrict__ items,
                                                             int count) {
    __shared__ int32_t smap[INIT_MAXCH][INIT_ROWS];
    __shared__ int32_t sch[INIT_MAXCH];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w = blockIdx.x * (THREADS / 32) + warp;
    const int4 it = items[min(w, count - 1)];
    const int s = items[blockIdx.x * (THREADS / 32)].x;   // all 8 items of a CTA share the front
    const int q = (w < count && it.x == s) ? it.y : -1;
    const Dims z = dims(d, s);
    const int pad = z.kp - z.k;
    const int qc = q < 0 ? -1 : (q < z.k ? q : (q < z.kp ? -1 : q - pad));   // local column
    T *F = front + d.foff[s] + (int64_t)max(q, 0) * z.ld;
    const int cb = d.child_ptr[s], ce = d.child_ptr[s + 1];
    // first row slice of the CTA: its smallest column
    const int qmin = items[blockIdx.x * (THREADS / 32)].y;
    for (int r0 = (qmin / INIT_ROWS) * INIT_ROWS; r0 < z.mp; r0 += INIT_ROWS) {
        T acc[INIT_ROWS / 32];
#pragma unroll
        for (int u = 0; u < INIT_ROWS / 32; ++u) acc[u] = T(0);
        for (int g0 = cb; g0 < ce; g0 += INIT_MAXCH) {
            const int ng = min(INIT_MAXCH, ce - g0);
            __syncthreads();
            if (threadIdx.x < ng) sch[threadIdx.x] = d.children[g0 + threadIdx.x];
            __syncthreads();
            for (int idx = threadIdx.x; idx < ng * INIT_ROWS; idx += THREADS) {
                const int gi = idx / INIT_ROWS, rr = idx % INIT_ROWS;
                const int fr = r0 + rr;
                const int r = fr < z.k ? fr : (fr < z.kp ? -1 : fr - pad);
                smap[gi][rr] = (fr < z.mp && r >= 0) ? d.relmap[d.mapoff[sch[gi]] + r] : -1;
            }
            __syncthreads();
            if (qc >= 0) {
                for (int gi = 0; gi < ng; ++gi) {
                    const int c = sch[gi];
                    const int ic = d.relmap[d.mapoff[c] + qc];
                    if (ic < 0) continue;
                    const int kpc = d.skp[c], ldc = d.sld[c];
                    const T *U = front + d.foff[c] + (int64_t)(kpc + ic) * ldc + kpc;
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
                if (fr >= q && fr < z.mp) F[fr] = acc[u];
            }
        }
    }
    __syncwarp();
    if (q >= 0 && q < z.k) {
        const int64_t j = d.sfirst[s] + q;
        const int64_t e0 = d.csr_diag[j], e1 = d.csr_ptr[j + 1], l0 = d.pcp[j];
        for (int64_t e = e0 + lane; e < e1; e += 32) F[d.alrow[l0 + (e - e0)]] += (T)d.csr_val[e];
    }
}

// ---------------------------------------------------------------------------
// Cholesky of an nb x nb diagonal block (nb <= NB = 64) and the inverse of the
// factor, written zero-padded as an NB x NB lower-triangular matrix
// (column-major) to Dinv.  Right-looking by sub-blocks of 16 (loop not
// unrolled, to keep the code small):
//   1. one warp factors the 16 x 16 diagonal sub-block, one row per lane in
//      registers (shuffles, no block barrier);
//   2. the rows below are solved against it, one row per thread;
//   3. the trailing lower part is updated with register tiles of 2 x 4.
// The inverse, by 16 x 16 blocks X(i, j) of Linv: the diagonal inverses
// X(i, i) (one warp each, one column per lane); then W(i, k) = X(i, i) L(i, k)
// for all i > k at once; then one barrier step per block row i = 1, 2, 3:
// X(i, j) = -sum_{k=j}^{i-1} W(i, k) X(k, j), which only reads block rows
// finished before.  A pivot that is not positive records its global column in
// *status (smallest wins) and is replaced by 1 so that the arithmetic stays
// finite.  Must be called by a block of POTRF_THREADS threads.
// ---------------------------------------------------------------------------
constexpr int SB = 16;
constexpr int POTRF_THREADS = 256;

// Pivot C of a 16 x 16 Cholesky held by one warp, one row per lane (v),
// then pivots C+1, ...: compile-time recursion, so every register index is a
// constant.  The first pivot that is not positive is kept in `bad` (the caller
// reports it), so the unrolled chain has no branch.
template <class T, int C>
struct WarpChol {
    static __device__ __forceinline__ void step(T (&v)[SB], T &myinv, int lane, int w, int &bad) {
        T dc = __shfl_sync(0xffffffffu, v[C], C);
        const bool fail = C < w && !(dc > T(0));
        bad = (fail && bad < 0) ? C : bad;
        dc = (fail || C >= w) ? T(1) : dc;
        T sc, ic;
        pivot_root(dc, sc, ic);
        v[C] = lane == C ? sc : (lane > C ? v[C] * ic : v[C]);
        myinv = lane == C ? ic : myinv;
#pragma unroll
        for (int c2 = C + 1; c2 < SB; ++c2) {
            const T lc = __shfl_sync(0xffffffffu, v[C], c2);
            if (lane >= c2) v[c2] -= v[C] * lc;
        }
        WarpChol<T, C + 1>::step(v, myinv, lane, w, bad);
    }
};
template <class T>
struct WarpChol<T, SB> {
    static __device__ __forceinline__ void step(T (&)[SB], T &, int, int, int &) {}
};

// Shared memory of the block factorization (element offsets): the factor
// A[NB][NB + 1]; the inverse stored transposed, XT[c * XLD + r] = Linv(r, c),
// with 16-byte aligned rows (XLD = NB + 4) so that four consecutive entries
// are one vector load; the reciprocal pivots.  The strictly lower 16 x 16
// blocks of XT (Linv's zero upper part) hold the products W(i, k).
constexpr int XLD = NB + 4;
constexpr int BP_XT = NB * (NB + 1);
constexpr int BP_INVD = BP_XT + NB * XLD;
constexpr int BP_ELEMS = BP_INVD + NB;

// Issues, without committing, the cp.async copies of the lower part of the
// nb x nb block at F (column-major, ld) into A (zero-filled outside it), and
// zeroes XT.
template <class T>
__device__ void block_load(const T *F, int ld, int nb, T *smem) {
    T(*A)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem);
    T *XT = smem + BP_XT;
    for (int idx = threadIdx.x; idx < NB * NB; idx += POTRF_THREADS) {
        const int r = idx % NB, c = idx / NB;
        cp_async_elem(&A[r][c], F + (int64_t)c * ld + r, r >= c && r < nb && c < nb);
        XT[c * XLD + r] = T(0);
    }
}

// Factors the block that block_load brought in (the caller has waited for
// the copies and synchronised), leaving L in A and Linv in XT; if `write`,
// stores L to Lout (ld NB, lower part) and Linv to Dinv.  Ends with XT final
// and visible to the whole block.
template <class T>
__device__ void block_potrf_inv(int nb, int64_t gcol0, status_t *status, T *Dinv, T *Lout, bool write,
                                T *smem) {
    T(*A)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem);
    T *XT = smem + BP_XT;
    T *invd = smem + BP_INVD;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
#pragma unroll 1
    for (int jb = 0; jb < nb; jb += SB) {
        const int w = min(SB, nb - jb);
        if (warp == 0) {
            T v[SB], myinv = T(1);
#pragma unroll 16
            for (int c = 0; c < SB; ++c) v[c] = (lane < w && c <= lane) ? A[jb + lane][jb + c] : T(0);
            int bad = -1;
            WarpChol<T, 0>::step(v, myinv, lane, w, bad);
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
            T x[SB];
#pragma unroll 16
            for (int c = 0; c < SB; ++c) x[c] = A[i][jb + c];
#pragma unroll 16
            for (int c = 0; c < SB; ++c) {
                T acc0 = x[c], acc1 = T(0);
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
        for (int q = tid; q < ntr * ntc; q += POTRF_THREADS) {
            const int bi = q % ntr, bj = q / ntr;
            const int r0 = t0 + 2 * bi, c0 = t0 + 4 * bj;
            if (r0 + 1 < c0) continue;
            T acc[2][4];
#pragma unroll 2
            for (int i = 0; i < 2; ++i)
#pragma unroll 4
                for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
#pragma unroll 4
            for (int p = 0; p < SB; ++p) {
                T ar[2], ac[4];
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
    // X(i, i): the diagonal 16 x 16 inverses, one warp each, one column per lane
    const int nsb = (nb + SB - 1) / SB;
    if (warp < nsb && lane < SB) {
        const int b0 = warp * SB, wv = min(SB, nb - b0), c = lane;
        T x[SB];
#pragma unroll 16
        for (int r = 0; r < SB; ++r) {
            T acc0 = (r == c) ? T(1) : T(0), acc1 = T(0);
#pragma unroll 8
            for (int p = 0; p + 1 < r; p += 2) {
                acc0 -= A[b0 + r][b0 + p] * x[p];
                acc1 -= A[b0 + r][b0 + p + 1] * x[p + 1];
            }
            if (r & 1) acc0 -= A[b0 + r][b0 + r - 1] * x[r - 1];
            x[r] = (r < wv && c < wv) ? (acc0 + acc1) * invd[min(b0 + r, NB - 1)] : T(0);
        }
#pragma unroll 16
        for (int r = 0; r < SB; ++r)
            if (r >= c) XT[(b0 + c) * XLD + b0 + r] = x[r];
    }
    __syncthreads();
    // W(i, k) = X(i, i) L(i, k), i > k, into XT's block (i, k); X(i, i)(r, t) is
    // zero for t > r, so the sum runs over the whole sub-block
    {
        const int r = tid % SB, q = tid / SB;
        for (int i = 1; i < nsb; ++i)
            for (int k = 0; k < i; ++k) {
                T acc0 = T(0), acc1 = T(0);
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
            for (int j = 0; j < i; ++j) {
                T acc[4] = {T(0), T(0), T(0), T(0)};
                for (int k = j; k < i; ++k) {
                    const T *w = XT + (SB * i + r) * XLD + SB * k;
                    const T *x = XT + (SB * j + c) * XLD + SB * k;
#pragma unroll
                    for (int q = 0; q < SB; q += 4) {
                        T wv[4], xv[4];
                        load4(wv, w + q);
                        load4(xv, x + q);
#pragma unroll
                        for (int u = 0; u < 4; ++u) acc[u] += wv[u] * xv[u];
                    }
                }
                XT[(SB * j + c) * XLD + SB * i + r] = -((acc[0] + acc[1]) + (acc[2] + acc[3]));
            }
            __syncthreads();
        }
    }
    if (write) {
        for (int idx = tid; idx < NB * NB; idx += POTRF_THREADS) {
            const int r = idx % NB, c = idx / NB;
            Lout[idx] = (r >= c && r < nb) ? A[r][c] : T(0);
            Dinv[idx] = (r >= c) ? XT[c * XLD + r] : T(0);
        }
    }
}

// the factored diagonal blocks (kept aside while the panels of a step still
// read the unfactored block) into the fronts: item = (s, first pivot column)
template <class T>
__global__ void __launch_bounds__(THREADS) diag_copy_kernel(DevSym d, T *__restrict__ front,
                                                            const T *__restrict__ ldiag,
                                                            const int4 *__restrict__ items) {
    const int4 it = items[blockIdx.x];
    const int s = it.x, j0 = it.y;
    const Dims z = dims(d, s);
    const int nb = min(NB, z.k - j0);
    const T *Lb = ldiag + d.dinvoff[s] + (int64_t)(j0 / NB) * NB * NB;
    T *F = front + d.foff[s] + (int64_t)j0 * z.ld + j0;
    for (int idx = threadIdx.x; idx < NB * NB; idx += THREADS) {
        const int r = idx % NB, c = idx / NB;
        if (r >= c && r < nb) F[(int64_t)c * z.ld + r] = Lb[idx];
    }
}

// ---------------------------------------------------------------------------
// potrf + panel of pivot block kb: every CTA factors the NB x NB diagonal block
// and inverts the factor itself (the pivot chain is latency-bound: doing it
// redundantly on many SMs costs nothing and saves a dependent launch per
// step); CTA rb = 0 stores the factor (aside, in ldiag, since other CTAs of
// the launch may still be reading the unfactored block) and the inverse.
// Then rows [r0, r0+RB) of columns [kb, kb+nb):  X := X Linv^T.  The rows
// start at kb+NB, or at kp when kb is the last block (rows [k, kp) are zero
// padding); a CTA may have no rows (its launch item only factors the block).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 3 : 1) panel_kernel(DevSym d, T *__restrict__ front,
                                                        T *__restrict__ dinv, T *__restrict__ ldiag,
                                                        unsigned char *__restrict__ pk,
                                                        const int4 *__restrict__ items, int kb,
                                                        status_t *status) {
    static_assert(THREADS == POTRF_THREADS, "the panel CTA runs the block factorization");
    static_assert(RB == 64 && NB == 64 && THREADS == 256, "4 x 4 register tiles cover the 64 x 64 panel block");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *Psm = reinterpret_cast<T *>(smem_raw);        // block factorization (BP_ELEMS)
    T *Xs = Psm + BP_ELEMS;                           // [p][r], ld RB
    const int4 it = items[blockIdx.x];
    const int s = it.x, rb = it.y;
    const Dims z = dims(d, s);
    const int nb = min(NB, z.k - kb);
    const int t0 = kb + nb;
    const int r0 = (t0 == z.k ? z.kp : t0) + rb * RB;
    T *F = front + d.foff[s];
    // the diagonal block first, in its own group: the pivot chain starts while
    // the panel rows are still in flight
    block_load<T>(F + (int64_t)kb * z.ld + kb, z.ld, nb, Psm);
    cp_async_commit();
    stage_tile<T, THREADS>(Xs, RB, F + (int64_t)kb * z.ld + r0, z.ld, RB, NB, z.mp - r0, nb);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const int64_t boff = d.dinvoff[s] + (int64_t)(kb / NB) * NB * NB;
    block_potrf_inv<T>(nb, d.sfirst[s] + kb, status, dinv + boff, ldiag + boff, rb == 0, Psm);
    cp_async_wait<0>();
    __syncthreads();
    // out[r][c] = sum_{p <= c} X[r][p] Linv(c, p), Linv(c, p) = XT[p][c];
    // thread: rows 4 (tid % 16) + i, columns 4 (tid / 16) + j, so both
    // operands of a step p are one 4-wide shared load, and p stops at the
    // thread's last column (Linv is lower triangular).
    const int tid = threadIdx.x;
    const T *LT = Psm + BP_XT;
    const int rq = tid % (RB / 4), cq = tid / (RB / 4);
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    const int pend = min(nb, 4 * cq + 4);
#pragma unroll 4
    for (int pp = 0; pp < pend; ++pp) {
        T xv[4], lv[4];
        load4(xv, Xs + pp * RB + 4 * rq);
        load4(lv, LT + pp * XLD + 4 * cq);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += xv[i] * lv[j];
    }
    // through shared memory ([c][r], ld RB) for whole-column stores
    __syncthreads();
    T *Os = Xs;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        T o[4] = {acc[0][j], acc[1][j], acc[2][j], acc[3][j]};
        store4(Os + (4 * cq + j) * RB + 4 * rq, o);
    }
    __syncthreads();
    for (int q = tid; q < RB * NB; q += THREADS) {
        const int rr = q % RB, c = q / RB;
        if (c < nb && r0 + rr < z.mp) F[(int64_t)(kb + c) * z.ld + r0 + rr] = Os[c * RB + rr];
    }
    if (pk != nullptr) {
        // packed tf32 hi/lo lines of these rows for the tensor-core updates
        unsigned char *P = pk + d.pkoff[s];
        const int prow = pack_rows(z.mp);
        for (int q = tid; q < RB * (NB / 4); q += THREADS) {
            const int rr = q % RB, g = q / RB;  // row, group of 4 columns
            const int row = r0 + rr;
            if (row >= z.mp) continue;
            const int kc = kb / 32 + g / 8, gg = g % 8;
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) split_tf32_bits((float)Os[(4 * g + j) * RB + rr], hi[j], lo[j]);
            const int64_t sw = (int64_t)((gg ^ (row & 7)) * 16);
            *reinterpret_cast<uint4 *>(P + pack_offset(kc, 0, row, prow) + sw) =
                make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(P + pack_offset(kc, 1, row, prow) + sw) =
                make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
}

// ---------------------------------------------------------------------------
// Schur tile: C(rows [r0, r0+BM), cols [c0, c0+BN)) -= A(rows, ka:ka+K) A(cols, ka:ka+K)^T
// restricted to r >= c, r < mp, c < cmax.  thread (tx, ty): rows tx + 16 i,
// columns ty + 16 j (i < 8, j < 4).
//   mode 0 (step):  base = kb + NB, ka = kb, K = NB, cmax = k
//   mode 1 (syrk):  base = kp, ka = 0, K = k, cmax = mp
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(THREADS) schur_kernel(DevSym d, T *__restrict__ front,
                                                        T *__restrict__ dinv,
                                                        const int4 *__restrict__ items, int kb,
                                                        int mode, status_t *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *As[2] = {sm, sm + BK * (BM + BN)};
    T *Bs[2] = {sm + BK * BM, sm + BK * (BM + BN) + BK * BM};
    const int4 it = items[blockIdx.x];
    const int s = it.x, ti = it.y, tj = it.z;
    const Dims z = dims(d, s);
    int base, ka, K, cmax;
    if (mode == 0) {
        base = kb + NB;
        ka = kb;
        K = NB;
        cmax = z.k;
    } else {
        base = z.kp;
        ka = 0;
        K = z.k;
        cmax = z.mp;
    }
    const int r0 = base + ti * BM, c0 = base + tj * BN;
    T *F = front + d.foff[s];
    const T *Ar = F + (int64_t)ka * z.ld + r0;
    const T *Bc = F + (int64_t)ka * z.ld + c0;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    T acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    const int nk = (K + BK - 1) / BK;
    stage_tile<T, THREADS>(As[0], BM, Ar, z.ld, BM, BK, z.mp - r0, min(BK, K));
    stage_tile<T, THREADS>(Bs[0], BN, Bc, z.ld, BN, BK, cmax - c0, min(BK, K));
    cp_async_commit();
    for (int kt = 0; kt < nk; ++kt) {
        const int cur = kt & 1;
        if (kt + 1 < nk) {
            const int k1 = (kt + 1) * BK;
            stage_tile<T, THREADS>(As[cur ^ 1], BM, Ar + (int64_t)k1 * z.ld, z.ld, BM, BK, z.mp - r0,
                                   min(BK, K - k1));
            stage_tile<T, THREADS>(Bs[cur ^ 1], BN, Bc + (int64_t)k1 * z.ld, z.ld, BN, BK, cmax - c0,
                                   min(BK, K - k1));
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const T *A = As[cur];
        const T *B = Bs[cur];
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
            T a[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = A[kk * BM + tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = B[kk * BN + ty + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = c0 + ty + 16 * j;
        if (c >= cmax) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = r0 + tx + 16 * i;
            if (r < z.mp && r >= c) F[(int64_t)c * z.ld + r] -= acc[i][j];
        }
    }
}

template <class T>
constexpr size_t panel_smem() { return sizeof(T) * (BP_ELEMS + NB * RB); }
template <class T>
constexpr size_t schur_smem() { return 2 * sizeof(T) * BK * (BM + BN); }

template <class T>
void set_smem_attrs() {
    static bool done = false;  // per instantiation and process
    if (done) return;
    cudaFuncSetAttribute(panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)panel_smem<T>());
    cudaFuncSetAttribute(schur_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)schur_smem<T>());
    done = true;
}

}  // namespace

void init_front_attributes() {
    set_smem_attrs<double>();
    set_smem_attrs<float>();
}

template <class T>
void launch_front_init(const DevSym &d, T *front, const int4 *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    const int warps = THREADS / 32;
    front_init_kernel<T><<<(count + warps - 1) / warps, THREADS, 0, st>>>(d, front, items, count);
}

template <class T>
void launch_panel(const DevSym &d, T *front, T *dinv, T *ldiag, unsigned char *pk, const int4 *items,
                  int count, int kb, status_t *status, cudaStream_t st) {
    if (count <= 0) return;
    set_smem_attrs<T>();
    panel_kernel<T><<<count, THREADS, panel_smem<T>(), st>>>(d, front, dinv, ldiag, pk, items, kb, status);
}

template <class T>
void launch_diag_copy(const DevSym &d, T *front, const T *ldiag, const int4 *items, int count,
                      cudaStream_t st) {
    if (count <= 0) return;
    diag_copy_kernel<T><<<count, THREADS, 0, st>>>(d, front, ldiag, items);
}

template <class T>
void launch_schur(const DevSym &d, T *front, T *dinv, const int4 *items, int count, int kb,
                  int mode, status_t *status, cudaStream_t st) {
    if (count <= 0) return;
    set_smem_attrs<T>();
    schur_kernel<T><<<count, THREADS, schur_smem<T>(), st>>>(d, front, dinv, items, kb, mode, status);
}

#define WD_INST(T)                                                                               \
    template void launch_front_init<T>(const DevSym &, T *, const int4 *, int, cudaStream_t);    \
    template void launch_panel<T>(const DevSym &, T *, T *, T *, unsigned char *, const int4 *, int,  \
                                  int, status_t *, cudaStream_t);                                \
    template void launch_diag_copy<T>(const DevSym &, T *, const T *, const int4 *, int,         \
                                      cudaStream_t);                                       \
    template void launch_schur<T>(const DevSym &, T *, T *, const int4 *, int, int, int,         \
                                  status_t *, cudaStream_t);
WD_INST(double)
WD_INST(float)
#undef WD_INST

}  // namespace wd
