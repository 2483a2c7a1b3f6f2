// Supernodal triangular solves by super-blocks of SB pivot columns.
//
// x = P^T L^-T L^-1 P b (the exact inverse of the compressed matrix applied to
// right-hand sides, Sections 1 and 5).  Both substitutions walk the supernodal
// tree level by level.  Inside a supernode they step over super-blocks of
// SB = 512 pivot columns, using the explicit inverse X of each super-block's
// diagonal block (lower triangular, built once per factorization from the
// stored 64 x 64 inverses), so a supernode of width k takes ceil(k / SB)
// dependent steps instead of ceil(k / 64):
//   forward:  y_B = X_B t_B;  t(rows below B) -= L(rows below, B) y_B
//   backward: t_B = y_B - L(rows below, B)^T x(rows below);  x_B = X_B^T t_B
// Rows below a supernode's pivot block go to its update vector, which the
// parent gathers through the extend-add row maps (no atomics).
//
// Buffers (column-major n x nrhs, factor order): Y holds b on entry and x on
// exit; Tt holds the pending right-hand side of pivot rows during the forward
// pass and t during the backward pass.
#include "dev_common.cuh"
#include "engine.h"

namespace wd {
namespace {

constexpr int THREADS = 256;

// ---------------------------------------------------------------------------
// super-block inverses
// ---------------------------------------------------------------------------
// X(t, t) = Dinv of pivot block sb*8 + t; item = (s, sb, t)
template <class T>
__global__ void __launch_bounds__(THREADS) sbinv_diag_kernel(DevSym d, const T *__restrict__ dinv,
                                                             T *__restrict__ xpool,
                                                             const int64_t *__restrict__ xsoff,
                                                             const int4 *__restrict__ items) {
    const int4 it = items[blockIdx.x];
    const int s = it.x, sb = it.y, t = it.z;
    const int k = d.sk[s];
    const int w = min(SB, k - sb * SB), wp = (w + NB - 1) / NB * NB;
    const T *D = dinv + d.dinvoff[s] + (int64_t)(sb * (SB / NB) + t) * NB * NB;
    T *X = xpool + xsoff[s] + (int64_t)sb * SB * SB + (int64_t)(t * NB) * wp + t * NB;
    for (int idx = threadIdx.x; idx < NB * NB; idx += THREADS) {
        const int r = idx % NB, c = idx / NB;
        X[(int64_t)c * wp + r] = D[idx];
    }
}

// X(t, bj) = -D_t sum_{p = bj}^{t-1} L(t, p) X(p, bj), 64 x 64 blocks of the
// super-block; item = (s, sb, bj), stage t = the launch argument
template <class T>
__global__ void __launch_bounds__(THREADS) sbinv_stage_kernel(DevSym d, const T *__restrict__ front,
                                                              const T *__restrict__ dinv,
                                                              T *__restrict__ xpool,
                                                              const int64_t *__restrict__ xsoff,
                                                              const int4 *__restrict__ items, int t) {
    constexpr int TK = 16;
    // staging of the product, then (after it) the 64 x 64 result
    __shared__ T smem[NB * (NB + 1)];
    static_assert(2 * TK * (NB + 1) <= NB * (NB + 1), "staging fits");
    T(*As)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem);
    T(*Bs)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem + TK * (NB + 1));
    T(*Ts)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem);
    const int4 it = items[blockIdx.x];
    const int s = it.x, sb = it.y, bj = it.z;
    const int k = d.sk[s], ld = d.sld[s];
    const int c0 = sb * SB;                          // first column of the super-block
    const int w = min(SB, k - c0), wp = (w + NB - 1) / NB * NB;
    const T *L = front + d.foff[s] + (int64_t)c0 * ld + c0;   // L(c0 + r, c0 + c) at L[c * ld + r]
    T *X = xpool + xsoff[s] + (int64_t)sb * SB * SB;
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    const int rmax = w - t * NB;                     // valid rows of block t
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    // T = sum_p L(t, p) X(p, bj) over p in [bj*64, t*64)
    for (int k0 = bj * NB; k0 < t * NB; k0 += TK) {
        for (int idx = tid; idx < TK * NB; idx += THREADS) {
            const int kk = idx / NB, r = idx % NB;      // rows of L contiguous
            As[kk][r] = (r < rmax) ? L[(int64_t)(k0 + kk) * ld + t * NB + r] : T(0);
        }
        for (int idx = tid; idx < TK * NB; idx += THREADS) {
            const int kk = idx % TK, r = idx / TK;      // rows of X contiguous
            Bs[kk][r] = X[(int64_t)(bj * NB + r) * wp + k0 + kk];
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < TK; ++kk) {
            T a[4], b[4];
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
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) Ts[tx + 16 * i][ty + 16 * j] = acc[i][j];
    __syncthreads();
    // X(t, bj) = -D_t T  (D_t lower triangular, column-major, zero beyond the block)
    const T *D = dinv + d.dinvoff[s] + (int64_t)(sb * (SB / NB) + t) * NB * NB;
    for (int idx = tid; idx < NB * NB; idx += THREADS) {
        const int r = idx % NB, c = idx / NB;
        T v = T(0);
        if (r < rmax)
            for (int p = 0; p <= r; ++p) v += D[(int64_t)p * NB + r] * Ts[p][c];
        X[(int64_t)(bj * NB + c) * wp + t * NB + r] = -v;
    }
}

// XT = X^T per super-block, 64 x 64 tiles: item = (s, sb, i, j), i >= j:
// XT(j, i) = X(i, j)^T
template <class T>
__global__ void __launch_bounds__(THREADS) sbinv_transpose_kernel(DevSym d, const T *__restrict__ xpool,
                                                                  T *__restrict__ xtpool,
                                                                  const int64_t *__restrict__ xsoff,
                                                                  const int4 *__restrict__ items) {
    __shared__ T tile[NB][NB + 1];
    const int4 it = items[blockIdx.x];
    const int s = it.x, sb = it.y, bi = it.z, bj = it.w;
    const int k = d.sk[s];
    const int w = min(SB, k - sb * SB), wp = (w + NB - 1) / NB * NB;
    const int64_t base = xsoff[s] + (int64_t)sb * SB * SB;
    const T *X = xpool + base + (int64_t)(bj * NB) * wp + bi * NB;   // X(bi, bj) tile
    T *XT = xtpool + base + (int64_t)(bi * NB) * wp + bj * NB;       // XT(bj, bi) tile
    for (int idx = threadIdx.x; idx < NB * NB; idx += THREADS) {
        const int r = idx % NB, c = idx / NB;
        tile[r][c] = X[(int64_t)c * wp + r];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < NB * NB; idx += THREADS) {
        const int r = idx % NB, c = idx / NB;
        XT[(int64_t)c * wp + r] = tile[c][r];
    }
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
// Right-hand-side tiles: RGT (64 or 16) columns per CTA; 256 threads = 64 rows
// (or pivot columns) x 4 groups of NPT = RGT / 4 right-hand sides.  Operand
// rows of right-hand sides are staged RHS-contiguous, so a thread reads its
// NPT values with 16-byte shared-memory loads.

// 16-byte vector of T
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
};

// acc[j] += a * v[j], j < NPT, v 16-byte aligned in shared memory
template <class T, int NPT>
__device__ __forceinline__ void axpy_row(T (&acc)[NPT], T a, const T *v) {
    using V = typename Vec16<T>::type;
    constexpr int E = Vec16<T>::n;
#pragma unroll
    for (int j = 0; j < NPT; j += E) {
        const V q = *reinterpret_cast<const V *>(v + j);
        const T *e = reinterpret_cast<const T *>(&q);
#pragma unroll
        for (int u = 0; u < E; ++u) acc[j + u] += a * e[u];
    }
}

// pivot rows: Tt = b_J + children's update vectors; rows below: W_s = the
// children's update vectors.  item = (s, 32-row block, rhs tile); lane = row,
// warp w takes right-hand sides w, w + 8, ... of the tile.
template <class T, int RGT>
__global__ void __launch_bounds__(THREADS) bfwd_gather_kernel(DevSym d, const T *__restrict__ Y,
                                                              T *__restrict__ Tt, T *__restrict__ W,
                                                              const int4 *__restrict__ items,
                                                              int nrhs) {
    constexpr int PW = RGT / 8;  // right-hand sides per thread
    const int4 it = items[blockIdx.x];
    const int s = it.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = it.y * 32 + lane;
    const int m = d.sm[s], k = d.sk[s];
    if (r >= m) return;
    const int64_t n = d.n;
    const int f = d.sfirst[s];
    const int c0 = it.z * RGT;
    T t[PW];
#pragma unroll
    for (int j = 0; j < PW; ++j) {
        const int c = c0 + warp + 8 * j;
        t[j] = (r < k && c < nrhs) ? Y[f + r + (int64_t)c * n] : T(0);
    }
    for (int ci = d.child_ptr[s]; ci < d.child_ptr[s + 1]; ++ci) {
        const int ch = d.children[ci];
        const int ic = d.relmap[d.mapoff[ch] + r];
        if (ic < 0) continue;
        const int ldc = d.sm[ch] - d.sk[ch];
        const T *Wc = W + d.woff[ch] * nrhs + ic;
#pragma unroll
        for (int j = 0; j < PW; ++j) {
            const int c = c0 + warp + 8 * j;
            if (c < nrhs) t[j] += Wc[(int64_t)c * ldc];
        }
    }
    T *Ws = W + d.woff[s] * nrhs;
#pragma unroll
    for (int j = 0; j < PW; ++j) {
        const int c = c0 + warp + 8 * j;
        if (c >= nrhs) continue;
        if (r < k) Tt[f + r + (int64_t)c * n] = t[j];
        else Ws[(int64_t)c * (m - k) + (r - k)] = t[j];
    }
}

// Tiles of the dependent solve products: ROWS rows (or pivot columns) x RHS
// right-hand sides per CTA; warp w owns RPW consecutive rows, lane l the
// right-hand sides l, l + 32, ... (RPL of them).  The matrix tile is staged
// with rows contiguous (A[p * lda + row]) and read by a whole warp at once
// (broadcast 16-byte loads), the right-hand-side tile is staged right-hand-
// side major with an odd stride (R[c * LDR + p]), so both the staging writes
// and the reads are free of bank conflicts.  The shape in use is 64 x 32 (8
// rows per warp, one right-hand side per lane); 128 x 64 tiles measured slower
// on the 2D 256^2 case (half the CTAs on the narrow tree levels).
template <int RPW_, int RPL_>
struct TileCfg {
    static constexpr int RPW = RPW_;
    static constexpr int RPL = RPL_;
    static constexpr int ROWS = 8 * RPW;
    static constexpr int RHS = 32 * RPL;
    static constexpr int LDO = ROWS + 1;     // stride of the staged result
    static constexpr int MINB = RPW * RPL > 8 ? 2 : 4;   // resident CTAs per SM (register budget)
};
using TileS = TileCfg<8, 1>;
constexpr int LDR = NB + 1;                  // stride of a staged right-hand side

template <class T, class C, int LDA>
__device__ __forceinline__ void tile_accumulate(T (&acc)[C::RPW][C::RPL], const T *A, const T *R, int np) {
    using V = typename Vec16<T>::type;
    constexpr int E = Vec16<T>::n;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T *a = A + C::RPW * w;
    const T *r = R + lane * LDR;
#pragma unroll 2
    for (int p = 0; p < np; ++p) {
        T x[C::RPL];
#pragma unroll
        for (int q = 0; q < C::RPL; ++q) x[q] = r[q * 32 * LDR + p];
#pragma unroll
        for (int j = 0; j < C::RPW; j += E) {
            const V v = *reinterpret_cast<const V *>(a + p * LDA + j);
            const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int u = 0; u < E; ++u)
#pragma unroll
                for (int q = 0; q < C::RPL; ++q) acc[j + u][q] += e[u] * x[q];
        }
    }
}

template <class T, class C>
__device__ __forceinline__ void tile_zero(T (&acc)[C::RPW][C::RPL]) {
#pragma unroll
    for (int i = 0; i < C::RPW; ++i)
#pragma unroll
        for (int q = 0; q < C::RPL; ++q) acc[i][q] = T(0);
}

// the CTA's result into O[c * LDO + r] (r = row of the tile, c = right-hand
// side), so that it can be written out with rows contiguous
template <class T, class C>
__device__ __forceinline__ void tile_to_smem(const T (&acc)[C::RPW][C::RPL], T *O) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < C::RPW; ++i)
#pragma unroll
        for (int q = 0; q < C::RPL; ++q) O[(lane + 32 * q) * C::LDO + C::RPW * w + i] = acc[i][q];
}

// rows [p0, p0 + 64) of right-hand sides c0 .. c0 + RHS - 1 (column-major,
// ld n, first row `row0`) into R[c * LDR + p]; rows >= valid (and columns
// >= nc) zero
template <class T, class C>
__device__ __forceinline__ void stage_rhs(T *R, const T *src, int64_t row0, int p0, int valid, int c0,
                                          int nc, int64_t n) {
    for (int idx = threadIdx.x; idx < NB * C::RHS; idx += THREADS) {
        const int p = idx % NB, c = idx / NB;
        const bool v = p0 + p < valid && c < nc;
        cp_async_elem(R + c * LDR + p, v ? src + row0 + p0 + p + (int64_t)(c0 + c) * n : src, v);
    }
}

template <class T, class C>
constexpr int tile_smem_elems() {
    return 2 * NB * C::ROWS + 2 * C::RHS * LDR + 8;
}

// out(B rows ROWS rb .. +ROWS) = X_B in_B (upper = 0) or X_B^T in_B (upper =
// 1, using the stored transpose); item = (s, sb, rb, rhs tile)
template <class T, class C>
__global__ void __launch_bounds__(THREADS, C::MINB) xapply_kernel(DevSym d, const T *__restrict__ xp,
                                                         const int64_t *__restrict__ xsoff,
                                                         const T *__restrict__ in, T *__restrict__ out,
                                                         const int4 *__restrict__ items, int upper,
                                                         int nrhs) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *Xs[2] = {sm, sm + NB * C::ROWS};                                    // [p][r], ld ROWS
    T *Rs[2] = {sm + 2 * NB * C::ROWS, sm + 2 * NB * C::ROWS + C::RHS * LDR};  // [c][p], ld LDR
    const int4 it = items[blockIdx.x];
    const int s = it.x, sb = it.y, rb = it.z, c0 = it.w * C::RHS;
    const int k = d.sk[s];
    const int b0 = sb * SB;
    const int w = min(SB, k - b0), wp = (w + NB - 1) / NB * NB;
    const int nb = wp / NB;
    const int nc = min(C::RHS, nrhs - c0);
    const int64_t n = d.n;
    const int64_t row0 = d.sfirst[s] + b0;
    const T *X = xp + xsoff[s] + (int64_t)sb * SB * SB;
    const int r0 = rb * C::ROWS, rvalid = wp - r0;
    const int q0 = upper ? r0 / NB : 0, q1 = upper ? nb : min(nb, (r0 + C::ROWS) / NB);
    auto stage = [&](int buf, int q) {
        stage_tile<T, THREADS>(Xs[buf], C::ROWS, X + (int64_t)(q * NB) * wp + r0, wp, C::ROWS, NB, rvalid, NB);
        stage_rhs<T, C>(Rs[buf], in, row0, q * NB, w, c0, nc, n);
        cp_async_commit();
    };
    T acc[C::RPW][C::RPL];
    tile_zero<T, C>(acc);
    stage(0, q0);
    for (int q = q0; q < q1; ++q) {
        const int cur = (q - q0) & 1;
        if (q + 1 < q1) {
            stage(cur ^ 1, q + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        tile_accumulate<T, C, C::ROWS>(acc, Xs[cur], Rs[cur], min(NB, w - q * NB));
        __syncthreads();
    }
    T *O = sm;
    tile_to_smem<T, C>(acc, O);
    __syncthreads();
    for (int idx = threadIdx.x; idx < C::ROWS * C::RHS; idx += THREADS) {
        const int r = idx % C::ROWS, c = idx / C::ROWS;
        const int rr = r0 + r;
        if (rr < w && c < nc) out[row0 + rr + (int64_t)(c0 + c) * n] = O[c * C::LDO + r];
    }
}

// rows below super-block B: target -= L(rows, B) y_B.  item = (s, sb, rb,
// tile + 65536 * seg): seg 0 = pivot rows after B (target Tt), seg 1 = rows
// of R (target the update vector W_s)
template <class T, class C>
__global__ void __launch_bounds__(THREADS, C::MINB) bupdate_kernel(DevSym d, const T *__restrict__ front,
                                                          const T *__restrict__ Y, T *__restrict__ Tt,
                                                          T *__restrict__ W, const int4 *__restrict__ items,
                                                          int nrhs) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *Ls[2] = {sm, sm + NB * C::ROWS};
    T *Rs[2] = {sm + 2 * NB * C::ROWS, sm + 2 * NB * C::ROWS + C::RHS * LDR};
    const int4 it = items[blockIdx.x];
    const int s = it.x, sb = it.y, rb = it.z, g = it.w & 0xFFFF, seg = it.w >> 16;
    const int m = d.sm[s], k = d.sk[s], kp = d.skp[s], ld = d.sld[s];
    const int b0 = sb * SB, w = min(SB, k - b0);
    const int c0 = g * C::RHS, nc = min(C::RHS, nrhs - c0);
    const int64_t n = d.n;
    const int f = d.sfirst[s];
    const int i0 = seg == 0 ? b0 + w + rb * C::ROWS : rb * C::ROWS;     // seg 1: index into R
    const int nrow = seg == 0 ? k - i0 : (m - k) - i0;
    const int mrow = seg == 0 ? i0 : kp + i0;
    const T *F = front + d.foff[s] + mrow;
    auto stage = [&](int buf, int p0) {
        stage_tile<T, THREADS>(Ls[buf], C::ROWS, F + (int64_t)(b0 + p0) * ld, ld, C::ROWS, NB, nrow, w - p0);
        stage_rhs<T, C>(Rs[buf], Y, f + b0, p0, w, c0, nc, n);
        cp_async_commit();
    };
    T *dst;
    int64_t ldd;
    if (seg == 0) {
        dst = Tt + f + i0;
        ldd = n;
    } else {
        dst = W + d.woff[s] * nrhs + i0;
        ldd = m - k;
    }
    constexpr int PE = C::ROWS * C::RHS / THREADS;   // target elements per thread
    // FP32 with the small tile has the registers to hold the target early
    constexpr bool PRE = sizeof(T) == 4 && C::RPW * C::RPL <= 8;
    T acc[C::RPW][C::RPL];
    tile_zero<T, C>(acc);
    const int nchunk = (w + NB - 1) / NB;
    stage(0, 0);
    // the target tile is read now, while the staging copies are in flight
    // (same element order as the write-back below: rows contiguous)
    T tpre[PE];
#pragma unroll
    for (int e = 0; e < PE; ++e) {
        const int idx = threadIdx.x + e * THREADS;
        const int r = idx % C::ROWS, c = idx / C::ROWS;
        tpre[e] = (PRE && r < nrow && c < nc) ? dst[r + (int64_t)(c0 + c) * ldd] : T(0);
    }
    for (int ch = 0; ch < nchunk; ++ch) {
        const int cur = ch & 1;
        if (ch + 1 < nchunk) {
            stage(cur ^ 1, (ch + 1) * NB);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        tile_accumulate<T, C, C::ROWS>(acc, Ls[cur], Rs[cur], min(NB, w - ch * NB));
        __syncthreads();
    }
    T *O = sm;
    tile_to_smem<T, C>(acc, O);
    if (!PRE) {
        // every old target value is read before the first store: a store may
        // alias a later element's load through the runtime stride, which
        // would make each read-modify-write a memory round trip of its own
#pragma unroll
        for (int e = 0; e < PE; ++e) {
            const int idx = threadIdx.x + e * THREADS;
            const int r = idx % C::ROWS, c = idx / C::ROWS;
            tpre[e] = (r < nrow && c < nc) ? dst[r + (int64_t)(c0 + c) * ldd] : T(0);
        }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < PE; ++e) {
        const int idx = threadIdx.x + e * THREADS;
        const int r = idx % C::ROWS, c = idx / C::ROWS;
        if (r < nrow && c < nc) dst[r + (int64_t)(c0 + c) * ldd] = tpre[e] - O[c * C::LDO + r];
    }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
constexpr int KSR = SOLVE_KSR;    // rows below B per split of the reduction

template <class C>
struct ReduceCfg {
    static constexpr int LDT = C::ROWS + 4;   // row stride of the staged L^T tile (16-byte multiple)
};

template <class T, class C>
constexpr int breduce_smem_elems() {
    return 2 * (64 * ReduceCfg<C>::LDT + C::RHS * LDR) + 8;
}

// Partial reduction of t_B = y_B - L(rows below B, B)^T x(rows below) over the
// rows [ks * KSR, (ks + 1) * KSR) of the "rows below" list (pivot rows after B,
// then the rows of R; x of a front row read at its global row):
// P[slot] (RHS x ROWS, [rhs][c]) = sum_i L(i, j0 + c) x(i, rhs), j0 = b0 +
// ROWS cb.  item = (s, sb * 8 + cb, tile + 65536 * ks, slot)
template <class T, class C>
__global__ void __launch_bounds__(THREADS, C::MINB) breduce_kernel(DevSym d, const T *__restrict__ front,
                                                          const T *__restrict__ Y, T *__restrict__ P,
                                                          const int4 *__restrict__ items, int nrhs) {
    constexpr int LDT = ReduceCfg<C>::LDT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    T *Ls[2] = {sm, sm + 64 * LDT};                                          // [rr][c], ld LDT
    T *Rs[2] = {sm + 2 * 64 * LDT, sm + 2 * 64 * LDT + C::RHS * LDR};        // [rhs][rr], ld LDR
    const int4 it = items[blockIdx.x];
    const int s = it.x, sb = it.y >> 3, cb = it.y & 7, g = it.z & 0xFFFF, ks = it.z >> 16;
    const int m = d.sm[s], k = d.sk[s], kp = d.skp[s], ld = d.sld[s];
    const int b0 = sb * SB, w = min(SB, k - b0);
    const int j0 = b0 + cb * C::ROWS, nb = min(C::ROWS, k - j0);
    const int c0 = g * C::RHS, nc = min(C::RHS, nrhs - c0);
    const int64_t n = d.n;
    const T *F = front + d.foff[s] + (int64_t)j0 * ld;
    const int32_t *rows = d.rows + d.rowptr[s];
    const int tid = threadIdx.x;
    const int nJ = k - (b0 + w), nbelow = nJ + (m - k);
    const int u0 = ks * KSR, u1 = min(nbelow, u0 + KSR);
    auto stage = [&](int buf, int ua) {
        for (int idx = tid; idx < 64 * C::ROWS; idx += THREADS) {
            const int rr = idx % 64, c = idx / 64;
            const int u = ua + rr;
            const bool v = u < u1 && c < nb;
            const int mrow = u < nJ ? b0 + w + u : kp + (u - nJ);
            cp_async_elem(Ls[buf] + rr * LDT + c, v ? F + (int64_t)c * ld + mrow : F, v);
        }
        for (int idx = tid; idx < 64 * C::RHS; idx += THREADS) {
            const int rr = idx % 64, c = idx / 64;
            const int u = ua + rr;
            const bool v = u < u1 && c < nc;
            const int lr = u < nJ ? b0 + w + u : k + (u - nJ);
            cp_async_elem(Rs[buf] + c * LDR + rr, v ? Y + rows[lr] + (int64_t)(c0 + c) * n : Y, v);
        }
        cp_async_commit();
    };
    T acc[C::RPW][C::RPL];
    tile_zero<T, C>(acc);
    const int nchunk = (u1 - u0 + 63) / 64;
    stage(0, u0);
    for (int ch = 0; ch < nchunk; ++ch) {
        const int cur = ch & 1;
        if (ch + 1 < nchunk) {
            stage(cur ^ 1, u0 + (ch + 1) * 64);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        tile_accumulate<T, C, LDT>(acc, Ls[cur], Rs[cur], min(64, u1 - u0 - ch * 64));
        __syncthreads();
    }
    T *O = sm;
    tile_to_smem<T, C>(acc, O);
    __syncthreads();
    T *Pt = P + (int64_t)it.w * C::RHS * C::ROWS;
    for (int idx = tid; idx < C::ROWS * C::RHS; idx += THREADS) {
        const int r = idx % C::ROWS, c = idx / C::ROWS;
        Pt[c * C::ROWS + r] = O[c * C::LDO + r];
    }
}

// Tt(B columns) = y - sum of the splits' partial sums, in split order; one
// element of the ROWS x RHS tile per thread.
// item = (s, sb * 8 + cb, tile + 65536 * nsplit, first slot)
template <class T, class C>
__global__ void __launch_bounds__(THREADS) breduce_finish_kernel(DevSym d, const T *__restrict__ Y,
                                                                 T *__restrict__ Tt, const T *__restrict__ P,
                                                                 const int4 *__restrict__ items, int nrhs) {
    constexpr int PER = C::ROWS * C::RHS / THREADS;   // CTAs per item
    const int4 it = items[blockIdx.x / PER];
    const int s = it.x, sb = it.y >> 3, cb = it.y & 7, g = it.z & 0xFFFF, nsplit = it.z >> 16;
    const int k = d.sk[s];
    const int j0 = sb * SB + cb * C::ROWS, nb = min(C::ROWS, k - j0);
    const int c0 = g * C::RHS, nc = min(C::RHS, nrhs - c0);
    const int64_t n = d.n;
    const int f = d.sfirst[s];
    const int idx = (blockIdx.x % PER) * THREADS + threadIdx.x;
    const int cl = idx % C::ROWS, c = idx / C::ROWS;
    if (cl >= nb || c >= nc) return;
    T sum = T(0);
    for (int q = 0; q < nsplit; ++q) sum += P[((int64_t)(it.w + q) * C::RHS + c) * C::ROWS + cl];
    const int64_t o = f + j0 + cl + (int64_t)(c0 + c) * n;
    Tt[o] = Y[o] - sum;
}

// ---------------------------------------------------------------------------
// Few right-hand sides (nrhs <= 8): the products are matrix-vector shaped, so
// lanes run over rows (coalesced columns of L or X) instead of right-hand
// sides.  A CTA covers NRW = 32 rows; its 8 warps split the columns (column p
// to warp p mod 8), the right-hand-side block is staged in shared memory
// (V[p * NR + c]), and the warps' partial sums are added in a fixed order.
// NR = nrhs rounded up to 1, 2, 4 or 8; columns c >= nrhs are zero.
// ---------------------------------------------------------------------------
constexpr int NRW = 32;
constexpr int NWARP = THREADS / 32;

// acc[c] += sum over p in [pa, pb) with p = warp (mod NWARP) of A[p * lda] V[p * NR + c]
// (A already offset to this lane's row; ok = the row is valid)
template <class T, int NR>
__device__ __forceinline__ void narrow_accumulate(T (&acc)[NR], const T *__restrict__ A, int64_t lda, bool ok,
                                                  const T *V, int pa, int pb) {
    const int warp = threadIdx.x >> 5;
    constexpr int U = 4;
    for (int p0 = pa + warp; p0 < pb; p0 += NWARP * U) {
        T a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int p = p0 + NWARP * u;
            a[u] = (ok && p < pb) ? A[(int64_t)p * lda] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int p = min(p0 + NWARP * u, pb - 1);
#pragma unroll
            for (int c = 0; c < NR; ++c) acc[c] += a[u] * V[p * NR + c];
        }
    }
}

// the warps' sums of row (tid % 32), column (tid / 32) in warp order, for
// tid < 32 NR (red: [NWARP][NRW][NR]); call after narrow_accumulate by all threads
template <class T, int NR>
__device__ __forceinline__ T narrow_reduce(const T (&acc)[NR], T *red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < NR; ++c) red[(warp * NRW + lane) * NR + c] = acc[c];
    __syncthreads();
    T sum = T(0);
    if (threadIdx.x < NRW * NR) {
        const int r = threadIdx.x % NRW, c = threadIdx.x / NRW;
        for (int g = 0; g < NWARP; ++g) sum += red[(g * NRW + r) * NR + c];
    }
    return sum;
}

// y_B rows [32 rb, 32 rb + 32) = X_B in_B (upper = 0) or X_B^T in_B (upper =
// 1, the stored transpose); item = (s, sb, rb, 0)
template <class T, int NR>
__global__ void __launch_bounds__(THREADS) xapply_narrow_kernel(DevSym d, const T *__restrict__ xp,
                                                                const int64_t *__restrict__ xsoff,
                                                                const T *__restrict__ in, T *__restrict__ out,
                                                                const int4 *__restrict__ items, int upper,
                                                                int nrhs) {
    __shared__ T V[SB * NR];
    __shared__ T red[NWARP * NRW * NR];
    const int4 it = items[blockIdx.x];
    const int s = it.x, sb = it.y, rb = it.z;
    const int k = d.sk[s];
    const int b0 = sb * SB, w = min(SB, k - b0), wp = (w + NB - 1) / NB * NB;
    const int64_t n = d.n;
    const int64_t row0 = d.sfirst[s] + b0;
    const T *X = xp + xsoff[s] + (int64_t)sb * SB * SB;
    for (int idx = threadIdx.x; idx < w * NR; idx += THREADS) {
        const int q = idx / NR, c = idx % NR;
        V[idx] = c < nrhs ? in[row0 + q + (int64_t)c * n] : T(0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, r0 = rb * NRW, r = r0 + lane;
    T acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = T(0);
    // lower: columns q <= r; upper: q >= r (the stored blocks are zero outside)
    const int qa = upper ? r0 : 0, qb = upper ? w : min(w, r0 + NRW);
    narrow_accumulate<T, NR>(acc, X + r, wp, r < w, V, qa, qb);
    const T sum = narrow_reduce<T, NR>(acc, red);
    if (threadIdx.x < NRW * NR) {
        const int rr = r0 + threadIdx.x % NRW, c = threadIdx.x / NRW;
        if (rr < w && c < nrhs) out[row0 + rr + (int64_t)c * n] = sum;
    }
}

// rows below super-block B: target -= L(rows, B) y_B, 32 rows per CTA; item =
// (s, sb, rb, 65536 * seg): seg 0 = pivot rows after B (target Tt), seg 1 =
// rows of R (target the update vector W_s)
template <class T, int NR>
__global__ void __launch_bounds__(THREADS) bupdate_narrow_kernel(DevSym d, const T *__restrict__ front,
                                                                 const T *__restrict__ Y, T *__restrict__ Tt,
                                                                 T *__restrict__ W, const int4 *__restrict__ items,
                                                                 int nrhs) {
    __shared__ T V[SB * NR];
    __shared__ T red[NWARP * NRW * NR];
    const int4 it = items[blockIdx.x];
    const int s = it.x, sb = it.y, rb = it.z, seg = it.w >> 16;
    const int m = d.sm[s], k = d.sk[s], kp = d.skp[s], ld = d.sld[s];
    const int b0 = sb * SB, w = min(SB, k - b0);
    const int64_t n = d.n;
    const int f = d.sfirst[s];
    const int i0 = seg == 0 ? b0 + w + rb * NRW : rb * NRW;
    const int nrow = seg == 0 ? k - i0 : (m - k) - i0;
    const int mrow = seg == 0 ? i0 : kp + i0;
    T *dst;
    int64_t ldd;
    if (seg == 0) {
        dst = Tt + f + i0;
        ldd = n;
    } else {
        dst = W + d.woff[s] * nrhs + i0;
        ldd = m - k;
    }
    for (int idx = threadIdx.x; idx < w * NR; idx += THREADS) {
        const int p = idx / NR, c = idx % NR;
        V[idx] = c < nrhs ? Y[f + b0 + p + (int64_t)c * n] : T(0);
    }
    // the target is read while the columns stream in
    T tpre = T(0);
    if (threadIdx.x < NRW * NR) {
        const int r = threadIdx.x % NRW, c = threadIdx.x / NRW;
        if (r < nrow && c < nrhs) tpre = dst[r + (int64_t)c * ldd];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    T acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = T(0);
    narrow_accumulate<T, NR>(acc, front + d.foff[s] + (int64_t)b0 * ld + mrow + lane, ld, lane < nrow, V, 0, w);
    const T sum = narrow_reduce<T, NR>(acc, red);
    if (threadIdx.x < NRW * NR) {
        const int r = threadIdx.x % NRW, c = threadIdx.x / NRW;
        if (r < nrow && c < nrhs) dst[r + (int64_t)c * ldd] = tpre - sum;
    }
}

// Partial reduction of t_B = y_B - L(rows below B, B)^T x(rows below) over the
// rows [ks KSR, (ks + 1) KSR) of the "rows below" list, for the 64 columns
// j0 = b0 + 64 cb ...: one warp per column (8 columns per warp), lanes over
// rows; P[slot] holds the sums in the 64 x 32 tile layout ([rhs][column]).
// item = (s, sb * 8 + cb, 65536 * ks, slot)
template <class T, int NR>
__global__ void __launch_bounds__(THREADS) breduce_narrow_kernel(DevSym d, const T *__restrict__ front,
                                                                 const T *__restrict__ Y, T *__restrict__ P,
                                                                 const int4 *__restrict__ items, int nrhs) {
    constexpr int RC = TileS::ROWS, RR = TileS::RHS;     // P tile: RR right-hand sides x RC columns
    __shared__ T xs[KSR * NR];
    const int4 it = items[blockIdx.x];
    const int s = it.x, sb = it.y >> 3, cb = it.y & 7, ks = it.z >> 16;
    const int m = d.sm[s], k = d.sk[s], kp = d.skp[s], ld = d.sld[s];
    const int b0 = sb * SB, w = min(SB, k - b0);
    const int j0 = b0 + cb * RC, nb = min(RC, k - j0);
    const int64_t n = d.n;
    const T *F = front + d.foff[s] + (int64_t)j0 * ld;
    const int32_t *rows = d.rows + d.rowptr[s];
    const int nJ = k - (b0 + w), nbelow = nJ + (m - k);
    const int u0 = ks * KSR, nu = min(nbelow, u0 + KSR) - u0;
    for (int idx = threadIdx.x; idx < nu * NR; idx += THREADS) {
        const int rr = idx / NR, c = idx % NR;
        const int u = u0 + rr;
        const int lr = u < nJ ? b0 + w + u : k + (u - nJ);
        xs[idx] = c < nrhs ? Y[rows[lr] + (int64_t)c * n] : T(0);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *Pt = P + (int64_t)it.w * RR * RC;
    for (int q = 0; q < RC / NWARP; ++q) {
        const int cl = warp * (RC / NWARP) + q;
        if (cl >= nb) break;
        T acc[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = T(0);
        const T *col = F + (int64_t)cl * ld;
#pragma unroll
        for (int rr = lane; rr < KSR; rr += 32) {
            if (rr < nu) {
                const int u = u0 + rr;
                const T a = col[u < nJ ? b0 + w + u : kp + (u - nJ)];
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[c] += a * xs[rr * NR + c];
            }
        }
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            T v = acc[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && c < nrhs) Pt[c * RC + cl] = v;
        }
    }
}

}  // namespace

template <class T, class C>
void set_blocked_attributes() {
    cudaFuncSetAttribute(xapply_kernel<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(tile_smem_elems<T, C>() * sizeof(T)));
    cudaFuncSetAttribute(bupdate_kernel<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(tile_smem_elems<T, C>() * sizeof(T)));
    cudaFuncSetAttribute(breduce_kernel<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(breduce_smem_elems<T, C>() * sizeof(T)));
}

void init_blocked_attributes() {
    static bool done = false;
    if (done) return;
    set_blocked_attributes<float, TileS>();
    set_blocked_attributes<double, TileS>();
    done = true;
}

// the partial-sum tile of the tensor-core backward products (128 columns x 64
// right-hand sides); only its ROWS and RHS are used
using TileTc = TileCfg<16, 2>;
int solve_tile_rows(int large) { return large == 1 ? TileTc::ROWS : TileS::ROWS; }
int solve_tile_rhs(int large) { return large == 1 ? TileTc::RHS : TileS::RHS; }
int solve_update_rows(int large) { return large == 2 ? NRW : solve_tile_rows(large); }

template <class T>
void launch_sbinv_diag(const DevSym &d, const T *dinv, T *xpool, const int64_t *xsoff, const int4 *items,
                       int count, cudaStream_t st) {
    if (count > 0) sbinv_diag_kernel<T><<<count, THREADS, 0, st>>>(d, dinv, xpool, xsoff, items);
}
template <class T>
void launch_sbinv_stage(const DevSym &d, const T *front, const T *dinv, T *xpool, const int64_t *xsoff,
                        const int4 *items, int count, int t, cudaStream_t st) {
    if (count > 0)
        sbinv_stage_kernel<T><<<count, THREADS, 0, st>>>(d, front, dinv, xpool, xsoff, items, t);
}
template <class T>
void launch_sbinv_transpose(const DevSym &d, const T *xpool, T *xtpool, const int64_t *xsoff,
                            const int4 *items, int count, cudaStream_t st) {
    if (count > 0) sbinv_transpose_kernel<T><<<count, THREADS, 0, st>>>(d, xpool, xtpool, xsoff, items);
}
template <class T>
void launch_bfwd_gather(const DevSym &d, const T *Y, T *Tt, T *W, const int4 *items, int count, int rgt,
                        int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    if (rgt == 64) bfwd_gather_kernel<T, 64><<<count, THREADS, 0, st>>>(d, Y, Tt, W, items, nrhs);
    else bfwd_gather_kernel<T, 16><<<count, THREADS, 0, st>>>(d, Y, Tt, W, items, nrhs);
}
template <class T, class C>
static void xapply_go(const DevSym &d, const T *xp, const int64_t *xsoff, const T *in, T *out,
                      const int4 *items, int count, int upper, int nrhs, cudaStream_t st) {
    xapply_kernel<T, C><<<count, THREADS, tile_smem_elems<T, C>() * sizeof(T), st>>>(d, xp, xsoff, in, out,
                                                                                   items, upper, nrhs);
}
template <class T, class C>
static void bupdate_go(const DevSym &d, const T *front, const T *Y, T *Tt, T *W, const int4 *items,
                       int count, int nrhs, cudaStream_t st) {
    bupdate_kernel<T, C><<<count, THREADS, tile_smem_elems<T, C>() * sizeof(T), st>>>(d, front, Y, Tt, W,
                                                                                    items, nrhs);
}
template <class T, class C>
static void breduce_go(const DevSym &d, const T *front, const T *Y, T *P, const int4 *items, int count,
                       int nrhs, cudaStream_t st) {
    breduce_kernel<T, C><<<count, THREADS, breduce_smem_elems<T, C>() * sizeof(T), st>>>(d, front, Y, P,
                                                                                       items, nrhs);
}
template <class T, class C>
static void finish_go(const DevSym &d, const T *Y, T *Tt, const T *P, const int4 *items, int count, int nrhs,
                      cudaStream_t st) {
    constexpr int PER = C::ROWS * C::RHS / THREADS;
    breduce_finish_kernel<T, C><<<count * PER, THREADS, 0, st>>>(d, Y, Tt, P, items, nrhs);
}

// large = 1 selects the 128 x 64 tiles (FP32 only)
template <class T>
void launch_xapply(const DevSym &d, const T *xp, const int64_t *xsoff, const T *in, T *out,
                   const int4 *items, int count, int upper, int large, int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    if (large == 2) {
        if (nrhs == 1) xapply_narrow_kernel<T, 1><<<count, THREADS, 0, st>>>(d, xp, xsoff, in, out, items, upper, nrhs);
        else if (nrhs == 2) xapply_narrow_kernel<T, 2><<<count, THREADS, 0, st>>>(d, xp, xsoff, in, out, items, upper, nrhs);
        else if (nrhs <= 4) xapply_narrow_kernel<T, 4><<<count, THREADS, 0, st>>>(d, xp, xsoff, in, out, items, upper, nrhs);
        else xapply_narrow_kernel<T, 8><<<count, THREADS, 0, st>>>(d, xp, xsoff, in, out, items, upper, nrhs);
        return;
    }
    xapply_go<T, TileS>(d, xp, xsoff, in, out, items, count, upper, nrhs, st);
}
template <class T>
void launch_bupdate(const DevSym &d, const T *front, const T *Y, T *Tt, T *W, const int4 *items, int count,
                    int large, int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    if (large == 2) {
        if (nrhs == 1) bupdate_narrow_kernel<T, 1><<<count, THREADS, 0, st>>>(d, front, Y, Tt, W, items, nrhs);
        else if (nrhs == 2) bupdate_narrow_kernel<T, 2><<<count, THREADS, 0, st>>>(d, front, Y, Tt, W, items, nrhs);
        else if (nrhs <= 4) bupdate_narrow_kernel<T, 4><<<count, THREADS, 0, st>>>(d, front, Y, Tt, W, items, nrhs);
        else bupdate_narrow_kernel<T, 8><<<count, THREADS, 0, st>>>(d, front, Y, Tt, W, items, nrhs);
        return;
    }
    bupdate_go<T, TileS>(d, front, Y, Tt, W, items, count, nrhs, st);
}
template <class T>
void launch_breduce(const DevSym &d, const T *front, const T *Y, T *P, const int4 *items, int count,
                    int large, int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    if (large == 2) {
        if (nrhs == 1) breduce_narrow_kernel<T, 1><<<count, THREADS, 0, st>>>(d, front, Y, P, items, nrhs);
        else if (nrhs == 2) breduce_narrow_kernel<T, 2><<<count, THREADS, 0, st>>>(d, front, Y, P, items, nrhs);
        else if (nrhs <= 4) breduce_narrow_kernel<T, 4><<<count, THREADS, 0, st>>>(d, front, Y, P, items, nrhs);
        else breduce_narrow_kernel<T, 8><<<count, THREADS, 0, st>>>(d, front, Y, P, items, nrhs);
        return;
    }
    breduce_go<T, TileS>(d, front, Y, P, items, count, nrhs, st);
}
template <class T>
void launch_breduce_finish(const DevSym &d, const T *Y, T *Tt, const T *P, const int4 *items, int count,
                           int large, int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    if (large == 1) finish_go<T, TileTc>(d, Y, Tt, P, items, count, nrhs, st);
    else finish_go<T, TileS>(d, Y, Tt, P, items, count, nrhs, st);
}

#define WD_BLOCKED_INST(T)                                                                              \
    template void launch_sbinv_diag<T>(const DevSym &, const T *, T *, const int64_t *, const int4 *, int, \
                                       cudaStream_t);                                                   \
    template void launch_sbinv_stage<T>(const DevSym &, const T *, const T *, T *, const int64_t *,      \
                                        const int4 *, int, int, cudaStream_t);                          \
    template void launch_sbinv_transpose<T>(const DevSym &, const T *, T *, const int64_t *, const int4 *, \
                                            int, cudaStream_t);                                         \
    template void launch_bfwd_gather<T>(const DevSym &, const T *, T *, T *, const int4 *, int, int, int, \
                                        cudaStream_t);                                                  \
    template void launch_xapply<T>(const DevSym &, const T *, const int64_t *, const T *, T *,           \
                                   const int4 *, int, int, int, int, cudaStream_t);                     \
    template void launch_bupdate<T>(const DevSym &, const T *, const T *, T *, T *, const int4 *, int,   \
                                    int, int, cudaStream_t);                                            \
    template void launch_breduce<T>(const DevSym &, const T *, const T *, T *, const int4 *, int, int,   \
                                    int, cudaStream_t);                                                 \
    template void launch_breduce_finish<T>(const DevSym &, const T *, T *, const T *, const int4 *, int, \
                                           int, int, cudaStream_t);
WD_BLOCKED_INST(float)
WD_BLOCKED_INST(double)

}  // namespace wd
