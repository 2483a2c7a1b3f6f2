// Permutations and transposes of right-hand sides, P^T L z, the FP64
// residual of the refinement and the reductions (norms, log det).  The
// triangular solves themselves are in solve_blocked.cu.
#include "dev_common.cuh"
#include "engine.h"

namespace wd {
namespace {

constexpr int THREADS = 256;

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

// out = values in CSR order; hi / lo (optional): the double-float split
// out = hi + lo (hi = out rounded to FP32, lo = the rest rounded to FP32)
__global__ void gather_values_kernel(const int32_t *__restrict__ src, const double *__restrict__ v,
                                     double *__restrict__ out, float *__restrict__ hi,
                                     float *__restrict__ lo, int64_t nnz) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double x = v[src[e]];
        out[e] = x;
        if (hi) {
            const float h = __double2float_rn(x);
            hi[e] = h;
            lo[e] = __double2float_rn(x - (double)h);
        }
    }
}

// Xp[t] = (hi, lo), hi + lo = X[t] (double-float split of the refinement
// vectors, the two halves side by side so that one 8-byte load fetches both)
__global__ void split_df_kernel(const double *__restrict__ X, float2 *__restrict__ Xp, int64_t cnt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double x = X[t];
        const float h = __double2float_rn(x);
        Xp[t] = make_float2(h, __double2float_rn(x - (double)h));
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

// Y += alpha G X on the full CSR of P A P^T with other values (G's, on the
// same structure; FP64; X and Y row-major n x nrhs, factor order): one warp
// per row, lanes over the row's entries, the lanes' sums added by a fixed
// shuffle tree, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) spmv_axpy_kernel(DevSym d, const double *__restrict__ vals,
                                                        const double *__restrict__ X, double alpha,
                                                        double *__restrict__ Y, int nrhs) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= d.n) return;
    const int64_t e0 = d.csr_ptr[row], e1 = d.csr_ptr[row + 1];
    for (int c0 = 0; c0 < nrhs; c0 += 8) {
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const double v = vals[e];
            const int64_t xo = (int64_t)d.csr_col[e] * nrhs;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c0 + c < nrhs) acc[c] += v * X[xo + c0 + c];
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            double t = acc[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0 && c0 + c < nrhs) Y[row * nrhs + c0 + c] += alpha * t;
        }
    }
}

// One step of the theta-scheme (Eq. (theta) with G = I), staged in factor
// order, row-major: Bp[i*nrhs + c] = a U[o] + g F[o] (F nullable) and
// X[i*nrhs + c] = x U[o], o = perm[i] + c*ld; the residual kernel then forms
// Bp - M X, the step's right-hand side.
__global__ void theta_stage_kernel(const double *__restrict__ U, const double *__restrict__ F, int64_t ld,
                                   const int32_t *__restrict__ perm, int64_t n, int64_t nrhs, double a,
                                   double x, double g, double *__restrict__ Bp, double *__restrict__ X) {
    const int64_t tot = n * nrhs;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / nrhs, c = t % nrhs;
        const int64_t o = perm[i] + c * ld;
        const double u = U[o];
        Bp[t] = F ? a * u + g * F[o] : a * u;
        X[t] = x * u;
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

// Double-float accumulator (hi, lo), about 48 significant bits.  Products of
// double-float operands are formed exactly up to the lo*lo term with FMA
// (Dekker / Ogita-Rump-Oishi TwoProd); a product is added to hi with Knuth's
// TwoSum and the two error terms are collected in lo without renormalising
// (the compensated dot product of Ogita, Rump and Oishi); df_renorm folds lo
// back every few terms so that it stays at the rounding level of hi.  All
// operations are explicitly rounded intrinsics, so nothing is contracted.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ void df_add_prod(DF &s, float ah, float al, float xh, float xl) {
    const float ph = __fmul_rn(ah, xh);
    float pl = __fmaf_rn(ah, xh, -ph);          // exact error of ah * xh
    pl = __fmaf_rn(ah, xl, pl);
    pl = __fmaf_rn(al, xh, pl);
    const float t = __fadd_rn(s.hi, ph);         // TwoSum(s.hi, ph)
    const float z = __fsub_rn(t, s.hi);
    const float e = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(ph, z));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(pl, e));
}
// (hi, lo) := TwoSum(hi, lo)
__device__ __forceinline__ void df_renorm(DF &s) {
    const float t = __fadd_rn(s.hi, s.lo);
    const float z = __fsub_rn(t, s.hi);
    s.lo = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(s.lo, z));
    s.hi = t;
}
// s += u (both double-float)
__device__ __forceinline__ void df_add(DF &s, DF u) {
    const float t = __fadd_rn(s.hi, u.hi);
    const float z = __fsub_rn(t, s.hi);
    float e = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(u.hi, z));
    e = __fadd_rn(e, __fadd_rn(s.lo, u.lo));
    s.hi = __fadd_rn(t, e);
    s.lo = __fsub_rn(e, __fsub_rn(s.hi, t));
}

// The many-right-hand-side residual in double-float arithmetic on the FP32
// pipes (about 48 bits: the residual of a refined solution is then exact to
// ~1e-14 of ||A|| ||x||, far below the 1e-12 backward-error target), same
// chunking as spmv_wide_kernel; partial and final sums in FP64.
__global__ void __launch_bounds__(THREADS, 4) spmv_df_kernel(DevSym d, const int4 *__restrict__ items,
                                                          int count, const float *__restrict__ vh,
                                                          const float *__restrict__ vl,
                                                          const float2 *__restrict__ Xp,
                                                          const double *__restrict__ Bp,
                                                          double *__restrict__ R, double *__restrict__ P,
                                                          int nrhs) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= count) return;
    const int4 it = items[w];
    const int64_t row = it.x;
    const int e0 = it.y, e1 = it.z, slot = it.w;
    for (int c0 = 0; c0 < nrhs; c0 += 64) {
        const int ca = c0 + lane, cb = c0 + 32 + lane;
        const bool va = ca < nrhs, vb = cb < nrhs;
        // entries are fetched 32 at a time (lane i loads entry eb + i) and
        // broadcast by shuffles; NS interleaved accumulation streams keep NS
        // independent chains and NS entries' x loads in flight
        constexpr int NS = 4;
        DF a[NS], b[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) a[q] = b[q] = DF{0.f, 0.f};
        for (int eb = e0; eb < e1; eb += 32) {
            const int my = eb + lane, cnt = min(32, e1 - eb);
            const int col = my < e1 ? d.csr_col[my] : 0;
            const float mh = my < e1 ? vh[my] : 0.f, ml = my < e1 ? vl[my] : 0.f;
            for (int j = 0; j < cnt; j += NS) {
                float xh[NS][2], xl[NS][2], ah[NS], al[NS];
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const int src = (j + q) & 31;
                    const int64_t xo = (int64_t)__shfl_sync(0xffffffffu, col, src) * nrhs;
                    ah[q] = __shfl_sync(0xffffffffu, mh, src);
                    al[q] = __shfl_sync(0xffffffffu, ml, src);
                    const bool ok = j + q < cnt;
                    const float2 pa = (ok && va) ? Xp[xo + ca] : make_float2(0.f, 0.f);
                    const float2 pb = (ok && vb) ? Xp[xo + cb] : make_float2(0.f, 0.f);
                    xh[q][0] = pa.x;
                    xl[q][0] = pa.y;
                    xh[q][1] = pb.x;
                    xl[q][1] = pb.y;
                }
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    if (j + q < cnt) {
                        df_add_prod(a[q], ah[q], al[q], xh[q][0], xl[q][0]);
                        df_add_prod(b[q], ah[q], al[q], xh[q][1], xl[q][1]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                df_renorm(a[q]);
                df_renorm(b[q]);
            }
        }
        df_add(a[0], a[1]);
        df_add(a[2], a[3]);
        df_add(a[0], a[2]);
        df_add(b[0], b[1]);
        df_add(b[2], b[3]);
        df_add(b[0], b[2]);
        const double sa = (double)a[0].hi + (double)a[0].lo, sb = (double)b[0].hi + (double)b[0].lo;
        if (slot < 0) {
            if (va) R[row * nrhs + ca] = Bp[row * nrhs + ca] - sa;
            if (vb) R[row * nrhs + cb] = Bp[row * nrhs + cb] - sb;
        } else {
            if (va) P[(int64_t)slot * nrhs + ca] = sa;
            if (vb) P[(int64_t)slot * nrhs + cb] = sb;
        }
    }
}

// s += (ah + al) x for x exactly an FP32 value: the product ah x is split
// exactly (TwoProd), al x is the small correction
__device__ __forceinline__ void df_add_prod1(DF &s, float ah, float al, float x) {
    const float ph = __fmul_rn(ah, x);
    float pl = __fmaf_rn(ah, x, -ph);
    pl = __fmaf_rn(al, x, pl);
    const float t = __fadd_rn(s.hi, ph);
    const float z = __fsub_rn(t, s.hi);
    const float e = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(t, z)), __fsub_rn(ph, z));
    s.hi = t;
    s.lo = __fadd_rn(s.lo, __fadd_rn(pl, e));
}

// R = S - A x for x held exactly in FP32 (row-major Xf), in double-float
// arithmetic as spmv_df_kernel: the first residual of a mixed-precision solve
// (x = the FP32 solution, S = b) and every later one by the recurrence
// r_{k+1} = r_k - A d_k (x = the FP32 correction d_k, S = R in place, so the
// refined x itself is never re-read).  Half the bytes of x per entry.  S and
// R may be the same array: each element is read and then written by one
// thread (chunked rows only write P here).
__global__ void __launch_bounds__(THREADS, 4) spmv_df32_kernel(DevSym d, const int4 *__restrict__ items,
                                                            int count, const float *__restrict__ vh,
                                                            const float *__restrict__ vl,
                                                            const float *__restrict__ Xf, const double *S,
                                                            double *R, double *__restrict__ P, int nrhs) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= count) return;
    const int4 it = items[w];
    const int64_t row = it.x;
    const int e0 = it.y, e1 = it.z, slot = it.w;
    for (int c0 = 0; c0 < nrhs; c0 += 64) {
        const int ca = c0 + lane, cb = c0 + 32 + lane;
        const bool va = ca < nrhs, vb = cb < nrhs;
        constexpr int NS = 4;
        DF a[NS], b[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q) a[q] = b[q] = DF{0.f, 0.f};
        for (int eb = e0; eb < e1; eb += 32) {
            const int my = eb + lane, cnt = min(32, e1 - eb);
            const int col = my < e1 ? d.csr_col[my] : 0;
            const float mh = my < e1 ? vh[my] : 0.f, ml = my < e1 ? vl[my] : 0.f;
            for (int j = 0; j < cnt; j += NS) {
                float xa[NS], xb[NS], ah[NS], al[NS];
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    const int src = (j + q) & 31;
                    const int64_t xo = (int64_t)__shfl_sync(0xffffffffu, col, src) * nrhs;
                    ah[q] = __shfl_sync(0xffffffffu, mh, src);
                    al[q] = __shfl_sync(0xffffffffu, ml, src);
                    const bool ok = j + q < cnt;
                    xa[q] = (ok && va) ? Xf[xo + ca] : 0.f;
                    xb[q] = (ok && vb) ? Xf[xo + cb] : 0.f;
                }
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    if (j + q < cnt) {
                        df_add_prod1(a[q], ah[q], al[q], xa[q]);
                        df_add_prod1(b[q], ah[q], al[q], xb[q]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                df_renorm(a[q]);
                df_renorm(b[q]);
            }
        }
        df_add(a[0], a[1]);
        df_add(a[2], a[3]);
        df_add(a[0], a[2]);
        df_add(b[0], b[1]);
        df_add(b[2], b[3]);
        df_add(b[0], b[2]);
        const double sa = (double)a[0].hi + (double)a[0].lo, sb = (double)b[0].hi + (double)b[0].lo;
        if (slot < 0) {
            if (va) R[row * nrhs + ca] = S[row * nrhs + ca] - sa;
            if (vb) R[row * nrhs + cb] = S[row * nrhs + cb] - sb;
        } else {
            if (va) P[(int64_t)slot * nrhs + ca] = sa;
            if (vb) P[(int64_t)slot * nrhs + cb] = sb;
        }
    }
}

// The same product for a multiple of 4 right-hand sides: a half-warp covers 64
// right-hand sides with one 16-byte load of x per lane, the two halves of the
// warp take alternate entries of the row chunk (their sums are added at the
// end), and the x row and the value of the next entry are fetched before the
// current one is accumulated.  Fewer instructions per (entry, right-hand
// side) term than the lane-per-right-hand-side form: one shuffle triple per
// four terms and one load per four.
__device__ __forceinline__ void spmv_x4_fetch(const int32_t col, const float mh, const float ml, int src,
                                              const float *__restrict__ Xf, int nrhs, int c, bool vc, float4 &x,
                                              float &ah, float &al) {
    const int cc = __shfl_sync(0xffffffffu, col, src);
    ah = __shfl_sync(0xffffffffu, mh, src);
    al = __shfl_sync(0xffffffffu, ml, src);
    x = vc ? *reinterpret_cast<const float4 *>(Xf + (int64_t)cc * nrhs + c) : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void spmv_x4_acc(DF (&a)[4], float ah, float al, float4 x) {
    df_add_prod1(a[0], ah, al, x.x);
    df_add_prod1(a[1], ah, al, x.y);
    df_add_prod1(a[2], ah, al, x.z);
    df_add_prod1(a[3], ah, al, x.w);
}

__global__ void __launch_bounds__(THREADS, 4) spmv_df32x4_kernel(DevSym d, const int4 *__restrict__ items,
                                                              int count, const float *__restrict__ vh,
                                                              const float *__restrict__ vl,
                                                              const float *__restrict__ Xf, const double *S,
                                                              double *R, double *__restrict__ P, int nrhs) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    if (w >= count) return;
    const int4 it = items[w];
    const int64_t row = it.x;
    const int e0 = it.y, e1 = it.z, slot = it.w;
    for (int c0 = 0; c0 < nrhs; c0 += 64) {
        const int c = c0 + 4 * hl;
        const bool vc = c < nrhs;
        DF a0[4], a1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) a0[q] = a1[q] = DF{0.f, 0.f};
        for (int eb = e0; eb < e1; eb += 32) {
            // entry eb + lane's column and value; lanes past the chunk hold
            // column 0 and value 0 (their products are exact zeros)
            const int my = eb + lane, cnt = min(32, e1 - eb);
            const int32_t col = my < e1 ? d.csr_col[my] : 0;
            const float mh = my < e1 ? vh[my] : 0.f, ml = my < e1 ? vl[my] : 0.f;
            const int npair = (cnt + 1) >> 1;   // entry 2 jj + half of the group
            float4 x;
            float ah, al;
            spmv_x4_fetch(col, mh, ml, half, Xf, nrhs, c, vc, x, ah, al);
            for (int jj = 0; jj < npair; jj += 2) {
                float4 xn;
                float ahn, aln;
                if (jj + 1 < npair) spmv_x4_fetch(col, mh, ml, 2 * (jj + 1) + half, Xf, nrhs, c, vc, xn, ahn, aln);
                spmv_x4_acc(a0, ah, al, x);
                if (jj + 1 < npair) {
                    if (jj + 2 < npair) spmv_x4_fetch(col, mh, ml, 2 * (jj + 2) + half, Xf, nrhs, c, vc, x, ah, al);
                    spmv_x4_acc(a1, ahn, aln, xn);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                df_renorm(a0[q]);
                df_renorm(a1[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            df_add(a0[q], a1[q]);
            const DF o{__shfl_xor_sync(0xffffffffu, a0[q].hi, 16), __shfl_xor_sync(0xffffffffu, a0[q].lo, 16)};
            df_add(a0[q], o);
        }
        if (half == 0 && vc) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double sq = (double)a0[q].hi + (double)a0[q].lo;
                if (slot < 0) R[row * nrhs + c + q] = S[row * nrhs + c + q] - sq;
                else P[(int64_t)slot * nrhs + c + q] = sq;
            }
        }
    }
}

// R = S - sum of a cut row's partial sums, in slot order (S may be R)
__global__ void spmv_finish_src_kernel(const int4 *__restrict__ items, int count, const double *S, double *R,
                                       const double *__restrict__ P, int nrhs) {
    const int i = blockIdx.x;
    if (i >= count) return;
    const int4 it = items[i];
    const int64_t row = it.x;
    for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
        double acc = 0.0;
        for (int q = 0; q < it.z; ++q) acc += P[(int64_t)(it.y + q) * nrhs + c];
        R[row * nrhs + c] = S[row * nrhs + c] - acc;
    }
}

// The FP32 solution (or correction) Y, column-major n x nrhs, into the
// row-major FP64 refinement vector X (=, or += if accumulate) and its FP32
// row-major copy Xf (the x of spmv_df32_kernel)
__global__ void xupdate_kernel(const float *__restrict__ Y, double *__restrict__ X, float *__restrict__ Xf,
                               int64_t n, int64_t nrhs, int accumulate) {
    __shared__ float tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int j = ty; j < 32; j += 8) {
        const int64_t i = i0 + tx, c = c0 + j;
        tile[j][tx] = (i < n && c < nrhs) ? Y[i + c * n] : 0.f;
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int64_t i = i0 + j, c = c0 + tx;
        if (i < n && c < nrhs) {
            const float v = tile[tx][j];
            const int64_t o = i * nrhs + c;
            X[o] = accumulate ? X[o] + (double)v : (double)v;
            Xf[o] = v;
        }
    }
}

// Few right-hand sides (<= 8): lanes over the entries of the chunk, NR (the
// number of right-hand sides rounded up to 1, 2, 4 or 8) accumulators per
// lane and U = 4 entries per lane in flight (their values, columns and x loads
// are all issued before the first product), which hides the dependent
// column -> x latency that one entry at a time leaves exposed.  Each lane adds
// its entries in the same order as one entry per step would.  Every address
// formed is in range: lanes past the end of the chunk re-read the lane's
// first entry with weight 0, accumulators past nrhs read right-hand side 0
// (never written out), and a column index outside [0, n) is skipped and its
// CSR position recorded in *bad (atomic minimum; the host clears and reads it).
template <int NR>
__global__ void __launch_bounds__(THREADS) spmv_narrow_kernel(DevSym d, const int4 *__restrict__ items,
                                                              int count, const double *__restrict__ X,
                                                              const double *__restrict__ Bp,
                                                              double *__restrict__ R,
                                                              double *__restrict__ P, int nrhs,
                                                              unsigned long long *__restrict__ bad) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= count) return;
    const int4 it = items[w];
    const int64_t row = it.x;
    const int slot = it.w;
    constexpr int U = 4;
    double acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = 0.0;
    for (int e0 = it.y + lane; e0 < it.z; e0 += 32 * U) {
        double v[U];
        int64_t xo[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int e = e0 + 32 * u;
            const bool in = e < it.z;
            const int ec = in ? e : e0;
            double val = __ldcs(d.csr_val + ec);
            const int col = __ldcs(d.csr_col + ec);
            const bool col_ok = (int64_t)(uint32_t)col < d.n;
            if (!col_ok && in) atomicMin(bad, (unsigned long long)e);
            if (!in || !col_ok) val = 0.0;
            v[u] = val;
            xo[u] = col_ok ? (int64_t)col * nrhs : 0;
        }
        double x[U][NR];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < NR; ++c) x[u][c] = X[xo[u] + (c < nrhs ? c : 0)];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < NR; ++c) acc[c] += v[u] * x[u][c];
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) {
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

}  // namespace

void init_solve_attributes() {}

void launch_gather_values(const int32_t *src, const double *values, double *out, float *hi, float *lo,
                          int64_t nnz, cudaStream_t st) {
    if (nnz <= 0) return;
    gather_values_kernel<<<grid_for(nnz), THREADS, 0, st>>>(src, values, out, hi, lo, nnz);
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
void launch_apply_L(const DevSym &d, const T *front, const T *Z, T *Out, T *W,
                    const int4 *items, int count, int nrhs, cudaStream_t st) {
    if (count <= 0) return;
    apply_L_kernel<T><<<count, THREADS, 0, st>>>(d, front, Z, Out, W, items, nrhs);
}

void launch_spmv_axpy(const DevSym &d, const double *vals, const double *X, double alpha, double *Y,
                      int64_t nrhs, cudaStream_t st) {
    const int64_t warps = d.n;
    spmv_axpy_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(d, vals, X, alpha, Y, (int)nrhs);
}

void launch_permute_in_rm(const double *B, int64_t ldb, double *Bp, const int32_t *perm, int64_t n,
                          int64_t nrhs, cudaStream_t st) {
    permute_in_rm_kernel<<<grid_for(n * nrhs), THREADS, 0, st>>>(B, ldb, Bp, perm, n, nrhs);
}

void launch_theta_stage(const double *U, const double *F, int64_t ld, const int32_t *perm, int64_t n,
                        int64_t nrhs, double a, double x, double g, double *Bp, double *X, cudaStream_t st) {
    theta_stage_kernel<<<grid_for(n * nrhs), THREADS, 0, st>>>(U, F, ld, perm, n, nrhs, a, x, g, Bp, X);
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
                          int64_t nrhs, unsigned long long *bad, cudaStream_t st) {
    const int blocks = (int)(((int64_t)nchunks * 32 + THREADS - 1) / THREADS);
    const int nr = (int)nrhs;
    if (nrhs == 1)
        spmv_narrow_kernel<1><<<blocks, THREADS, 0, st>>>(d, chunks, nchunks, X, Bp, R, P, nr, bad);
    else if (nrhs == 2)
        spmv_narrow_kernel<2><<<blocks, THREADS, 0, st>>>(d, chunks, nchunks, X, Bp, R, P, nr, bad);
    else if (nrhs <= 4)
        spmv_narrow_kernel<4><<<blocks, THREADS, 0, st>>>(d, chunks, nchunks, X, Bp, R, P, nr, bad);
    else if (nrhs <= 8)
        spmv_narrow_kernel<8><<<blocks, THREADS, 0, st>>>(d, chunks, nchunks, X, Bp, R, P, nr, bad);
    else
        spmv_wide_kernel<<<blocks, THREADS, 0, st>>>(d, chunks, nchunks, X, Bp, R, P, (int)nrhs);
    if (nfin > 0) spmv_finish_kernel<<<nfin, 64, 0, st>>>(fin, nfin, Bp, R, P, (int)nrhs);
}

void launch_spmv_residual_df(const DevSym &d, const int4 *chunks, int nchunks, const int4 *fin, int nfin,
                             const float *vh, const float *vl, const double *X, float2 *Xp,
                             const double *Bp, double *R, double *P, int64_t nrhs, cudaStream_t st) {
    const int64_t cnt = d.n * nrhs;
    split_df_kernel<<<grid_for(cnt), THREADS, 0, st>>>(X, Xp, cnt);
    const int blocks = (int)(((int64_t)nchunks * 32 + THREADS - 1) / THREADS);
    spmv_df_kernel<<<blocks, THREADS, 0, st>>>(d, chunks, nchunks, vh, vl, Xp, Bp, R, P, (int)nrhs);
    if (nfin > 0) spmv_finish_kernel<<<nfin, 64, 0, st>>>(fin, nfin, Bp, R, P, (int)nrhs);
}

void launch_spmv_residual_df32(const DevSym &d, const int4 *chunks, int nchunks, const int4 *fin, int nfin,
                               const float *vh, const float *vl, const float *Xf, const double *S, double *R,
                               double *P, int64_t nrhs, cudaStream_t st) {
    const int blocks = (int)(((int64_t)nchunks * 32 + THREADS - 1) / THREADS);
    if (nrhs % 4 == 0)
        spmv_df32x4_kernel<<<blocks, THREADS, 0, st>>>(d, chunks, nchunks, vh, vl, Xf, S, R, P, (int)nrhs);
    else
        spmv_df32_kernel<<<blocks, THREADS, 0, st>>>(d, chunks, nchunks, vh, vl, Xf, S, R, P, (int)nrhs);
    if (nfin > 0) spmv_finish_src_kernel<<<nfin, 64, 0, st>>>(fin, nfin, S, R, P, (int)nrhs);
}

void launch_xupdate(const float *Y, double *X, float *Xf, int64_t n, int64_t nrhs, int accumulate,
                    cudaStream_t st) {
    const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((nrhs + 31) / 32));
    xupdate_kernel<<<grid, dim3(32, 8), 0, st>>>(Y, X, Xf, n, nrhs, accumulate);
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
