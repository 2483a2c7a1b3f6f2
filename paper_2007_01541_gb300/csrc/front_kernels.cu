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

template <class T>
__device__ __forceinline__ T dev_sqrt(T x);
template <>
__device__ __forceinline__ double dev_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dev_sqrt<float>(float x) { return sqrtf(x); }

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
// assemble + extend-add, one warp per front column
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(THREADS) front_init_kernel(DevSym d, T *__restrict__ front,
                                                             const int4 *__restrict__ items,
                                                             int count) {
    const int w = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= count) return;
    const int4 it = items[w];
    const int s = it.x, q = it.y;
    const Dims z = dims(d, s);
    const int pad = z.kp - z.k;
    const int qc = q < z.k ? q : (q < z.kp ? -1 : q - pad);  // local column
    T *F = front + d.foff[s] + (int64_t)q * z.ld;
    const int cb = d.child_ptr[s], ce = d.child_ptr[s + 1];
    for (int r0 = q; r0 < z.mp; r0 += 128) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        if (qc >= 0) {
            for (int ci = cb; ci < ce; ++ci) {
                const int c = d.children[ci];
                const int32_t *map = d.relmap + d.mapoff[c];
                const int ic = map[qc];
                if (ic < 0) continue;
                const int kpc = d.skp[c], ldc = d.sld[c];
                const T *U = front + d.foff[c] + (int64_t)(kpc + ic) * ldc + kpc;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int fr = r0 + u * 32 + lane;
                    const int r = fr < z.k ? fr : (fr < z.kp ? -1 : fr - pad);
                    if (fr < z.mp && r >= 0) {
                        const int ir = map[r];
                        if (ir >= 0) acc[u] += U[ir];
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int fr = r0 + u * 32 + lane;
            if (fr < z.mp) F[fr] = acc[u];
        }
    }
    __syncwarp();
    if (q < z.k) {
        const int64_t j = d.sfirst[s] + q;
        const int64_t e0 = d.csr_diag[j], e1 = d.csr_ptr[j + 1], l0 = d.pcp[j];
        for (int64_t e = e0 + lane; e < e1; e += 32) F[d.alrow[l0 + (e - e0)]] += (T)d.csr_val[e];
    }
}

// ---------------------------------------------------------------------------
// Cholesky of an nb x nb diagonal block (nb <= NB = 64) and the inverse of the
// factor, written zero-padded as an NB x NB lower-triangular matrix
// (column-major) to Dinv.  2 x 2 blocks of 32: each 32 x 32 diagonal block is
// factored by one warp with one row per lane in registers (shuffles, no block
// barrier); the off-diagonal block is solved and the trailing block updated
// by both warps; the two diagonal inverses are computed one column per lane,
// and X21 = -X22 L21 X11.  A pivot that is not positive records its global
// column in *status (smallest wins) and is replaced by 1 so that the
// arithmetic stays finite.  Must be called by a block of exactly NB threads.
// ---------------------------------------------------------------------------
constexpr int HB = 32;

// factor A[o:o+w, o:o+w] in place (w <= 32); one warp, lane = row
template <class T>
__device__ __forceinline__ void chol32_warp(T (*A)[NB + 1], int o, int w, int64_t gcol0,
                                            status_t *status, T *invd) {
    const int lane = threadIdx.x & 31;
    T a[HB];
#pragma unroll
    for (int c = 0; c < HB; ++c) a[c] = (lane < w && c <= lane) ? A[o + lane][o + c] : T(0);
#pragma unroll
    for (int j = 0; j < HB; ++j) {
        if (j < w) {
            T dj = __shfl_sync(0xffffffffu, a[j], j);
            if (!(dj > T(0))) {
                if (lane == 0) atomicMin(status, (status_t)(gcol0 + o + j));
                dj = T(1);
            }
            const T sj = dev_sqrt(dj);
            if (lane == j) a[j] = sj;
            else if (lane > j) a[j] = a[j] / sj;
#pragma unroll
            for (int c = j + 1; c < HB; ++c) {
                const T lc = __shfl_sync(0xffffffffu, a[j], c);
                if (lane >= c) a[c] -= a[j] * lc;
            }
        }
    }
    if (lane < w) {
#pragma unroll
        for (int c = 0; c < HB; ++c)
            if (c <= lane) A[o + lane][o + c] = a[c];
        invd[o + lane] = T(1) / a[lane];
    }
}

// column `lane` of inv(A[o:o+w, o:o+w]) (lower) into X[o:o+w, o+lane]
template <class T>
__device__ __forceinline__ void inv32_warp(const T (*A)[NB + 1], T (*X)[NB + 1], int o, int w,
                                           const T *invd) {
    const int c = threadIdx.x & 31;
    T x[HB];
#pragma unroll
    for (int r = 0; r < HB; ++r) {
        T acc0 = (r == c) ? T(1) : T(0), acc1 = T(0);
#pragma unroll
        for (int p = 0; p + 1 < r; p += 2) {
            acc0 -= A[o + r][o + p] * x[p];
            acc1 -= A[o + r][o + p + 1] * x[p + 1];
        }
        if (r & 1) acc0 -= A[o + r][o + r - 1] * x[r - 1];
        x[r] = (r >= c && r < w && c < w) ? (acc0 + acc1) * invd[o + r] : T(0);
    }
#pragma unroll
    for (int r = 0; r < HB; ++r) X[o + r][o + c] = x[r];
}

template <class T>
__device__ void block_potrf_inv(T *F, int ld, int nb, int64_t gcol0, status_t *status, T *Dinv,
                                T *smem) {
    T(*A)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem);
    T(*X)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem + NB * (NB + 1));
    T *invd = smem + 2 * NB * (NB + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int w1 = min(HB, nb), w2 = nb - w1;
    for (int c = 0; c < nb; ++c)
        if (tid >= c && tid < nb) cp_async_elem(&A[tid][c], F + (int64_t)c * ld + tid, true);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    if (warp == 0) chol32_warp<T>(A, 0, w1, gcol0, status, invd);
    __syncthreads();
    if (w2 > 0) {
        // L21 = A21 L11^-T, one row per thread of warp 1
        if (warp == 1 && lane < w2) {
            const int r = HB + lane;
            T x[HB];
#pragma unroll
            for (int c = 0; c < HB; ++c) x[c] = A[r][c];
#pragma unroll
            for (int c = 0; c < HB; ++c) {
                T acc0 = x[c], acc1 = T(0);
#pragma unroll
                for (int p = 0; p + 1 < c; p += 2) {
                    acc0 -= x[p] * A[c][p];
                    acc1 -= x[p + 1] * A[c][p + 1];
                }
                if (c & 1) acc0 -= x[c - 1] * A[c][c - 1];
                x[c] = (acc0 + acc1) * invd[c];
            }
#pragma unroll
            for (int c = 0; c < HB; ++c) A[r][c] = x[c];
        }
        if (warp == 0) inv32_warp<T>(A, X, 0, w1, invd);
        __syncthreads();
        // A22 -= L21 L21^T (lower)
        for (int idx = tid; idx < HB * HB; idx += NB) {
            const int r = idx % HB, c = idx / HB;
            if (r >= c && r < w2) {
                T acc0 = T(0), acc1 = T(0);
#pragma unroll
                for (int p = 0; p < HB; p += 2) {
                    acc0 += A[HB + r][p] * A[HB + c][p];
                    acc1 += A[HB + r][p + 1] * A[HB + c][p + 1];
                }
                A[HB + r][HB + c] -= acc0 + acc1;
            }
        }
        __syncthreads();
        if (warp == 1) {
            chol32_warp<T>(A, HB, w2, gcol0, status, invd);
            __syncwarp();
            inv32_warp<T>(A, X, HB, w2, invd);
        }
        __syncthreads();
        // X21 = -X22 (L21 X11): first T = L21 X11 into X[HB + r][c]
        for (int idx = tid; idx < HB * HB; idx += NB) {
            const int r = idx % HB, c = idx / HB;
            T acc = T(0);
            if (r < w2 && c < w1)
                for (int p = c; p < HB; ++p) acc += A[HB + r][p] * X[p][c];
            X[HB + r][c] = acc;
        }
        __syncthreads();
        T out[HB * HB / NB];
#pragma unroll
        for (int q = 0; q < HB * HB / NB; ++q) {
            const int idx = tid + q * NB, r = idx % HB, c = idx / HB;
            T acc = T(0);
            for (int p = 0; p <= r; ++p) acc += X[HB + r][HB + p] * X[HB + p][c];
            out[q] = -acc;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < HB * HB / NB; ++q) {
            const int idx = tid + q * NB, r = idx % HB, c = idx / HB;
            X[HB + r][c] = (r < w2 && c < w1) ? out[q] : T(0);
        }
    } else {
        if (warp == 0) inv32_warp<T>(A, X, 0, w1, invd);
        for (int idx = tid; idx < NB * NB; idx += NB) {
            const int r = idx % NB, c = idx / NB;
            if (r >= HB || c >= HB) X[r][c] = T(0);
        }
    }
    __syncthreads();
    for (int c = 0; c < nb; ++c)
        if (tid >= c && tid < nb) F[(int64_t)c * ld + tid] = A[tid][c];
    for (int c = 0; c < NB; ++c) Dinv[(int64_t)c * NB + tid] = (tid >= c) ? X[tid][c] : T(0);
    __syncthreads();
}

// diagonal block starting at pivot column j0 = item.y of front item.x
template <class T>
__global__ void __launch_bounds__(NB, 1) potrf_kernel(DevSym d, T *__restrict__ front,
                                                   T *__restrict__ dinv,
                                                   const int4 *__restrict__ items,
                                                   status_t *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int4 it = items[blockIdx.x];
    const int s = it.x, j0 = it.y;
    const Dims z = dims(d, s);
    block_potrf_inv<T>(front + d.foff[s] + (int64_t)j0 * z.ld + j0, z.ld, min(NB, z.k - j0),
                       d.sfirst[s] + j0, status, dinv + d.dinvoff[s] + (int64_t)(j0 / NB) * NB * NB,
                       reinterpret_cast<T *>(smem_raw));
}

// ---------------------------------------------------------------------------
// panel: rows [r0, r0+RB) of columns [kb, kb+nb):  X := X Linv^T.  The rows
// start at kb+NB, or at kp when kb is the last block (rows [k, kp) are zero
// padding).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(THREADS) panel_kernel(DevSym d, T *__restrict__ front,
                                                        const T *__restrict__ dinv,
                                                        const int4 *__restrict__ items, int kb) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);         // [p][r], ld RB
    T *Ds = Xs + NB * RB;                            // [p][c] = Linv(c, p), ld NB
    const int4 it = items[blockIdx.x];
    const int s = it.x, rb = it.y;
    const Dims z = dims(d, s);
    const int nb = min(NB, z.k - kb);
    const int t0 = kb + nb;
    const int r0 = (t0 == z.k ? z.kp : t0) + rb * RB;
    T *F = front + d.foff[s];
    stage_tile<T, THREADS>(Xs, RB, F + (int64_t)kb * z.ld + r0, z.ld, RB, NB, z.mp - r0, nb);
    stage_tile<T, THREADS>(Ds, NB, dinv + d.dinvoff[s] + (int64_t)(kb / NB) * NB * NB, NB, NB, NB,
                           NB, NB);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    // out[r][c] = sum_{p <= c} X[r][p] Linv(c, p); thread: row tid % 64, 16 cols
    const int tid = threadIdx.x;
    const int r = tid % RB, cg = tid / RB;
    T acc[NB / 4];
#pragma unroll
    for (int u = 0; u < NB / 4; ++u) acc[u] = T(0);
    for (int p = 0; p < nb; ++p) {
        const T x = Xs[p * RB + r];
#pragma unroll
        for (int u = 0; u < NB / 4; ++u) acc[u] += x * Ds[p * NB + cg + 4 * u];
    }
    if (r0 + r < z.mp) {
#pragma unroll
        for (int u = 0; u < NB / 4; ++u) {
            const int c = cg + 4 * u;
            if (c < nb) F[(int64_t)(kb + c) * z.ld + r0 + r] = acc[u];
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
constexpr size_t potrf_smem() { return sizeof(T) * (2 * NB * (NB + 1) + NB); }
template <class T>
constexpr size_t panel_smem() { return sizeof(T) * (NB * RB + NB * NB); }
template <class T>
constexpr size_t schur_smem() { return 2 * sizeof(T) * BK * (BM + BN); }

template <class T>
void set_smem_attrs() {
    static bool done = false;  // per instantiation and process
    if (done) return;
    cudaFuncSetAttribute(potrf_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)potrf_smem<T>());
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
void launch_potrf(const DevSym &d, T *front, T *dinv, const int4 *items, int count,
                  status_t *status, cudaStream_t st) {
    if (count <= 0) return;
    set_smem_attrs<T>();
    potrf_kernel<T><<<count, NB, potrf_smem<T>(), st>>>(d, front, dinv, items, status);
}

template <class T>
void launch_panel(const DevSym &d, T *front, const T *dinv, const int4 *items, int count, int kb,
                  cudaStream_t st) {
    if (count <= 0) return;
    set_smem_attrs<T>();
    panel_kernel<T><<<count, THREADS, panel_smem<T>(), st>>>(d, front, dinv, items, kb);
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
    template void launch_potrf<T>(const DevSym &, T *, T *, const int4 *, int, status_t *,       \
                                  cudaStream_t);                                                 \
    template void launch_panel<T>(const DevSym &, T *, const T *, const int4 *, int, int,        \
                                  cudaStream_t);                                                 \
    template void launch_schur<T>(const DevSym &, T *, T *, const int4 *, int, int, int,         \
                                  status_t *, cudaStream_t);
WD_INST(double)
WD_INST(float)
#undef WD_INST

}  // namespace wd
