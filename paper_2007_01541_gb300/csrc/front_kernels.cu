// Multifrontal numeric factorization kernels (FP64 and FP32 fronts).
//
// Each supernode s owns a dense front F_s of order m_s (column-major, lower
// triangle used).  Its first k_s columns become the supernode's columns of L;
// its trailing block becomes the update matrix U_s = F22 - L21 L21^T that the
// parent gathers (extend-add).  This is the block form of P A P^T under
// nested dissection (Section 4): fronts of disjoint subtrees are independent,
// so every level of the supernodal tree is processed by one launch per phase.
//
// Phases for the fronts of one level:
//   front_init   assemble A's entries and gather the children's update
//                matrices through relative row maps (no atomics: every front
//                entry is written by exactly one thread)
//   potrf_first  Cholesky of the first NB x NB diagonal block
//   per pivot block kb = 0, NB, 2NB, ... < k_s:
//     panel      L21 := F21 L11^-T for the rows below the diagonal block
//     update     trailing lower tiles -= L21 L21^T; the tile holding the next
//                diagonal block also factors it (so no extra launch)
#include "engine.h"

#include <cstdio>

namespace wd {
namespace {

constexpr int THREADS = 256;
constexpr int KC = 32;  // k-chunk of the Schur tile update

template <class T>
__device__ __forceinline__ T dev_sqrt(T x);
template <>
__device__ __forceinline__ double dev_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dev_sqrt<float>(float x) { return sqrtf(x); }

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
    const int m = d.sm[s], k = d.sk[s];
    T *F = front + d.foff[s] + (int64_t)q * m;
    const int cb = d.child_ptr[s], ce = d.child_ptr[s + 1];
    for (int r0 = q; r0 < m; r0 += 128) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int ci = cb; ci < ce; ++ci) {
            const int c = d.children[ci];
            const int32_t *map = d.relmap + d.mapoff[c];
            const int ic = map[q];
            if (ic < 0) continue;
            const int mc = d.sm[c], kc = d.sk[c];
            const T *U = front + d.foff[c] + (int64_t)(kc + ic) * mc + kc;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int r = r0 + u * 32 + lane;
                if (r < m) {
                    const int ir = map[r];
                    if (ir >= 0) acc[u] += U[ir];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = r0 + u * 32 + lane;
            if (r < m) F[r] = acc[u];
        }
    }
    __syncwarp();
    if (q < k) {
        const int64_t j = d.sfirst[s] + q;
        const int64_t e0 = d.csr_diag[j], e1 = d.csr_ptr[j + 1], l0 = d.pcp[j];
        for (int64_t e = e0 + lane; e < e1; e += 32) F[d.alrow[l0 + (e - e0)]] += (T)d.csr_val[e];
    }
}

// ---------------------------------------------------------------------------
// Cholesky of an nb x nb diagonal block (nb <= NB) in shared memory.  A pivot
// that is not positive records its global column in *status (smallest wins)
// and is replaced by 1 so that the arithmetic stays finite.
// Must be called by all THREADS threads of the block.
// ---------------------------------------------------------------------------
template <class T>
__device__ void block_potrf(T *F, int ld, int nb, int64_t gcol0, status_t *status, T *smem) {
    T(*A)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem);
    const int tid = threadIdx.x;
    for (int idx = tid; idx < nb * nb; idx += THREADS) {
        const int r = idx % nb, c = idx / nb;
        if (r >= c) A[r][c] = F[(int64_t)c * ld + r];
    }
    __syncthreads();
    const int r = tid % NB, cg = tid / NB;
    for (int j = 0; j < nb; ++j) {
        if (tid == 0) {
            T dj = A[j][j];
            if (!(dj > T(0))) {
                atomicMin(status, (status_t)(gcol0 + j));
                dj = T(1);
            }
            A[j][j] = dev_sqrt(dj);
        }
        __syncthreads();
        if (cg == 0 && r > j && r < nb) A[r][j] = A[r][j] / A[j][j];
        __syncthreads();
        if (r > j && r < nb) {
            const T arj = A[r][j];
            for (int c = j + 1 + cg; c <= r; c += THREADS / NB) A[r][c] -= arj * A[c][j];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < nb * nb; idx += THREADS) {
        const int rr = idx % nb, c = idx / nb;
        if (rr >= c) F[(int64_t)c * ld + rr] = A[rr][c];
    }
    __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(THREADS) potrf_first_kernel(DevSym d, T *__restrict__ front,
                                                              const int4 *__restrict__ items,
                                                              status_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int s = items[blockIdx.x].x;
    const int m = d.sm[s], k = d.sk[s];
    block_potrf<T>(front + d.foff[s], m, min(NB, k), d.sfirst[s], status,
                   reinterpret_cast<T *>(smem_raw));
}

// ---------------------------------------------------------------------------
// panel: rows [r0, r1) of columns [kb, kb+nb):  X := X L11^-T
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(THREADS) panel_kernel(DevSym d, T *__restrict__ front,
                                                        const int4 *__restrict__ items, int kb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*D)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);
    T(*X)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw + sizeof(T) * NB * (NB + 1));
    const int4 it = items[blockIdx.x];
    const int s = it.x, rb = it.y;
    const int m = d.sm[s], k = d.sk[s];
    const int nb = min(NB, k - kb);
    const int r0 = kb + nb + rb * RB;
    const int nr = min(RB, m - r0);
    const T *Fc = front + d.foff[s];
    T *F = front + d.foff[s];
    const int tid = threadIdx.x;
    for (int idx = tid; idx < nb * nb; idx += THREADS) {
        const int r = idx % nb, c = idx / nb;
        if (r >= c) D[r][c] = Fc[(int64_t)(kb + c) * m + kb + r];
    }
    for (int idx = tid; idx < RB * nb; idx += THREADS) {
        const int r = idx % RB, c = idx / RB;
        if (r < nr) X[r][c] = Fc[(int64_t)(kb + c) * m + r0 + r];
    }
    __syncthreads();
    const int r = tid % RB, cg = tid / RB;
    for (int j = 0; j < nb; ++j) {
        if (cg == 0 && r < nr) X[r][j] = X[r][j] / D[j][j];
        __syncthreads();
        if (r < nr) {
            const T xrj = X[r][j];
            for (int c = j + 1 + cg; c < nb; c += THREADS / RB) X[r][c] -= xrj * D[c][j];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < RB * nb; idx += THREADS) {
        const int rr = idx % RB, c = idx / RB;
        if (rr < nr) F[(int64_t)(kb + c) * m + r0 + rr] = X[rr][c];
    }
}

// ---------------------------------------------------------------------------
// Schur update of one NB x NB lower tile of the trailing matrix:
//   C(rows I, cols J) -= L(I, kb:kb+nb) L(J, kb:kb+nb)^T
// thread (tx, ty) owns rows tx + 16 i and columns ty + 16 j (i, j < 4).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(THREADS) update_kernel(DevSym d, T *__restrict__ front,
                                                         const int4 *__restrict__ items, int kb,
                                                         status_t *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*As)[NB] = reinterpret_cast<T(*)[NB]>(smem_raw);
    T(*Bs)[NB] = reinterpret_cast<T(*)[NB]>(smem_raw + sizeof(T) * KC * NB);
    const int4 it = items[blockIdx.x];
    const int s = it.x, ti = it.y, tj = it.z;
    const int m = d.sm[s], k = d.sk[s];
    const int nb = min(NB, k - kb);
    const int t0 = kb + nb;
    const int rbase = t0 + ti * NB, cbase = t0 + tj * NB;
    T *F = front + d.foff[s];
    const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < nb; k0 += KC) {
        const int kc = min(KC, nb - k0);
        for (int idx = tid; idx < KC * NB; idx += THREADS) {
            const int kk = idx / NB, rr = idx % NB;
            const int64_t col = (int64_t)(kb + k0 + kk) * m;
            As[kk][rr] = (kk < kc && rbase + rr < m) ? F[col + rbase + rr] : T(0);
            Bs[kk][rr] = (kk < kc && cbase + rr < m) ? F[col + cbase + rr] : T(0);
        }
        __syncthreads();
        for (int kk = 0; kk < kc; ++kk) {
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
    for (int j = 0; j < 4; ++j) {
        const int c = cbase + ty + 16 * j;
        if (c >= m) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = rbase + tx + 16 * i;
            if (r < m && r >= c) F[(int64_t)c * m + r] -= acc[i][j];
        }
    }
    if (ti == 0 && tj == 0 && t0 < k) {
        __syncthreads();
        block_potrf<T>(F + (int64_t)t0 * m + t0, m, min(NB, k - t0), d.sfirst[s] + t0, status,
                       reinterpret_cast<T *>(smem_raw));
    }
}

template <class T>
constexpr size_t potrf_smem() { return sizeof(T) * NB * (NB + 1); }
template <class T>
constexpr size_t panel_smem() { return sizeof(T) * (NB + RB) * (NB + 1); }
template <class T>
constexpr size_t update_smem() {
    return (2 * sizeof(T) * KC * NB > potrf_smem<T>()) ? 2 * sizeof(T) * KC * NB : potrf_smem<T>();
}

template <class T>
void set_smem_attrs() {
    static bool done = false;  // per instantiation and process
    if (done) return;
    cudaFuncSetAttribute(panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)panel_smem<T>());
    done = true;
}

}  // namespace

template <class T>
void launch_front_init(const DevSym &d, T *front, const int4 *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    const int warps = THREADS / 32;
    front_init_kernel<T><<<(count + warps - 1) / warps, THREADS, 0, st>>>(d, front, items, count);
}

template <class T>
void launch_potrf_first(const DevSym &d, T *front, const int4 *items, int count,
                        status_t *status, cudaStream_t st) {
    if (count <= 0) return;
    potrf_first_kernel<T><<<count, THREADS, potrf_smem<T>(), st>>>(d, front, items, status);
}

template <class T>
void launch_panel(const DevSym &d, T *front, const int4 *items, int count, int kb,
                  cudaStream_t st) {
    if (count <= 0) return;
    set_smem_attrs<T>();
    panel_kernel<T><<<count, THREADS, panel_smem<T>(), st>>>(d, front, items, kb);
}

template <class T>
void launch_update(const DevSym &d, T *front, const int4 *items, int count, int kb,
                   status_t *status, cudaStream_t st) {
    if (count <= 0) return;
    update_kernel<T><<<count, THREADS, update_smem<T>(), st>>>(d, front, items, kb, status);
}

#define WD_INST(T)                                                                              \
    template void launch_front_init<T>(const DevSym &, T *, const int4 *, int, cudaStream_t);   \
    template void launch_potrf_first<T>(const DevSym &, T *, const int4 *, int, status_t *,     \
                                        cudaStream_t);                                          \
    template void launch_panel<T>(const DevSym &, T *, const int4 *, int, int, cudaStream_t);   \
    template void launch_update<T>(const DevSym &, T *, const int4 *, int, int, status_t *,     \
                                   cudaStream_t);
WD_INST(double)
WD_INST(float)
#undef WD_INST

}  // namespace wd
