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
//   diag_factor  pivot block 0 of every front: L11 = chol(F11) and L11^-1
//   per pivot block kb = 0, NB, 2NB, ... < k_s:
//     panel      L21 := F21 L11^-T  as a product with the stored inverse
//     update     pivot columns [kb+NB, k) of the trailing rows -= L21 L21^T;
//                the CTA of the tile holding the next diagonal block then
//                factors that block (the next step's L11 and L11^-1), so
//                each step is two dependent launches
//   syrk         U = F22 - L(R, 0:k) L(R, 0:k)^T, one product with the whole
//                pivot width as inner dimension
// Tiles are staged into shared memory with cp.async (many loads in flight
// per thread) and double buffered along the inner dimension.
#include "dev_common.cuh"
#include "engine.h"
#include "front_block.cuh"

namespace wd {
namespace {

constexpr int THREADS = 256;
constexpr int BM = SCHUR_BM;   // rows of a Schur tile
constexpr int BN = SCHUR_BN;   // columns of a Schur tile
constexpr int BK = 32;         // inner-dimension chunk

using blk::load4;
// four consecutive shared-memory elements (16-byte aligned for float,
// two 16-byte halves for double)
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
// diagonal block kb of front s (item = (s, kb)): L11 and L11^-1 (the first
// pivot block of every front of a level; the later ones are factored by the
// update launch of the step before).  FP32 fronts whose width is at least
// diag64_min_k (> 0) factor the block in FP64.
// ---------------------------------------------------------------------------
template <class T, bool HAS64>
__global__ void __launch_bounds__(THREADS) diag_factor_kernel(DevSym d, T *__restrict__ front,
                                                              T *__restrict__ dinv,
                                                              const int4 *__restrict__ items,
                                                              int diag64_min_k, status_t *status) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int4 it = items[blockIdx.x];
    const int s = it.x, kb = it.y;
    if (HAS64 && sizeof(T) == 4 && diag64_min_k > 0 && d.sk[s] >= diag64_min_k)
        blk::factor_diag_block<double, T, THREADS>(d, front, dinv, s, kb, status, smem_raw);
    else
        blk::factor_diag_block<T, T, THREADS>(d, front, dinv, s, kb, status, smem_raw);
}

// ---------------------------------------------------------------------------
// panel of pivot block kb: rows [r0, r0+RB) of columns [kb, kb+nb) become
// X := X L11^-T, with L11^-1 already in dinv.  The rows start at kb+NB, or
// at kp when kb is the last block (rows [k, kp) are zero padding); a CTA may
// have no rows.
// ---------------------------------------------------------------------------
constexpr int XLD = blk::XLD;
template <class T>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 4 : 2) panel_kernel(DevSym d, T *__restrict__ front,
                                                        const T *__restrict__ dinv,
                                                        unsigned char *__restrict__ pk,
                                                        const int4 *__restrict__ items, int kb) {
    static_assert(RB == 64 && NB == 64 && THREADS == 256, "4 x 4 register tiles cover the 64 x 64 panel block");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *LT = reinterpret_cast<T *>(smem_raw);         // LT[p * XLD + c] = Linv(c, p)
    T *Xs = LT + NB * XLD;                            // [p][r], ld RB
    const int4 it = items[blockIdx.x];
    const int s = it.x, rb = it.y;
    const Dims z = dims(d, s);
    const int nb = min(NB, z.k - kb);
    const int t0 = kb + nb;
    const int r0 = (t0 == z.k ? z.kp : t0) + rb * RB;
    T *F = front + d.foff[s];
    {
        // Linv is stored column-major (Dv[c + p NB] = Linv(c, p)), so LT's rows
        // are Dv's columns: 16-byte copies
        const T *Dv = dinv + d.dinvoff[s] + (int64_t)(kb / NB) * NB * NB;
        constexpr int V = 16 / sizeof(T);
        for (int idx = threadIdx.x; idx < NB * NB / V; idx += THREADS) {
            const int p = idx / (NB / V), c = (idx % (NB / V)) * V;
            cp_async16(LT + p * XLD + c, Dv + p * NB + c, 16);
        }
    }
    stage_tile<T, THREADS>(Xs, RB, F + (int64_t)kb * z.ld + r0, z.ld, RB, NB, z.mp - r0, nb);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    // out[r][c] = sum_{p <= c} X[r][p] Linv(c, p), Linv(c, p) = XT[p][c];
    // thread: rows 4 (tid % 16) + i, columns 4 (tid / 16) + j, so both
    // operands of a step p are one 4-wide shared load, and p stops at the
    // thread's last column (Linv is lower triangular).
    const int tid = threadIdx.x;
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
// In mode 0 the CTA of tile (0, 0), which holds the whole next diagonal
// block, then factors that block (L11 and L11^-1 of step kb + NB).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(THREADS) schur_kernel(DevSym d, T *__restrict__ front,
                                                        T *__restrict__ dinv,
                                                        const int4 *__restrict__ items, int kb,
                                                        int mode, status_t *status) {
    static_assert(BM >= NB && BN >= NB, "tile (0, 0) covers the next diagonal block");
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
    if (mode == 0 && ti == 0 && tj == 0 && kb + NB < z.k) {
        __syncthreads();   // the block's updated entries, written above, visible to the CTA
        blk::factor_diag_block<T, T, THREADS>(d, front, dinv, s, kb + NB, status, smem_raw);
    }
}

template <class T>
constexpr size_t panel_smem() { return sizeof(T) * (NB * XLD + NB * RB); }
constexpr size_t cmax_size(size_t a, size_t b) { return a > b ? a : b; }
template <class T>
constexpr size_t schur_smem() { return cmax_size(2 * sizeof(T) * BK * (BM + BN), blk::block_smem_bytes<T>()); }
constexpr size_t diag_smem() { return blk::block_smem_bytes<double>(); }

template <class T>
void set_smem_attrs() {
    static bool done = false;  // per instantiation and process
    if (done) return;
    cudaFuncSetAttribute(panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)panel_smem<T>());
    cudaFuncSetAttribute(schur_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)schur_smem<T>());
    cudaFuncSetAttribute(diag_factor_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)diag_smem());
    cudaFuncSetAttribute(diag_factor_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)diag_smem());
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
void launch_diag_factor(const DevSym &d, T *front, T *dinv, const int4 *items, int count, int diag64_min_k,
                        status_t *status, cudaStream_t st) {
    if (count <= 0) return;
    set_smem_attrs<T>();
    if (sizeof(T) == 4 && diag64_min_k > 0)
        diag_factor_kernel<T, true><<<count, THREADS, diag_smem(), st>>>(d, front, dinv, items, diag64_min_k, status);
    else
        diag_factor_kernel<T, false><<<count, THREADS, diag_smem(), st>>>(d, front, dinv, items, diag64_min_k, status);
}

template <class T>
void launch_panel(const DevSym &d, T *front, const T *dinv, unsigned char *pk, const int4 *items, int count,
                  int kb, cudaStream_t st) {
    if (count <= 0) return;
    set_smem_attrs<T>();
    panel_kernel<T><<<count, THREADS, panel_smem<T>(), st>>>(d, front, dinv, pk, items, kb);
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
    template void launch_diag_factor<T>(const DevSym &, T *, T *, const int4 *, int, int, status_t *, \
                                        cudaStream_t);                                           \
    template void launch_panel<T>(const DevSym &, T *, const T *, unsigned char *, const int4 *, int, \
                                  int, cudaStream_t);                                            \
    template void launch_schur<T>(const DevSym &, T *, T *, const int4 *, int, int, int,         \
                                  status_t *, cudaStream_t);
WD_INST(double)
WD_INST(float)
#undef WD_INST

}  // namespace wd
