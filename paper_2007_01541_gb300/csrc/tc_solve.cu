// Products of the supernodal substitutions on the 5th-generation tensor cores
// (FP32 fronts, many right-hand sides): the exact inverse of the compressed
// matrix applied to a block of right-hand sides (Sections 1 and 5) by
// super-blocks of 512 pivot columns, with the three products of a step
//   xapply   y_B = X_B t_B            (forward, X_B the super-block inverse)
//            x_B = X_B^T t_B          (backward)
//   bupdate  t(rows below B) -= L(rows below, B) y_B
//   breduce  partial sums of L(rows below, B)^T x(rows below), per split of
//            the rows below (added in a fixed order by breduce_finish)
// as D = A B^T with A: 128 x K, B: 64 right-hand sides x K, in 3xTF32 (every
// FP32 operand value x = hi + lo, hi = x rounded to tf32, lo = the rest
// rounded to tf32; D += A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation
// in tensor memory).
//
// Operands reach shared memory in the 128-byte-swizzled K-major layout of the
// MMA.  bupdate's A (rows of L) is copied in pre-split by the bulk-copy engine
// from the packed tf32 lines the panel kernel wrote; every other operand is
// read from its FP32 array (the super-block inverses, the fronts' columns, the
// right-hand-side columns), split by the CTA's threads and stored swizzled.
// The loads of the next 32-wide chunk of the inner dimension are issued before
// the current chunk is split and stored; two shared-memory stages alternate,
// the MMAs of a chunk running while the next one is prepared.
//
// Every wait is bounded; on expiry the CTA records the timeout status, waits
// (with a fixed bound) for its copies and products in flight, frees its tensor
// memory and returns without writing.
#include "dev_common.cuh"
#include "engine.h"
#include "tc_common.cuh"

namespace wd {
namespace {

constexpr int TM = 128, TN = 64, TK = 32;
constexpr int NTH = 256;
constexpr int A_BYTES = TM * TK * 4;           // one plane of A: 16 KB
constexpr int B_BYTES = TN * TK * 4;           // one plane of B: 8 KB
constexpr int STG_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int NSTG = 2;
constexpr uint32_t WAIT_DEFAULT = 1u << 26;
constexpr uint32_t DRAIN_LIMIT = 1u << 26;

enum { OP_XAPPLY = 0, OP_BUPDATE = 1, OP_BREDUCE = 2 };

__device__ __forceinline__ void bulk_copy(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            tc::smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tc::smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// four values of one operand row -> tf32 hi / lo planes at the swizzled
// position of (row, k .. k+3) (k a multiple of 4)
__device__ __forceinline__ void put4(unsigned char *hi, unsigned char *lo, int row, int k, const float (&v)[4]) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) tc::split_tf32(v[i], h[i], l[i]);
    const uint32_t off = tc::sw128_offset(row, k);
    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Per-item geometry of the three products (see the plan in api.cpp).
struct Geo {
    int s, k, m, kp, mp, ld, f;
    int b0, w, wp;       // super-block: first column, width, width rounded to 64
    int c0, nc;          // right-hand sides of the tile
    int kc0, nchunk;     // first 32-wide chunk of the inner dimension (in its own index), chunks
    // xapply
    int r0;
    // bupdate
    int seg, i0, nrow, mrow;
    // breduce
    int j0, nb, q0, q1, slot;
};

template <int OP>
__device__ __forceinline__ Geo geometry(const DevSym &d, const TcSolveArgs &a, int4 it) {
    Geo g;
    g.s = it.x;
    g.k = d.sk[g.s];
    g.m = d.sm[g.s];
    g.kp = d.skp[g.s];
    g.mp = g.kp + g.m - g.k;
    g.ld = d.sld[g.s];
    g.f = d.sfirst[g.s];
    const int sb = OP == OP_BREDUCE ? (it.y >> 3) : it.y;
    g.b0 = sb * SB;
    g.w = min(SB, g.k - g.b0);
    g.wp = (g.w + NB - 1) / NB * NB;
    const int gt = OP == OP_BREDUCE ? (it.z & 0xFFFF) : (it.w & 0xFFFF);
    g.c0 = gt * TN;
    g.nc = min(TN, a.nrhs - g.c0);
    if (OP == OP_XAPPLY) {
        g.r0 = it.z * TM;
        // lower (forward): columns [0, r0 + TM); upper (backward): [r0, wp)
        const int ka = a.upper ? g.r0 : 0, kb = a.upper ? g.wp : min(g.wp, g.r0 + TM);
        g.kc0 = ka / TK;
        g.nchunk = (kb - ka + TK - 1) / TK;
    } else if (OP == OP_BUPDATE) {
        g.seg = it.w >> 16;
        if (g.seg == 0) {
            g.i0 = g.b0 + g.w + it.z * TM;   // pivot rows after B
            g.nrow = g.k - g.i0;
            g.mrow = g.i0;
        } else {
            g.i0 = it.z * TM;                // rows of R
            g.nrow = (g.m - g.k) - g.i0;
            g.mrow = g.kp + g.i0;
        }
        g.kc0 = g.b0 / TK;
        g.nchunk = (g.w + TK - 1) / TK;
    } else {
        const int cb = it.y & 7, ks = it.z >> 16;
        g.j0 = g.b0 + cb * TM;
        g.nb = min(TM, g.b0 + g.w - g.j0);
        const int kbeg = (g.b0 + g.w) & ~(TK - 1);   // storage rows below B, from a 32-row boundary
        g.q0 = kbeg + ks * SOLVE_KSR_TC;
        g.q1 = min(g.mp, g.q0 + SOLVE_KSR_TC);
        g.kc0 = g.q0 / TK;
        g.nchunk = (g.q1 - g.q0 + TK - 1) / TK;
        g.slot = it.w;
    }
    return g;
}

// Loads of chunk c of the FP32 operands into registers: A (16 consecutive
// inner values of row tid / 2) where it is read from an array, B (8
// consecutive inner values of right-hand side tid / 4).
template <int OP>
__device__ __forceinline__ void load_chunk(const DevSym &d, const TcSolveArgs &a, const Geo &g, int c,
                                           float (&ra)[16], float (&rb)[8]) {
    const int tid = threadIdx.x;
    const int kk0 = (g.kc0 + c) * TK;   // first inner index of the chunk
    if (OP != OP_BUPDATE) {
        const int r = tid >> 1, kh = (tid & 1) * 16;
        const float *src = nullptr;
        bool ok;
        if (OP == OP_XAPPLY) {
            // row r0 + r of X (forward: the stored X^T, column-major, holds X's
            // rows as its columns; backward: X itself holds the rows of X^T)
            ok = g.r0 + r < g.wp;
            src = a.xp + a.xsoff[g.s] + (int64_t)(g.b0 / SB) * SB * SB + (int64_t)(g.r0 + r) * g.wp + kk0 + kh;
        } else {
            // column j0 + r of L over storage rows kk0 + kh ..
            ok = r < g.nb;
            src = a.front + d.foff[g.s] + (int64_t)(g.j0 + r) * g.ld + kk0 + kh;
        }
        const int lim = OP == OP_XAPPLY ? g.wp : g.mp;   // inner extent stored
        // xapply: only the 64 x 64 blocks on the stored side of the diagonal
        // are written (X lower, X^T upper); the others are read as zero
        const int rblk = (g.r0 + r) / NB;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int kblk = (kk0 + kh + 4 * q) / NB;
            const bool side = OP != OP_XAPPLY || (a.upper ? kblk >= rblk : kblk <= rblk);
            const bool v = ok && side && kk0 + kh + 4 * q < lim;
            const float4 t = v ? *reinterpret_cast<const float4 *>(src + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
            ra[4 * q] = t.x, ra[4 * q + 1] = t.y, ra[4 * q + 2] = t.z, ra[4 * q + 3] = t.w;
        }
    }
    const int j = tid >> 2, kq = (tid & 3) * 8;
    const bool vj = j < g.nc;
    const int64_t coff = (int64_t)(g.c0 + j) * d.n;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int kk = kk0 + kq + q;
        float v = 0.f;
        if (OP == OP_XAPPLY) {
            // t_B (pending right-hand side of the super-block's pivot rows)
            if (vj && kk < g.w) v = a.in[g.f + g.b0 + kk + coff];
        } else if (OP == OP_BUPDATE) {
            // the chunk index counts the packed panel's 32-column chunks from
            // the supernode's first column; y_B is indexed inside the super-block
            const int kr = kk - g.b0;
            if (vj && kr < g.w) v = a.in[g.f + g.b0 + kr + coff];   // y_B
        } else {
            // x at storage row kk: a pivot row after B, or a row of R
            if (vj && kk >= g.b0 + g.w && kk < g.q1) {
                if (kk < g.k) v = a.in[g.f + kk + coff];
                else if (kk >= g.kp) v = a.in[d.rows[d.rowptr[g.s] + g.k + (kk - g.kp)] + coff];
            }
        }
        rb[q] = v;
    }
}

template <int OP>
__global__ void __launch_bounds__(NTH, 1) tc_solve_kernel(DevSym d, TcSolveArgs a, const int4 *__restrict__ items) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + NSTG * STG_BYTES);
    uint64_t *empty = full + NSTG;
    uint64_t *done = empty + NSTG;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    const uint32_t limit = a.wait_limit ? a.wait_limit : WAIT_DEFAULT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Geo g = geometry<OP>(d, a, items[blockIdx.x]);
    const int prow = pack_rows(g.mp);
    const unsigned char *P = OP == OP_BUPDATE ? a.pk + d.pkoff[g.s] : nullptr;

    if (tid == 0) {
        for (int i = 0; i < NSTG; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(tslot, TN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    int fills[NSTG] = {0, 0};   // thread 0: bulk fills issued per stage
    float ra[16], rb[8], na[16], nbv[8];
    if (g.nchunk > 0) load_chunk<OP>(d, a, g, 0, ra, rb);
    const uint32_t idesc = tc::idesc_tf32(TM, TN);
    for (int c = 0; c < g.nchunk; ++c) {
        const int st = c & 1;
        if (c + 1 < g.nchunk) load_chunk<OP>(d, a, g, c + 1, na, nbv);
        if (tid == 0 && c >= NSTG && !tc::mbar_wait(&empty[st], ((c >> 1) - 1) & 1, limit))
            atomicExch(abort_flag, 1);
        __syncthreads();
        if (*(volatile int *)abort_flag) break;
        unsigned char *stg = sm + st * STG_BYTES;
        unsigned char *Ah = stg, *Al = stg + A_BYTES, *Bh = stg + 2 * A_BYTES, *Bl = Bh + B_BYTES;
        if (OP == OP_BUPDATE) {
            if (tid == 0) {
                ++fills[st];
                mbar_expect_tx(&full[st], 2 * A_BYTES);
                bulk_copy(Ah, P + pack_offset(g.kc0 + c, 0, g.mrow, prow), A_BYTES, &full[st]);
                bulk_copy(Al, P + pack_offset(g.kc0 + c, 1, g.mrow, prow), A_BYTES, &full[st]);
            }
        } else {
            const int r = tid >> 1, kh = (tid & 1) * 16;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float v4[4] = {ra[4 * q], ra[4 * q + 1], ra[4 * q + 2], ra[4 * q + 3]};
                put4(Ah, Al, r, kh + 4 * q, v4);
            }
        }
        {
            const int j = tid >> 2, kq = (tid & 3) * 8;
            const float v0[4] = {rb[0], rb[1], rb[2], rb[3]}, v1[4] = {rb[4], rb[5], rb[6], rb[7]};
            put4(Bh, Bl, j, kq, v0);
            put4(Bh, Bl, j, kq + 4, v1);
        }
        tc::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            bool ok = true;
            if (OP == OP_BUPDATE) ok = tc::mbar_wait(&full[st], (fills[st] - 1) & 1, limit);
            if (ok) {
                tc::tc_fence_after();
                const uint32_t a0 = tc::smem_u32(stg);
#pragma unroll
                for (int kk = 0; kk < TK / 8; ++kk) {
                    const uint64_t ah = tc::desc_kmajor_sw128(a0 + 32 * kk);
                    const uint64_t al = tc::desc_kmajor_sw128(a0 + A_BYTES + 32 * kk);
                    const uint64_t bh = tc::desc_kmajor_sw128(a0 + 2 * A_BYTES + 32 * kk);
                    const uint64_t bl = tc::desc_kmajor_sw128(a0 + 2 * A_BYTES + B_BYTES + 32 * kk);
                    tc::mma_tf32(tmem, ah, bh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
                    tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                    tc::mma_tf32(tmem, al, bh, idesc, 1u);
                }
            } else {
                atomicExch(abort_flag, 1);
            }
            tc::mma_commit(&empty[st]);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) ra[i] = na[i];
#pragma unroll
        for (int i = 0; i < 8; ++i) rb[i] = nbv[i];
    }
    // every MMA issued above has completed once `done` arrives
    if (tid == 0) tc::mma_commit(done);
    if (!tc::mbar_wait(done, 0, limit)) atomicExch(abort_flag, 1);
    tc::tc_fence_after();
    __syncthreads();
    const bool aborted = *(volatile int *)abort_flag != 0;
    if (!aborted) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its 32 rows of the
        // tile) and right-hand sides 32 (w / 4) .. +32
        const int lg = warp & 3, half = warp >> 2;
        const int r = 32 * lg + lane;
        float v[32];
        if (g.nchunk > 0) {
            float t[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + 32 * half, t);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = t[i];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + 32 * half + 16, t);
#pragma unroll
            for (int i = 0; i < 16; ++i) v[16 + i] = t[i];
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 0.f;
        }
        const int jb = 32 * half;
        if (OP == OP_XAPPLY) {
            if (g.r0 + r < g.w) {
                float *o = a.out + g.f + g.b0 + g.r0 + r + (int64_t)g.c0 * d.n;
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (jb + i < g.nc) o[(int64_t)(jb + i) * d.n] = v[i];
            }
        } else if (OP == OP_BUPDATE) {
            if (r < g.nrow) {
                float *o;
                int64_t ldd;
                if (g.seg == 0) {
                    o = a.out + g.f + g.i0 + r + (int64_t)g.c0 * d.n;
                    ldd = d.n;
                } else {
                    o = a.W + d.woff[g.s] * a.nrhs + g.i0 + r + (int64_t)g.c0 * (g.m - g.k);
                    ldd = g.m - g.k;
                }
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (jb + i < g.nc) o[(int64_t)(jb + i) * ldd] -= v[i];
            }
        } else {
            float *o = a.out + ((int64_t)g.slot * TN + jb) * TM + r;
#pragma unroll
            for (int i = 0; i < 32; ++i) o[(int64_t)i * TM] = v[i];
        }
    } else if (tid == 0) {
        // after a timeout: the issued fills have landed and the issued MMAs
        // have completed before the shared memory and TMEM are given up
        for (int st = 0; st < NSTG; ++st)
            if (fills[st] > 0) tc::mbar_wait(&full[st], (fills[st] - 1) & 1, DRAIN_LIMIT);
        tc::mbar_wait(done, 0, DRAIN_LIMIT);
        atomicMax(a.tstatus, 1ull);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, TN);
}

constexpr size_t tc_solve_smem() { return (size_t)NSTG * STG_BYTES + 1024 + 128; }

template <int OP>
void set_attr() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(tc_solve_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_solve_smem());
    done = true;
}

}  // namespace

void init_tc_solve_attributes() {
    set_attr<OP_XAPPLY>();
    set_attr<OP_BUPDATE>();
    set_attr<OP_BREDUCE>();
}

void launch_tc_xapply(const DevSym &d, const TcSolveArgs &a, const int4 *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    set_attr<OP_XAPPLY>();
    tc_solve_kernel<OP_XAPPLY><<<count, NTH, tc_solve_smem(), st>>>(d, a, items);
}
void launch_tc_bupdate(const DevSym &d, const TcSolveArgs &a, const int4 *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    set_attr<OP_BUPDATE>();
    tc_solve_kernel<OP_BUPDATE><<<count, NTH, tc_solve_smem(), st>>>(d, a, items);
}
void launch_tc_breduce(const DevSym &d, const TcSolveArgs &a, const int4 *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    set_attr<OP_BREDUCE>();
    tc_solve_kernel<OP_BREDUCE><<<count, NTH, tc_solve_smem(), st>>>(d, a, items);
}

}  // namespace wd
