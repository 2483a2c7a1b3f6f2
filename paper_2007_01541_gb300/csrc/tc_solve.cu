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
// The asynchronous copies of a 32-wide chunk of the inner dimension are issued
// ahead into a ring of shared-memory stages, straight to the values' swizzled
// places; each thread then splits the values it copied in place (hi) and into
// the lo plane, and one thread issues the chunk's MMAs while the next chunks
// are in flight.  The ring has three stages, two chunks ahead (144 KB), except
// in a bupdate launch of more CTAs than SMs (the many short products of the
// lower levels, a few chunks each): there it has two stages, one chunk ahead
// (96 KB), so that two CTAs share an SM and one's set-up, waits and epilogue
// overlap the other's copies.  The stage count changes no arithmetic.
//
// A launch with few output tiles (the top of the tree: a few super-blocks of
// one or two fronts) splits the inner dimension of xapply and bupdate over up
// to four CTAs per tile: each computes the product over its part of the
// chunks, and the last CTA of the tile to arrive (an atomic counter, no
// waiting) adds the partial tiles in a fixed order and writes the result.
// The serial chain of chunks per CTA, which sets the time of these launches,
// shrinks by the split factor.
//
// Every wait is bounded; on expiry the CTA records the timeout status, waits
// (with a fixed bound) for its copies and products in flight, frees its tensor
// memory and returns without writing (the output of a split tile whose CTA
// timed out is unspecified; the call reports the timeout).
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
constexpr int NSTG = 3;                         // most stages of the ring (chunks issued ahead: stages - 1)
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

// Per-item geometry of the three products (see the plan in api.cpp).
struct Geo {
    int s, k, m, kp, mp, ld, f;
    int b0, w, wp;       // super-block: first column, width, width rounded to 64
    int c0, nc;          // right-hand sides of the tile
    int kc0, nchunk;     // first 32-wide chunk of the inner dimension (in its own index), chunks
    int ks, nks;         // xapply / bupdate: this CTA's part of the inner dimension, parts
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
    g.ks = 0;
    g.nks = 1;
    if (OP != OP_BREDUCE) {
        g.ks = (it.z >> 16) & 0xFF;
        g.nks = max(1, it.z >> 24);
    }
    const int rb = it.z & 0xFFFF;
    if (OP == OP_XAPPLY) {
        g.r0 = rb * TM;
        // lower (forward): columns [0, r0 + TM); upper (backward): [r0, wp)
        const int ka = a.upper ? g.r0 : 0, kb = a.upper ? g.wp : min(g.wp, g.r0 + TM);
        g.kc0 = ka / TK;
        g.nchunk = (kb - ka + TK - 1) / TK;
    } else if (OP == OP_BUPDATE) {
        g.seg = it.w >> 16;
        if (g.seg == 0) {
            g.i0 = g.b0 + g.w + rb * TM;     // pivot rows after B
            g.nrow = g.k - g.i0;
            g.mrow = g.i0;
        } else {
            g.i0 = rb * TM;                  // rows of R
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
    if (g.nks > 1) {
        // chunks [ks cps, (ks + 1) cps) of the inner dimension
        const int cps = (g.nchunk + g.nks - 1) / g.nks;
        const int cb = min(g.nchunk, g.ks * cps);
        g.kc0 += cb;
        g.nchunk = min(g.nchunk - cb, cps);
    }
    return g;
}

// Issues the asynchronous copies of chunk c of the FP32 operands into a stage,
// each value to its swizzled place in the hi plane (split later in place):
// A, where it is read from an array, as 16-byte copies (row tid / 2, inner
// values (tid % 2) 16 .. +16), B as 4-byte copies (right-hand side tid / 4,
// inner values (tid % 4) 8 .. +8).  Values outside the operand are zero-filled.
template <int OP>
__device__ __forceinline__ void issue_chunk(const DevSym &d, const TcSolveArgs &a, const Geo &g, int c,
                                            unsigned char *Ah, unsigned char *Bh) {
    const int tid = threadIdx.x;
    const int kk0 = (g.kc0 + c) * TK;   // first inner index of the chunk
    if (OP != OP_BUPDATE) {
        const int r = tid >> 1, kh = (tid & 1) * 16;
        const float *src;
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
            cp_async16(Ah + tc::sw128_offset(r, kh + 4 * q), v ? src + 4 * q : a.front, v ? 16 : 0);
        }
    }
    const int j = tid >> 2, kq = (tid & 3) * 8;
    const bool vj = j < g.nc;
    const int64_t coff = (int64_t)(g.c0 + j) * d.n;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int kk = kk0 + kq + q;
        const float *src = nullptr;
        if (OP == OP_XAPPLY) {
            // t_B (pending right-hand side of the super-block's pivot rows)
            if (vj && kk < g.w) src = a.in + g.f + g.b0 + kk + coff;
        } else if (OP == OP_BUPDATE) {
            // the chunk index counts the packed panel's 32-column chunks from
            // the supernode's first column; y_B is indexed inside the super-block
            const int kr = kk - g.b0;
            if (vj && kr < g.w) src = a.in + g.f + g.b0 + kr + coff;
        } else {
            // x at storage row kk: a pivot row after B, or a row of R
            if (vj && kk >= g.b0 + g.w && kk < g.q1) {
                if (kk < g.k) src = a.in + g.f + kk + coff;
                else if (kk >= g.kp) src = a.in + d.rows[d.rowptr[g.s] + g.k + (kk - g.kp)] + coff;
            }
        }
        cp_async4(Bh + tc::sw128_offset(j, kq + q), src ? src : a.in, src ? 4 : 0);
    }
}

// x -> (hi, lo) in place for four values: hi = x rounded to tf32 back into the
// hi plane, lo = (x - hi) rounded to tf32 into the lo plane
__device__ __forceinline__ void split4_inplace(unsigned char *hi, unsigned char *lo, uint32_t off) {
    const uint4 x = *reinterpret_cast<const uint4 *>(hi + off);
    const float v[4] = {__uint_as_float(x.x), __uint_as_float(x.y), __uint_as_float(x.z), __uint_as_float(x.w)};
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) tc::split_tf32(v[i], h[i], l[i]);
    *reinterpret_cast<uint4 *>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Splits the values this thread copied in issue_chunk (its own copies are
// complete after cp.async.wait_group, so no barrier is needed before).
template <int OP>
__device__ __forceinline__ void split_chunk(unsigned char *Ah, unsigned char *Al, unsigned char *Bh,
                                            unsigned char *Bl) {
    const int tid = threadIdx.x;
    if (OP != OP_BUPDATE) {
        const int r = tid >> 1, kh = (tid & 1) * 16;
#pragma unroll
        for (int q = 0; q < 4; ++q) split4_inplace(Ah, Al, tc::sw128_offset(r, kh + 4 * q));
    }
    const int j = tid >> 2, kq = (tid & 3) * 8;
    split4_inplace(Bh, Bl, tc::sw128_offset(j, kq));
    split4_inplace(Bh, Bl, tc::sw128_offset(j, kq + 4));
}

// NS: stages of the ring (3, or 2 for bupdate launches of more CTAs than SMs)
template <int OP, int NS>
__global__ void __launch_bounds__(NTH, NS == 2 ? 2 : 1) tc_solve_kernel(DevSym d, TcSolveArgs a,
                                                                       const int4 *__restrict__ items) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int nst = NS;     // the dynamic shared memory holds nst stages
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + nst * STG_BYTES);
    uint64_t *empty = full + NSTG;
    uint64_t *done = empty + NSTG;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    int *last_flag = abort_flag + 1;
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

    const uint32_t idesc = tc::idesc_tf32(TM, TN);
    // chunk cc goes to stage cc % nst; before it is issued, the MMAs of the
    // chunk that used the stage last (cc - nst) must have completed
    int issued = 0;
    auto issue = [&](int cc) {
        const int st = cc % nst;
        if (cc >= nst && !tc::mbar_wait(&empty[st], ((cc / nst) - 1) & 1, limit)) {
            atomicExch(abort_flag, 1);
            return;
        }
        unsigned char *stg = sm + st * STG_BYTES;
        if (OP == OP_BUPDATE && tid == 0) {
            mbar_expect_tx(&full[st], 2 * A_BYTES);
            bulk_copy(stg, P + pack_offset(g.kc0 + cc, 0, g.mrow, prow), A_BYTES, &full[st]);
            bulk_copy(stg + A_BYTES, P + pack_offset(g.kc0 + cc, 1, g.mrow, prow), A_BYTES, &full[st]);
        }
        issue_chunk<OP>(d, a, g, cc, stg, stg + 2 * A_BYTES);
        issued = cc + 1;
    };
    for (int cc = 0; cc < nst - 1; ++cc) {
        if (cc < g.nchunk) issue(cc);
        cp_async_commit();
    }
    for (int c = 0; c < g.nchunk; ++c) {
        const int st = c % nst;
        unsigned char *stg = sm + st * STG_BYTES;
        cp_async_wait<nst - 2>();     // this thread's copies of chunk c have landed
        split_chunk<OP>(stg, stg + A_BYTES, stg + 2 * A_BYTES, stg + 2 * A_BYTES + B_BYTES);
        tc::fence_async_smem();
        __syncthreads();
        if (*(volatile int *)abort_flag) break;
        if (tid == 0) {
            bool ok = true;
            if (OP == OP_BUPDATE) ok = tc::mbar_wait(&full[st], (c / nst) & 1, limit);
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
        if (c + nst - 1 < g.nchunk) issue(c + nst - 1);
        cp_async_commit();
    }
    cp_async_wait<0>();
    // every MMA issued above has completed once `done` arrives
    if (tid == 0) tc::mma_commit(done);
    if (!tc::mbar_wait(done, 0, limit)) atomicExch(abort_flag, 1);
    tc::tc_fence_after();
    __syncthreads();
    const bool aborted = *(volatile int *)abort_flag != 0;
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (its 32 rows of the
    // tile) and right-hand sides 32 (w / 4) .. +32
    const int lg = warp & 3, half = warp >> 2;
    const int r = 32 * lg + lane;
    const int jb = 32 * half;
    float v[32];
    if (!aborted && g.nchunk > 0) {
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
    if (aborted && tid == 0) {
        // after a timeout: the issued bulk fills have landed and the issued
        // MMAs have completed before the shared memory and TMEM are given up
        // (every thread's own copies were waited for above)
        if (OP == OP_BUPDATE)
            for (int cc = (issued > nst ? issued - nst : 0); cc < issued; ++cc)
                tc::mbar_wait(&full[cc % nst], (cc / nst) & 1, DRAIN_LIMIT);
        tc::mbar_wait(done, 0, DRAIN_LIMIT);
        atomicMax(a.tstatus, 1ull);
    }
    bool write = !aborted;
    if (OP != OP_BREDUCE && g.nks > 1) {
        // split inner dimension: every CTA of the tile stores its partial
        // product and counts itself in; the last to arrive adds the partials
        // in split order (the same sum whichever CTA is last) and writes the
        // tile, then resets the counter for the next launch.  A CTA that
        // timed out takes part with a zero partial (the call reports the
        // timeout; its output is unspecified).
        const int tile = blockIdx.x - g.ks;
        float *mine = a.ksw + (int64_t)blockIdx.x * TC_SOLVE_TILE + r;
#pragma unroll
        for (int i = 0; i < 32; ++i) mine[(jb + i) * TM] = v[i];
        __threadfence();
        __syncthreads();
        if (tid == 0) *last_flag = atomicAdd(a.kcnt + tile, 1) == g.nks - 1;
        __syncthreads();
        write = *(volatile int *)last_flag != 0;
        if (write) {
            __threadfence();
            const float *base = a.ksw + (int64_t)tile * TC_SOLVE_TILE + r;
            float acc[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[i] = 0.f;
            for (int q = 0; q < g.nks; ++q) {
                const volatile float *pq = base + (int64_t)q * TC_SOLVE_TILE;
#pragma unroll
                for (int i = 0; i < 32; ++i) acc[i] += pq[(jb + i) * TM];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = acc[i];
            if (tid == 0) a.kcnt[tile] = 0;
        }
    }
    if (write) {
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
                // 16 old values are read before the first of their stores: a
                // store may alias a later column's load through the runtime
                // stride, which would make each of the 32 read-modify-writes
                // a memory round trip of its own
#pragma unroll
                for (int h = 0; h < 32; h += 16) {
                    float old[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        old[i] = jb + h + i < g.nc ? o[(int64_t)(jb + h + i) * ldd] : 0.f;
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (jb + h + i < g.nc) o[(int64_t)(jb + h + i) * ldd] = old[i] - v[h + i];
                }
            }
        } else {
            float *o = a.out + ((int64_t)g.slot * TN + jb) * TM + r;
#pragma unroll
            for (int i = 0; i < 32; ++i) o[(int64_t)i * TM] = v[i];
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, TN);
}

constexpr size_t tc_solve_smem(int nst) { return (size_t)nst * STG_BYTES + 1024 + 128; }

template <int OP, int NS>
void set_attr() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(tc_solve_kernel<OP, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc_solve_smem(NS));
    cudaFuncSetAttribute(tc_solve_kernel<OP, NS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    done = true;
}

}  // namespace

void init_tc_solve_attributes() {
    set_attr<OP_XAPPLY, NSTG>();
    set_attr<OP_BUPDATE, NSTG>();
    set_attr<OP_BUPDATE, 2>();
    set_attr<OP_BREDUCE, NSTG>();
}

void launch_tc_xapply(const DevSym &d, const TcSolveArgs &a, const int4 *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    set_attr<OP_XAPPLY, NSTG>();
    tc_solve_kernel<OP_XAPPLY, NSTG><<<count, NTH, tc_solve_smem(NSTG), st>>>(d, a, items);
}
void launch_tc_bupdate(const DevSym &d, const TcSolveArgs &a, const int4 *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    // more CTAs than SMs (the lower levels: one super-block, a few chunks
    // per CTA): two stages, two CTAs per SM
    if (a.sms > 0 && count > a.sms) {
        set_attr<OP_BUPDATE, 2>();
        tc_solve_kernel<OP_BUPDATE, 2><<<count, NTH, tc_solve_smem(2), st>>>(d, a, items);
    } else {
        set_attr<OP_BUPDATE, NSTG>();
        tc_solve_kernel<OP_BUPDATE, NSTG><<<count, NTH, tc_solve_smem(NSTG), st>>>(d, a, items);
    }
}
void launch_tc_breduce(const DevSym &d, const TcSolveArgs &a, const int4 *items, int count, cudaStream_t st) {
    if (count <= 0) return;
    set_attr<OP_BREDUCE, NSTG>();
    tc_solve_kernel<OP_BREDUCE, NSTG><<<count, NTH, tc_solve_smem(NSTG), st>>>(d, a, items);
}

}  // namespace wd
