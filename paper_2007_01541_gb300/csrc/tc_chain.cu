// Pivot columns of FP32 fronts in one launch per level: the factorization
// P A P^T = L L^T of Section 4 restricted to each front's k pivot columns,
// as tasks ordered by dependency instead of one (panel, update) launch pair
// per 64-column step.
//
// Task (s, c, ti): front s, column block c (columns [64c, 64c + 64) of the
// front's pivot part), row tile ti (front rows [64c + 128 ti, ... + 128)).
// It computes
//   X = F(tile rows, block c) - sum_{j < c} L(tile rows, block j) L(block c rows, block j)^T
// on the tensor cores (3xTF32 products of the packed tf32 hi/lo lines of L
// that earlier tasks wrote; one tensor-memory accumulator per block j, and
// the epilogue subtracts each in FP32 while the next one runs, the update
// order of the right-looking factorization), then
//   ti = 0:  the tile's first 64 rows are the diagonal block: L11 = chol(X11)
//            and L11^-1 (front_block.cuh); L11^-1 is published as a tf32
//            hi / lo tensor-core operand for the column's other tasks;
//   ti > 0:  waits for it and fetches it with one bulk copy;
// then the panel rows L = X L11^-T are one more tensor-core product (3xTF32,
// the tile as the A operand), read from tensor memory straight into the
// front and the packed lines, after which the task publishes its two 64-row
// blocks.  A task reads only what earlier tasks (in launch order: c, then ti,
// then s) publish, and each CTA takes the next task from a counter when it
// starts, so every task it waits for is held by a CTA that is already
// running: the launch cannot deadlock, whatever the number of resident CTAs.
//
// Dependencies are words in global memory (zeroed before each factorization),
// set with release stores after a fence that also orders the generic-proxy
// stores before later bulk copies (async proxy) of other CTAs, and polled with
// acquire loads.  Every wait is bounded (wait_limit polls); a CTA whose wait
// expires records the timeout, raises a launch-wide abort word that the other
// CTAs' waits also watch, waits (bounded) for its own copies and products in
// flight, frees its tensor memory and returns.
//
// Thread roles (320 threads): warp 0 lane 0 polls the dependencies and issues
// the bulk copies into a 2-stage ring; warp 1 allocates 128 TMEM columns
// and one lane issues the MMAs; warps 2-9 hold one tile row and 32 columns
// each (F loaded while the products run, then X -= acc per block, then the
// panel rows); all threads take part in the block factorization.
#include "engine.h"
#include "front_block.cuh"
#include "tc_common.cuh"

namespace wd {
namespace {

constexpr int CM = 128, CN = 64, CKC = 32;   // tile rows, tile columns, inner chunk
constexpr int CSTAGES = 2;
constexpr int A_PLANE = CM * CKC * 4;        // 16 KB: one plane (hi or lo) of the A operand
constexpr int B_PLANE = CN * CKC * 4;        // 8 KB: one plane of the B operand
constexpr int CSTAGE_BYTES = 2 * A_PLANE + 2 * B_PLANE;
constexpr int CT = 320;
constexpr uint32_t WAIT_LIMIT = 1u << 26;    // default bound of a wait (polls)
constexpr uint32_t DRAIN_LIMIT = 1u << 26;   // bound of the waits for work in flight after a timeout
// after the products the stage memory holds, for the panel product on the
// tensor cores: the tile X as the A operand (tf32 hi / lo planes of 128 rows
// x 32 columns, 128-byte swizzled) and L11^-1 as the B operand (64 rows x 32
// columns per plane, row n = row n of L11^-1); before that, the diagonal
// task's block factorization (front_block.cuh) uses the A operand's place
constexpr int AOP_BYTES = 4 * A_PLANE;                       // 64 KB
constexpr int LPACK = 4 * B_PLANE;                            // 32 KB: L11^-1 as the B operand
constexpr int BOP_OFF = AOP_BYTES;
constexpr int DATA_BYTES = (CSTAGES * CSTAGE_BYTES > BOP_OFF + LPACK) ? CSTAGES * CSTAGE_BYTES : BOP_OFF + LPACK;
static_assert((int)blk::block_smem_bytes<float>() <= AOP_BYTES, "the block factorization fits below the B operand");
static_assert(CN == NB, "a task's column block is one pivot block");

__device__ __forceinline__ void bulk_copy(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            tc::smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tc::smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
// orders this thread's generic-proxy global accesses with async-proxy ones
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
}
// bounded wait for *f != 0; false when the bound expires or another CTA of
// the launch has given up
__device__ bool wait_flag(const unsigned *f, uint32_t limit, const unsigned *gabort) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (ld_acquire(f) != 0u) return true;
        if (*(volatile const unsigned *)gabort != 0u) return false;
        if (i >= 256) __nanosleep(64);   // a short spin first: the dependency is often about to be set
    }
    return false;
}
// bounded mbarrier wait that also gives up once this CTA has aborted
__device__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, uint32_t limit, const int *abort_flag) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if (*(volatile const int *)abort_flag) return false;
    }
    return false;
}

__global__ void __launch_bounds__(CT, 1)
    tc_chain_kernel(DevSym d, float *__restrict__ front, unsigned char *__restrict__ pk,
                    const int4 *__restrict__ items, int count, int level, ChainArgs a) {
    const uint32_t limit = a.wait_limit ? a.wait_limit : WAIT_LIMIT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + DATA_BYTES);
    uint64_t *empty = full + CSTAGES;
    uint64_t *tfull = empty + CSTAGES;     // accumulator b holds a finished column block
    uint64_t *tempty = tfull + 2;          // accumulator b has been read by the epilogue
    uint64_t *done = tempty + 2;           // every issued MMA has completed
    uint64_t *lbar = done + 1;             // the B operand (L11^-1) has landed
    uint64_t *pdone = lbar + 1;            // the panel product has completed
    uint32_t *tslot = reinterpret_cast<uint32_t *>(pdone + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    int *task_sm = abort_flag + 1;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        // the next task in launch order: all earlier ones are held by CTAs
        // that have started
        *task_sm = (int)atomicAdd(a.counter + level, 1u);
        for (int i = 0; i < CSTAGES; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&tfull[i], 1);
            tc::mbar_init(&tempty[i], 8);   // one arrival per epilogue warp
        }
        tc::mbar_init(done, 1);
        tc::mbar_init(lbar, 1);
        tc::mbar_init(pdone, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (*task_sm >= count) return;   // the counter was not zero at launch: nothing to take
    const int4 it = items[*task_sm];
    const int s = it.x, c = it.y, ti = it.z;
    const int k = d.sk[s], m = d.sm[s], kp = d.skp[s], ld = d.sld[s];
    const int mp = kp + m - k;
    const int c0 = c * NB;                 // first column of the block = first row of its diagonal block
    const int nbc = min(NB, k - c0);       // columns of the block
    const int R0 = c0 + ti * CM;           // first front row of the tile
    const int nk = 2 * c;                  // 32-wide chunks of the inner dimension [0, c0)
    const int prow = pack_rows(mp);
    unsigned char *P = pk + d.pkoff[s];
    const int nrb = (mp + NB - 1) / NB + 1;     // row blocks per column block in the flag array
    const int ncb = (k + NB - 1) / NB;
    unsigned *fl = a.flags + a.flagoff[s];      // ready[j * nrb + rb], then diag[j]
    unsigned *diagf = fl + ncb * nrb;

    if (warp == 1) tc::tmem_alloc(tslot, 2 * CN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    int fills[CSTAGES] = {};   // producer lane: fills issued per stage
    float cur[32];
    const int lg = warp & 3, half = (warp - 2) >> 2;
    const int lr = 32 * lg + lane;         // epilogue: local row
    const int cb = 32 * half;              // epilogue: first local column
    if (warp == 0) {
        if (lane == 0 && nk > 0) {
            const int rbA = R0 / NB;
            const int nrbv = (mp + NB - 1) / NB;   // row blocks that hold rows below mp
            for (int j = 0; j < c; ++j) {
                const unsigned *fj = fl + j * nrb;
                const bool ok = wait_flag(fj + c, limit, a.gabort) && wait_flag(fj + rbA, limit, a.gabort) &&
                                (rbA + 1 >= nrbv || wait_flag(fj + rbA + 1, limit, a.gabort));
                if (!ok) {
                    atomicExch(abort_flag, 1);
                    break;
                }
                fence_proxy_async_global();
                bool stop = false;
                for (int h = 0; h < 2 && !stop; ++h) {
                    const int kt = 2 * j + h, st = kt % CSTAGES;
                    if (kt >= CSTAGES &&
                        !mbar_wait_or_abort(&empty[st], ((kt / CSTAGES) - 1) & 1, limit, abort_flag)) {
                        atomicExch(abort_flag, 1);
                        stop = true;
                        break;
                    }
                    if (*(volatile int *)abort_flag) {
                        stop = true;
                        break;
                    }
                    ++fills[st];
                    unsigned char *stg = sm + st * CSTAGE_BYTES;
                    mbar_expect_tx(&full[st], CSTAGE_BYTES);
                    bulk_copy(stg, P + pack_offset(kt, 0, R0, prow), A_PLANE, &full[st]);
                    bulk_copy(stg + A_PLANE, P + pack_offset(kt, 1, R0, prow), A_PLANE, &full[st]);
                    bulk_copy(stg + 2 * A_PLANE, P + pack_offset(kt, 0, c0, prow), B_PLANE, &full[st]);
                    bulk_copy(stg + 2 * A_PLANE + B_PLANE, P + pack_offset(kt, 1, c0, prow), B_PLANE, &full[st]);
                }
                if (stop) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && nk > 0) {
            // column block j accumulates into TMEM columns 64 (j & 1): two
            // accumulators, so the epilogue subtracts block j in FP32 while
            // the products of block j + 1 run (the update order of the
            // right-looking factorization, one 64-column block at a time)
            const uint32_t idesc = tc::idesc_tf32(CM, CN);
            bool ok = true;
            for (int j = 0; j < c && ok; ++j) {
                const int b = j & 1;
                if (j >= 2 && !mbar_wait_or_abort(&tempty[b], ((j >> 1) - 1) & 1, limit, abort_flag)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(CN * b);
                for (int h = 0; h < 2; ++h) {
                    const int kt = 2 * j + h, st = kt % CSTAGES;
                    if (!mbar_wait_or_abort(&full[st], (kt / CSTAGES) & 1, limit, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_u32(sm + st * CSTAGE_BYTES);
#pragma unroll
                    for (int q = 0; q < CKC / 8; ++q) {
                        const uint64_t ah = tc::desc_kmajor_sw128(a0 + 32 * q);
                        const uint64_t al = tc::desc_kmajor_sw128(a0 + A_PLANE + 32 * q);
                        const uint64_t bh = tc::desc_kmajor_sw128(a0 + 2 * A_PLANE + 32 * q);
                        const uint64_t bl = tc::desc_kmajor_sw128(a0 + 2 * A_PLANE + B_PLANE + 32 * q);
                        tc::mma_tf32(acc, ah, bh, idesc, (h > 0 || q > 0) ? 1u : 0u);
                        tc::mma_tf32(acc, ah, bl, idesc, 1u);
                        tc::mma_tf32(acc, al, bh, idesc, 1u);
                    }
                    tc::mma_commit(&empty[st]);
                }
                if (ok) tc::mma_commit(&tfull[b]);
            }
            if (!ok) atomicExch(abort_flag, 1);
            // arrives once every MMA issued above has completed (also after
            // an abort, so that none is in flight when TMEM is freed)
            tc::mma_commit(done);
        }
    } else {
        // X = F - acc for this thread's row and 32 columns; entries above the
        // diagonal, padding rows [k, kp) and rows past the front are zero
        const int r = R0 + lr;
        const bool rowok = r < mp && !(r >= k && r < kp);
        const int ncol = rowok ? max(0, min(min(32, nbc - cb), r - c0 - cb + 1)) : 0;
        const float *rowp = front + d.foff[s] + (int64_t)(c0 + cb) * ld + r;
#pragma unroll
        for (int i = 0; i < 32; ++i) cur[i] = (i < ncol) ? rowp[(int64_t)i * ld] : 0.0f;
        for (int j = 0; j < c; ++j) {
            // X -= L(tile rows, block j) L(block c rows, block j)^T, rounded in FP32
            const int b = j & 1;
            bool ok = mbar_wait_or_abort(&tfull[b], (j >> 1) & 1, limit, abort_flag);
            tc::tc_fence_after();
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) atomicExch(abort_flag, 1);
                break;
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(CN * b) + cb + 16 * q, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) cur[16 * q + i] -= v[i];
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[b]);
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) cur[i] = (i < ncol) ? cur[i] : 0.0f;
        if (nk > 0) {
            // every product has completed before TMEM is given up
            const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(done, 0, limit));
            if (!ok && lane == 0) atomicExch(abort_flag, 1);
        }
        if (a.gate != nullptr && tid == 64) {
            // test of the timeout path: a gate that nothing opens
            bool open = false;
            for (uint32_t i = 0; i < limit && !open; ++i) {
                open = *(volatile const unsigned *)a.gate != 0u;
                if (!open) __nanosleep(256);
            }
            if (!open) atomicExch(abort_flag, 1);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    bool aborted = *(volatile int *)abort_flag != 0;
    bool lcopy = false, panel = false;     // tid 0: B operand copy issued; all: panel product entered
    unsigned char *Lp = a.lpack + (d.dinvoff[s] / (NB * NB) + c) * (int64_t)LPACK;   // published L11^-1 operand
    unsigned char *Bs = sm + BOP_OFF;
    if (!aborted) {
        if (ti == 0) {
            // ---- diagonal task: L11 = chol(X11) and L11^-1 -------------------------------
            float *Bk = reinterpret_cast<float *>(sm);
            float(*A11)[NB + 1] = reinterpret_cast<float(*)[NB + 1]>(Bk);
            float *XT = Bk + blk::BP_XT;
            // the epilogue threads keep their rows of X in registers meanwhile
            if (warp >= 2) {
                if (lr < NB) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) A11[lr][cb + i] = (lr < nbc) ? cur[i] : 0.0f;
                }
            }
            for (int idx = tid; idx < NB * blk::XLD; idx += CT) XT[idx] = 0.0f;
            __syncthreads();
            blk::block_potrf_inv<float, CT>(nbc, d.sfirst[s] + c0, a.status, Bk);
            // L11^-1 as the B operand: to the column's other tasks (global) and
            // to this task's own panel product (shared memory)
            for (int q = tid; q < NB * (NB / 4); q += CT) {
                const int n = q % NB, g = q / NB;           // row of L11^-1, group of 4 columns
                const int ch = g / 8, gg = g % 8;
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)   // XT's strictly upper part holds scratch products
                    tc::split_tf32((4 * g + j <= n) ? XT[(4 * g + j) * blk::XLD + n] : 0.0f, hi[j], lo[j]);
                const int off = n * 128 + ((gg ^ (n & 7)) * 16);
                const uint4 vh = make_uint4(hi[0], hi[1], hi[2], hi[3]), vl = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                *reinterpret_cast<uint4 *>(Lp + (2 * ch) * B_PLANE + off) = vh;
                *reinterpret_cast<uint4 *>(Lp + (2 * ch + 1) * B_PLANE + off) = vl;
                *reinterpret_cast<uint4 *>(Bs + (2 * ch) * B_PLANE + off) = vh;
                *reinterpret_cast<uint4 *>(Bs + (2 * ch + 1) * B_PLANE + off) = vl;
            }
            fence_proxy_async_global();
            __syncthreads();
            if (tid == 0) {
                // the barrier orders the block's stores before this release
                st_release(diagf + c, 1u);
            }
            // L11 into the front; L11^-1 (column-major) for the solves
            float *Fm = front + d.foff[s];
            float *Dv = a.dinv + d.dinvoff[s] + (int64_t)c * NB * NB;
            for (int idx = tid; idx < NB * NB; idx += CT) {
                const int rr = idx % NB, cc = idx / NB;
                if (rr >= cc && rr < nbc) Fm[(int64_t)(c0 + cc) * ld + c0 + rr] = A11[rr][cc];
                Dv[idx] = (rr >= cc) ? XT[cc * blk::XLD + rr] : 0.0f;
            }
            // (the diagonal block's rows of the product below are not used)
            __syncthreads();
        } else {
            // ---- other tasks: wait for L11^-1 of the block and fetch it ---------------
            if (tid == 0) {
                bool ok = wait_flag(diagf + c, limit, a.gabort);
                if (ok) {
                    fence_proxy_async_global();
                    mbar_expect_tx(lbar, LPACK);
                    bulk_copy(Bs, Lp, LPACK, lbar);
                    lcopy = true;
                } else {
                    *abort_flag = 1;
                }
            }
        }
        // ---- the tile as the A operand (tf32 hi / lo, swizzled) ------------------------
        if (warp >= 2) {
            const int atom = (lr >> 3) * 1024 + (lr & 7) * 128;
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                uint32_t hi[4], lo[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) tc::split_tf32(cur[4 * g + j], hi[j], lo[j]);
                const int off = atom + ((g ^ (lr & 7)) * 16);
                *reinterpret_cast<uint4 *>(sm + (2 * half) * A_PLANE + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                *reinterpret_cast<uint4 *>(sm + (2 * half + 1) * A_PLANE + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            }
        }
        tc::fence_async_smem();
        __syncthreads();
        aborted = *(volatile int *)abort_flag != 0;
    }
    if (!aborted) {
        // ---- panel product L(tile rows, block c) = X L11^-T on the tensor cores ---------
        panel = true;
        if (warp == 1 && lane == 0) {
            bool ok = ti == 0 || mbar_wait_or_abort(lbar, 0, limit, abort_flag);
            if (ok) {
                tc::tc_fence_after();
                const uint32_t idesc = tc::idesc_tf32(CM, CN);
                const uint32_t a0 = tc::smem_u32(sm), b0 = tc::smem_u32(Bs);
#pragma unroll
                for (int ch = 0; ch < 2; ++ch)
#pragma unroll
                    for (int q = 0; q < CKC / 8; ++q) {
                        const uint64_t ah = tc::desc_kmajor_sw128(a0 + (2 * ch) * A_PLANE + 32 * q);
                        const uint64_t al = tc::desc_kmajor_sw128(a0 + (2 * ch + 1) * A_PLANE + 32 * q);
                        const uint64_t bh = tc::desc_kmajor_sw128(b0 + (2 * ch) * B_PLANE + 32 * q);
                        const uint64_t bl = tc::desc_kmajor_sw128(b0 + (2 * ch + 1) * B_PLANE + 32 * q);
                        tc::mma_tf32(tmem, ah, bh, idesc, (ch > 0 || q > 0) ? 1u : 0u);
                        tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                        tc::mma_tf32(tmem, al, bh, idesc, 1u);
                    }
            } else {
                atomicExch(abort_flag, 1);
            }
            tc::mma_commit(pdone);
        }
        float v[32];
        const int r = R0 + lr;
        const bool mine = warp >= 2 && r < mp && (ti > 0 || lr >= nbc);   // a panel row of this thread
        if (warp >= 2) {
            const bool ok = __all_sync(0xffffffffu, mbar_wait_or_abort(pdone, 0, limit, abort_flag));
            tc::tc_fence_after();
            if (ok && *(volatile int *)abort_flag == 0) {
                tc::tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + cb, *reinterpret_cast<float(*)[16]>(v));
                tc::tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + cb + 16, *reinterpret_cast<float(*)[16]>(v + 16));
                if (mine) {
                    // this row's 128-byte line of chunk 2c + half (columns past
                    // nbc are zero): what the later tasks read
                    const int kc = 2 * c + half;
                    unsigned char *Lh = P + pack_offset(kc, 0, r, prow), *Ll = P + pack_offset(kc, 1, r, prow);
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        uint32_t hi[4], lo[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) tc::split_tf32(v[4 * g + j], hi[j], lo[j]);
                        const int off = (g ^ (r & 7)) * 16;
                        *reinterpret_cast<uint4 *>(Lh + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                        *reinterpret_cast<uint4 *>(Ll + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                    }
                }
            } else if (lane == 0) {
                atomicExch(abort_flag, 1);
            }
            fence_proxy_async_global();
        }
        tc::tc_fence_before();
        __syncthreads();
        aborted = *(volatile int *)abort_flag != 0;
        if (!aborted) {
            if (tid == 0) {
                // the barrier orders the block's stores before these releases
                unsigned *fc = fl + c * nrb + R0 / NB;
                st_release(fc, 1u);
                st_release(fc + 1, 1u);
            }
            // the FP32 panel rows into the front (read by the solves only),
            // column-major: a warp's stores cover 32 consecutive rows
            if (mine) {
                float *Fr = front + d.foff[s] + (int64_t)(c0 + cb) * ld + r;
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (cb + i < nbc) Fr[(int64_t)i * ld] = v[i];
            }
        }
    }
    if (aborted && tid == 0) {
        // every issued fill and copy has landed and every issued MMA has
        // completed before the shared memory and TMEM are given up
        for (int st = 0; st < CSTAGES; ++st)
            if (fills[st] > 0) tc::mbar_wait(&full[st], (fills[st] - 1) & 1, DRAIN_LIMIT);
        if (nk > 0) tc::mbar_wait(done, 0, DRAIN_LIMIT);
        if (lcopy) tc::mbar_wait(lbar, 0, DRAIN_LIMIT);
        if (panel) tc::mbar_wait(pdone, 0, DRAIN_LIMIT);
        atomicMax(a.tstatus, 1ull);
        atomicExch(a.gabort, 1u);
    }
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 1) tc::tmem_dealloc(tmem, 2 * CN);
}

}  // namespace

size_t tc_chain_smem() { return (size_t)DATA_BYTES + 1024 + 128; }

void init_chain_attributes() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(tc_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_chain_smem());
    done = true;
}

void launch_tc_chain(const DevSym &d, float *front, unsigned char *pk, const int4 *items, int count, int level,
                     const ChainArgs &a, cudaStream_t st) {
    if (count <= 0) return;
    init_chain_attributes();
    tc_chain_kernel<<<count, CT, tc_chain_smem(), st>>>(d, front, pk, items, count, level, a);
}

}  // namespace wd
