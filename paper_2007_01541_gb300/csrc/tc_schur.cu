// Schur updates of FP32 fronts on the 5th-generation tensor cores (tcgen05),
// 3xTF32: every L value x is split into x = hi + lo (tf32 each) and
//   C -= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
// with FP32 accumulation in tensor memory (the lo*lo term is dropped), which
// keeps FP32-level accuracy (the mixed path is then refined in FP64).
//
// Operands come pre-split and pre-swizzled: when the panel kernel finishes a
// block of L it also writes the block's rows as tf32 hi/lo lines in the
// 128-byte-swizzled K-major layout of the MMA (see pack_offset below), so a
// 128-row x 32-column operand tile is one contiguous 16 KB range that the
// Tensor Memory Accelerator copies into shared memory with a single bulk copy.
//
// One CTA per 128 x 128 output tile, warp-specialized:
//   warp 0: producer (bulk copies of A_hi, A_lo, B_hi, B_lo per 32-wide
//           chunk of the inner dimension into a 3-stage ring)
//   warp 1: allocates 128 TMEM columns; one lane issues the 12 MMAs of a
//           chunk and commits them to the stage's "empty" barrier
//   warps 2-9: epilogue, each thread one row and 64 columns of the tile: its
//           part of C is loaded into registers while the MMAs run, then
//           C -= acc (TMEM -> registers), lower part only
// In mode 0 (the pivot-column update of step kb) the CTA of tile (0, 0),
// which holds the whole next diagonal block, then factors that block with all
// its threads (L11 and L11^-1 of step kb + 64, in FP64 for wide fronts), so
// the next panel launch only multiplies by the stored inverse.
//
// Every wait is bounded (wait_limit polls); on expiry the CTA records the
// timeout status, waits (with a fixed bound) for its copies and products in
// flight, frees its TMEM and returns without writing its tile.
#include "engine.h"
#include "front_block.cuh"
#include "tc_common.cuh"

namespace wd {
namespace {

constexpr int TBM = 128, TBN = 128, TBK = 32;
constexpr int STAGES = 3;
constexpr int TILE_BYTES = TBM * TBK * 4;           // 16 KB per operand plane
constexpr int STAGE_BYTES = 4 * TILE_BYTES;          // A hi, A lo, B hi, B lo
constexpr int TC_THREADS = 320;
constexpr uint32_t WAIT_LIMIT = 1u << 26;    // default bound of a wait (polls)
constexpr uint32_t DRAIN_LIMIT = 1u << 26;   // bound of the waits for work in flight after a timeout
static_assert(STAGES * STAGE_BYTES >= blk::block_smem_bytes<double>(), "the stages hold the block factorization");

__device__ __forceinline__ void bulk_copy(void *dst_smem, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
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

// HAS64: the launch may factor diagonal blocks in FP64 (instantiated apart,
// so that the usual FP32 kernel carries only the FP32 block factorization)
template <bool HAS64>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_schur_kernel(DevSym d, float *__restrict__ front, const unsigned char *__restrict__ pk,
                    const int4 *__restrict__ items, int kb, int mode, TcArgs a) {
    const uint32_t limit = a.wait_limit ? a.wait_limit : WAIT_LIMIT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 it = items[blockIdx.x];
    const int s = it.x, ti = it.y, tj = it.z;
    const int k = d.sk[s], m = d.sm[s], kp = d.skp[s], ld = d.sld[s];
    const int mp = kp + m - k;
    int base, ka, K, cmax;
    if (mode == 0) {
        base = kb + NB;
        ka = kb;
        K = NB;
        cmax = k;
    } else {
        base = kp;
        ka = 0;
        K = k;
        cmax = mp;
    }
    const int r0 = base + ti * TBM, c0 = base + tj * TBN;
    const int nk = (K + TBK - 1) / TBK;
    const int prow = pack_rows(mp);
    const unsigned char *P = pk + d.pkoff[s];

    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) tc::tmem_alloc(tslot, TBN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    int fills[STAGES] = {};   // producer lane: fills issued per stage
    if (warp == 0) {
        if (lane == 0) {
            for (int kt = 0; kt < nk; ++kt) {
                const int st = kt % STAGES;
                if (kt >= STAGES && !tc::mbar_wait(&empty[st], ((kt / STAGES) - 1) & 1, limit)) {
                    atomicExch(abort_flag, 1);
                    break;
                }
                if (*(volatile int *)abort_flag) break;
                ++fills[st];
                unsigned char *stg = sm + st * STAGE_BYTES;
                const int kc = (ka / TBK) + kt;
                mbar_expect_tx(&full[st], STAGE_BYTES);
                bulk_copy(stg, P + pack_offset(kc, 0, r0, prow), TILE_BYTES, &full[st]);
                bulk_copy(stg + TILE_BYTES, P + pack_offset(kc, 1, r0, prow), TILE_BYTES, &full[st]);
                bulk_copy(stg + 2 * TILE_BYTES, P + pack_offset(kc, 0, c0, prow), TILE_BYTES, &full[st]);
                bulk_copy(stg + 3 * TILE_BYTES, P + pack_offset(kc, 1, c0, prow), TILE_BYTES, &full[st]);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(TBM, TBN);
            bool ok = true;
            for (int kt = 0; kt < nk; ++kt) {
                const int st = kt % STAGES;
                if (!tc::mbar_wait(&full[st], (kt / STAGES) & 1, limit)) {
                    atomicExch(abort_flag, 1);
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t a0 = tc::smem_u32(sm + st * STAGE_BYTES);
#pragma unroll
                for (int j = 0; j < TBK / 8; ++j) {
                    const uint64_t ah = tc::desc_kmajor_sw128(a0 + 32 * j);
                    const uint64_t al = tc::desc_kmajor_sw128(a0 + TILE_BYTES + 32 * j);
                    const uint64_t bh = tc::desc_kmajor_sw128(a0 + 2 * TILE_BYTES + 32 * j);
                    const uint64_t bl = tc::desc_kmajor_sw128(a0 + 3 * TILE_BYTES + 32 * j);
                    tc::mma_tf32(tmem, ah, bh, idesc, (kt > 0 || j > 0) ? 1u : 0u);
                    tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                    tc::mma_tf32(tmem, al, bh, idesc, 1u);
                }
                tc::mma_commit(&empty[st]);
            }
            // arrives once every MMA issued above has completed (also after a
            // timeout, so that no product is in flight when TMEM is freed)
            tc::mma_commit(done);
            (void)ok;
        }
    } else {
        // epilogue: warps 2..9; TMEM lane group = warp % 4, column half = (warp - 2) / 4
        const int lg = warp & 3, half = (warp - 2) >> 2;
        const int r = r0 + 32 * lg + lane;
        const int cb0 = c0 + 64 * half;
        // this thread's row of the tile, columns cb0 .. cb0+63 (stride ld)
        float *rowp = front + d.foff[s] + (int64_t)cb0 * ld + r;
        const int cend = min(64, cmax - cb0);     // columns below cmax
        const int cdiag = r - cb0 + 1;            // columns with c <= r
        const int nc = (r < mp) ? max(0, min(cend, cdiag)) : 0;
        float cur[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) cur[i] = (i < nc) ? rowp[i * ld] : 0.0f;
        bool ok = tc::mbar_wait(done, 0, limit);
        tc::tc_fence_after();
        if (ok && a.gate != nullptr) {
            // test of the timeout path: a gate that nothing opens
            int open = 0;
            if (lane == 0)
                for (uint32_t i = 0; i < limit && !open; ++i) {
                    open = *(volatile const unsigned *)a.gate != 0u;
                    if (!open) __nanosleep(256);
                }
            ok = __shfl_sync(0xffffffffu, open, 0) != 0;
        }
        if (ok && *(volatile int *)abort_flag == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + 64 * half + 16 * q, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) cur[16 * q + i] -= v[i];
            }
#pragma unroll
            for (int i = 0; i < 64; ++i)
                if (i < nc) rowp[i * ld] = cur[i];
        } else if (lane == 0) {
            atomicExch(abort_flag, 1);
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    const bool aborted = *(volatile int *)abort_flag != 0;
    if (aborted && tid == 0) {
        // after a timeout: every issued fill has landed and every issued MMA
        // has completed before the shared memory and TMEM are given up
        for (int st = 0; st < STAGES; ++st)
            if (fills[st] > 0) tc::mbar_wait(&full[st], (fills[st] - 1) & 1, DRAIN_LIMIT);
        tc::mbar_wait(done, 0, DRAIN_LIMIT);
    }
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 1) tc::tmem_dealloc(tmem, TBN);
    if (aborted) {
        if (tid == 0) atomicMax(a.tstatus, 1ull);
        return;
    }
    if (mode == 0 && ti == 0 && tj == 0 && kb + NB < k) {
        // the next diagonal block lies inside this tile, written above
        if (HAS64 && a.diag64_min_k > 0 && k >= a.diag64_min_k)
            blk::factor_diag_block<double, float, TC_THREADS>(d, front, a.dinv, s, kb + NB, a.status, sm);
        else
            blk::factor_diag_block<float, float, TC_THREADS>(d, front, a.dinv, s, kb + NB, a.status, sm);
    }
}


// The fronts' trailing blocks (mode 1, U = F22 - L21 L21^T with K = k) as a
// persistent launch: one CTA per SM takes the tiles blockIdx.x, blockIdx.x +
// gridDim.x, ...  The stage ring runs on across tiles, and two TMEM
// accumulators alternate, so a tile's epilogue (read-modify-write of its
// part of C) overlaps the next tile's copies and products; the per-CTA
// set-up (barriers, TMEM allocation) is paid once per SM instead of once per
// tile, which is what the many narrow fronts of the deep levels (K <= 64,
// two chunks per tile) spent their time on.  Arithmetic and bounded waits as
// in tc_schur_kernel.
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_syrk_persistent_kernel(DevSym d, float *__restrict__ front, const unsigned char *__restrict__ pk,
                              const int4 *__restrict__ items, int count, TcArgs a) {
    const uint32_t limit = a.wait_limit ? a.wait_limit : WAIT_LIMIT;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;      // accumulator b holds a finished tile
    uint64_t *tempty = tfull + 2;          // accumulator b has been read
    uint64_t *done = tempty + 2;           // every issued MMA has completed
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&tfull[i], 1);
            tc::mbar_init(&tempty[i], 8);   // one arrival per epilogue warp
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) tc::tmem_alloc(tslot, 2 * TBN);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    int fills[STAGES] = {};   // producer lane: fills issued per stage
    if (warp == 0) {
        if (lane == 0) {
            int kt = 0;   // chunk counter across the CTA's tiles
            for (int t = blockIdx.x; t < count && !*(volatile int *)abort_flag; t += gridDim.x) {
                const int4 it = items[t];
                const int s = it.x, k = d.sk[s], m = d.sm[s], kp = d.skp[s];
                const int mp = kp + m - k;
                const int r0 = kp + it.y * TBM, c0 = kp + it.z * TBN;
                const int nk = (k + TBK - 1) / TBK, prow = pack_rows(mp);
                const unsigned char *P = pk + d.pkoff[s];
                bool stop = false;
                for (int kc = 0; kc < nk; ++kc, ++kt) {
                    const int st = kt % STAGES;
                    if (kt >= STAGES && !tc::mbar_wait(&empty[st], ((kt / STAGES) - 1) & 1, limit)) {
                        atomicExch(abort_flag, 1);
                        stop = true;
                        break;
                    }
                    if (*(volatile int *)abort_flag) {
                        stop = true;
                        break;
                    }
                    ++fills[st];
                    unsigned char *stg = sm + st * STAGE_BYTES;
                    mbar_expect_tx(&full[st], STAGE_BYTES);
                    bulk_copy(stg, P + pack_offset(kc, 0, r0, prow), TILE_BYTES, &full[st]);
                    bulk_copy(stg + TILE_BYTES, P + pack_offset(kc, 1, r0, prow), TILE_BYTES, &full[st]);
                    bulk_copy(stg + 2 * TILE_BYTES, P + pack_offset(kc, 0, c0, prow), TILE_BYTES, &full[st]);
                    bulk_copy(stg + 3 * TILE_BYTES, P + pack_offset(kc, 1, c0, prow), TILE_BYTES, &full[st]);
                }
                if (stop) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(TBM, TBN);
            int kt = 0, i = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < count && ok; t += gridDim.x, ++i) {
                const int k = d.sk[items[t].x];
                const int nk = (k + TBK - 1) / TBK;
                const int b = i & 1;
                if (i >= 2 && !tc::mbar_wait(&tempty[b], ((i >> 1) - 1) & 1, limit)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(TBN * b);
                for (int kc = 0; kc < nk; ++kc, ++kt) {
                    const int st = kt % STAGES;
                    if (!tc::mbar_wait(&full[st], (kt / STAGES) & 1, limit) || *(volatile int *)abort_flag) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t a0 = tc::smem_u32(sm + st * STAGE_BYTES);
#pragma unroll
                    for (int j = 0; j < TBK / 8; ++j) {
                        const uint64_t ah = tc::desc_kmajor_sw128(a0 + 32 * j);
                        const uint64_t al = tc::desc_kmajor_sw128(a0 + TILE_BYTES + 32 * j);
                        const uint64_t bh = tc::desc_kmajor_sw128(a0 + 2 * TILE_BYTES + 32 * j);
                        const uint64_t bl = tc::desc_kmajor_sw128(a0 + 3 * TILE_BYTES + 32 * j);
                        tc::mma_tf32(acc, ah, bh, idesc, (kc > 0 || j > 0) ? 1u : 0u);
                        tc::mma_tf32(acc, ah, bl, idesc, 1u);
                        tc::mma_tf32(acc, al, bh, idesc, 1u);
                    }
                    tc::mma_commit(&empty[st]);
                }
                if (ok) tc::mma_commit(&tfull[b]);
            }
            if (!ok) atomicExch(abort_flag, 1);
            // arrives once every MMA issued above has completed
            tc::mma_commit(done);
        }
    } else {
        // epilogue: warps 2..9; TMEM lane group = warp % 4, column half = (warp - 2) / 4
        const int lg = warp & 3, half = (warp - 2) >> 2;
        int i = 0;
        for (int t = blockIdx.x; t < count; t += gridDim.x, ++i) {
            const int4 it = items[t];
            const int s = it.x, k = d.sk[s], m = d.sm[s], kp = d.skp[s], ld = d.sld[s];
            const int mp = kp + m - k;
            const int r0 = kp + it.y * TBM, c0 = kp + it.z * TBN;
            const int r = r0 + 32 * lg + lane;
            const int cb0 = c0 + 64 * half;
            float *rowp = front + d.foff[s] + (int64_t)cb0 * ld + r;
            const int cend = min(64, mp - cb0);
            const int nc = (r < mp) ? max(0, min(cend, r - cb0 + 1)) : 0;
            float cur[64];
#pragma unroll
            for (int q = 0; q < 64; ++q) cur[q] = (q < nc) ? rowp[q * ld] : 0.0f;
            const int b = i & 1;
            bool ok = tc::mbar_wait(&tfull[b], (i >> 1) & 1, limit);
            tc::tc_fence_after();
            if (ok && a.gate != nullptr) {
                // test of the timeout path: a gate that nothing opens
                int open = 0;
                if (lane == 0)
                    for (uint32_t g = 0; g < limit && !open; ++g) {
                        open = *(volatile const unsigned *)a.gate != 0u;
                        if (!open) __nanosleep(256);
                    }
                ok = __shfl_sync(0xffffffffu, open, 0) != 0;
            }
            ok = __all_sync(0xffffffffu, ok && *(volatile int *)abort_flag == 0);
            if (!ok) {
                if (lane == 0) atomicExch(abort_flag, 1);
                break;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(TBN * b) + 64 * half + 16 * q, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) cur[16 * q + j] -= v[j];
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[b]);
#pragma unroll
            for (int q = 0; q < 64; ++q)
                if (q < nc) rowp[q * ld] = cur[q];
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    const bool aborted = *(volatile int *)abort_flag != 0;
    if (tid == 0) {
        // every issued fill has landed and every issued MMA has completed
        // before the shared memory and TMEM are given up (after a timeout;
        // otherwise these waits return at once)
        if (aborted)
            for (int st = 0; st < STAGES; ++st)
                if (fills[st] > 0) tc::mbar_wait(&full[st], (fills[st] - 1) & 1, DRAIN_LIMIT);
        tc::mbar_wait(done, 0, DRAIN_LIMIT);
        if (aborted) atomicMax(a.tstatus, 1ull);
    }
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 1) tc::tmem_dealloc(tmem, 2 * TBN);
}
}  // namespace

size_t tc_schur_smem() { return (size_t)STAGES * STAGE_BYTES + 1024 + 128; }

void init_tc_attributes() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(tc_schur_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc_schur_smem());
    cudaFuncSetAttribute(tc_schur_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc_schur_smem());
    cudaFuncSetAttribute(tc_syrk_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc_schur_smem());
    done = true;
}

void launch_tc_schur(const DevSym &d, float *front, const unsigned char *pk, const int4 *items,
                     int count, int kb, int mode, const TcArgs &a, cudaStream_t st) {
    if (count <= 0) return;
    init_tc_attributes();
    if (mode == 1 && a.ctas > 0) {
        tc_syrk_persistent_kernel<<<min(count, a.ctas), TC_THREADS, tc_schur_smem(), st>>>(d, front, pk, items, count,
                                                                                          a);
        return;
    }
    if (a.diag64_min_k > 0 && mode == 0)
        tc_schur_kernel<true><<<count, TC_THREADS, tc_schur_smem(), st>>>(d, front, pk, items, kb, mode, a);
    else
        tc_schur_kernel<false><<<count, TC_THREADS, tc_schur_smem(), st>>>(d, front, pk, items, kb, mode, a);
}

}  // namespace wd
