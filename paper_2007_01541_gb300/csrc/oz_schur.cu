// Schur updates of FP64 fronts on the 5th-generation tensor cores, emulating
// FP64 with bf16 slices (the splitting scheme of Ozaki et al.): the FP64
// counterpart of the 3xTF32 updates of the FP32 fronts, for the update
// C -= L21 L21^T of the block form of P A P^T = L L^T (Section 4).
//
// Slicing.  After the panel of pivot block b is final, every panel row r of
// the block (64 values) gets a scale 2^e_r >= max |L_rk| and is written as
// eight integer digits of 7 bits, L_rk = 2^e_r sum_i q_i(r, k) 2^(-7 i),
// i = 1..8 (|q_1| <= 128, |q_i| <= 64 else, each exact in bf16; the rounding
// of the last digit is 2^-57 of the scale).  The digits go to eight bf16
// planes in the 128-byte-swizzled K-major layout of the MMA operands (one
// 128-byte line per row and plane, 64 values), the scales to an int16 array.
//
// Product.  For rows r and columns c of a tile,
//   sum_k L_rk L_ck = 2^(e_r + e_c) sum_d 2^(-7 d) D_d(r, c),
//   D_d = sum_{i + j = d} sum_k q_i(r, k) q_j(c, k),   d = 2..9,
// where every D_d is an integer below 2^23 in magnitude (at most 8 slice
// pairs, 64 terms, products below 2^14), so it accumulates EXACTLY in the
// FP32 accumulators of the MMA, in any order.  The pairs with i + j > 9 are
// dropped: at most 2^-47 of 2^(e_r + e_c) per 64-column block, at the level
// of FP64's own rounding bound for such a sum (64 u max|L_r| max|L_c|).  The
// 36 slice-pair products of a 64-column block are 144 tcgen05.mma kind::f16
// instructions (128 x 64 x 16 each) into eight TMEM accumulators of 64
// columns (all 512 columns of the SM's tensor memory).  The epilogue reads
// them, adds the eight terms in double-float arithmetic on the FP32 pipes
// (exact powers of two as scales, TwoSum), turns the pair into two doubles
// scaled by 2^(e_r + e_c) with integer operations on the bits, and adds them
// to an FP64 register accumulator (two FP64 additions: GB300's FP64 pipe is
// the scarce one); after the last block C -= acc in FP64.
//
// One CTA per 128 x 64 output tile (the tiles of the SIMT FP64 kernel):
//   warp 0: producer (bulk copies of the 8 + 8 slice planes of a block)
//   warp 1: allocates the 512 TMEM columns; one lane issues the MMAs
//   warps 2-9: epilogue, a thread = one row and 32 columns
// mode 0: the pivot-block update of step kb (one block), after which the CTA
// of tile (0, 0) factors the next diagonal block (FP64, as the SIMT kernel);
// mode 1: the fronts' trailing blocks (all blocks of the supernode).
//
// Every wait is bounded; on expiry the CTA records the timeout status, waits
// (with a fixed bound) for its copies and products in flight, frees its TMEM
// and returns without writing its tile.
#include <cuda_bf16.h>

#include "dev_common.cuh"
#include "engine.h"
#include "front_block.cuh"
#include "tc_common.cuh"

namespace wd {
namespace {

constexpr int OM = 128, ON = 64;                 // tile rows, columns (one 64-column block of K per pass)
constexpr int NSL = 8;                           // slices (digits of 7 bits)
constexpr int NACC = 8;                          // accumulators: d = i + j = 2..9
constexpr int A_PLANE = OM * 128;                // 16 KB: 128 rows x 64 bf16
constexpr int B_PLANE = ON * 128;                // 8 KB
constexpr int STAGE = NSL * (A_PLANE + B_PLANE); // 192 KB
constexpr int OZ_THREADS = 320;
constexpr uint32_t WAIT_LIMIT = 1u << 26;
constexpr uint32_t DRAIN_LIMIT = 1u << 26;
static_assert(STAGE >= (int)blk::block_smem_bytes<double>(), "the stage holds the block factorization");

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
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::smem_u32(bar)) : "memory");
}

// 2^e as a double (0 below the normal range)
__device__ __forceinline__ double pow2(int e) {
    return e < -1022 ? 0.0 : __longlong_as_double((long long)(1023 + min(e, 1023)) << 52);
}

// f 2^e as a double, built from f's bits on the integer pipes (no FP64
// conversion or multiply): zero and FP32 subnormals give 0, so do results
// below the FP64 normal range
__device__ __forceinline__ double f2d_scaled(float f, int e) {
    const uint32_t u = __float_as_uint(f);
    const int ex = (int)((u >> 23) & 0xFFu) - 127 + 1023 + e;
    const bool zero = ((u >> 23) & 0xFFu) == 0u || ex < 1;
    const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)min(ex, 2046) << 52) |
                          ((uint64_t)(u & 0x7FFFFFu) << 29);
    return zero ? 0.0 : __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void two_sum(float &h, float &l, float t) {
    const float s = __fadd_rn(h, t);
    const float bb = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(t, bb));
    h = s;
    l = __fadd_rn(l, err);
}

// ---------------------------------------------------------------------------
// slices of the panel rows of pivot block kb (the panel kernel's items: 64
// rows per CTA, one warp per row at a time, lane l columns 2l and 2l + 1)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) oz_slice_kernel(DevSym d, const double *__restrict__ front, OzArgs a,
                                                       const int4 *__restrict__ items, int kb) {
    const int4 it = items[blockIdx.x];
    const int s = it.x, rb = it.y;
    const int k = d.sk[s], m = d.sm[s], kp = d.skp[s], ld = d.sld[s];
    const int mp = kp + m - k;
    const int nb = min(NB, k - kb), t0 = kb + nb;
    const int r0 = (t0 == k ? kp : t0) + rb * RB;
    const int srow = pack_rows(mp), bb = kb / NB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double *F = front + d.foff[s] + (int64_t)kb * ld;
    unsigned char *Sl = a.sl + a.soff[s];
    int16_t *E = a.ex + a.eoff[s];
    const int c = 2 * lane;
    for (int rr = 0; rr < RB / 8; ++rr) {
        const int row = r0 + warp * (RB / 8) + rr;
        if (row >= mp) break;
        const double v0 = c < nb ? F[(int64_t)c * ld + row] : 0.0;
        const double v1 = c + 1 < nb ? F[(int64_t)(c + 1) * ld + row] : 0.0;
        double mx = fmax(fabs(v0), fabs(v1));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const int e = mx > 0.0 ? ilogb(mx) + 1 : 0;   // 2^e > max |v|
        const double sc = pow2(56 - e);
        long long x0 = __double2ll_rn(v0 * sc), x1 = __double2ll_rn(v1 * sc);   // |x| <= 2^56
        const int64_t line0 = ((int64_t)bb * NSL * srow + row) * 128;
        const int off = ((lane >> 2) ^ (row & 7)) * 16 + (c & 7) * 2;
#pragma unroll
        for (int q = 0; q < NSL; ++q) {
            const int sh = 49 - 7 * q;
            long long q0 = x0, q1 = x1;
            if (sh > 0) {
                q0 = (x0 + (1LL << (sh - 1))) >> sh;   // nearest digit (ties up)
                q1 = (x1 + (1LL << (sh - 1))) >> sh;
            }
            x0 -= q0 * (1LL << sh);
            x1 -= q1 * (1LL << sh);
            const __nv_bfloat162 pr = __floats2bfloat162_rn((float)q0, (float)q1);
            *reinterpret_cast<__nv_bfloat162 *>(Sl + line0 + (int64_t)q * srow * 128 + off) = pr;
        }
        if (lane == 0) E[(int64_t)bb * srow + row] = (int16_t)e;
    }
}

// ---------------------------------------------------------------------------
// the product (see the header); mode 0: base = kb + NB, block kb / NB,
// cmax = k; mode 1: base = kp, blocks 0 .. ceil(k / NB) - 1, cmax = mp
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_schur_kernel(DevSym d, double *__restrict__ front,
                                                                 const int4 *__restrict__ items, int kb, int mode,
                                                                 OzArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + STAGE);
    uint64_t *mdone = full + 1;   // a block's MMAs completed: the epilogue may read TMEM
    uint64_t *sfree = full + 2;   // a block's MMAs completed: the producer may refill the stage
    uint64_t *tfree = full + 3;   // the epilogue has read a block's accumulators
    uint64_t *fin = full + 4;     // every MMA issued has completed (committed once, at the end)
    uint32_t *tslot = reinterpret_cast<uint32_t *>(full + 5);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    const uint32_t limit = a.wait_limit ? a.wait_limit : WAIT_LIMIT;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int4 it = items[blockIdx.x];
    const int s = it.x, ti = it.y, tj = it.z;
    const int k = d.sk[s], m = d.sm[s], kp = d.skp[s], ld = d.sld[s];
    const int mp = kp + m - k;
    const int base = mode == 0 ? kb + NB : kp;
    const int b0 = mode == 0 ? kb / NB : 0;
    const int nblk = mode == 0 ? 1 : (k + NB - 1) / NB;
    const int cmax = mode == 0 ? k : mp;
    const int r0 = base + ti * OM, c0 = base + tj * ON;
    const int srow = pack_rows(mp);
    const unsigned char *Sl = a.sl + a.soff[s];
    const int16_t *E = a.ex + a.eoff[s];

    if (tid == 0) {
        tc::mbar_init(full, 1);
        tc::mbar_init(mdone, 1);
        tc::mbar_init(sfree, 1);
        tc::mbar_init(tfree, 8);
        tc::mbar_init(fin, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) tc::tmem_alloc(tslot, 512);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tslot;

    int fills = 0;     // producer lane: blocks whose copies were issued
    if (warp == 0) {
        if (lane == 0) {
            for (int b = 0; b < nblk; ++b) {
                if (b > 0 && !tc::mbar_wait(sfree, (b - 1) & 1, limit)) {
                    atomicExch(abort_flag, 1);
                    break;
                }
                if (*(volatile int *)abort_flag) break;
                const int64_t blk0 = (int64_t)(b0 + b) * NSL * srow;
                mbar_expect_tx(full, STAGE);
                for (int q = 0; q < NSL; ++q)
                    bulk_copy(sm + q * A_PLANE, Sl + (blk0 + (int64_t)q * srow + r0) * 128, A_PLANE, full);
                for (int q = 0; q < NSL; ++q)
                    bulk_copy(sm + NSL * A_PLANE + q * B_PLANE, Sl + (blk0 + (int64_t)q * srow + c0) * 128, B_PLANE,
                              full);
                ++fills;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(OM, ON);
            const uint32_t sa = tc::smem_u32(sm), sb = tc::smem_u32(sm + NSL * A_PLANE);
            for (int b = 0; b < nblk; ++b) {
                if (!tc::mbar_wait(full, b & 1, limit) || (b > 0 && !tc::mbar_wait(tfree, (b - 1) & 1, limit))) {
                    atomicExch(abort_flag, 1);
                    break;
                }
                tc::tc_fence_after();
#pragma unroll 1
                for (int dd = 0; dd < NACC; ++dd) {
                    const int dsum = dd + 2;
                    const uint32_t acc = tmem + dd * ON;
                    uint32_t accum = 0u;
                    for (int i = max(1, dsum - NSL); i <= min(NSL, dsum - 1); ++i) {
                        const int j = dsum - i;
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            const uint64_t ad = tc::desc_kmajor_sw128(sa + (i - 1) * A_PLANE + 32 * ks);
                            const uint64_t bd = tc::desc_kmajor_sw128(sb + (j - 1) * B_PLANE + 32 * ks);
                            tc::mma_bf16(acc, ad, bd, idesc, accum);
                            accum = 1u;
                        }
                    }
                }
                tc::mma_commit(mdone);
                tc::mma_commit(sfree);
            }
            // also after a timeout, so that no product is in flight when TMEM is freed
            tc::mma_commit(fin);
        }
    } else {
        // epilogue: TMEM lane group = warp % 4 (32 rows), column half = (warp - 2) / 4
        const int lg = warp & 3, half = (warp - 2) >> 2;
        const int r = r0 + 32 * lg + lane;
        const int cb = c0 + 32 * half;
        double acc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = 0.0;
        bool ok = true;
        for (int b = 0; b < nblk && ok; ++b) {
            ok = tc::mbar_wait(mdone, b & 1, limit) && *(volatile int *)abort_flag == 0;
            if (!ok) break;
            tc::tc_fence_after();
            const int16_t *Eb = E + (int64_t)(b0 + b) * srow;
            const int er = Eb[r];   // rows up to mp + 127 exist (zero scales past mp)
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float D[NACC][8];
#pragma unroll
                for (int dd = 0; dd < NACC; ++dd)
                    tc::tmem_ld8(tmem + ((uint32_t)(32 * lg) << 16) + dd * ON + 32 * half + 8 * g, D[dd]);
#pragma unroll
                for (int cc = 0; cc < 8; ++cc) {
                    // sum_d 2^(-7 d) D_d, smallest term first
                    float h = D[NACC - 1][cc] * 0x1p-63f, l = 0.0f;
#pragma unroll
                    for (int dd = NACC - 2; dd >= 0; --dd) two_sum(h, l, D[dd][cc] * __int_as_float((127 - 7 * (dd + 2)) << 23));
                    const int esc = er + Eb[cb + 8 * g + cc];
                    acc[8 * g + cc] += f2d_scaled(h, esc);
                    acc[8 * g + cc] += f2d_scaled(l, esc);
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tfree);
        }
        if (!ok) {
            if (lane == 0) atomicExch(abort_flag, 1);
        } else if (r < mp) {
            double *rowp = front + d.foff[s] + (int64_t)cb * ld + r;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int c = cb + i;
                if (c <= r && c < cmax) rowp[(int64_t)i * ld] -= acc[i];
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    const bool aborted = *(volatile int *)abort_flag != 0;
    if (aborted && tid == 0) {
        // after a timeout: the issued copies have landed and the issued MMAs
        // have completed before the shared memory and TMEM are given up
        if (fills > 0) tc::mbar_wait(full, (fills - 1) & 1, DRAIN_LIMIT);
        tc::mbar_wait(fin, 0, DRAIN_LIMIT);
    }
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 1) tc::tmem_dealloc(tmem, 512);
    if (aborted) {
        if (tid == 0) atomicMax(a.tstatus, 1ull);
        return;
    }
    if (mode == 0 && ti == 0 && tj == 0 && kb + NB < k) {
        // the next diagonal block lies inside this tile, written above
        blk::factor_diag_block<double, double, OZ_THREADS>(d, front, a.dinv, s, kb + NB, a.status, sm);
    }
}

constexpr size_t oz_smem() { return (size_t)STAGE + 1024 + 128; }

}  // namespace

void init_oz_attributes() {
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(oz_schur_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem());
    done = true;
}

void launch_oz_slice(const DevSym &d, const double *front, const OzArgs &a, const int4 *items, int count, int kb,
                     cudaStream_t st) {
    if (count > 0) oz_slice_kernel<<<count, 256, 0, st>>>(d, front, a, items, kb);
}

void launch_oz_schur(const DevSym &d, double *front, const int4 *items, int count, int kb, int mode,
                     const OzArgs &a, cudaStream_t st) {
    if (count <= 0) return;
    init_oz_attributes();
    oz_schur_kernel<<<count, OZ_THREADS, oz_smem(), st>>>(d, front, items, kb, mode, a);
}

}  // namespace wd
