// Per-instance reductions of a batch of independent systems analyzed as one
// block-diagonal matrix (wd_analyze_batch): instance i owns the permuted rows
// [coff[i], coff[i+1]) and the supernodes [soff[i], soff[i+1]).  One block per
// instance, fixed reduction order (deterministic).
#include "engine.h"

namespace wd {
namespace {

constexpr int THREADS = 256;

__device__ __forceinline__ double block_max(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = lane < THREADS / 32 ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    v = lane < THREADS / 32 ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// instance owning permuted row r: coff[i] <= r < coff[i + 1]
__device__ __forceinline__ int instance_of(const int64_t *coff, int count, int64_t r) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (coff[mid] <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

// out[inst] = max over the instance's rows of sum_j |a_ij|: the chunk items of
// the residual product (row, first entry, end, slot), one warp each; rows cut
// into several chunks leave their partial sums in partial[slot] for the finish
// kernel.  out must be zeroed; the maximum is order-independent.
__global__ void __launch_bounds__(THREADS) seg_norm_chunks_kernel(DevSym d, const int4 *__restrict__ items,
                                                                  int nchunks, double *__restrict__ partial,
                                                                  const int64_t *__restrict__ coff, int count,
                                                                  double *__restrict__ out) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nchunks) return;
    const int4 it = items[w];
    double acc = 0.0;
    for (int e = it.y + lane; e < it.z; e += 32) acc += fabs(d.csr_val[e]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        if (it.w < 0) atomic_max_nonneg(out + instance_of(coff, count, it.x), acc);
        else partial[it.w] = acc;
    }
}

// rows cut into chunks: item = (row, first slot, number of slots)
__global__ void seg_norm_finish_kernel(const int4 *__restrict__ fin, int nfin, const double *__restrict__ partial,
                                       const int64_t *__restrict__ coff, int count, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nfin) return;
    double acc = 0.0;
    for (int q = 0; q < fin[i].z; ++q) acc += partial[fin[i].y + q];
    atomic_max_nonneg(out + instance_of(coff, count, fin[i].x), acc);
}

// out[(inst * nrhs + c) * 3 + {0, 1, 2}] = max |R|, |X|, |B| over the
// instance's rows of column c (row-major n x nrhs arrays)
__global__ void __launch_bounds__(THREADS) seg_colmax3_kernel(const double *__restrict__ R,
                                                              const double *__restrict__ X,
                                                              const double *__restrict__ B,
                                                              const int64_t *__restrict__ coff, int nrhs,
                                                              double *__restrict__ out) {
    __shared__ double red[THREADS / 32];
    const int inst = blockIdx.x;
    for (int c = 0; c < nrhs; ++c) {
        double a = 0.0, b = 0.0, e = 0.0;
        for (int64_t r = coff[inst] + threadIdx.x; r < coff[inst + 1]; r += THREADS) {
            a = fmax(a, fabs(R[r * nrhs + c]));
            b = fmax(b, fabs(X[r * nrhs + c]));
            e = fmax(e, fabs(B[r * nrhs + c]));
        }
        a = block_max(a, red);
        b = block_max(b, red);
        e = block_max(e, red);
        if (threadIdx.x == 0) {
            double *o = out + ((int64_t)inst * nrhs + c) * 3;
            o[0] = a;
            o[1] = b;
            o[2] = e;
        }
    }
}

// sdl[s] = 2 sum log L_jj over the pivots of supernode s, one warp each
template <class T>
__global__ void __launch_bounds__(THREADS) snode_logdet_kernel(DevSym d, const T *__restrict__ front,
                                                               double *__restrict__ sdl) {
    const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (s >= d.ns) return;
    const int k = d.sk[s], ld = d.sld[s];
    const T *F = front + d.foff[s];
    double acc = 0.0;
    for (int j = lane; j < k; j += 32) acc += 2.0 * log((double)F[(int64_t)j * ld + j]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sdl[s] = acc;
}

// out[i] = sum of sdl over the instance's supernodes (fixed order)
__global__ void __launch_bounds__(THREADS) seg_sum_kernel(const double *__restrict__ sdl,
                                                          const int32_t *__restrict__ soff,
                                                          double *__restrict__ out) {
    __shared__ double red[THREADS / 32];
    const int inst = blockIdx.x;
    double acc = 0.0;
    for (int s = soff[inst] + threadIdx.x; s < soff[inst + 1]; s += THREADS) acc += sdl[s];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[inst] = acc;
}

}  // namespace

void launch_seg_norm_inf(const DevSym &d, const int4 *chunks, int nchunks, const int4 *fin, int nfin,
                         double *partial, const int64_t *coff, int count, double *out, cudaStream_t st) {
    cudaMemsetAsync(out, 0, count * sizeof(double), st);
    seg_norm_chunks_kernel<<<(int)(((int64_t)nchunks * 32 + THREADS - 1) / THREADS), THREADS, 0, st>>>(
        d, chunks, nchunks, partial, coff, count, out);
    if (nfin > 0) seg_norm_finish_kernel<<<(nfin + 127) / 128, 128, 0, st>>>(fin, nfin, partial, coff, count, out);
}

void launch_seg_colmax3(const double *R, const double *X, const double *B, const int64_t *coff, int count,
                        int nrhs, double *out, cudaStream_t st) {
    seg_colmax3_kernel<<<count, THREADS, 0, st>>>(R, X, B, coff, nrhs, out);
}

template <class T>
void launch_seg_logdet(const DevSym &d, const T *front, const int32_t *soff, int count, double *sdl,
                       double *out, cudaStream_t st) {
    snode_logdet_kernel<T><<<(int)(((int64_t)d.ns * 32 + THREADS - 1) / THREADS), THREADS, 0, st>>>(d, front,
                                                                                                   sdl);
    seg_sum_kernel<<<count, THREADS, 0, st>>>(sdl, soff, out);
}
template void launch_seg_logdet<double>(const DevSym &, const double *, const int32_t *, int, double *,
                                        double *, cudaStream_t);
template void launch_seg_logdet<float>(const DevSym &, const float *, const int32_t *, int, double *,
                                       double *, cudaStream_t);

}  // namespace wd
