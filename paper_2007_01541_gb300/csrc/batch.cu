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

// out[i] = max over the instance's rows of sum_j |a_ij| (full CSR of P A P^T)
__global__ void __launch_bounds__(THREADS) seg_norm_inf_kernel(DevSym d, const int64_t *__restrict__ coff,
                                                               double *__restrict__ out) {
    __shared__ double red[THREADS / 32];
    const int inst = blockIdx.x;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double mx = 0.0;
    for (int64_t r = coff[inst] + w; r < coff[inst + 1]; r += THREADS / 32) {
        double acc = 0.0;
        for (int64_t e = d.csr_ptr[r] + lane; e < d.csr_ptr[r + 1]; e += 32) acc += fabs(d.csr_val[e]);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        mx = fmax(mx, acc);
    }
    mx = block_max(mx, red);
    if (threadIdx.x == 0) out[inst] = mx;
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

// out[i] = 2 sum log L_jj over the instance's supernodes
template <class T>
__global__ void __launch_bounds__(THREADS) seg_logdet_kernel(DevSym d, const T *__restrict__ front,
                                                             const int32_t *__restrict__ soff,
                                                             double *__restrict__ out) {
    __shared__ double red[THREADS / 32];
    const int inst = blockIdx.x;
    double acc = 0.0;
    for (int s = soff[inst]; s < soff[inst + 1]; ++s) {
        const int k = d.sk[s], ld = d.sld[s];
        const T *F = front + d.foff[s];
        for (int j = threadIdx.x; j < k; j += THREADS) acc += 2.0 * log((double)F[(int64_t)j * ld + j]);
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[inst] = acc;
}

}  // namespace

void launch_seg_norm_inf(const DevSym &d, const int64_t *coff, int count, double *out, cudaStream_t st) {
    seg_norm_inf_kernel<<<count, THREADS, 0, st>>>(d, coff, out);
}

void launch_seg_colmax3(const double *R, const double *X, const double *B, const int64_t *coff, int count,
                        int nrhs, double *out, cudaStream_t st) {
    seg_colmax3_kernel<<<count, THREADS, 0, st>>>(R, X, B, coff, nrhs, out);
}

template <class T>
void launch_seg_logdet(const DevSym &d, const T *front, const int32_t *soff, int count, double *out,
                       cudaStream_t st) {
    seg_logdet_kernel<T><<<count, THREADS, 0, st>>>(d, front, soff, out);
}
template void launch_seg_logdet<double>(const DevSym &, const double *, const int32_t *, int, double *,
                                        cudaStream_t);
template void launch_seg_logdet<float>(const DevSym &, const float *, const int32_t *, int, double *,
                                       cudaStream_t);

}  // namespace wd
