// Small device helpers shared by the kernels of the solver.
#pragma once
#include <cstdint>

namespace wd {

// Asynchronous global -> shared copies (cp.async): the copy does not occupy a
// register, so a thread can have many of them in flight.  Bytes beyond
// src_bytes are filled with zeros (src_bytes = 0 reads nothing).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Copy one element of type T with zero fill (valid = false -> zero).
template <class T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem, bool valid) {
    if (sizeof(T) == 8) cp_async8(smem, valid ? gmem : smem, valid ? 8 : 0);
    else cp_async4(smem, valid ? gmem : smem, valid ? 4 : 0);
}

// Stage a tile of `rows` x `cols` elements, column c starting at g + c*ldg
// (columns contiguous in global memory, 16-byte aligned, rows a multiple of
// the vector width), into shared memory s + c*lds (lds a multiple of the
// vector width).  Rows >= rvalid (and columns >= cvalid) are zero-filled.
// Issues cp.async only; the caller commits and waits.
template <class T, int THREADS>
__device__ __forceinline__ void stage_tile(T *s, int lds, const T *g, int64_t ldg, int rows,
                                           int cols, int rvalid, int cvalid) {
    constexpr int V = 16 / sizeof(T);  // elements per 16-byte vector
    const int vpc = rows / V;          // vectors per column
    const int total = vpc * cols;
    for (int idx = threadIdx.x; idx < total; idx += THREADS) {
        const int c = idx / vpc, r = (idx % vpc) * V;
        int valid = (c < cvalid) ? rvalid - r : 0;
        valid = valid < 0 ? 0 : (valid > V ? V : valid);
        const T *src = valid ? g + (int64_t)c * ldg + r : g;
        cp_async16(s + c * lds + r, src, valid * (int)sizeof(T));
    }
}

}  // namespace wd
