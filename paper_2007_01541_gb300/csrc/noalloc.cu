// Scratch memory of the allocation-free export of the factor
// (wd_export_L_noalloc).  The panel offsets live in a file-scope device array
// of fixed size instead of a buffer allocated per call, so the call never
// asks the CUDA allocator for memory.  Its users: a caller whose device memory
// is held by another allocator (a framework's caching allocator, a memory
// cap), where a factor-sized cudaMalloc would fail, and a caller that cannot
// take the device-wide synchronization that cudaMalloc / cudaFree imply.
//
// One array per device (a __device__ variable exists once in every context);
// its address is looked up once per device with cudaGetSymbolAddress and
// cached.  Calls whose executions overlap (different streams without
// ordering, or different host threads) share the array and race on it.
#include <mutex>

#include "engine.h"

namespace wd {
namespace {

constexpr int SCAN_THREADS = 1024;

// offsets of the supernodes' panels: g_panel_off[s] = sum_{t < s} m_t k_t,
// g_panel_off[ns] = total.  Every call rewrites entries 0..ns before they are
// read, so nothing in it has to start at zero.
static __device__ __align__(256) int64_t g_panel_off[NOALLOC_MAX_SUPERNODES + 1];

// exclusive prefix sum of m_s k_s over the supernodes, one block: each thread
// sums a contiguous run of supernodes, the block scans the run totals
__global__ void __launch_bounds__(SCAN_THREADS) panel_offsets_kernel(DevSym d) {
    __shared__ int64_t part[SCAN_THREADS];
    const int ns = d.ns, tid = threadIdx.x;
    const int per = (ns + SCAN_THREADS - 1) / SCAN_THREADS;
    const int s0 = min(ns, tid * per), s1 = min(ns, s0 + per);
    int64_t sum = 0;
    for (int s = s0; s < s1; ++s) sum += (int64_t)d.sm[s] * d.sk[s];
    part[tid] = sum;
    __syncthreads();
    // Hillis-Steele inclusive scan of the run totals
    for (int o = 1; o < SCAN_THREADS; o <<= 1) {
        const int64_t v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int64_t off = part[tid] - sum;
    for (int s = s0; s < s1; ++s) {
        g_panel_off[s] = off;
        off += (int64_t)d.sm[s] * d.sk[s];
    }
    if (tid == SCAN_THREADS - 1) g_panel_off[ns] = part[tid];
}

std::mutex g_lock;
constexpr int MAX_DEVICES = 64;
int64_t *g_addr[MAX_DEVICES] = {};

}  // namespace

cudaError_t noalloc_panel_offsets(int device, int64_t **addr) {
    *addr = nullptr;
    if (device < 0 || device >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_lock);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_panel_off);
        if (e != cudaSuccess) return e;
        g_addr[device] = static_cast<int64_t *>(p);
    }
    *addr = g_addr[device];
    return cudaSuccess;
}

void launch_panel_offsets_noalloc(const DevSym &d, cudaStream_t st) {
    panel_offsets_kernel<<<1, SCAN_THREADS, 0, st>>>(d);
}

}  // namespace wd
