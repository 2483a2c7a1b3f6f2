// C ABI of the solver: handle, analysis, launch plans and the numeric calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <thread>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/wd.h"
#include "engine.h"
#include "symbolic.h"

using wd::DevSym;
using wd::NB;
using wd::RB;
using wd::status_t;

namespace {

constexpr int ROWS_PER_CTA = 256;  // one thread per front row (gather / apply_L)

enum LaunchKind {
    K_INIT, K_PANEL, K_UPDATE, K_SYRK, K_UPDATE_TC, K_SYRK_TC, K_DIAG,      // factor
    K_SBINV_DIAG, K_SBINV_STAGE, K_SBINV_T,                    // super-block inverses
    K_FWD_GATHER, K_FWD_XAPPLY, K_FWD_BUPDATE,                 // forward solve
    K_BWD_REDUCE, K_BWD_FINISH, K_BWD_XAPPLY,                  // backward solve
    K_APPLY_L,
    K_LU_INIT, K_LU_DIAG, K_LU_PANEL, K_LU_UPDATE,               // LU factor
    K_LU_GATHER, K_LU_FWD, K_LU_BWD,                             // LU substitutions
    K_OZ_SLICE, K_OZ_UPDATE, K_OZ_SYRK,                          // FP64 updates on the tensor cores
    K_CHAIN_TC                                                   // pivot columns of a level, one launch
};

struct Launch {
    int kind;
    int64_t off;   // into the item array
    int count;
    int arg;       // kb or ib
    double flops = 0;        // algorithmic flops of the launch
    double elems = 0;        // front / vector elements moved (x sizeof(T))
    double bytes = 0;        // other bytes (A values and indices)
};

const char *kind_name(int k) {
    static const char *names[] = {"front_init", "panel", "schur_update", "schur_syrk",
                                  "tc_schur_update", "tc_schur_syrk", "diag_factor", "sbinv_diag",
                                  "sbinv_stage", "sbinv_transpose", "fwd_gather", "fwd_xapply",
                                  "fwd_bupdate", "bwd_reduce", "bwd_finish", "bwd_xapply",
                                  "apply_L", "lu_init", "lu_diag", "lu_panel", "lu_update",
                                  "lu_gather", "lu_fwd", "lu_bwd", "oz_slice", "oz_schur_update",
                                  "oz_schur_syrk", "tc_chain"};
    return names[k];
}

struct KStat {
    int64_t launches = 0;
    double ms = 0, flops = 0, bytes = 0;
};

struct Plan {
    std::vector<int4> items;
    std::vector<Launch> launches;
    int4 *d_items = nullptr;
    int rgt = 16;            // solve plans: right-hand sides per gather CTA
    int large = 0;           // solve plans: product mode (0: 64 x 32 tiles, 2: few right-hand sides)
    int64_t slots = 0;       // solve plans: partial-sum slots of the largest split step
    int64_t ksplit = 0;      // solve plans: CTAs of the largest launch split over the inner dimension
};

struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int64_t key = -1;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key = -1;
    }
};

struct DevMem {
    std::vector<void *> ptrs;
    // test hook (wd_options.test_fail_alloc): the handle's allocations so far
    // and the one that fails as if device memory ran out (0: none)
    int64_t *count = nullptr;
    int64_t fail_at = 0;
    cudaError_t alloc(void **p, size_t bytes) {
        *p = nullptr;
        if (bytes == 0) bytes = 16;
        if (count && ++*count == fail_at) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release(void *p) {
        if (!p) return;
        auto it = std::find(ptrs.begin(), ptrs.end(), p);
        if (it != ptrs.end()) {
            cudaFree(p);
            ptrs.erase(it);
        }
    }
    void free_all() {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

}  // namespace

struct wd_ctx {
    wd_options opt;
    int device = 0;
    bool analyzed = false, factored = false;
    wd_precision prec = WD_FP64;
    wd::Symbolic S;
    DevMem mem;        // analysis lifetime
    DevMem work;       // numeric workspaces (factor / solve)
    int64_t allocs = 0;   // device allocations made by this handle (test hook)
    DevSym dsym{};
    int32_t *d_csr_src = nullptr;
    double *d_csr_val = nullptr;
    // LU without pivoting (wd_factor_lu, FP64): position codes of the full
    // CSR, both values per position, U11^-1 blocks, plans
    bool lu_factored = false;
    bool ldlt = false;          // the LU factor is that of a symmetric matrix (wd_factor_ldlt)
    bool front_dirty = false;   // the fronts' upper parts hold an LU factor
    std::vector<int8_t> h_csr_code;
    int8_t *d_lu_code = nullptr;
    double *d_vrow = nullptr, *d_vcol = nullptr, *d_uinv = nullptr, *d_lu_part = nullptr;
    double *d_upper_stage = nullptr;
    Plan fplan_lu, splan_lu_f, splan_lu_b;
    double *d_gcsr = nullptr;   // mass matrix G on the full CSR (wd_set_mass; nullptr: G = I)
    double *mass_buf = nullptr; // its storage (analysis lifetime)
    float *d_csr_vh = nullptr, *d_csr_vl = nullptr;   // double-float split of csr_val
    double *d_values_stage = nullptr;
    void *d_front = nullptr;
    size_t front_elems = 0;
    void *d_dinv = nullptr;        // inverses of the NB x NB diagonal blocks
    size_t dinv_elems = 0;
    void *d_xs = nullptr, *d_xts = nullptr;  // super-block inverses and their transposes
    int64_t *d_xsoff = nullptr;
    // FP64 updates on the tensor cores: bf16 slice planes and row-scale
    // exponents per supernode and 64-column block (wd_options.fp64_tc_schur)
    unsigned char *d_oz_sl = nullptr;
    int16_t *d_oz_ex = nullptr;
    int64_t *d_oz_soff = nullptr, *d_oz_eoff = nullptr;
    int64_t oz_sl_bytes = 0, oz_ex_elems = 0;
    size_t xs_elems = 0;
    unsigned char *d_pack = nullptr;  // packed tf32 panel lines (FP32 fronts)
    int64_t pack_total = 0;
    // one launch per level for the FP32 fronts' pivot columns: dependency
    // words of every supernode (offsets chain_flagoff), then one task counter
    // per level and the launch-wide abort word; zeroed before each factor
    bool chain = false;
    std::vector<int8_t> level_step;   // per level: 1 keeps the launch pairs (wd_set_level_schedule)
    unsigned *d_chain_flags = nullptr;
    int64_t *d_chain_flagoff = nullptr;
    unsigned char *d_chain_lpack = nullptr;   // L11^-1 blocks as tensor-core operands (32 KB each)
    int64_t chain_words = 0, chain_ctr = 0;
    status_t *d_tstatus = nullptr;    // nonzero: a bounded device wait expired
    unsigned *d_gate = nullptr;       // a device word that stays zero (wd_options.test_closed_gate)
    cudaStream_t cap_stream = nullptr;
    // wd_export_L_noalloc returns without waiting; this event, recorded on its
    // stream, orders that read of the fronts before the next call that
    // rewrites or frees them (wd_factor, wd_analyze, wd_destroy)
    cudaEvent_t export_ev = nullptr;
    bool export_pending = false;
    GraphCache g_factor, g_solve;
    status_t *d_status = nullptr;
    double *d_scalars = nullptr;   // [0] = ||A||_inf, [1] = logdet, [2..] partials
    Plan fplan;        // FP64 fronts (SIMT Schur tiles)
    Plan fplan_tc;     // FP32 fronts (tensor-core Schur tiles)
    Plan splan;
    int splan_nrhs = -1;
    Plan aplan;
    int aplan_nrhs = -1;
    // solve workspaces (sized for ws_cols right-hand sides)
    int64_t ws_cols = 0;
    void *d_Y = nullptr, *d_W = nullptr, *d_T = nullptr;
    void *d_part = nullptr;        // partial sums of the backward split reduction
    int64_t part_elems = 0;
    // tensor-core solve products split over the inner dimension: one partial
    // tile per CTA and one arrival counter per output tile (kept at zero
    // between launches)
    float *d_ksw = nullptr;
    int *d_kcnt = nullptr;
    int64_t ksw_items = 0;
    int sms = 152;                 // multiprocessors of the device
    double *d_B = nullptr, *d_Bp = nullptr, *d_X = nullptr, *d_R = nullptr, *d_cm = nullptr;
    float2 *d_Xp = nullptr;   // double-float split of the refinement vectors, (hi, lo) pairs
    int64_t W_rows = 0;   // sum of (m_s - k_s)
    int64_t nnz_full = 0;  // stored entries of the full CSR of P A P^T
    int4 *d_spmv_chunks = nullptr, *d_spmv_fin = nullptr;
    int n_spmv_chunks = 0, n_spmv_fin = 0, n_spmv_slots = 0;
    double *d_P = nullptr;  // partial sums of chunked rows (slots x nrhs)
    double *d_norm_part = nullptr;  // partial row sums of |a| of chunked rows
    double normA = 0.0;
    // selected inverse (built on first use; pointers into mem)
    struct SelStep {
        int kind;  // 0 trinv, 1 gemm, 2 zgather
        int64_t off;
        int count;
    };
    std::vector<SelStep> sel_steps;
    bool sel_ready = false;
    double *d_zpool = nullptr, *d_xw = nullptr, *d_sel_out = nullptr;
    int64_t *d_xoff = nullptr, *d_upoff = nullptr;
    int32_t *d_upmap = nullptr, *d_col2s = nullptr, *d_prow = nullptr, *d_psrc = nullptr;
    int4 *d_sel_items = nullptr;
    wd::GemmItem *d_sel_gemm = nullptr;
    double sel_flops = 0.0;
    // batch of independent instances (wd_analyze_batch): column and supernode offsets
    int32_t batch_count = 0;
    std::vector<int64_t> batch_coff;
    std::vector<int32_t> batch_soff;
    int32_t *d_batch_soff = nullptr;
    int64_t *d_batch_coff = nullptr;
    double *d_batch_norm = nullptr;   // per-instance ||A_i||_inf
    double *d_batch_ld = nullptr;     // per-instance log det
    double *d_batch_sdl = nullptr;    // per-supernode log det terms
    unsigned long long *d_spmv_bad = nullptr;   // residual: first bad column index position
    double *d_batch_cm = nullptr;     // per-instance column maxima (solve workspace)
    std::vector<double> batch_normA;
    std::vector<int64_t> h_foff;   // host copies of the front layout
    std::vector<int32_t> h_sld;
    wd_info info{};
    // profiling
    int64_t launches = 0;  // kernels launched by this handle
    std::vector<cudaEvent_t> prof_ev;
    cudaEvent_t single_ev[2] = {nullptr, nullptr};
    std::vector<std::pair<std::string, KStat>> prof;
    std::string msg;
    int64_t errcol = -1;
};

static wd_status fail(wd_handle h, wd_status s, const std::string &m, int64_t col = -1) {
    if (h) {
        h->msg = m;
        h->errcol = col;
    }
    return s;
}

static wd_status cuda_fail(wd_handle h, cudaError_t e, const char *where) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(h, WD_ERR_OOM, std::string(where) + ": " + cudaGetErrorString(e));
    }
    return fail(h, WD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                     \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
    } while (0)

extern "C" {

const char *wd_status_string(wd_status s) {
    switch (s) {
        case WD_OK: return "WD_OK";
        case WD_ERR_INVALID_ARG: return "WD_ERR_INVALID_ARG";
        case WD_ERR_PATTERN: return "WD_ERR_PATTERN";
        case WD_ERR_STATE: return "WD_ERR_STATE";
        case WD_ERR_NOT_SPD: return "WD_ERR_NOT_SPD";
        case WD_ERR_OOM: return "WD_ERR_OOM";
        case WD_ERR_CUDA: return "WD_ERR_CUDA";
        case WD_ERR_TIMEOUT: return "WD_ERR_TIMEOUT";
        case WD_ERR_NO_CONVERGENCE: return "WD_ERR_NO_CONVERGENCE";
    }
    return "unknown";
}

void wd_default_options(wd_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->nd_leaf = 128;
    o->relax_k = 64;
    o->relax_pct = 10;
    o->ir_max_iter = 10;
    o->ir_tol = 1e-12;
    o->use_graphs = 1;
}

wd_status wd_create(wd_handle *out, const wd_options *opt) {
    if (!out) return WD_ERR_INVALID_ARG;
    *out = nullptr;
    wd_ctx *h = new (std::nothrow) wd_ctx();
    if (!h) return WD_ERR_OOM;
    wd_default_options(&h->opt);
    if (opt) h->opt = *opt;
    if (h->opt.nd_leaf < 1 || h->opt.relax_k < 0 || h->opt.relax_pct < 0 || h->opt.ir_max_iter < 0 ||
        !(h->opt.ir_tol > 0) || h->opt.diag64_min_k < 0 || h->opt.wait_limit < 0 ||
        h->opt.test_fail_alloc < 0 || h->opt.fp64_tc_schur < 0 || h->opt.fp64_tc_schur > 1 ||
        h->opt.step_launches < 0 || h->opt.step_launches > 1) {
        delete h;
        return WD_ERR_INVALID_ARG;
    }
    h->mem.count = h->work.count = &h->allocs;
    h->mem.fail_at = h->work.fail_at = h->opt.test_fail_alloc;
    if (!h->opt.symbolic_only &&
        (cudaGetDevice(&h->device) != cudaSuccess ||
         cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)) {
        cudaGetLastError();
        delete h;
        return WD_ERR_CUDA;
    }
    *out = h;
    return WD_OK;
}

// waits (host side) for the last wd_export_L_noalloc's read of the fronts
static void wait_export(wd_handle h) {
    if (h->export_pending) {
        cudaEventSynchronize(h->export_ev);
        h->export_pending = false;
    }
}

void wd_destroy(wd_handle h) {
    if (!h) return;
    if (!h->opt.symbolic_only) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(h->device);
        wait_export(h);
        if (h->export_ev) cudaEventDestroy(h->export_ev);
        for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
        for (cudaEvent_t e : h->single_ev)
            if (e) cudaEventDestroy(e);
        h->g_factor.reset();
        h->g_solve.reset();
        if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
        h->work.free_all();
        h->mem.free_all();
        cudaSetDevice(prev);
    }
    delete h;
}

wd_status wd_status_detail(wd_handle h, int64_t *column, char *msg, size_t len) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (column) *column = h->errcol;
    if (msg && len) {
        std::snprintf(msg, len, "%s", h->msg.c_str());
    }
    return WD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
static void add_launch(Plan &p, int kind, size_t first, int arg, double flops = 0,
                       double elems = 0, double bytes = 0) {
    const int count = (int)(p.items.size() - first);
    if (count > 0) {
        Launch L;
        L.kind = kind;
        L.off = (int64_t)first;
        L.count = count;
        L.arg = arg;
        L.flops = flops;
        L.elems = elems;
        L.bytes = bytes;
        p.launches.push_back(L);
    }
}

// lower-triangle entries (r >= c) of the tile rows [r0, r1) x cols [c0, c1)
static double lower_count(int64_t r0, int64_t r1, int64_t c0, int64_t c1) {
    double cnt = 0;
    for (int64_t c = c0; c < c1; ++c) cnt += (double)std::max<int64_t>(0, r1 - std::max(r0, c));
    return cnt;
}

static int kpad(int k) { return (k + 31) / 32 * 32; }
// rows of a front: pivot rows, zero padding to a multiple of 32, rows below
static int front_order(const wd::Symbolic &S, int s) { return kpad(S.k(s)) + S.m(s) - S.k(s); }

// oz (FP64 fronts): the Schur updates through bf16 slices on the tensor
// cores, each panel launch followed by the slicing of its rows.
// chain (FP32 fronts on the tensor cores): the pivot columns of a level in
// one launch of dependency-ordered tasks (tc_chain.cu) instead of the diagonal
// block launch and a (panel, update) launch pair per pivot block.
// level_step (nullable, one flag per level): levels whose flag is set keep
// the (panel, update) launch pairs although chain is on.
static void build_factor_plan(const wd::Symbolic &S, Plan &p, bool tc, bool oz = false, bool chain = false,
                              const int8_t *level_step = nullptr) {
    const int SCHUR_BM = tc ? wd::TC_BM : wd::SCHUR_BM;
    const int SCHUR_BN = tc ? wd::TC_BN : wd::SCHUR_BN;
    p.items.clear();
    p.launches.clear();
    for (int l = 0; l < S.nlevels; ++l) {
        const int b = S.level_ptr[l], e = S.level_ptr[l + 1];
        size_t f0 = p.items.size();
        double el = 0, by = 0;
        for (int i = b; i < e; ++i) {
            const int s = S.level_nodes[i];
            const double m = S.m(s);
            const int mp = front_order(S, s);
            // 8 columns per CTA, never two fronts in one CTA (padding items: q = -1)
            for (int q = 0; q < (mp + 7) / 8 * 8; ++q) p.items.push_back({s, q < mp ? q : -1, 0, 0});
            el += m * (m + 1) / 2;  // every lower front entry written once
            for (int c = S.child_ptr[s]; c < S.child_ptr[s + 1]; ++c) {
                const double u = S.m(S.children[c]) - S.k(S.children[c]);
                el += u * (u + 1) / 2;  // every child update entry read once
            }
            by += 12.0 * (double)(S.pcp[S.sfirst[s + 1]] - S.pcp[S.sfirst[s]]);
        }
        add_launch(p, K_INIT, f0, 0, 0, el, by);
        // factorization and inverse of a diagonal block of nb columns
        auto diag_flops = [](double nb) { return 2.0 * nb * nb * nb / 3; };
        int kmax = 0;
        double fl = 0;
        for (int i = b; i < e; ++i) kmax = std::max(kmax, S.k(S.level_nodes[i]));
        if (tc && chain && !(level_step && level_step[l])) {
            // tasks (s, c, ti): column block c, row tile ti (128 rows from row
            // 64 c); in order of c, then ti, then front, so that every task
            // depends only on earlier ones
            f0 = p.items.size();
            fl = el = 0;
            for (int cbk = 0; cbk * NB < kmax; ++cbk) {
                int tmax = 0;
                for (int i = b; i < e; ++i) {
                    const int s = S.level_nodes[i];
                    if (S.k(s) > cbk * NB) tmax = std::max(tmax, (front_order(S, s) - cbk * NB + 127) / 128);
                }
                for (int ti = 0; ti < tmax; ++ti)
                    for (int i = b; i < e; ++i) {
                        const int s = S.level_nodes[i];
                        if (S.k(s) > cbk * NB && cbk * NB + ti * 128 < front_order(S, s))
                            p.items.push_back({s, cbk, ti, 0});
                    }
            }
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i], k = S.k(s), m = S.m(s);
                for (int kb = 0; kb < k; kb += NB) {
                    const int nb = std::min(NB, k - kb), t0 = kb + nb;
                    const double cw = k - t0, below = m - k;
                    const double ent = cw * (cw + 1) / 2 + below * cw;
                    fl += diag_flops(nb) + (double)(m - t0) * nb * nb + 2.0 * nb * ent;
                    el += 2.0 * (m - kb) * nb;
                }
            }
            add_launch(p, K_CHAIN_TC, f0, l, fl, el, 0);
        } else {
        // the first diagonal block of every front of the level
        f0 = p.items.size();
        fl = el = 0;
        for (int i = b; i < e; ++i) {
            const int s = S.level_nodes[i], nb = std::min(NB, S.k(s));
            p.items.push_back({s, 0, 0, 0});
            fl += diag_flops(nb);
            el += nb * (nb + 1) + 2.0 * NB * NB;
        }
        add_launch(p, K_DIAG, f0, 0, fl, el, 0);
        for (int kb = 0; kb < kmax; kb += NB) {
            // panel rows: L21 = F21 L11^-T with the stored inverse
            f0 = p.items.size();
            fl = el = 0;
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i], k = S.k(s), m = S.m(s);
                if (k <= kb) continue;
                const int nb = std::min(NB, k - kb);
                const int t0 = kb + nb;
                const int mp = front_order(S, s);
                const int rs = (t0 == k) ? kpad(k) : t0;
                const int nrb = (mp - rs + RB - 1) / RB;
                for (int rb = 0; rb < nrb; ++rb) p.items.push_back({s, rb, 0, 0});
                fl += (double)(m - t0) * nb * nb;
                el += 2.0 * (m - t0) * nb + (double)NB * NB;
            }
            add_launch(p, K_PANEL, f0, kb, fl, el, 0);
            if (oz) {
                // the same rows, sliced for the updates
                const size_t g0 = p.items.size(), g1 = p.items.size() - f0;
                for (size_t q = 0; q < g1; ++q) {
                    const int4 itq = p.items[f0 + q];
                    p.items.push_back(itq);
                }
                add_launch(p, K_OZ_SLICE, g0, kb, 0, el, 0);
            }
            // trailing pivot columns; the CTA of tile (0, 0) also factors the
            // next diagonal block
            f0 = p.items.size();
            fl = el = 0;
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i], k = S.k(s), m = S.m(s);
                if (k <= kb) continue;
                const int nb = std::min(NB, k - kb);
                const int t0 = kb + nb;
                if (t0 >= k) continue;
                const int nrt = (front_order(S, s) - t0 + SCHUR_BM - 1) / SCHUR_BM;
                const int nct = (k - t0 + SCHUR_BN - 1) / SCHUR_BN;
                for (int tj = 0; tj < nct; ++tj)
                    for (int ti = (tj * SCHUR_BN) / SCHUR_BM; ti < nrt; ++ti)
                        p.items.push_back({s, ti, tj, 0});
                const double cw = k - t0, below = m - k;
                const double ent = cw * (cw + 1) / 2 + below * cw;
                const int nb2 = std::min(NB, k - t0);
                fl += 2.0 * nb * ent + diag_flops(nb2);
                el += 2.0 * ent + (double)(m - t0) * nb + nb2 * (nb2 + 1) + 2.0 * NB * NB;
            }
            add_launch(p, tc ? K_UPDATE_TC : (oz ? K_OZ_UPDATE : K_UPDATE), f0, kb, fl, el, 0);
        }
        }
        f0 = p.items.size();
        fl = el = 0;
        for (int i = b; i < e; ++i) {
            const int s = S.level_nodes[i], k = S.k(s), m = S.m(s);
            if (m <= k) continue;
            const int u = m - k;
            const int nrt = (u + SCHUR_BM - 1) / SCHUR_BM;
            const int nct = (u + SCHUR_BN - 1) / SCHUR_BN;
            for (int tj = 0; tj < nct; ++tj)
                for (int ti = (tj * SCHUR_BN) / SCHUR_BM; ti < nrt; ++ti)
                    p.items.push_back({s, ti, tj, 0});
            const double tri = (double)u * (u + 1) / 2;
            fl += 2.0 * k * tri;
            el += 2.0 * tri + (double)u * k;
        }
        add_launch(p, tc ? K_SYRK_TC : (oz ? K_OZ_SYRK : K_SYRK), f0, 0, fl, el, 0);
    }
    // explicit inverses of the super-blocks' diagonal blocks (for the solves)
    constexpr int BPS = wd::SB / NB;  // 64-blocks per super-block
    auto nblk_of = [&](int s, int sb) { return (std::min(wd::SB, S.k(s) - sb * wd::SB) + NB - 1) / NB; };
    {
        const size_t f0 = p.items.size();
        double el = 0;
        for (int s = 0; s < S.ns; ++s)
            for (int sb = 0; sb * wd::SB < S.k(s); ++sb)
                for (int t = 0; t < nblk_of(s, sb); ++t) {
                    p.items.push_back({s, sb, t, 0});
                    el += 2.0 * NB * NB;
                }
        add_launch(p, K_SBINV_DIAG, f0, 0, 0, el, 0);
    }
    for (int t = 1; t < BPS; ++t) {
        const size_t f0 = p.items.size();
        double fl = 0, el = 0;
        for (int s = 0; s < S.ns; ++s)
            for (int sb = 0; sb * wd::SB < S.k(s); ++sb) {
                if (nblk_of(s, sb) <= t) continue;
                for (int bj = 0; bj < t; ++bj) {
                    p.items.push_back({s, sb, bj, 0});
                    fl += 2.0 * NB * NB * NB * (t - bj) + (double)NB * NB * NB;
                    el += 2.0 * NB * NB * (t - bj) + 2.0 * NB * NB;
                }
            }
        add_launch(p, K_SBINV_STAGE, f0, t, fl, el, 0);
    }
    {
        const size_t f0 = p.items.size();
        double el = 0;
        for (int s = 0; s < S.ns; ++s)
            for (int sb = 0; sb * wd::SB < S.k(s); ++sb) {
                const int nb = nblk_of(s, sb);
                for (int bi = 0; bi < nb; ++bi)
                    for (int bj = 0; bj <= bi; ++bj) {
                        p.items.push_back({s, sb, bi, bj});
                        el += 2.0 * NB * NB;
                    }
            }
        add_launch(p, K_SBINV_T, f0, 0, 0, el, 0);
    }
}

// Tensor-core product launches with few output tiles split the inner
// dimension (up to 512 columns of a super-block) over up to four CTAs per
// tile, so that a launch fills about one wave of the device; the item's z
// carries the split (row block | split << 16 | splits << 24).
static void split_inner(Plan &p, size_t f0, int sms) {
    const int64_t tiles = (int64_t)(p.items.size() - f0);
    if (tiles <= 0 || 2 * tiles > sms) return;
    const int nks = (int)std::min<int64_t>(4, sms / tiles);
    std::vector<int4> split;
    split.reserve(tiles * nks);
    for (size_t i = f0; i < p.items.size(); ++i)
        for (int ks = 0; ks < nks; ++ks) {
            int4 q = p.items[i];
            q.z = q.z | (ks << 16) | (nks << 24);
            split.push_back(q);
        }
    p.items.resize(f0);
    p.items.insert(p.items.end(), split.begin(), split.end());
    p.ksplit = std::max<int64_t>(p.ksplit, (int64_t)split.size());
}

static void build_solve_plan(const wd::Symbolic &S, int nrhs, int large, int sms, Plan &p) {
    p.items.clear();
    p.launches.clear();
    p.ksplit = 0;
    const int rgt = nrhs >= 48 ? 64 : 16;   // right-hand sides per gather CTA
    p.rgt = rgt;
    p.large = large;
    p.slots = 0;
    const int ngg = (nrhs + rgt - 1) / rgt;
    const int TRW = wd::solve_tile_rows(large), TNW = wd::solve_tile_rhs(large);
    const int TRX = wd::solve_update_rows(large);   // rows per CTA of the xapply / bupdate items
    const int ng = (nrhs + TNW - 1) / TNW;
    const double R = nrhs;
    const int SBW = wd::SB, KSR = large == 1 ? wd::SOLVE_KSR_TC : wd::SOLVE_KSR;
    auto nsb = [&](int s) { return (S.k(s) + SBW - 1) / SBW; };
    auto width = [&](int s, int sb) { return std::min(SBW, S.k(s) - sb * SBW); };
    auto wpad = [&](int s, int sb) { return (width(s, sb) + NB - 1) / NB * NB; };
    for (int l = 0; l < S.nlevels; ++l) {
        const int b = S.level_ptr[l], e = S.level_ptr[l + 1];
        size_t f0 = p.items.size();
        int maxsb = 0;
        double el = 0, fl = 0;
        for (int i = b; i < e; ++i) {
            const int s = S.level_nodes[i];
            for (int rc = 0; rc * 32 < S.m(s); ++rc)
                for (int g = 0; g < ngg; ++g) p.items.push_back({s, rc, g, 0});
            maxsb = std::max(maxsb, nsb(s));
            el += R * (S.m(s) + S.k(s));
            for (int c = S.child_ptr[s]; c < S.child_ptr[s + 1]; ++c)
                el += R * (S.m(S.children[c]) - S.k(S.children[c]));
        }
        add_launch(p, K_FWD_GATHER, f0, 0, 0, el, 0);
        for (int sb = 0; sb < maxsb; ++sb) {
            f0 = p.items.size();
            el = fl = 0;
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i];
                if (nsb(s) <= sb) continue;
                const int w = width(s, sb), wp = wpad(s, sb);
                for (int rb = 0; rb * TRX < wp; ++rb)
                    for (int g = 0; g < ng; ++g) p.items.push_back({s, sb, rb, g});
                fl += (double)w * (w + 1) * R;
                el += (double)w * (w + 1) / 2 + 2.0 * w * R;
            }
            if (large == 1) split_inner(p, f0, sms);
            add_launch(p, K_FWD_XAPPLY, f0, sb, fl, el, 0);
            f0 = p.items.size();
            el = fl = 0;
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i];
                if (nsb(s) <= sb) continue;
                const int k = S.k(s), m = S.m(s), w = width(s, sb);
                const int nJ = k - (sb * SBW + w), nR = m - k;
                for (int rb = 0; rb * TRX < nJ; ++rb)
                    for (int g = 0; g < ng; ++g) p.items.push_back({s, sb, rb, g});
                for (int rb = 0; rb * TRX < nR; ++rb)
                    for (int g = 0; g < ng; ++g) p.items.push_back({s, sb, rb, g + 65536});
                fl += 2.0 * (nJ + nR) * w * R;
                el += (double)(nJ + nR) * w + 2.0 * (nJ + nR) * R + w * R;
            }
            if (large == 1) split_inner(p, f0, sms);
            add_launch(p, K_FWD_BUPDATE, f0, sb, fl, el, 0);
        }
    }
    for (int l = S.nlevels - 1; l >= 0; --l) {
        const int b = S.level_ptr[l], e = S.level_ptr[l + 1];
        int maxsb = 0;
        for (int i = b; i < e; ++i) maxsb = std::max(maxsb, nsb(S.level_nodes[i]));
        for (int sb = maxsb - 1; sb >= 0; --sb) {
            // partial sums over splits of the rows below the super-block
            size_t f0 = p.items.size();
            double el = 0, fl = 0;
            int slot = 0;
            std::vector<int4> fin;
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i];
                if (nsb(s) <= sb) continue;
                const int m = S.m(s), w = width(s, sb);
                const int below = m - (sb * SBW + w);
                // tensor-core splits run over the front's storage rows from the
                // 32-row boundary at or above the super-block's end
                const int kbeg = (sb * SBW + w) & ~31;
                const int nsplit = large == 1 ? (below > 0 ? (front_order(S, s) - kbeg + KSR - 1) / KSR : 0)
                                              : (below + KSR - 1) / KSR;
                for (int cb = 0; cb * TRW < w; ++cb)
                    for (int g = 0; g < ng; ++g) {
                        fin.push_back({s, sb * 8 + cb, g + 65536 * nsplit, slot});
                        for (int ks = 0; ks < nsplit; ++ks)
                            p.items.push_back({s, sb * 8 + cb, g + 65536 * ks, slot++});
                    }
                fl += 2.0 * below * w * R;
                el += (double)below * w + below * R;
            }
            p.slots = std::max<int64_t>(p.slots, slot);
            add_launch(p, K_BWD_REDUCE, f0, sb, fl, el, 0);
            f0 = p.items.size();
            el = 0;
            for (const int4 &q : fin) {
                p.items.push_back(q);
                el += 2.0 * TRW * R + (double)(q.z >> 16) * TRW * TNW;
            }
            add_launch(p, K_BWD_FINISH, f0, sb, 0, el, 0);
            f0 = p.items.size();
            el = fl = 0;
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i];
                if (nsb(s) <= sb) continue;
                const int w = width(s, sb), wp = wpad(s, sb);
                for (int rb = 0; rb * TRX < wp; ++rb)
                    for (int g = 0; g < ng; ++g) p.items.push_back({s, sb, rb, g});
                fl += (double)w * (w + 1) * R;
                el += (double)w * (w + 1) / 2 + 2.0 * w * R;
            }
            if (large == 1) split_inner(p, f0, sms);
            add_launch(p, K_BWD_XAPPLY, f0, sb, fl, el, 0);
        }
    }
}

static void build_apply_plan(const wd::Symbolic &S, Plan &p) {
    p.items.clear();
    p.launches.clear();
    for (int l = 0; l < S.nlevels; ++l) {
        size_t f0 = p.items.size();
        for (int i = S.level_ptr[l]; i < S.level_ptr[l + 1]; ++i) {
            const int s = S.level_nodes[i];
            for (int rc = 0; rc * ROWS_PER_CTA < S.m(s); ++rc) p.items.push_back({s, rc, 0, 0});
        }
        add_launch(p, K_APPLY_L, f0, 0);
    }
}

static wd_status upload_plan(wd_handle h, DevMem &mem, Plan &p) {
    if (p.d_items) mem.release(p.d_items);
    p.d_items = nullptr;
    CK(mem.alloc((void **)&p.d_items, p.items.size() * sizeof(int4)), "plan alloc");
    CK(cudaMemcpy(p.d_items, p.items.data(), p.items.size() * sizeof(int4), cudaMemcpyHostToDevice),
       "plan upload");
    return WD_OK;
}

template <class V>
static wd_status upload(wd_handle h, const std::vector<V> &v, const V **dst) {
    V *p = nullptr;
    CK(h->mem.alloc((void **)&p, v.size() * sizeof(V)), "analysis alloc");
    if (!v.empty()) CK(cudaMemcpy(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice), "upload");
    *dst = p;
    return WD_OK;
}

#define UP(vec, field)                                  \
    do {                                                \
        wd_status s_ = upload(h, vec, &(field));        \
        if (s_ != WD_OK) return s_;                     \
    } while (0)

static void fill_info(wd_handle h, int64_t nnzl, int maxm, int maxk,
                      std::chrono::steady_clock::time_point t0) {
    const wd::Symbolic &S = h->S;
    wd_info &I = h->info;
    std::memset(&I, 0, sizeof(I));
    I.n = S.n;
    I.nnz_A_lower = nnzl;
    I.nnz_L = S.nnzL;
    I.nnz_L_stored = S.nnzL_stored;
    I.flops_factor = S.flops;
    I.nsuper = S.ns;
    I.nlevels = S.nlevels;
    I.max_front = maxm;
    I.max_width = maxk;
    I.front_bytes = (int64_t)h->front_elems * 8;
    I.factor_launches = (int64_t)h->fplan_tc.launches.size();
    I.analyze_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// drop everything of a previous analysis; set up the device and stream
static wd_status reset_analysis(wd_handle h) {
    const bool host_only = h->opt.symbolic_only != 0;
    if (!host_only) {
        CK(cudaSetDevice(h->device), "set device");
        wd::init_kernel_attributes();
        if (!h->cap_stream)
            CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "stream");
        if (!h->export_ev) CK(cudaEventCreateWithFlags(&h->export_ev, cudaEventDisableTiming), "event");
        wait_export(h);
    }
    h->analyzed = h->factored = false;
    if (!host_only) {
        h->work.free_all();
        h->mem.free_all();
    }
    h->fplan = Plan();
    h->fplan_tc = Plan();
    h->d_pack = nullptr;
    h->d_chain_flags = nullptr;
    h->d_chain_flagoff = nullptr;
    h->d_chain_lpack = nullptr;
    h->chain_words = h->chain_ctr = 0;
    h->splan = Plan();
    h->aplan = Plan();
    h->splan_nrhs = h->aplan_nrhs = -1;
    h->ws_cols = 0;
    h->d_ksw = nullptr;
    h->d_kcnt = nullptr;
    h->ksw_items = 0;
    h->d_front = nullptr;
    h->d_dinv = nullptr;
    h->d_gcsr = h->mass_buf = nullptr;
    h->lu_factored = h->front_dirty = false;
    h->d_lu_code = nullptr;
    h->d_vrow = h->d_vcol = h->d_uinv = h->d_lu_part = h->d_upper_stage = nullptr;
    h->fplan_lu = Plan();
    h->splan_lu_f = Plan();
    h->splan_lu_b = Plan();
    h->d_xs = h->d_xts = nullptr;
    h->d_xsoff = nullptr;
    h->d_oz_sl = nullptr;
    h->d_oz_ex = nullptr;
    h->d_oz_soff = h->d_oz_eoff = nullptr;
    h->oz_sl_bytes = h->oz_ex_elems = 0;
    h->xs_elems = 0;
    h->d_values_stage = nullptr;
    h->front_elems = 0;
    h->g_factor.reset();
    h->g_solve.reset();
    h->sel_ready = false;
    h->sel_steps.clear();
    h->d_zpool = h->d_xw = h->d_sel_out = nullptr;
    h->d_xoff = h->d_upoff = nullptr;
    h->d_upmap = h->d_col2s = h->d_prow = h->d_psrc = nullptr;
    h->d_sel_items = nullptr;
    h->d_sel_gemm = nullptr;
    h->batch_count = 0;
    h->batch_coff.clear();
    h->batch_soff.clear();
    h->d_batch_soff = nullptr;
    h->d_batch_coff = nullptr;
    h->d_batch_norm = nullptr;
    h->d_batch_ld = nullptr;
    h->d_batch_sdl = nullptr;
    h->d_spmv_bad = nullptr;
    h->d_batch_cm = nullptr;
    h->batch_normA.clear();
    return WD_OK;
}

static wd_status finish_analysis(wd_handle h, std::chrono::steady_clock::time_point t0);

static wd_status check_geometry(wd_handle h, const wd_geometry *geom) {
    if (geom && (geom->dim < 0 || geom->dim > 3))
        return fail(h, WD_ERR_INVALID_ARG, "unsupported geometry");
    return WD_OK;
}

static int analyze_one(wd_handle h, wd::Symbolic &S, int64_t n, const int64_t *colptr,
                       const int32_t *rowidx, const wd_geometry *geom, std::string &msg) {
    const int dim = geom ? geom->dim : 0;
    return wd::analyze(S, n, colptr, rowidx, dim, geom ? geom->level : nullptr,
                       geom ? geom->box_lo : nullptr, geom ? geom->box_side : nullptr,
                       geom ? geom->patch : nullptr, h->opt.nd_leaf, h->opt.relax_k, h->opt.relax_pct,
                       msg);
}

extern "C" wd_status wd_analyze(wd_handle h, int64_t n, const int64_t *colptr, const int32_t *rowidx,
                                const wd_geometry *geom) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (n <= 0 || !colptr || !rowidx) return fail(h, WD_ERR_INVALID_ARG, "bad size or null pattern");
    wd_status st = check_geometry(h, geom);
    if (st != WD_OK) return st;
    auto t0 = std::chrono::steady_clock::now();
    st = reset_analysis(h);
    if (st != WD_OK) return st;
    std::string msg;
    int rc = analyze_one(h, h->S, n, colptr, rowidx, geom, msg);
    if (rc) return fail(h, (wd_status)rc, msg);
    return finish_analysis(h, t0);
}

extern "C" wd_status wd_analyze_batch(wd_handle h, int32_t count, const int64_t *n,
                                      const int64_t *const *colptr, const int32_t *const *rowidx,
                                      const wd_geometry *geom) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (count <= 0 || !n || !colptr || !rowidx) return fail(h, WD_ERR_INVALID_ARG, "bad batch");
    for (int32_t i = 0; i < count; ++i) {
        if (n[i] <= 0 || !colptr[i] || !rowidx[i])
            return fail(h, WD_ERR_INVALID_ARG, "bad size or null pattern of instance " + std::to_string(i));
        wd_status st = check_geometry(h, geom ? geom + i : nullptr);
        if (st != WD_OK) return st;
    }
    auto t0 = std::chrono::steady_clock::now();
    wd_status st = reset_analysis(h);
    if (st != WD_OK) return st;
    // instances with the same pattern and geometry arrays (same pointers) share one analysis
    std::vector<int32_t> uniq(count, -1);
    std::vector<int32_t> reps;
    for (int32_t i = 0; i < count; ++i) {
        for (size_t q = 0; q < reps.size(); ++q) {
            const int32_t r = reps[q];
            const bool same_geom =
                (!geom) || (geom[r].dim == geom[i].dim && geom[r].level == geom[i].level &&
                            geom[r].box_lo == geom[i].box_lo && geom[r].box_side == geom[i].box_side &&
                            geom[r].patch == geom[i].patch);
            if (n[r] == n[i] && colptr[r] == colptr[i] && rowidx[r] == rowidx[i] && same_geom) {
                uniq[i] = (int32_t)q;
                break;
            }
        }
        if (uniq[i] < 0) {
            uniq[i] = (int32_t)reps.size();
            reps.push_back(i);
        }
    }
    std::vector<wd::Symbolic> parts(reps.size());
    std::vector<int> rcs(reps.size(), 0);
    std::vector<std::string> msgs(reps.size());
    {
        const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        std::atomic<size_t> next{0};
        auto work = [&]() {
            for (size_t q = next++; q < reps.size(); q = next++) {
                const int32_t i = reps[q];
                rcs[q] = analyze_one(h, parts[q], n[i], colptr[i], rowidx[i], geom ? geom + i : nullptr,
                                     msgs[q]);
            }
        };
        std::vector<std::thread> pool;
        for (unsigned t = 1; t < std::min<size_t>(hw, reps.size()); ++t) pool.emplace_back(work);
        work();
        for (auto &t : pool) t.join();
    }
    for (size_t q = 0; q < reps.size(); ++q)
        if (rcs[q]) return fail(h, (wd_status)rcs[q], "instance " + std::to_string(reps[q]) + ": " + msgs[q]);
    std::vector<const wd::Symbolic *> seq(count);
    for (int32_t i = 0; i < count; ++i) seq[i] = &parts[uniq[i]];
    std::string msg;
    int rc = wd::merge(h->S, seq, msg);
    if (rc) return fail(h, (wd_status)rc, msg);
    h->batch_count = count;
    h->batch_coff.assign(count + 1, 0);
    h->batch_soff.assign(count + 1, 0);
    for (int32_t i = 0; i < count; ++i) {
        h->batch_coff[i + 1] = h->batch_coff[i] + seq[i]->n;
        h->batch_soff[i + 1] = h->batch_soff[i] + seq[i]->ns;
    }
    return finish_analysis(h, t0);
}

static wd_status finish_analysis(wd_handle h, std::chrono::steady_clock::time_point t0) {
    const bool host_only = h->opt.symbolic_only != 0;
    wd::Symbolic &S = h->S;
    const int64_t n = S.n;
    const int ns = S.ns;
    // per-supernode arrays
    std::vector<int32_t> sk(ns), sm(ns), skp(ns), sld(ns);
    std::vector<int64_t> foff(ns), woff(ns), dioff(ns), pkoff(ns);
    int64_t fo = 0, wo = 0, dio = 0, pko = 0;
    int maxm = 0, maxk = 0;
    for (int s = 0; s < ns; ++s) {
        sk[s] = S.k(s);
        sm[s] = S.m(s);
        skp[s] = (sk[s] + 31) / 32 * 32;
        const int mp = skp[s] + sm[s] - sk[s];
        sld[s] = (mp + 31) / 32 * 32;
        foff[s] = fo;
        woff[s] = wo;
        dioff[s] = dio;
        fo += (int64_t)sld[s] * mp;
        wo += sm[s] - sk[s];
        dio += (int64_t)((sk[s] + NB - 1) / NB) * NB * NB;
        pkoff[s] = pko;
        pko += wd::pack_bytes(sk[s], mp);
        maxm = std::max(maxm, sm[s]);
        maxk = std::max(maxk, sk[s]);
    }
    h->front_elems = (size_t)fo;
    std::vector<int64_t> xsoff(ns);
    {
        int64_t xo = 0;
        for (int s = 0; s < ns; ++s) {
            xsoff[s] = xo;
            const int nsb = (sk[s] + wd::SB - 1) / wd::SB;
            const int wl = sk[s] - (nsb - 1) * wd::SB, wpl = (wl + NB - 1) / NB * NB;
            xo += (int64_t)(nsb - 1) * wd::SB * wd::SB + (int64_t)wpl * wpl;
        }
        h->xs_elems = (size_t)xo;
    }
    h->h_foff = foff;
    h->h_sld = sld;
    h->dinv_elems = (size_t)dio;
    h->pack_total = pko;
    h->W_rows = wo;
    // full CSR of P A P^T with the source index of every value
    std::vector<int64_t> cptr(n + 1, 0), cdiag(n);
    const int64_t nnzl = S.pcp[n];
    for (int64_t j = 0; j < n; ++j)
        for (int64_t e = S.pcp[j]; e < S.pcp[j + 1]; ++e) {
            ++cptr[S.prow[e] + 1];
            if (S.prow[e] != j) ++cptr[j + 1];
        }
    for (int64_t i = 0; i < n; ++i) cptr[i + 1] += cptr[i];
    const int64_t nnzf = cptr[n];
    h->nnz_full = nnzf;
    std::vector<int32_t> ccol(nnzf), csrc(nnzf);
    h->h_csr_code.assign(nnzf, 0);
    {
        std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
        // row i gets, in column order: entries (i, j<i) from lower columns j,
        // then the diagonal and (i, j>i) from lower column i.  The code of a
        // position tells a nonsymmetric matrix's values apart (LU): which of
        // the source's two values is the entry and which its transpose
        for (int64_t j = 0; j < n; ++j)
            for (int64_t e = S.pcp[j] + 1; e < S.pcp[j + 1]; ++e) {
                const int32_t i = S.prow[e];
                ccol[fill[i]] = (int32_t)j;
                h->h_csr_code[fill[i]] = S.pswap[e] ? 1 : 0;
                csrc[fill[i]++] = S.psrc[e];
            }
        for (int64_t j = 0; j < n; ++j) {
            cdiag[j] = fill[j];
            for (int64_t e = S.pcp[j]; e < S.pcp[j + 1]; ++e) {
                ccol[fill[j]] = S.prow[e];
                h->h_csr_code[fill[j]] = S.prow[e] == j ? 2 : (S.pswap[e] ? 0 : 1);
                csrc[fill[j]++] = S.psrc[e];
            }
        }
    }
    build_factor_plan(S, h->fplan, false, h->opt.fp64_tc_schur != 0);
    h->chain = !h->opt.step_launches && h->opt.diag64_min_k <= 0;
    h->level_step.assign(S.nlevels, 0);
    build_factor_plan(S, h->fplan_tc, true, false, h->chain);
    std::vector<int64_t> chain_off(ns);
    {
        int64_t cw = 0;
        for (int s = 0; s < ns; ++s) {
            chain_off[s] = cw;
            cw += wd::chain_flag_words(sk[s], skp[s] + sm[s] - sk[s]);
        }
        h->chain_ctr = cw;
        h->chain_words = cw + S.nlevels + 1;
    }
    if (host_only) {
        fill_info(h, nnzl, maxm, maxk, t0);
        h->analyzed = true;
        return WD_OK;
    }
    DevSym &d = h->dsym;
    d.n = n;
    d.ns = ns;
    UP(S.sfirst, d.sfirst);
    UP(sk, d.sk);
    UP(sm, d.sm);
    UP(skp, d.skp);
    UP(sld, d.sld);
    UP(foff, d.foff);
    UP(S.srowptr, d.rowptr);
    UP(S.srows, d.rows);
    UP(S.child_ptr, d.child_ptr);
    UP(S.children, d.children);
    UP(S.mapoff, d.mapoff);
    UP(S.relmap, d.relmap);
    UP(S.pcp, d.pcp);
    {
        std::vector<int32_t> afr(S.alrow.size());
        for (int s = 0; s < ns; ++s)
            for (int j = S.sfirst[s]; j < S.sfirst[s + 1]; ++j)
                for (int64_t e = S.pcp[j]; e < S.pcp[j + 1]; ++e) {
                    const int r = S.alrow[e];
                    afr[e] = r < sk[s] ? r : r + skp[s] - sk[s];
                }
        UP(afr, d.alrow);
    }
    UP(cptr, d.csr_ptr);
    UP(ccol, d.csr_col);
    UP(cdiag, d.csr_diag);
    UP(woff, d.woff);
    UP(dioff, d.dinvoff);
    UP(pkoff, d.pkoff);
    UP(S.perm, d.perm);
    {
        const int64_t *p = nullptr;
        UP(chain_off, p);
        h->d_chain_flagoff = const_cast<int64_t *>(p);
        CK(h->mem.alloc((void **)&h->d_chain_flags, h->chain_words * sizeof(unsigned)), "dependency words alloc");
        CK(h->mem.alloc((void **)&h->d_chain_lpack, (h->dinv_elems / (NB * NB)) * (size_t)32768), "operand alloc");
    }
    {
        const int64_t *p = nullptr;
        UP(xsoff, p);
        h->d_xsoff = const_cast<int64_t *>(p);
    }
    if (h->opt.fp64_tc_schur) {
        std::vector<int64_t> so(ns), eo(ns);
        int64_t sb = 0, eb = 0;
        for (int s = 0; s < ns; ++s) {
            const int64_t nblk = (sk[s] + NB - 1) / NB, srow = wd::pack_rows(skp[s] + sm[s] - sk[s]);
            so[s] = sb;
            eo[s] = eb;
            sb += nblk * 8 * srow * 128;
            eb += nblk * srow;
        }
        h->oz_sl_bytes = std::max<int64_t>(sb, 128);
        h->oz_ex_elems = std::max<int64_t>(eb, 1);
        const int64_t *p = nullptr;
        UP(so, p);
        h->d_oz_soff = const_cast<int64_t *>(p);
        UP(eo, p);
        h->d_oz_eoff = const_cast<int64_t *>(p);
    }
    {
        const int32_t *p = nullptr;
        UP(csrc, p);
        h->d_csr_src = const_cast<int32_t *>(p);
    }
    CK(h->mem.alloc((void **)&h->d_csr_val, nnzf * sizeof(double)), "values alloc");
    CK(h->mem.alloc((void **)&h->d_csr_vh, nnzf * sizeof(float)), "values alloc");
    CK(h->mem.alloc((void **)&h->d_csr_vl, nnzf * sizeof(float)), "values alloc");
    {
        // residual work items: rows cut into chunks of at most SPMV_CHUNK entries
        std::vector<int4> ch, fin;
        int slots = 0;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t b0 = cptr[i], b1 = cptr[i + 1];
            const int64_t nc = (b1 - b0 + wd::SPMV_CHUNK - 1) / wd::SPMV_CHUNK;
            if (nc <= 1) {
                ch.push_back({(int)i, (int)b0, (int)b1, -1});
                continue;
            }
            fin.push_back({(int)i, slots, (int)nc, 0});
            for (int64_t q = 0; q < nc; ++q) {
                const int64_t e0 = b0 + q * wd::SPMV_CHUNK;
                ch.push_back({(int)i, (int)e0, (int)std::min(b1, e0 + wd::SPMV_CHUNK), slots++});
            }
        }
        h->n_spmv_chunks = (int)ch.size();
        h->n_spmv_fin = (int)fin.size();
        h->n_spmv_slots = slots;
        CK(h->mem.alloc((void **)&h->d_spmv_chunks, ch.size() * sizeof(int4)), "spmv items");
        CK(cudaMemcpy(h->d_spmv_chunks, ch.data(), ch.size() * sizeof(int4), cudaMemcpyHostToDevice), "upload");
        CK(h->mem.alloc((void **)&h->d_spmv_fin, std::max<size_t>(fin.size(), 1) * sizeof(int4)), "spmv items");
        if (!fin.empty())
            CK(cudaMemcpy(h->d_spmv_fin, fin.data(), fin.size() * sizeof(int4), cudaMemcpyHostToDevice), "upload");
        CK(h->mem.alloc((void **)&h->d_norm_part, std::max(slots, 1) * sizeof(double)), "norm partials");
        CK(h->mem.alloc((void **)&h->d_spmv_bad, sizeof(unsigned long long)), "spmv check");
    }
    d.csr_val = h->d_csr_val;
    CK(h->mem.alloc((void **)&h->d_status, sizeof(status_t)), "status alloc");
    CK(h->mem.alloc((void **)&h->d_scalars, 1024 * sizeof(double)), "scalars alloc");
    {
        wd_status st = upload_plan(h, h->mem, h->fplan);
        if (st != WD_OK) return st;
        st = upload_plan(h, h->mem, h->fplan_tc);
        if (st != WD_OK) return st;
    }
    CK(h->mem.alloc((void **)&h->d_tstatus, sizeof(status_t)), "status alloc");
    if (h->opt.test_closed_gate) {
        CK(h->mem.alloc((void **)&h->d_gate, sizeof(unsigned)), "gate alloc");
        CK(cudaMemset(h->d_gate, 0, sizeof(unsigned)), "gate clear");
    }
    if (h->batch_count > 0) {
        const int64_t *pc = nullptr;
        const int32_t *ps = nullptr;
        UP(h->batch_coff, pc);
        UP(h->batch_soff, ps);
        h->d_batch_coff = const_cast<int64_t *>(pc);
        h->d_batch_soff = const_cast<int32_t *>(ps);
        CK(h->mem.alloc((void **)&h->d_batch_norm, h->batch_count * sizeof(double)), "batch alloc");
        CK(h->mem.alloc((void **)&h->d_batch_ld, h->batch_count * sizeof(double)), "batch alloc");
        CK(h->mem.alloc((void **)&h->d_batch_sdl, std::max(ns, 1) * sizeof(double)), "batch alloc");
    }
    fill_info(h, nnzl, maxm, maxk, t0);
    h->analyzed = true;
    return WD_OK;
}

extern "C" wd_status wd_symbolic_export(wd_handle h, int32_t *perm, int32_t *parent,
                                        int64_t *colcount, int32_t *super_first,
                                        int64_t *super_rowptr, int32_t *super_rows) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->analyzed) return fail(h, WD_ERR_STATE, "not analyzed");
    const wd::Symbolic &S = h->S;
    if (perm) std::memcpy(perm, S.perm.data(), S.n * sizeof(int32_t));
    if (parent) std::memcpy(parent, S.parent.data(), S.n * sizeof(int32_t));
    if (colcount) std::memcpy(colcount, S.colcount.data(), S.n * sizeof(int64_t));
    if (super_first) std::memcpy(super_first, S.sfirst.data(), S.sfirst.size() * sizeof(int32_t));
    if (super_rowptr) std::memcpy(super_rowptr, S.srowptr.data(), S.srowptr.size() * sizeof(int64_t));
    if (super_rows) std::memcpy(super_rows, S.srows.data(), S.srows.size() * sizeof(int32_t));
    return WD_OK;
}

extern "C" wd_status wd_get_info(wd_handle h, wd_info *info) {
    if (!h || !info) return WD_ERR_INVALID_ARG;
    if (!h->analyzed) return fail(h, WD_ERR_STATE, "not analyzed");
    *info = h->info;
    return WD_OK;
}

// ---------------------------------------------------------------------------
// factor
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// profiling: events around every launch of a plan, accumulated per kernel
// ---------------------------------------------------------------------------
// inside a stream capture an event becomes a timing node of the graph only
// with cudaEventRecordExternal; outside a capture the plain record is used
static void record_event(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
}

static bool prof_begin(wd_handle h, size_t nlaunch) {
    if (!h->opt.profile) return false;
    while (h->prof_ev.size() < 2 * nlaunch) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return false;
        h->prof_ev.push_back(e);
    }
    return true;
}

static void prof_end(wd_handle h, const Plan &p, size_t elem_size, const char *suffix) {
    const size_t nl = p.launches.size();
    if (nl == 0) return;
    cudaEventSynchronize(h->prof_ev[2 * nl - 1]);
    for (size_t i = 0; i < nl; ++i) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]) != cudaSuccess) {
            cudaGetLastError();  // a profiling failure must not poison later calls
            ms = 0;
        }
        const Launch &L = p.launches[i];
        std::string name = std::string(kind_name(L.kind)) + suffix;
        KStat *st = nullptr;
        for (auto &kv : h->prof)
            if (kv.first == name) st = &kv.second;
        if (!st) {
            h->prof.push_back({name, KStat()});
            st = &h->prof.back().second;
        }
        st->launches += 1;
        st->ms += ms;
        st->flops += L.flops;
        st->bytes += L.elems * (double)elem_size + L.bytes;
    }
}

// profiling of a single launch outside the plans (events, synchronizing)
static void prof_single(wd_handle h, const char *name, double flops, double bytes, cudaStream_t st,
                        bool begin) {
    if (!h->opt.profile) return;
    if (h->single_ev[0] == nullptr) {
        if (cudaEventCreate(&h->single_ev[0]) != cudaSuccess ||
            cudaEventCreate(&h->single_ev[1]) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
    }
    if (begin) {
        cudaEventRecord(h->single_ev[0], st);
        return;
    }
    cudaEventRecord(h->single_ev[1], st);
    cudaEventSynchronize(h->single_ev[1]);
    float ms = 0;
    if (cudaEventElapsedTime(&ms, h->single_ev[0], h->single_ev[1]) != cudaSuccess) {
        cudaGetLastError();
        ms = 0;
    }
    KStat *stt = nullptr;
    for (auto &kv : h->prof)
        if (kv.first == name) stt = &kv.second;
    if (!stt) {
        h->prof.push_back({name, KStat()});
        stt = &h->prof.back().second;
    }
    stt->launches += 1;
    stt->ms += ms;
    stt->flops += flops;
    stt->bytes += bytes;
}

extern "C" wd_status wd_launch_count(wd_handle h, int64_t *count, int reset) {
    if (!h || !count) return WD_ERR_INVALID_ARG;
    *count = h->launches;
    if (reset) h->launches = 0;
    return WD_OK;
}

extern "C" wd_status wd_kernel_stats(wd_handle h, wd_kernel_stat *out, int32_t cap, int32_t *count,
                                     int reset) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (count) *count = (int32_t)h->prof.size();
    for (int32_t i = 0; out && i < cap && i < (int32_t)h->prof.size(); ++i) {
        std::memset(&out[i], 0, sizeof(out[i]));
        std::snprintf(out[i].name, sizeof(out[i].name), "%s", h->prof[i].first.c_str());
        out[i].launches = h->prof[i].second.launches;
        out[i].milliseconds = h->prof[i].second.ms;
        out[i].flops = h->prof[i].second.flops;
        out[i].bytes = h->prof[i].second.bytes;
    }
    if (reset) h->prof.clear();
    return WD_OK;
}

template <class T>
static void enqueue_factor_plan(wd_handle h, cudaStream_t st, bool prof) {
    T *F = static_cast<T *>(h->d_front);
    T *Dv = static_cast<T *>(h->d_dinv);
    const DevSym &d = h->dsym;
    const bool fp32 = sizeof(T) == 4;
    const Plan &P = fp32 ? h->fplan_tc : h->fplan;
    unsigned char *pk = fp32 ? h->d_pack : nullptr;
    wd::TcArgs ta{};
    ta.dinv = reinterpret_cast<float *>(Dv);
    ta.status = h->d_status;
    ta.tstatus = h->d_tstatus;
    ta.diag64_min_k = h->opt.diag64_min_k;
    ta.wait_limit = (uint32_t)std::max(0, h->opt.wait_limit);
    ta.gate = h->opt.test_closed_gate ? h->d_gate : nullptr;
    ta.ctas = h->sms;       // the fronts' trailing blocks: one persistent CTA per SM
    wd::OzArgs oa{};
    oa.sl = h->d_oz_sl;
    oa.ex = h->d_oz_ex;
    oa.soff = h->d_oz_soff;
    oa.eoff = h->d_oz_eoff;
    oa.dinv = reinterpret_cast<double *>(Dv);
    oa.status = h->d_status;
    oa.tstatus = h->d_tstatus;
    oa.wait_limit = ta.wait_limit;
    wd::ChainArgs ca{};
    ca.dinv = reinterpret_cast<float *>(Dv);
    ca.lpack = h->d_chain_lpack;
    ca.status = h->d_status;
    ca.tstatus = h->d_tstatus;
    ca.wait_limit = ta.wait_limit;
    ca.gate = ta.gate;
    ca.flags = h->d_chain_flags;
    ca.flagoff = h->d_chain_flagoff;
    ca.counter = h->d_chain_flags + h->chain_ctr;
    ca.gabort = h->d_chain_flags + h->chain_words - 1;
    if (fp32 && h->chain)
        cudaMemsetAsync(h->d_chain_flags, 0, h->chain_words * sizeof(unsigned), st);
    size_t li = 0;
    for (const Launch &L : P.launches) {
        const int4 *it = P.d_items + L.off;
        if (prof) record_event(h->prof_ev[2 * li], st);
        switch (L.kind) {
            case K_CHAIN_TC:
                wd::launch_tc_chain(d, reinterpret_cast<float *>(F), pk, it, L.count, L.arg, ca, st);
                break;
            case K_INIT: wd::launch_front_init<T>(d, F, it, L.count, st); break;
            case K_DIAG:
                wd::launch_diag_factor<T>(d, F, Dv, it, L.count, h->opt.diag64_min_k, h->d_status, st);
                break;
            case K_PANEL: wd::launch_panel<T>(d, F, Dv, pk, it, L.count, L.arg, st); break;
            case K_UPDATE: wd::launch_schur<T>(d, F, Dv, it, L.count, L.arg, 0, h->d_status, st); break;
            case K_SYRK: wd::launch_schur<T>(d, F, Dv, it, L.count, 0, 1, h->d_status, st); break;
            case K_UPDATE_TC:
                wd::launch_tc_schur(d, reinterpret_cast<float *>(F), pk, it, L.count, L.arg, 0, ta, st);
                break;
            case K_SYRK_TC:
                wd::launch_tc_schur(d, reinterpret_cast<float *>(F), pk, it, L.count, 0, 1, ta, st);
                break;
            case K_OZ_SLICE:
                wd::launch_oz_slice(d, reinterpret_cast<const double *>(F), oa, it, L.count, L.arg, st);
                break;
            case K_OZ_UPDATE:
                wd::launch_oz_schur(d, reinterpret_cast<double *>(F), it, L.count, L.arg, 0, oa, st);
                break;
            case K_OZ_SYRK: wd::launch_oz_schur(d, reinterpret_cast<double *>(F), it, L.count, 0, 1, oa, st); break;
            case K_SBINV_DIAG:
                wd::launch_sbinv_diag<T>(d, Dv, static_cast<T *>(h->d_xs), h->d_xsoff, it, L.count, st);
                break;
            case K_SBINV_STAGE:
                wd::launch_sbinv_stage<T>(d, F, Dv, static_cast<T *>(h->d_xs), h->d_xsoff, it, L.count, L.arg,
                                          st);
                break;
            case K_SBINV_T:
                wd::launch_sbinv_transpose<T>(d, static_cast<const T *>(h->d_xs), static_cast<T *>(h->d_xts),
                                              h->d_xsoff, it, L.count, st);
                break;
        }
        if (prof) record_event(h->prof_ev[2 * li + 1], st);
        ++li;
    }
}

// Run a launch sequence: captured once into a CUDA graph (keyed), replayed on
// the caller's stream; or launched directly when graphs are disabled.
template <class Body>
static wd_status run_graph(wd_handle h, GraphCache &gc, int64_t key, cudaStream_t st, Body body) {
    if (!h->opt.use_graphs) {
        body(st);
        CK(cudaGetLastError(), "launch");
        return WD_OK;
    }
    if (gc.key != key || !gc.exec) {
        gc.reset();
        CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "capture");
        body(h->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
        if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
        e = cudaGraphInstantiate(&gc.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            gc.exec = nullptr;
            return cuda_fail(h, e, "graph instantiate");
        }
        gc.key = key;
    }
    CK(cudaGraphLaunch(gc.exec, st), "graph launch");
    return WD_OK;
}

template <class T>
static wd_status run_factor_plan(wd_handle h, cudaStream_t st) {
    const Plan &P = sizeof(T) == 4 ? h->fplan_tc : h->fplan;
    const bool prof = prof_begin(h, P.launches.size());
    const int64_t key = (sizeof(T) == 8 ? 1 : 2) + (prof ? 10 : 0);
    wd_status s = run_graph(h, h->g_factor, key, st,
                            [&](cudaStream_t cs) { enqueue_factor_plan<T>(h, cs, prof); });
    if (s != WD_OK) return s;
    h->launches += (int64_t)P.launches.size();
    if (prof) prof_end(h, P, sizeof(T), sizeof(T) == 8 ? "_fp64" : "_fp32");
    return WD_OK;
}

extern "C" wd_status wd_factor(wd_handle h, const double *values, int values_on_device,
                               wd_precision prec, void *stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->analyzed || h->opt.symbolic_only)
        return fail(h, WD_ERR_STATE, "wd_factor before wd_analyze (or on a host-only handle)");
    if (!values || (prec != WD_FP64 && prec != WD_MIXED))
        return fail(h, WD_ERR_INVALID_ARG, "null values or bad precision");
    CK(cudaSetDevice(h->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wait_export(h);   // a pending allocation-free export still reads the fronts
    h->factored = false;
    h->lu_factored = false;
    if (h->front_dirty && h->d_front) {
        // an LU factor filled the upper parts that the Cholesky kernels keep zero
        CK(cudaMemsetAsync(h->d_front, 0, h->front_elems * sizeof(double), st), "front pool clear");
        h->front_dirty = false;
    }
    const int64_t nnzl = h->S.pcp[h->S.n];
    if (!h->d_front) {
        CK(h->mem.alloc(&h->d_front, h->front_elems * sizeof(double)), "front pool alloc");
        CK(h->mem.alloc(&h->d_dinv, h->dinv_elems * sizeof(double)), "inverse blocks alloc");
        CK(h->mem.alloc(&h->d_xs, h->xs_elems * sizeof(double)), "super-block inverse alloc");
        CK(h->mem.alloc(&h->d_xts, h->xs_elems * sizeof(double)), "super-block inverse alloc");
        // padding rows stay zero forever: no kernel writes them
        CK(cudaMemsetAsync(h->d_front, 0, h->front_elems * sizeof(double), st), "front pool clear");
    }
    if (prec == WD_FP64 && h->opt.fp64_tc_schur && !h->d_oz_sl) {
        CK(h->mem.alloc((void **)&h->d_oz_sl, h->oz_sl_bytes), "slice planes alloc");
        CK(h->mem.alloc((void **)&h->d_oz_ex, h->oz_ex_elems * sizeof(int16_t)), "slice scales alloc");
        // rows no slicing writes (padding, the window past the front) stay zero
        CK(cudaMemsetAsync(h->d_oz_sl, 0, h->oz_sl_bytes, st), "slice planes clear");
        CK(cudaMemsetAsync(h->d_oz_ex, 0, h->oz_ex_elems * sizeof(int16_t), st), "slice scales clear");
        h->g_factor.reset();
    }
    if (prec == WD_MIXED && !h->d_pack) {
        CK(h->mem.alloc((void **)&h->d_pack, h->pack_total), "packed panel alloc");
        // rows no panel writes (slack, padding of the last block) stay zero
        CK(cudaMemsetAsync(h->d_pack, 0, h->pack_total, st), "packed panel clear");
        h->g_factor.reset();
    }
    const double *vals = values;
    if (!values_on_device) {
        if (!h->d_values_stage)
            CK(h->mem.alloc((void **)&h->d_values_stage, nnzl * sizeof(double)), "stage alloc");
        CK(cudaMemcpyAsync(h->d_values_stage, values, nnzl * sizeof(double), cudaMemcpyHostToDevice, st),
           "values H2D");
        vals = h->d_values_stage;
    }
    wd::launch_gather_values(h->d_csr_src, vals, h->d_csr_val, h->d_csr_vh, h->d_csr_vl, h->nnz_full, st);
    h->launches += 1;
    CK(cudaMemsetAsync(h->d_status, 0xFF, sizeof(status_t), st), "status reset");
    CK(cudaMemsetAsync(h->d_tstatus, 0, sizeof(status_t), st), "status reset");
    {
        wd_status fs = (prec == WD_FP64) ? run_factor_plan<double>(h, st) : run_factor_plan<float>(h, st);
        if (fs != WD_OK) return fs;
    }
    wd::launch_norm_inf_rows(h->dsym, h->d_spmv_chunks, h->n_spmv_chunks, h->d_spmv_fin, h->n_spmv_fin,
                             h->d_norm_part, h->d_scalars, st);
    h->launches += h->n_spmv_fin > 0 ? 2 : 1;
    if (h->batch_count > 0) {
        wd::launch_seg_norm_inf(h->dsym, h->d_spmv_chunks, h->n_spmv_chunks, h->d_spmv_fin, h->n_spmv_fin,
                                h->d_norm_part, h->d_batch_coff, h->batch_count, h->d_batch_norm, st);
        h->launches += 1;
        h->batch_normA.resize(h->batch_count);
        CK(cudaMemcpyAsync(h->batch_normA.data(), h->d_batch_norm, h->batch_count * sizeof(double),
                           cudaMemcpyDeviceToHost, st),
           "norm D2H");
    }
    CK(cudaGetLastError(), "factor launch");
    status_t status = 0, tstatus = 0;
    CK(cudaMemcpyAsync(&status, h->d_status, sizeof(status_t), cudaMemcpyDeviceToHost, st), "status D2H");
    CK(cudaMemcpyAsync(&tstatus, h->d_tstatus, sizeof(status_t), cudaMemcpyDeviceToHost, st), "status D2H");
    CK(cudaMemcpyAsync(&h->normA, h->d_scalars, sizeof(double), cudaMemcpyDeviceToHost, st), "norm D2H");
    CK(cudaStreamSynchronize(st), "factor");
    if (tstatus != 0) return fail(h, WD_ERR_TIMEOUT, "a bounded wait of the tensor-core update expired");
    if (status != ~0ULL) {
        std::string where = "pivot not positive at column " + std::to_string(status);
        if (h->batch_count > 0) {
            const auto it = std::upper_bound(h->batch_coff.begin(), h->batch_coff.end(), (int64_t)status);
            const int64_t inst = (it - h->batch_coff.begin()) - 1;
            where += " (instance " + std::to_string(inst) + ", its column " +
                     std::to_string((int64_t)status - h->batch_coff[inst]) + " in factor order)";
        }
        return fail(h, WD_ERR_NOT_SPD, where, (int64_t)status);
    }
    h->prec = prec;
    h->factored = true;
    return WD_OK;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
static wd_status ensure_solve_ws(wd_handle h, int64_t nrhs) {
    if (h->ws_cols >= nrhs) return WD_OK;
    h->work.free_all();
    h->d_Y = h->d_W = h->d_T = h->d_part = nullptr;
    h->part_elems = 0;
    h->d_B = h->d_Bp = h->d_X = h->d_R = h->d_cm = h->d_P = nullptr;
    h->d_Xp = nullptr;
    h->d_ksw = nullptr;
    h->d_kcnt = nullptr;
    h->ksw_items = 0;
    h->splan = Plan();
    h->aplan = Plan();
    h->splan_nrhs = h->aplan_nrhs = -1;
    h->g_solve.reset();
    const int64_t n = h->S.n;
    CK(h->work.alloc(&h->d_Y, n * nrhs * sizeof(double)), "solve ws");
    CK(h->work.alloc(&h->d_T, n * nrhs * sizeof(double)), "solve ws");
    CK(h->work.alloc(&h->d_W, std::max<int64_t>(h->W_rows, 1) * nrhs * sizeof(double)), "solve ws");
    CK(h->work.alloc((void **)&h->d_B, n * nrhs * sizeof(double)), "solve ws");
    CK(h->work.alloc((void **)&h->d_Bp, n * nrhs * sizeof(double)), "solve ws");
    CK(h->work.alloc((void **)&h->d_X, n * nrhs * sizeof(double)), "solve ws");
    CK(h->work.alloc((void **)&h->d_Xp, n * nrhs * sizeof(float2)), "solve ws");
    CK(h->work.alloc((void **)&h->d_R, n * nrhs * sizeof(double)), "solve ws");
    CK(h->work.alloc((void **)&h->d_cm, 3 * nrhs * sizeof(double)), "solve ws");
    CK(h->work.alloc((void **)&h->d_P, std::max(h->n_spmv_slots, 1) * nrhs * sizeof(double)), "solve ws");
    h->d_batch_cm = nullptr;
    if (h->batch_count > 0)
        CK(h->work.alloc((void **)&h->d_batch_cm, 3 * (int64_t)h->batch_count * nrhs * sizeof(double)),
           "solve ws");
    h->ws_cols = nrhs;
    return WD_OK;
}

template <class T>
static void enqueue_solve_plan(wd_handle h, T *Y, int nrhs, cudaStream_t st, bool prof) {
    const T *F = static_cast<const T *>(h->d_front);
    const T *Xs = static_cast<const T *>(h->d_xs);
    const T *XTs = static_cast<const T *>(h->d_xts);
    T *W = static_cast<T *>(h->d_W);
    T *Tt = static_cast<T *>(h->d_T);
    T *P = static_cast<T *>(h->d_part);
    const DevSym &d = h->dsym;
    const int rgt = h->splan.rgt;
    const int lg = h->splan.large;
    // tensor-core products (FP32 only): forward xapply reads X's rows from the
    // stored X^T, backward reads X^T's rows from X
    wd::TcSolveArgs ta{};
    ta.front = reinterpret_cast<const float *>(F);
    ta.pk = h->d_pack;
    ta.xsoff = h->d_xsoff;
    ta.W = reinterpret_cast<float *>(W);
    ta.tstatus = h->d_tstatus;
    ta.nrhs = nrhs;
    ta.wait_limit = (uint32_t)std::max(0, h->opt.wait_limit);
    ta.ksw = h->d_ksw;
    ta.kcnt = h->d_kcnt;
    ta.sms = h->sms;
    const bool tc = lg == 1 && sizeof(T) == 4;
    size_t li = 0;
    for (const Launch &L : h->splan.launches) {
        const int4 *it = h->splan.d_items + L.off;
        if (prof) record_event(h->prof_ev[2 * li], st);
        switch (L.kind) {
            case K_FWD_GATHER: wd::launch_bfwd_gather<T>(d, Y, Tt, W, it, L.count, rgt, nrhs, st); break;
            case K_FWD_XAPPLY:
                if (tc) {
                    wd::TcSolveArgs a = ta;
                    a.xp = reinterpret_cast<const float *>(XTs);
                    a.in = reinterpret_cast<const float *>(Tt);
                    a.out = reinterpret_cast<float *>(Y);
                    a.upper = 0;
                    wd::launch_tc_xapply(d, a, it, L.count, st);
                } else {
                    wd::launch_xapply<T>(d, Xs, h->d_xsoff, Tt, Y, it, L.count, 0, lg, nrhs, st);
                }
                break;
            case K_FWD_BUPDATE:
                if (tc) {
                    wd::TcSolveArgs a = ta;
                    a.in = reinterpret_cast<const float *>(Y);
                    a.out = reinterpret_cast<float *>(Tt);
                    wd::launch_tc_bupdate(d, a, it, L.count, st);
                } else {
                    wd::launch_bupdate<T>(d, F, Y, Tt, W, it, L.count, lg, nrhs, st);
                }
                break;
            case K_BWD_REDUCE:
                if (tc) {
                    wd::TcSolveArgs a = ta;
                    a.in = reinterpret_cast<const float *>(Y);
                    a.out = reinterpret_cast<float *>(P);
                    wd::launch_tc_breduce(d, a, it, L.count, st);
                } else {
                    wd::launch_breduce<T>(d, F, Y, P, it, L.count, lg, nrhs, st);
                }
                break;
            case K_BWD_FINISH: wd::launch_breduce_finish<T>(d, Y, Tt, P, it, L.count, lg, nrhs, st); break;
            case K_BWD_XAPPLY:
                if (tc) {
                    wd::TcSolveArgs a = ta;
                    a.xp = reinterpret_cast<const float *>(Xs);
                    a.in = reinterpret_cast<const float *>(Tt);
                    a.out = reinterpret_cast<float *>(Y);
                    a.upper = 1;
                    wd::launch_tc_xapply(d, a, it, L.count, st);
                } else {
                    wd::launch_xapply<T>(d, XTs, h->d_xsoff, Tt, Y, it, L.count, 1, lg, nrhs, st);
                }
                break;
        }
        if (prof) record_event(h->prof_ev[2 * li + 1], st);
        ++li;
    }
}

template <class T>
static wd_status run_solve_plan(wd_handle h, T *Y, int nrhs, cudaStream_t st) {
    const bool prof = prof_begin(h, h->splan.launches.size());
    const int64_t key = ((int64_t)nrhs << 8) + (sizeof(T) == 8 ? 1 : 2) + (prof ? 10 : 0);
    wd_status s = run_graph(h, h->g_solve, key, st,
                            [&](cudaStream_t cs) { enqueue_solve_plan<T>(h, Y, nrhs, cs, prof); });
    if (s != WD_OK) return s;
    h->launches += (int64_t)h->splan.launches.size();
    if (prof) prof_end(h, h->splan, sizeof(T), sizeof(T) == 8 ? "_fp64" : "_fp32");
    return WD_OK;
}

// R = Bp - A X (row-major n x nrhs, factor order) to FP64 accuracy: FP64 up
// to 8 columns (with the device check of the column indices, read back by the
// caller from d_spmv_bad), double-float arithmetic beyond
static wd_status launch_residual(wd_handle h, const double *X, int64_t nrhs, cudaStream_t st,
                                 const float *Xf = nullptr, const double *S = nullptr) {
    const int64_t n = h->S.n;
    const double nf = (double)h->nnz_full;
    if (nrhs > 8 && Xf != nullptr) {
        // x exactly FP32: R = S - A x (S = b, or R itself for the recurrence)
        prof_single(h, "spmv_residual_df32", 0, 0, st, true);
        wd::launch_spmv_residual_df32(h->dsym, h->d_spmv_chunks, h->n_spmv_chunks, h->d_spmv_fin,
                                      h->n_spmv_fin, h->d_csr_vh, h->d_csr_vl, Xf, S, h->d_R, h->d_P, nrhs, st);
        prof_single(h, "spmv_residual_df32", 2.0 * nf * nrhs, 12.0 * nf + 20.0 * n * nrhs, st, false);
        h->launches += h->n_spmv_fin > 0 ? 2 : 1;
    } else if (nrhs > 8) {
        // many right-hand sides: double-float arithmetic on the FP32 pipes
        prof_single(h, "spmv_residual_df", 0, 0, st, true);
        wd::launch_spmv_residual_df(h->dsym, h->d_spmv_chunks, h->n_spmv_chunks, h->d_spmv_fin,
                                    h->n_spmv_fin, h->d_csr_vh, h->d_csr_vl, X, h->d_Xp, h->d_Bp,
                                    h->d_R, h->d_P, nrhs, st);
        prof_single(h, "spmv_residual_df", 2.0 * nf * nrhs, 12.0 * nf + 24.0 * n * nrhs, st, false);
        h->launches += h->n_spmv_fin > 0 ? 3 : 2;
    } else {
        CK(cudaMemsetAsync(h->d_spmv_bad, 0xff, sizeof(unsigned long long), st), "spmv check");
        prof_single(h, "spmv_residual_fp64", 0, 0, st, true);
        wd::launch_spmv_residual(h->dsym, h->d_spmv_chunks, h->n_spmv_chunks, h->d_spmv_fin,
                                 h->n_spmv_fin, X, h->d_Bp, h->d_R, h->d_P, nrhs, h->d_spmv_bad, st);
        prof_single(h, "spmv_residual_fp64", 2.0 * nf * nrhs, 12.0 * nf + 24.0 * n * nrhs, st, false);
        h->launches += h->n_spmv_fin > 0 ? 2 : 1;
    }
    CK(cudaGetLastError(), "residual launch");
    return WD_OK;
}

// R = Bp - A X (FP64, row-major n x nrhs) and the largest normwise backward
// error over the columns
static wd_status backward_errors(wd_handle h, const double *X, int64_t nrhs, cudaStream_t st,
                                 double *be_max, const float *Xf = nullptr, const double *S = nullptr) {
    const int64_t n = h->S.n;
    unsigned long long bad = ~0ULL;
    wd_status rs = launch_residual(h, X, nrhs, st, Xf, S);
    if (rs != WD_OK) return rs;
    if (h->batch_count > 0) {
        // per instance and column: each instance is its own system
        const int cnt = h->batch_count;
        wd::launch_seg_colmax3(h->d_R, X, h->d_Bp, h->d_batch_coff, cnt, (int)nrhs, h->d_batch_cm, st);
        h->launches += 2;
        std::vector<double> cm(3 * (size_t)cnt * nrhs);
        if (nrhs <= 8)
            CK(cudaMemcpyAsync(&bad, h->d_spmv_bad, sizeof(bad), cudaMemcpyDeviceToHost, st), "spmv check");
        CK(cudaMemcpyAsync(cm.data(), h->d_batch_cm, cm.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
           "be D2H");
        CK(cudaStreamSynchronize(st), "backward error");
        if (bad != ~0ULL)
            return fail(h, WD_ERR_CUDA, "residual: column index out of range at CSR position " + std::to_string(bad));
        double mx = 0.0;
        for (int i = 0; i < cnt; ++i)
            for (int64_t c = 0; c < nrhs; ++c) {
                const double *q = cm.data() + ((size_t)i * nrhs + c) * 3;
                const double den = h->batch_normA[i] * q[1] + q[2];
                mx = std::max(mx, den > 0 ? q[0] / den : 0.0);
            }
        *be_max = mx;
        return WD_OK;
    }
    wd::launch_colmax3(h->d_R, X, h->d_Bp, n, nrhs, h->d_cm, st);
    h->launches += 2;
    std::vector<double> cm(3 * nrhs);
    if (nrhs <= 8)
        CK(cudaMemcpyAsync(&bad, h->d_spmv_bad, sizeof(bad), cudaMemcpyDeviceToHost, st), "spmv check");
    CK(cudaMemcpyAsync(cm.data(), h->d_cm, cm.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "be D2H");
    CK(cudaStreamSynchronize(st), "backward error");
    if (bad != ~0ULL)
        return fail(h, WD_ERR_CUDA, "residual: column index out of range at CSR position " + std::to_string(bad));
    double mx = 0.0;
    for (int64_t c = 0; c < nrhs; ++c) {
        const double den = h->normA * cm[3 * c + 1] + cm[3 * c + 2];
        const double be = den > 0 ? cm[3 * c] / den : 0.0;
        mx = std::max(mx, be);
    }
    *be_max = mx;
    return WD_OK;
}

// workspaces and the launch plan of solves with nrhs right-hand sides
static wd_status prepare_solve(wd_handle h, int64_t nrhs) {
    wd_status s = ensure_solve_ws(h, nrhs);
    if (s != WD_OK) return s;
    // tiles of 64 rows x 32 right-hand sides; FP32 with more than 8
    // right-hand sides: tensor-core tiles of 128 rows x 64 right-hand sides
    // (unless wd_options.solve_simt); up to 8 right-hand sides:
    // matrix-vector shaped kernels, lanes over rows
    const int large = nrhs <= 8 ? 2 : (h->prec == WD_MIXED && !h->opt.solve_simt ? 1 : 0);
    if (h->splan_nrhs != nrhs || h->splan.large != large) {
        build_solve_plan(h->S, (int)nrhs, large, h->sms, h->splan);
        s = upload_plan(h, h->work, h->splan);
        if (s != WD_OK) return s;
        if (h->splan.ksplit > h->ksw_items) {
            if (h->d_ksw) h->work.release(h->d_ksw);
            if (h->d_kcnt) h->work.release(h->d_kcnt);
            h->d_ksw = nullptr;
            h->d_kcnt = nullptr;
            h->ksw_items = 0;
            CK(h->work.alloc((void **)&h->d_ksw, h->splan.ksplit * wd::TC_SOLVE_TILE * sizeof(float)), "solve ws");
            CK(h->work.alloc((void **)&h->d_kcnt, h->splan.ksplit * sizeof(int)), "solve ws");
            CK(cudaMemset(h->d_kcnt, 0, h->splan.ksplit * sizeof(int)), "solve ws clear");
            h->ksw_items = h->splan.ksplit;
        }
        const int64_t need = std::max<int64_t>(h->splan.slots, 1) * wd::solve_tile_rows(large) *
                             wd::solve_tile_rhs(large);
        if (need > h->part_elems) {
            if (h->d_part) h->work.release(h->d_part);
            h->d_part = nullptr;
            h->part_elems = 0;
            CK(h->work.alloc(&h->d_part, need * sizeof(double)), "solve ws");
            h->part_elems = need;
        }
        h->splan_nrhs = (int)nrhs;
        h->g_solve.reset();
    }
    return WD_OK;
}

// The solve of the right-hand sides staged in d_Bp (factor order, row-major,
// FP64): both substitutions, refinement in mixed precision, the result into
// Bd (device, column-major, ld); when B is a host array (B_on_device = 0,
// Bd = d_B) it is copied back to B (ldb).  Synchronous.
static wd_status solve_core(wd_handle h, double *Bd, int64_t ld, double *B, int64_t ldb, int B_on_device,
                            int64_t nrhs, cudaStream_t st, wd_solve_info *info) {
    const int64_t n = h->S.n;
    const int nr = (int)nrhs;
    wd_status s;
    if (h->prec == WD_FP64) {
        double *Y = static_cast<double *>(h->d_Y);
        wd::launch_transpose<double>(Y, h->d_Bp, n, nrhs, 0, 0, st);
        h->launches += 1;
        s = run_solve_plan<double>(h, Y, nr, st);
        if (s != WD_OK) return s;
        if (info) {
            wd::launch_transpose<double>(Y, h->d_X, n, nrhs, 1, 0, st);
            h->launches += 1;
            double be;
            s = backward_errors(h, h->d_X, nrhs, st, &be);
            if (s != WD_OK) return s;
            info->backward_error = be;
        }
        wd::launch_permute_out<double>(Y, Bd, ld, h->dsym.perm, n, nrhs, st);
        h->launches += 1;
    } else {
        float *Y = static_cast<float *>(h->d_Y);
        CK(cudaMemsetAsync(h->d_tstatus, 0, sizeof(status_t), st), "status reset");
        wd::launch_transpose<float>(Y, h->d_Bp, n, nrhs, 0, 0, st);
        s = run_solve_plan<float>(h, Y, nr, st);
        if (s != WD_OK) return s;
        // many right-hand sides: the solution and every correction are exactly
        // FP32, so r_0 = b - A x_0 and r_{k+1} = r_k - A d_k take the FP32
        // values (Xf, in the double-float split buffer) and never re-read the
        // refined FP64 x; up to 8: the FP64 residual of x itself
        float *Xf = nrhs > 8 ? reinterpret_cast<float *>(h->d_Xp) : nullptr;
        if (Xf) wd::launch_xupdate(Y, h->d_X, Xf, n, nrhs, 0, st);
        else wd::launch_transpose<float>(Y, h->d_X, n, nrhs, 1, 0, st);
        h->launches += 2;
        CK(cudaGetLastError(), "solve launch");
        double be = 1.0;
        int it = 0;
        for (;;) {
            s = backward_errors(h, h->d_X, nrhs, st, &be, Xf, it == 0 ? h->d_Bp : h->d_R);
            if (s != WD_OK) return s;
            if (be <= h->opt.ir_tol || it >= h->opt.ir_max_iter) break;
            wd::launch_transpose<float>(Y, h->d_R, n, nrhs, 0, 0, st);
            s = run_solve_plan<float>(h, Y, nr, st);
            if (s != WD_OK) return s;
            if (Xf) wd::launch_xupdate(Y, h->d_X, Xf, n, nrhs, 1, st);
            else wd::launch_transpose<float>(Y, h->d_X, n, nrhs, 1, 1, st);
            h->launches += 2;
            CK(cudaGetLastError(), "refinement launch");
            ++it;
        }
        if (info) {
            info->iterations = it;
            info->backward_error = be;
        }
        wd::launch_permute_out_rm(h->d_X, Bd, ld, h->dsym.perm, n, nrhs, st);
        h->launches += 1;
        status_t tstatus = 0;
        CK(cudaMemcpyAsync(&tstatus, h->d_tstatus, sizeof(status_t), cudaMemcpyDeviceToHost, st), "status D2H");
        CK(cudaStreamSynchronize(st), "solve");
        if (tstatus != 0) return fail(h, WD_ERR_TIMEOUT, "a bounded wait of a tensor-core solve product expired");
        if (be > h->opt.ir_tol) {
            if (!B_on_device)
                cudaMemcpy2DAsync(B, ldb * sizeof(double), h->d_B, n * sizeof(double), n * sizeof(double),
                                  nrhs, cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            return fail(h, WD_ERR_NO_CONVERGENCE,
                        "refinement stopped at backward error " + std::to_string(be) + " after " +
                            std::to_string(it) + " steps");
        }
    }
    if (!B_on_device)
        CK(cudaMemcpy2DAsync(B, ldb * sizeof(double), h->d_B, n * sizeof(double), n * sizeof(double), nrhs,
                             cudaMemcpyDeviceToHost, st),
           "B D2H");
    CK(cudaStreamSynchronize(st), "solve");
    return WD_OK;
}

extern "C" wd_status wd_solve(wd_handle h, double *B, int64_t nrhs, int64_t ldb, int B_on_device,
                              void *stream, wd_solve_info *info) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->factored) return fail(h, WD_ERR_STATE, "wd_solve before a successful wd_factor");
    const int64_t n = h->S.n;
    if (!B || nrhs < 0 || ldb < n || nrhs > (1 << 20)) return fail(h, WD_ERR_INVALID_ARG, "bad B");
    if (info) {
        info->iterations = 0;
        info->backward_error = -1.0;
    }
    if (nrhs == 0) return WD_OK;
    CK(cudaSetDevice(h->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wd_status s = prepare_solve(h, nrhs);
    if (s != WD_OK) return s;
    double *Bd = B;
    int64_t ld = ldb;
    if (!B_on_device) {
        CK(cudaMemcpy2DAsync(h->d_B, n * sizeof(double), B, ldb * sizeof(double), n * sizeof(double),
                             nrhs, cudaMemcpyHostToDevice, st),
           "B H2D");
        Bd = h->d_B;
        ld = n;
    }
    // right-hand sides in factor order, row-major, FP64
    wd::launch_permute_in_rm(Bd, ld, h->d_Bp, h->dsym.perm, n, nrhs, st);
    h->launches += 1;
    return solve_core(h, Bd, ld, B, ldb, B_on_device, nrhs, st, info);
}

// One theta-scheme step (Section 5, Eq. (theta)) with the factored matrix
// M = I + theta dt K: U <- M^-1 [(1/theta) U - ((1 - theta)/theta) M U + dt F],
// which is (I + theta dt K) U_new = (I - (1 - theta) dt K) U + dt F.
extern "C" wd_status wd_theta_step(wd_handle h, double *U, const double *F, int64_t nrhs, int64_t ld,
                                   double theta, double dt, int on_device, void *stream,
                                   wd_solve_info *info) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->factored) return fail(h, WD_ERR_STATE, "wd_theta_step before a successful wd_factor");
    const int64_t n = h->S.n;
    if (!U || nrhs < 0 || ld < n || nrhs > (1 << 20)) return fail(h, WD_ERR_INVALID_ARG, "bad U");
    if (!(theta > 0.0 && theta <= 1.0) || !(dt >= 0.0) || !std::isfinite(dt))
        return fail(h, WD_ERR_INVALID_ARG, "theta must lie in (0, 1] and dt be finite and >= 0");
    if (info) {
        info->iterations = 0;
        info->backward_error = -1.0;
    }
    if (nrhs == 0) return WD_OK;
    CK(cudaSetDevice(h->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wd_status s = prepare_solve(h, nrhs);
    if (s != WD_OK) return s;
    double *Ud = U;
    const double *Fd = F;
    int64_t ldd = ld;
    if (!on_device) {
        // U into d_B, F into d_Y (free until the substitutions start)
        CK(cudaMemcpy2DAsync(h->d_B, n * sizeof(double), U, ld * sizeof(double), n * sizeof(double), nrhs,
                             cudaMemcpyHostToDevice, st),
           "U H2D");
        if (F) {
            CK(cudaMemcpy2DAsync(h->d_Y, n * sizeof(double), F, ld * sizeof(double), n * sizeof(double), nrhs,
                                 cudaMemcpyHostToDevice, st),
               "F H2D");
            Fd = static_cast<const double *>(h->d_Y);
        }
        Ud = h->d_B;
        ldd = n;
    }
    if (h->d_gcsr) {
        // G != I: Bp = dt F, then Bp += (1/theta) G U (U in factor order, in R)
        wd::launch_theta_stage(Ud, Fd, ldd, h->dsym.perm, n, nrhs, 0.0, (1.0 - theta) / theta, dt, h->d_Bp,
                               h->d_X, st);
        wd::launch_permute_in_rm(Ud, ldd, h->d_R, h->dsym.perm, n, nrhs, st);
        wd::launch_spmv_axpy(h->dsym, h->d_gcsr, h->d_R, 1.0 / theta, h->d_Bp, nrhs, st);
        h->launches += 3;
    } else {
        wd::launch_theta_stage(Ud, Fd, ldd, h->dsym.perm, n, nrhs, 1.0 / theta, (1.0 - theta) / theta, dt,
                               h->d_Bp, h->d_X, st);
        h->launches += 1;
    }
    if (theta < 1.0) {
        s = launch_residual(h, h->d_X, nrhs, st);
        if (s != WD_OK) return s;
        unsigned long long bad = ~0ULL;
        if (nrhs <= 8)
            CK(cudaMemcpyAsync(&bad, h->d_spmv_bad, sizeof(bad), cudaMemcpyDeviceToHost, st), "spmv check");
        CK(cudaMemcpyAsync(h->d_Bp, h->d_R, n * nrhs * sizeof(double), cudaMemcpyDeviceToDevice, st),
           "step right-hand side");
        CK(cudaStreamSynchronize(st), "theta step");
        if (bad != ~0ULL)
            return fail(h, WD_ERR_CUDA, "residual: column index out of range at CSR position " + std::to_string(bad));
    }
    return solve_core(h, Ud, ldd, U, ld, on_device, nrhs, st, info);
}

extern "C" wd_status wd_set_mass(wd_handle h, const double *gvalues, int on_device) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->analyzed || h->opt.symbolic_only)
        return fail(h, WD_ERR_STATE, "wd_set_mass before wd_analyze (or on a host-only handle)");
    CK(cudaSetDevice(h->device), "set device");
    if (!gvalues) {
        h->d_gcsr = nullptr;   // the allocation stays with the analysis; G = I from now on
        return WD_OK;
    }
    const int64_t nnzl = h->S.pcp[h->S.n];
    if (!h->mass_buf) CK(h->mem.alloc((void **)&h->mass_buf, h->nnz_full * sizeof(double)), "mass alloc");
    const double *src = gvalues;
    if (!on_device) {
        if (!h->d_values_stage)
            CK(h->mem.alloc((void **)&h->d_values_stage, nnzl * sizeof(double)), "stage alloc");
        CK(cudaMemcpy(h->d_values_stage, gvalues, nnzl * sizeof(double), cudaMemcpyHostToDevice), "G H2D");
        src = h->d_values_stage;
    }
    wd::launch_gather_values(h->d_csr_src, src, h->mass_buf, nullptr, nullptr, h->nnz_full, 0);
    h->launches += 1;
    CK(cudaDeviceSynchronize(), "mass gather");
    h->d_gcsr = h->mass_buf;
    return WD_OK;
}

extern "C" wd_status wd_backward_error(wd_handle h, const double *X, const double *B, int64_t nrhs,
                                       int64_t ld, int on_device, void *stream, double *be) {
    if (!h || !be) return WD_ERR_INVALID_ARG;
    if (!h->factored) return fail(h, WD_ERR_STATE, "wd_backward_error before a successful wd_factor");
    const int64_t n = h->S.n;
    if (!X || !B || nrhs <= 0 || ld < n) return fail(h, WD_ERR_INVALID_ARG, "bad arguments");
    CK(cudaSetDevice(h->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wd_status s = ensure_solve_ws(h, nrhs);
    if (s != WD_OK) return s;
    const double *Xd = X, *Bd = B;
    int64_t ldd = ld;
    if (!on_device) {
        // stage both through the solve workspaces (column-major, ld n)
        CK(cudaMemcpy2DAsync(h->d_B, n * sizeof(double), B, ld * sizeof(double), n * sizeof(double), nrhs,
                             cudaMemcpyHostToDevice, st),
           "B H2D");
        CK(cudaMemcpy2DAsync(h->d_R, n * sizeof(double), X, ld * sizeof(double), n * sizeof(double), nrhs,
                             cudaMemcpyHostToDevice, st),
           "X H2D");
        Bd = h->d_B;
        Xd = h->d_R;
        ldd = n;
    }
    wd::launch_permute_in_rm(Bd, ldd, h->d_Bp, h->dsym.perm, n, nrhs, st);
    wd::launch_permute_in_rm(Xd, ldd, h->d_X, h->dsym.perm, n, nrhs, st);
    h->launches += 2;
    CK(cudaGetLastError(), "permute launch");
    return backward_errors(h, h->d_X, nrhs, st, be);
}

extern "C" wd_status wd_logdet(wd_handle h, double *out) {
    if (!h || !out) return WD_ERR_INVALID_ARG;
    if (!h->factored) return fail(h, WD_ERR_STATE, "wd_logdet before a successful wd_factor");
    CK(cudaSetDevice(h->device), "set device");
    const int nb = 256;
    double *partial = h->d_scalars + 8;
    if (h->prec == WD_FP64)
        wd::launch_logdet_partial<double>(h->dsym, static_cast<const double *>(h->d_front), partial, nb, 0);
    else
        wd::launch_logdet_partial<float>(h->dsym, static_cast<const float *>(h->d_front), partial, nb, 0);
    wd::launch_sum_final(partial, nb, h->d_scalars + 1, 0);
    h->launches += 2;
    CK(cudaGetLastError(), "logdet launch");
    CK(cudaMemcpy(out, h->d_scalars + 1, sizeof(double), cudaMemcpyDeviceToHost), "logdet D2H");
    return WD_OK;
}

extern "C" wd_status wd_logdet_batch(wd_handle h, double *out) {
    if (!h || !out) return WD_ERR_INVALID_ARG;
    if (!h->factored) return fail(h, WD_ERR_STATE, "wd_logdet_batch before a successful wd_factor");
    if (h->batch_count == 0) return fail(h, WD_ERR_STATE, "not a batch (use wd_analyze_batch)");
    CK(cudaSetDevice(h->device), "set device");
    double *dst = h->d_batch_ld;
    if (h->prec == WD_FP64)
        wd::launch_seg_logdet<double>(h->dsym, static_cast<const double *>(h->d_front), h->d_batch_soff,
                                      h->batch_count, h->d_batch_sdl, dst, 0);
    else
        wd::launch_seg_logdet<float>(h->dsym, static_cast<const float *>(h->d_front), h->d_batch_soff,
                                     h->batch_count, h->d_batch_sdl, dst, 0);
    h->launches += 2;
    CK(cudaGetLastError(), "logdet launch");
    CK(cudaMemcpy(out, dst, h->batch_count * sizeof(double), cudaMemcpyDeviceToHost), "logdet D2H");
    return WD_OK;
}

extern "C" wd_status wd_apply_L(wd_handle h, const double *Z, double *S_out, int64_t nrhs, int64_t ld,
                                int on_device, void *stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->factored) return fail(h, WD_ERR_STATE, "wd_apply_L before a successful wd_factor");
    const int64_t n = h->S.n;
    if (!Z || !S_out || nrhs < 0 || ld < n) return fail(h, WD_ERR_INVALID_ARG, "bad arguments");
    if (nrhs == 0) return WD_OK;
    CK(cudaSetDevice(h->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wd_status s = ensure_solve_ws(h, nrhs);
    if (s != WD_OK) return s;
    if (h->aplan_nrhs < 0) {
        build_apply_plan(h->S, h->aplan);
        s = upload_plan(h, h->work, h->aplan);
        if (s != WD_OK) return s;
        h->aplan_nrhs = 1;
    }
    const double *Zd = Z;
    double *Sd = S_out;
    if (!on_device) {
        CK(cudaMemcpy2DAsync(h->d_B, n * sizeof(double), Z, ld * sizeof(double), n * sizeof(double), nrhs,
                             cudaMemcpyHostToDevice, st),
           "Z H2D");
        Zd = h->d_B;
        Sd = h->d_B;
    }
    const int64_t ldo = on_device ? ld : n;
    // Z is indexed in factor order: copy it (column by column) into Bp with ld = n
    CK(cudaMemcpy2DAsync(h->d_Bp, n * sizeof(double), Zd, (on_device ? ld : n) * sizeof(double),
                         n * sizeof(double), nrhs, cudaMemcpyDeviceToDevice, st),
       "Z copy");
    const DevSym &d = h->dsym;
    if (h->prec == WD_FP64) {
        double *Out = static_cast<double *>(h->d_Y);
        for (const Launch &L : h->aplan.launches)
            wd::launch_apply_L<double>(d, static_cast<const double *>(h->d_front), h->d_Bp, Out,
                                       static_cast<double *>(h->d_W), h->aplan.d_items + L.off, L.count,
                                       (int)nrhs, st);
        wd::launch_permute_out<double>(Out, Sd, ldo, d.perm, n, nrhs, st);
        h->launches += (int64_t)h->aplan.launches.size() + 1;
    } else {
        float *Zf = reinterpret_cast<float *>(h->d_R);
        wd::launch_cast<float>(h->d_Bp, Zf, n * nrhs, st);
        float *Out = static_cast<float *>(h->d_Y);
        for (const Launch &L : h->aplan.launches)
            wd::launch_apply_L<float>(d, static_cast<const float *>(h->d_front), Zf, Out,
                                      static_cast<float *>(h->d_W), h->aplan.d_items + L.off, L.count,
                                      (int)nrhs, st);
        wd::launch_permute_out<float>(Out, Sd, ldo, d.perm, n, nrhs, st);
        h->launches += (int64_t)h->aplan.launches.size() + 2;
    }
    CK(cudaGetLastError(), "apply_L launch");
    if (!on_device)
        CK(cudaMemcpy2DAsync(S_out, ld * sizeof(double), h->d_B, n * sizeof(double), n * sizeof(double), nrhs,
                             cudaMemcpyDeviceToHost, st),
           "S D2H");
    CK(cudaStreamSynchronize(st), "apply_L");
    return WD_OK;
}

extern "C" wd_status wd_export_L(wd_handle h, double *panels) {
    if (!h || !panels) return WD_ERR_INVALID_ARG;
    if (!h->factored) return fail(h, WD_ERR_STATE, "wd_export_L before a successful wd_factor");
    CK(cudaSetDevice(h->device), "set device");
    const wd::Symbolic &S = h->S;
    std::vector<int64_t> poff(S.ns);
    int64_t tot = 0;
    for (int s = 0; s < S.ns; ++s) {
        poff[s] = tot;
        tot += (int64_t)S.m(s) * S.k(s);
    }
    int64_t *d_poff = nullptr;
    double *d_out = nullptr;
    CK(cudaMalloc((void **)&d_poff, S.ns * sizeof(int64_t)), "export alloc");
    if (cudaMalloc((void **)&d_out, tot * sizeof(double)) != cudaSuccess) {
        cudaFree(d_poff);
        return cuda_fail(h, cudaErrorMemoryAllocation, "export alloc");
    }
    cudaMemcpy(d_poff, poff.data(), S.ns * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (h->prec == WD_FP64)
        wd::launch_export_panels<double>(h->dsym, static_cast<const double *>(h->d_front), d_out, d_poff, 0);
    else
        wd::launch_export_panels<float>(h->dsym, static_cast<const float *>(h->d_front), d_out, d_poff, 0);
    cudaError_t e = cudaMemcpy(panels, d_out, tot * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d_out);
    cudaFree(d_poff);
    if (e != cudaSuccess) return cuda_fail(h, e, "export");
    return WD_OK;
}

// ---------------------------------------------------------------------------
// selected inverse (Takahashi recurrences, supernodal, FP64)
// ---------------------------------------------------------------------------
static wd_status upload_pattern_maps(wd_handle h) {
    const wd::Symbolic &S = h->S;
    if (!h->d_prow) {
        const int32_t *p = nullptr;
        UP(S.prow, p);
        h->d_prow = const_cast<int32_t *>(p);
        UP(S.psrc, p);
        h->d_psrc = const_cast<int32_t *>(p);
    }
    return WD_OK;
}

// X_s = L_JJ^-1 and W_s = L_RJ X_s depend on the factor only; Z_JJ starts as
// X^T X; then, top-down by tree level: gather Z_RR from the parent's Z front,
// Z_RJ = -Z_RR W, Z_JJ -= W^T Z_RJ.  Items carry device pointers of the front,
// Z and X/W pools, which stay put until the next wd_analyze.
static wd_status build_selinv(wd_handle h) {
    const wd::Symbolic &S = h->S;
    const int ns = S.ns;
    std::vector<int64_t> xoff(ns), upoff(ns, 0);
    int64_t xw = 0, up = 0;
    for (int s = 0; s < ns; ++s) {
        xoff[s] = xw;
        xw += (int64_t)S.m(s) * S.k(s);
        upoff[s] = up;
        up += S.m(s) - S.k(s);
        if (S.sparent[s] < 0 && S.m(s) != S.k(s))
            return fail(h, WD_ERR_STATE, "root supernode with update rows");
    }
    std::vector<int32_t> upmap(std::max<int64_t>(up, 1), -1), col2s(S.n);
    for (int c = 0; c < ns; ++c) {
        for (int j = S.sfirst[c]; j < S.sfirst[c + 1]; ++j) col2s[j] = c;
        const int p = S.sparent[c];
        if (p < 0) continue;
        const int kp_p = kpad(S.k(p)), k_p = S.k(p);
        for (int r = 0; r < S.m(p); ++r) {
            const int i = S.relmap[S.mapoff[c] + r];
            if (i >= 0) upmap[upoff[c] + i] = r < k_p ? r : r + kp_p - k_p;
        }
    }
    for (int c = 0; c < ns; ++c)
        for (int i = 0; i < S.m(c) - S.k(c); ++i)
            if (upmap[upoff[c] + i] < 0) return fail(h, WD_ERR_STATE, "update row missing in parent front");
    CK(h->mem.alloc((void **)&h->d_zpool, h->front_elems * sizeof(double)), "selinv alloc");
    CK(h->mem.alloc((void **)&h->d_xw, std::max<int64_t>(xw, 1) * sizeof(double)), "selinv alloc");
    CK(cudaMemset(h->d_xw, 0, std::max<int64_t>(xw, 1) * sizeof(double)), "selinv clear");
    CK(cudaMemset(h->d_zpool, 0, h->front_elems * sizeof(double)), "selinv clear");
    {
        const int64_t *p64 = nullptr;
        const int32_t *p32 = nullptr;
        UP(xoff, p64);
        h->d_xoff = const_cast<int64_t *>(p64);
        UP(upoff, p64);
        h->d_upoff = const_cast<int64_t *>(p64);
        UP(upmap, p32);
        h->d_upmap = const_cast<int32_t *>(p32);
        UP(col2s, p32);
        h->d_col2s = const_cast<int32_t *>(p32);
    }
    {
        wd_status st = upload_pattern_maps(h);
        if (st != WD_OK) return st;
    }
    CK(h->mem.alloc((void **)&h->d_sel_out, std::max<int64_t>(S.pcp[S.n], 1) * sizeof(double)),
       "selinv alloc");

    const double *F = static_cast<const double *>(h->d_front);
    double *Z = h->d_zpool, *XW = h->d_xw;
    std::vector<int4> items;
    std::vector<wd::GemmItem> gemm;
    auto &steps = h->sel_steps;
    steps.clear();
    double flops = 0.0;
    auto push_step = [&](int kind, int64_t off, int64_t end) {
        if (end > off) steps.push_back({kind, off, (int)(end - off)});
    };
    auto tiles = [](int x) { return (x + 63) / 64; };
    // 1) X = L_JJ^-1 by block rows
    int maxblk = 0;
    for (int s = 0; s < ns; ++s) maxblk = std::max(maxblk, tiles(S.k(s)));
    for (int t = 0; t < maxblk; ++t) {
        const int64_t o = (int64_t)items.size();
        for (int s = 0; s < ns; ++s)
            if (tiles(S.k(s)) > t)
                for (int bj = 0; bj <= t; ++bj) items.push_back({s, t, bj, 0});
        push_step(0, o, (int64_t)items.size());
    }
    auto gi = [](const double *A, int64_t ars, int64_t acs, const double *B, int64_t brs, int64_t bcs,
                 double *C, int64_t crs, int64_t ccs, int M, int N, int p0, int p1, int i0, int j0,
                 int flags, double alpha) {
        wd::GemmItem g;
        g.A = A;
        g.B = B;
        g.C = C;
        g.a_rs = ars;
        g.a_cs = acs;
        g.b_rs = brs;
        g.b_cs = bcs;
        g.c_rs = crs;
        g.c_cs = ccs;
        g.M = M;
        g.N = N;
        g.p0 = p0;
        g.p1 = p1;
        g.i0 = i0;
        g.j0 = j0;
        g.flags = flags;
        g.pad = 0;
        g.alpha = alpha;
        return g;
    };
    // 2) W = L_RJ X (X lower triangular: p from the tile's first column) and
    //    Z_JJ = X^T X (lower tiles, p from the tile's first row)
    {
        const int64_t o = (int64_t)gemm.size();
        for (int s = 0; s < ns; ++s) {
            const int k = S.k(s), r = S.m(s) - S.k(s), kp = kpad(k), ld = h->h_sld[s];
            const int64_t fo = h->h_foff[s];
            double *X = XW + xoff[s], *W = X + (int64_t)k * k;
            for (int ti = 0; ti < tiles(r); ++ti)
                for (int tj = 0; tj < tiles(k); ++tj)
                    gemm.push_back(gi(F + fo + kp, 1, ld, X, k, 1, W, 1, r, r, k, 64 * tj, k, 64 * ti,
                                      64 * tj, 0, 1.0));
            flops += (double)r * k * k;
            for (int ti = 0; ti < tiles(k); ++ti)
                for (int tj = 0; tj <= ti; ++tj)
                    gemm.push_back(gi(X, k, 1, X, k, 1, Z + fo, 1, ld, k, k, 64 * ti, k, 64 * ti, 64 * tj,
                                      wd::GEMM_C_LOWER, 1.0));
            flops += (double)k * k * k / 3.0;
        }
        push_step(1, o, (int64_t)gemm.size());
    }
    // 3) top-down over the tree levels
    for (int lv = S.nlevels - 1; lv >= 0; --lv) {
        const int64_t oz = (int64_t)items.size();
        for (int q = S.level_ptr[lv]; q < S.level_ptr[lv + 1]; ++q) {
            const int s = S.level_nodes[q];
            const int r = S.m(s) - S.k(s);
            for (int j = 0; j < r; ++j) items.push_back({s, j, S.sparent[s], 0});
        }
        push_step(2, oz, (int64_t)items.size());
        const int64_t o1 = (int64_t)gemm.size();
        for (int q = S.level_ptr[lv]; q < S.level_ptr[lv + 1]; ++q) {
            const int s = S.level_nodes[q];
            const int k = S.k(s), r = S.m(s) - S.k(s), kp = kpad(k), ld = h->h_sld[s];
            if (r == 0) continue;
            const int64_t fo = h->h_foff[s];
            const double *W = XW + xoff[s] + (int64_t)k * k;
            // Z_RJ = -Z_RR W
            for (int ti = 0; ti < tiles(r); ++ti)
                for (int tj = 0; tj < tiles(k); ++tj)
                    gemm.push_back(gi(Z + fo + (int64_t)kp * ld + kp, 1, ld, W, r, 1, Z + fo + kp, 1, ld, r,
                                      k, 0, r, 64 * ti, 64 * tj, wd::GEMM_A_SYM_LOWER, -1.0));
            flops += 2.0 * r * r * k;
        }
        push_step(1, o1, (int64_t)gemm.size());
        const int64_t o2 = (int64_t)gemm.size();
        for (int q = S.level_ptr[lv]; q < S.level_ptr[lv + 1]; ++q) {
            const int s = S.level_nodes[q];
            const int k = S.k(s), r = S.m(s) - S.k(s), kp = kpad(k), ld = h->h_sld[s];
            if (r == 0) continue;
            const int64_t fo = h->h_foff[s];
            const double *W = XW + xoff[s] + (int64_t)k * k;
            // Z_JJ -= W^T Z_RJ (lower)
            for (int ti = 0; ti < tiles(k); ++ti)
                for (int tj = 0; tj <= ti; ++tj)
                    gemm.push_back(gi(W, r, 1, Z + fo + kp, ld, 1, Z + fo, 1, ld, k, k, 0, r, 64 * ti,
                                      64 * tj, wd::GEMM_C_LOWER | wd::GEMM_ACCUMULATE, -1.0));
            flops += (double)r * k * k;
        }
        push_step(1, o2, (int64_t)gemm.size());
    }
    CK(h->mem.alloc((void **)&h->d_sel_items, std::max<size_t>(items.size(), 1) * sizeof(int4)),
       "selinv alloc");
    if (!items.empty())
        CK(cudaMemcpy(h->d_sel_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice),
           "selinv upload");
    CK(h->mem.alloc((void **)&h->d_sel_gemm, std::max<size_t>(gemm.size(), 1) * sizeof(wd::GemmItem)),
       "selinv alloc");
    if (!gemm.empty())
        CK(cudaMemcpy(h->d_sel_gemm, gemm.data(), gemm.size() * sizeof(wd::GemmItem),
                      cudaMemcpyHostToDevice),
           "selinv upload");
    h->sel_flops = flops;
    h->sel_ready = true;
    return WD_OK;
}

// Z at A's stored entries into dst (device), enqueued on st
static wd_status selinv_enqueue(wd_handle h, double *dst, cudaStream_t st) {
    if (!h->sel_ready) {
        wd_status s = build_selinv(h);
        if (s != WD_OK) return s;
    }
    const DevSym &d = h->dsym;
    const double *F = static_cast<const double *>(h->d_front);
    const double *Dv = static_cast<const double *>(h->d_dinv);
    prof_single(h, "selinv_fp64", 0, 0, st, true);
    for (const auto &sp : h->sel_steps) {
        switch (sp.kind) {
            case 0:
                wd::launch_trinv(d, F, Dv, h->d_xw, h->d_xoff, h->d_sel_items + sp.off, sp.count, st);
                break;
            case 1: wd::launch_gemm_items(h->d_sel_gemm + sp.off, sp.count, st); break;
            case 2:
                wd::launch_zgather(d, h->d_zpool, h->d_upmap, h->d_upoff, h->d_sel_items + sp.off, sp.count,
                                   st);
                break;
        }
    }
    wd::launch_zextract(d, h->d_zpool, h->d_col2s, h->d_psrc, dst, st);
    prof_single(h, "selinv_fp64", h->sel_flops, 0, st, false);
    h->launches += (int64_t)h->sel_steps.size() + 1;
    CK(cudaGetLastError(), "selinv launch");
    return WD_OK;
}

extern "C" wd_status wd_selinv(wd_handle h, double *out, int on_device, void *stream) {
    if (!h || !out) return WD_ERR_INVALID_ARG;
    if (!h->factored || h->prec != WD_FP64)
        return fail(h, WD_ERR_STATE, "wd_selinv needs a successful WD_FP64 factorization");
    CK(cudaSetDevice(h->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!h->sel_ready) {
        wd_status s = build_selinv(h);
        if (s != WD_OK) return s;
    }
    wd_status s = selinv_enqueue(h, on_device ? out : h->d_sel_out, st);
    if (s != WD_OK) return s;
    if (!on_device)
        CK(cudaMemcpyAsync(out, h->d_sel_out, h->S.pcp[h->S.n] * sizeof(double), cudaMemcpyDeviceToHost, st),
           "selinv D2H");
    CK(cudaStreamSynchronize(st), "selinv");
    return WD_OK;
}

// out = alpha * pattern(U V^T + V U^T) + zscale * w * Z (zscale != 0 needs the
// FP64 factor); host or device operands
static wd_status pattern_outer(wd_handle h, const double *U, const double *V, int64_t ncols, int64_t ld,
                               double alpha, double zscale, double *out, int on_device, void *stream) {
    const int64_t n = h->S.n, nnz = h->S.pcp[n];
    if (!out || ncols < 0 || (ncols > 0 && (!U || !V || ld < n)))
        return fail(h, WD_ERR_INVALID_ARG, "bad arguments");
    if (ncols == 0) ld = n;
    CK(cudaSetDevice(h->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wd_status s = upload_pattern_maps(h);
    if (s != WD_OK) return s;
    const double *Zsel = nullptr;
    if (zscale != 0.0) {
        if (!h->factored || h->prec != WD_FP64)
            return fail(h, WD_ERR_STATE, "the log-determinant term needs a WD_FP64 factorization");
        if (!h->sel_ready) {
            s = build_selinv(h);
            if (s != WD_OK) return s;
        }
        s = selinv_enqueue(h, h->d_sel_out, st);
        if (s != WD_OK) return s;
        Zsel = h->d_sel_out;
    }
    const double *Ud = U, *Vd = V;
    double *Od = out;
    DevMem tmp;
    if (!on_device) {
        double *u = nullptr, *v = nullptr, *o = nullptr;
        CK(tmp.alloc((void **)&u, std::max<int64_t>(n * ncols, 1) * sizeof(double)), "outer alloc");
        CK(tmp.alloc((void **)&v, std::max<int64_t>(n * ncols, 1) * sizeof(double)), "outer alloc");
        CK(tmp.alloc((void **)&o, std::max<int64_t>(nnz, 1) * sizeof(double)), "outer alloc");
        if (ncols > 0) {
            CK(cudaMemcpy2DAsync(u, n * sizeof(double), U, ld * sizeof(double), n * sizeof(double), ncols,
                                 cudaMemcpyHostToDevice, st),
               "U H2D");
            CK(cudaMemcpy2DAsync(v, n * sizeof(double), V, ld * sizeof(double), n * sizeof(double), ncols,
                                 cudaMemcpyHostToDevice, st),
               "V H2D");
        }
        Ud = u;
        Vd = v;
        Od = o;
        ld = n;
    }
    wd::launch_sym_outer(h->dsym, h->d_prow, h->d_psrc, Ud, Vd, ncols, ld, alpha, Zsel, zscale, Od, st);
    h->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(out, Od, nnz * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    tmp.free_all();
    if (e != cudaSuccess) return cuda_fail(h, e, "pattern outer product");
    return WD_OK;
}

extern "C" wd_status wd_sym_pattern_outer(wd_handle h, const double *U, const double *V, int64_t ncols,
                                          int64_t ld, double *out, int on_device, void *stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->analyzed || h->opt.symbolic_only)
        return fail(h, WD_ERR_STATE, "wd_sym_pattern_outer before wd_analyze (or on a host-only handle)");
    return pattern_outer(h, U, V, ncols, ld, 1.0, 0.0, out, on_device, stream);
}

extern "C" wd_status wd_value_gradient(wd_handle h, double g_logdet, const double *X, const double *G,
                                       int64_t ncols, int64_t ld, double *out, int on_device, void *stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->factored) return fail(h, WD_ERR_STATE, "wd_value_gradient before a successful wd_factor");
    return pattern_outer(h, G, X, ncols, ld, -1.0, g_logdet, out, on_device, stream);
}

// ---------------------------------------------------------------------------
// LU without pivoting (FP64)
// ---------------------------------------------------------------------------
static void build_lu_plans(const wd::Symbolic &S, Plan &fp, Plan &sf, Plan &sb) {
    fp = Plan();
    sf = Plan();
    sb = Plan();
    constexpr int TL = 64;
    for (int l = 0; l < S.nlevels; ++l) {
        const int b = S.level_ptr[l], e = S.level_ptr[l + 1];
        size_t f0 = fp.items.size();
        double el = 0;
        for (int i = b; i < e; ++i) {
            const int s = S.level_nodes[i];
            const int mp = front_order(S, s);
            for (int q = 0; q < (mp + 7) / 8 * 8; ++q) fp.items.push_back({s, q < mp ? q : -1, 0, 0});
            el += (double)mp * mp;
        }
        add_launch(fp, K_LU_INIT, f0, 0, 0, el, 0);
        int kmax = 0;
        for (int i = b; i < e; ++i) kmax = std::max(kmax, S.k(S.level_nodes[i]));
        for (int kb = 0; kb < kmax; kb += NB) {
            f0 = fp.items.size();
            double fl = 0;
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i];
                if (S.k(s) <= kb) continue;
                const double nb = std::min(NB, S.k(s) - kb);
                fp.items.push_back({s, 0, 0, 0});
                fl += 2.0 * nb * nb * nb / 3 + 2.0 * nb * nb * nb / 3;
            }
            add_launch(fp, K_LU_DIAG, f0, kb, fl, 0, 0);
            f0 = fp.items.size();
            fl = 0;
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i], k = S.k(s);
                if (k <= kb) continue;
                const int nb = std::min(NB, k - kb), t0 = kb + nb, mp = front_order(S, s);
                const int start = (t0 == k) ? kpad(k) : t0;
                const int nblk = (mp - start + TL - 1) / TL;
                for (int side = 0; side < 2; ++side)
                    for (int q = 0; q < nblk; ++q) fp.items.push_back({s, q, side, 0});
                fl += 2.0 * (double)(S.m(s) - t0) * nb * nb;
            }
            add_launch(fp, K_LU_PANEL, f0, kb, fl, 0, 0);
            f0 = fp.items.size();
            fl = 0;
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i], k = S.k(s);
                if (k <= kb) continue;
                const int nb = std::min(NB, k - kb), base = kb + nb, mp = front_order(S, s);
                const int T = (mp - base + TL - 1) / TL;
                for (int tj = 0; tj < T; ++tj)
                    for (int ti = 0; ti < T; ++ti) fp.items.push_back({s, ti, tj, 0});
                const double r = S.m(s) - base;
                fl += 2.0 * r * r * nb;
            }
            add_launch(fp, K_LU_UPDATE, f0, kb, fl, 0, 0);
        }
        // substitutions: gather, then the pivot blocks of the level in order
        f0 = sf.items.size();
        for (int i = b; i < e; ++i) {
            const int s = S.level_nodes[i];
            for (int rc = 0; rc * 32 < S.m(s); ++rc) sf.items.push_back({s, rc, 0, 0});
        }
        add_launch(sf, K_LU_GATHER, f0, 0, 0, 0, 0);
        for (int kb = 0; kb < kmax; kb += NB) {
            f0 = sf.items.size();
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i], k = S.k(s);
                if (k <= kb) continue;
                const int t0 = kb + std::min(NB, k - kb);
                const int nblk = 1 + (S.m(s) - t0 + TL - 1) / TL;
                for (int q = 0; q < nblk; ++q) sf.items.push_back({s, q, 0, 0});
            }
            add_launch(sf, K_LU_FWD, f0, kb, 0, 0, 0);
        }
    }
    for (int l = S.nlevels - 1; l >= 0; --l) {
        const int b = S.level_ptr[l], e = S.level_ptr[l + 1];
        int kmax = 0;
        for (int i = b; i < e; ++i) kmax = std::max(kmax, S.k(S.level_nodes[i]));
        for (int kb = (kmax - 1) / NB * NB; kb >= 0; kb -= NB) {
            const size_t f0 = sb.items.size();
            for (int i = b; i < e; ++i) {
                const int s = S.level_nodes[i];
                if (S.k(s) > kb) sb.items.push_back({s, 0, 0, 0});
            }
            add_launch(sb, K_LU_BWD, f0, kb, 0, 0, 0);
        }
    }
}

extern "C" wd_status wd_factor_lu(wd_handle h, const double *lower, const double *upper, int on_device,
                                  void *stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->analyzed || h->opt.symbolic_only)
        return fail(h, WD_ERR_STATE, "wd_factor_lu before wd_analyze (or on a host-only handle)");
    if (!lower || !upper) return fail(h, WD_ERR_INVALID_ARG, "null values");
    if (h->batch_count > 0) return fail(h, WD_ERR_INVALID_ARG, "wd_factor_lu takes a single matrix");
    CK(cudaSetDevice(h->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    wait_export(h);
    h->factored = false;
    h->lu_factored = false;
    h->ldlt = false;
    const int64_t nnzl = h->S.pcp[h->S.n];
    if (!h->d_front) {
        CK(h->mem.alloc(&h->d_front, h->front_elems * sizeof(double)), "front pool alloc");
        CK(h->mem.alloc(&h->d_dinv, h->dinv_elems * sizeof(double)), "inverse blocks alloc");
        CK(h->mem.alloc(&h->d_xs, h->xs_elems * sizeof(double)), "super-block inverse alloc");
        CK(h->mem.alloc(&h->d_xts, h->xs_elems * sizeof(double)), "super-block inverse alloc");
        CK(cudaMemsetAsync(h->d_front, 0, h->front_elems * sizeof(double), st), "front pool clear");
    }
    if (!h->d_uinv) {
        CK(h->mem.alloc((void **)&h->d_uinv, h->dinv_elems * sizeof(double)), "inverse blocks alloc");
        CK(h->mem.alloc((void **)&h->d_vrow, h->nnz_full * sizeof(double)), "values alloc");
        CK(h->mem.alloc((void **)&h->d_vcol, h->nnz_full * sizeof(double)), "values alloc");
        CK(h->mem.alloc((void **)&h->d_lu_part, 2 * 64 * sizeof(double)), "logdet alloc");
        const int8_t *p = nullptr;
        wd_status us = upload(h, h->h_csr_code, &p);
        if (us != WD_OK) return us;
        h->d_lu_code = const_cast<int8_t *>(p);
        build_lu_plans(h->S, h->fplan_lu, h->splan_lu_f, h->splan_lu_b);
        for (Plan *P : {&h->fplan_lu, &h->splan_lu_f, &h->splan_lu_b}) {
            wd_status ps = upload_plan(h, h->mem, *P);
            if (ps != WD_OK) return ps;
        }
    }
    const double *lo = lower, *up = upper;
    if (!on_device) {
        if (!h->d_values_stage)
            CK(h->mem.alloc((void **)&h->d_values_stage, nnzl * sizeof(double)), "stage alloc");
        if (!h->d_upper_stage)
            CK(h->mem.alloc((void **)&h->d_upper_stage, nnzl * sizeof(double)), "stage alloc");
        CK(cudaMemcpyAsync(h->d_values_stage, lower, nnzl * sizeof(double), cudaMemcpyHostToDevice, st), "H2D");
        CK(cudaMemcpyAsync(h->d_upper_stage, upper, nnzl * sizeof(double), cudaMemcpyHostToDevice, st), "H2D");
        lo = h->d_values_stage;
        up = h->d_upper_stage;
    }
    wd::launch_lu_gather(h->d_csr_src, h->d_lu_code, lo, up, h->d_vrow, h->d_vcol, h->nnz_full, st);
    CK(cudaMemsetAsync(h->d_status, 0xFF, sizeof(status_t), st), "status reset");
    h->front_dirty = true;
    double *F = static_cast<double *>(h->d_front);
    double *Li = static_cast<double *>(h->d_dinv);
    const DevSym &d = h->dsym;
    const Plan &P = h->fplan_lu;
    for (const Launch &L : P.launches) {
        const int4 *it = P.d_items + L.off;
        switch (L.kind) {
            case K_LU_INIT: wd::launch_lu_init(d, F, h->d_vrow, h->d_vcol, it, L.count, st); break;
            case K_LU_DIAG: wd::launch_lu_diag(d, F, Li, h->d_uinv, it, L.count, L.arg, h->d_status, st); break;
            case K_LU_PANEL: wd::launch_lu_panel(d, F, Li, h->d_uinv, it, L.count, L.arg, st); break;
            case K_LU_UPDATE: wd::launch_lu_update(d, F, it, L.count, L.arg, st); break;
        }
    }
    h->launches += 1 + (int64_t)P.launches.size();
    CK(cudaGetLastError(), "LU factor launch");
    status_t status = 0;
    CK(cudaMemcpyAsync(&status, h->d_status, sizeof(status_t), cudaMemcpyDeviceToHost, st), "status D2H");
    CK(cudaStreamSynchronize(st), "LU factor");
    if (status != ~0ULL)
        return fail(h, WD_ERR_NOT_SPD, "zero pivot at column " + std::to_string(status) + " (LU without pivoting)",
                    (int64_t)status);
    h->lu_factored = true;
    return WD_OK;
}

extern "C" wd_status wd_set_level_schedule(wd_handle h, const int8_t *step, int32_t nlevels) {
    if (!h || !step) return WD_ERR_INVALID_ARG;
    if (!h->analyzed) return fail(h, WD_ERR_STATE, "wd_set_level_schedule before wd_analyze");
    if (nlevels != h->S.nlevels) return fail(h, WD_ERR_INVALID_ARG, "one flag per level of the analysis");
    for (int32_t l = 0; l < nlevels; ++l)
        if (step[l] != 0 && step[l] != 1) return fail(h, WD_ERR_INVALID_ARG, "level flags are 0 or 1");
    h->level_step.assign(step, step + nlevels);
    build_factor_plan(h->S, h->fplan_tc, true, false, h->chain, h->level_step.data());
    if (!h->opt.symbolic_only) {
        CK(cudaSetDevice(h->device), "set device");
        wait_export(h);
        const wd_status us = upload_plan(h, h->mem, h->fplan_tc);
        if (us != WD_OK) return us;
        h->g_factor.reset();
        h->factored = false;
    }
    return WD_OK;
}

extern "C" wd_status wd_get_level_schedule(wd_handle h, int8_t *step, int32_t nlevels) {
    if (!h || !step) return WD_ERR_INVALID_ARG;
    if (!h->analyzed) return fail(h, WD_ERR_STATE, "wd_get_level_schedule before wd_analyze");
    if (nlevels != h->S.nlevels) return fail(h, WD_ERR_INVALID_ARG, "one flag per level of the analysis");
    for (int32_t l = 0; l < nlevels; ++l) step[l] = h->chain ? h->level_step[l] : 1;
    return WD_OK;
}

extern "C" wd_status wd_factor_ldlt(wd_handle h, const double *values, int on_device, void *stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    // the LU decomposition without pivoting of the symmetric matrix: L, and
    // U = D L^T (the same values for both triangles)
    const wd_status s = wd_factor_lu(h, values, values, on_device, stream);
    h->ldlt = s == WD_OK;
    return s;
}

// number of negative pivots of the LU factor (grid-stride partial counts)
static wd_status lu_pivot_stats(wd_handle h, double *logabs, int64_t *nneg) {
    CK(cudaSetDevice(h->device), "set device");
    constexpr int NBLK = 64;
    wd::launch_lu_logdet(h->dsym, static_cast<const double *>(h->d_front), h->d_lu_part, NBLK, 0);
    double part[2 * NBLK];
    CK(cudaMemcpy(part, h->d_lu_part, sizeof(part), cudaMemcpyDeviceToHost), "logdet D2H");
    double sum = 0.0, neg = 0.0;
    for (int b = 0; b < NBLK; ++b) {
        sum += part[b];
        neg += part[NBLK + b];
    }
    *logabs = sum;
    *nneg = (int64_t)neg;
    return WD_OK;
}

extern "C" wd_status wd_inertia(wd_handle h, int64_t *npos, int64_t *nneg) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->lu_factored || !h->ldlt) return fail(h, WD_ERR_STATE, "wd_inertia before a successful wd_factor_ldlt");
    double la = 0.0;
    int64_t neg = 0;
    const wd_status s = lu_pivot_stats(h, &la, &neg);
    if (s != WD_OK) return s;
    if (npos) *npos = h->S.n - neg;
    if (nneg) *nneg = neg;
    return WD_OK;
}

extern "C" wd_status wd_solve_lu(wd_handle h, double *B, int64_t nrhs, int64_t ldb, int B_on_device,
                                 void *stream) {
    if (!h) return WD_ERR_INVALID_ARG;
    if (!h->lu_factored) return fail(h, WD_ERR_STATE, "wd_solve_lu before a successful wd_factor_lu");
    const int64_t n = h->S.n;
    if (!B || nrhs < 0 || ldb < n || nrhs > (1 << 20)) return fail(h, WD_ERR_INVALID_ARG, "bad B");
    if (nrhs == 0) return WD_OK;
    CK(cudaSetDevice(h->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    constexpr int CH = 16;                      // right-hand sides per pass
    wd_status s = ensure_solve_ws(h, CH);
    if (s != WD_OK) return s;
    double *Bd = B;          // host arrays go through d_B in chunks of CH columns
    const int64_t ld = ldb;
    double *Y = static_cast<double *>(h->d_Y), *Tt = static_cast<double *>(h->d_T);
    double *W = static_cast<double *>(h->d_W);
    const double *F = static_cast<const double *>(h->d_front);
    const double *Li = static_cast<const double *>(h->d_dinv);
    const DevSym &d = h->dsym;
    for (int64_t c0 = 0; c0 < nrhs; c0 += CH) {
        const int nc = (int)std::min<int64_t>(CH, nrhs - c0);
        if (B_on_device) {
            wd::launch_permute_in<double>(Bd + c0 * ld, ld, Y, d.perm, n, nc, st);
        } else {
            CK(cudaMemcpy2DAsync(h->d_B, n * sizeof(double), B + c0 * ldb, ldb * sizeof(double), n * sizeof(double),
                                 nc, cudaMemcpyHostToDevice, st),
               "B H2D");
            wd::launch_permute_in<double>(h->d_B, n, Y, d.perm, n, nc, st);
        }
        for (const Launch &L : h->splan_lu_f.launches) {
            const int4 *it = h->splan_lu_f.d_items + L.off;
            if (L.kind == K_LU_GATHER) wd::launch_bfwd_gather<double>(d, Y, Tt, W, it, L.count, 16, nc, st);
            else wd::launch_lu_fwd(d, F, Li, Y, Tt, W, it, L.count, L.arg, nc, st);
        }
        for (const Launch &L : h->splan_lu_b.launches)
            wd::launch_lu_bwd(d, F, h->d_uinv, Y, h->splan_lu_b.d_items + L.off, L.count, L.arg, nc, st);
        if (B_on_device) {
            wd::launch_permute_out<double>(Y, Bd + c0 * ld, ld, d.perm, n, nc, st);
        } else {
            wd::launch_permute_out<double>(Y, h->d_B, n, d.perm, n, nc, st);
            CK(cudaMemcpy2DAsync(B + c0 * ldb, ldb * sizeof(double), h->d_B, n * sizeof(double), n * sizeof(double),
                                 nc, cudaMemcpyDeviceToHost, st),
               "B D2H");
        }
        h->launches += 2 + (int64_t)h->splan_lu_f.launches.size() + (int64_t)h->splan_lu_b.launches.size();
    }
    CK(cudaGetLastError(), "LU solve launch");
    CK(cudaStreamSynchronize(st), "LU solve");
    return WD_OK;
}

extern "C" wd_status wd_logdet_lu(wd_handle h, double *logabs, int32_t *sign) {
    if (!h || !logabs || !sign) return WD_ERR_INVALID_ARG;
    if (!h->lu_factored) return fail(h, WD_ERR_STATE, "wd_logdet_lu before a successful wd_factor_lu");
    int64_t neg = 0;
    const wd_status s = lu_pivot_stats(h, logabs, &neg);
    if (s != WD_OK) return s;
    *sign = (neg % 2 == 0) ? 1 : -1;
    return WD_OK;
}

extern "C" wd_status wd_export_LU(wd_handle h, double *lpanels, double *utpanels) {
    if (!h || !lpanels || !utpanels) return WD_ERR_INVALID_ARG;
    if (!h->lu_factored) return fail(h, WD_ERR_STATE, "wd_export_LU before a successful wd_factor_lu");
    CK(cudaSetDevice(h->device), "set device");
    const wd::Symbolic &S = h->S;
    std::vector<int64_t> poff(S.ns);
    int64_t tot = 0;
    for (int s = 0; s < S.ns; ++s) {
        poff[s] = tot;
        tot += (int64_t)S.m(s) * S.k(s);
    }
    int64_t *d_poff = nullptr;
    double *d_out = nullptr;
    CK(cudaMalloc((void **)&d_poff, S.ns * sizeof(int64_t)), "export alloc");
    if (cudaMalloc((void **)&d_out, 2 * tot * sizeof(double)) != cudaSuccess) {
        cudaFree(d_poff);
        return cuda_fail(h, cudaErrorMemoryAllocation, "export alloc");
    }
    cudaMemcpy(d_poff, poff.data(), S.ns * sizeof(int64_t), cudaMemcpyHostToDevice);
    wd::launch_lu_export(h->dsym, static_cast<const double *>(h->d_front), d_out, d_out + tot, d_poff, 0);
    cudaError_t e = cudaMemcpy(lpanels, d_out, tot * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(utpanels, d_out + tot, tot * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d_out);
    cudaFree(d_poff);
    if (e != cudaSuccess) return cuda_fail(h, e, "export");
    return WD_OK;
}

extern "C" wd_status wd_export_L_noalloc(wd_handle h, double *panels, void *stream) {
    if (!h || !panels) return WD_ERR_INVALID_ARG;
    if (!h->factored) return fail(h, WD_ERR_STATE, "wd_export_L_noalloc before a successful wd_factor");
    if (h->S.ns > wd::NOALLOC_MAX_SUPERNODES)
        return fail(h, WD_ERR_INVALID_ARG,
                    std::to_string(h->S.ns) + " supernodes exceed the static scratch of " +
                        std::to_string(wd::NOALLOC_MAX_SUPERNODES) + " panel offsets");
    int prev = -1;
    CK(cudaGetDevice(&prev), "get device");
    CK(cudaSetDevice(h->device), "set device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t *poff = nullptr;
    cudaError_t e = wd::noalloc_panel_offsets(h->device, &poff);
    if (e == cudaSuccess) {
        wd::launch_panel_offsets_noalloc(h->dsym, st);
        if (h->prec == WD_FP64)
            wd::launch_export_panels<double>(h->dsym, static_cast<const double *>(h->d_front), panels, poff, st);
        else
            wd::launch_export_panels<float>(h->dsym, static_cast<const float *>(h->d_front), panels, poff, st);
        h->launches += 2;
        e = cudaGetLastError();
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (e == cudaSuccess) e = cudaStreamIsCapturing(st, &cs);
        if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            // (a captured export runs when its graph is launched: ordering
            // those launches is the caller's)
            e = cudaEventRecord(h->export_ev, st);
            if (e == cudaSuccess) h->export_pending = true;
        }
    }
    cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(h, e, "allocation-free export");
    return WD_OK;
}
