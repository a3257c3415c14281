// C ABI of libsgspm.so: handle lifetime, set-up (plans, twiddles, Newell spectrum), the
// per-step pass programs and their CUDA-graph capture.  See include/sgspm.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "../../include/sgspm.h"
#include "common.cuh"
#include "passes.cuh"
#include "launch.cuh"
#include "misc.cu"
#include "newell.cu"
#include "noalloc.cu"
#include "adjoint.cu"

namespace sgspm {

// real field slots: the forward step's, then (allocated by sgspm_record) the recorded
// intermediates of a step and the adjoint accumulators
enum {
    M1 = 0, M2, M3, A1, A2, A3, B1, B2, E3N, E1S, E3SS, D1, D2, D3, HS1, HS2, HS3, NSLOT_FWD,
    D2N = NSLOT_FWD, D2S, D2SS, V1, V2, V3, MN1, MN2, MN3, ERS1, ERS2, ERS3,
    G1, G2, G3, bM1, bM2, bM3, bA1, bA2, bA3, bB1, bB2, bD2N, bE3N, bE1S, bD2S, bE3SS, bD2SS,
    RB1, RB2, RB3, FB1, FB2, FB3, bHE1, bHE2, bHE3, NSLOT
};
static_assert(NSLOT <= kMaxSlots, "slot table too small");
// slots a recorded step leaves for its reverse (the forward step's and the recorded intermediates)
constexpr int kRecSlots = G1;
// spectral slots
enum { S1 = 0, S2, S3, H1, H2, H3, NSPEC_FWD, SA1 = NSPEC_FWD, SA2, SA3, NSPEC };

struct Launch {
    int kind;   // 0 xz, 1 y heat, 2 y stray, 3 step counter, 4 adj GS, 5 adj f, 6 adj ew, 7 adj proj, 8 adj alpha
    XZProg xz;
    YProg y;
    AdjGS gs;
    AdjF af;
    AdjEw ew;
    AdjProj pj;
    AdjAlpha al;
};

}  // namespace sgspm

using namespace sgspm;

struct sgspm_ctx {
    int nfilm = 0;
    int flags = 0;
    bool fp64 = false;
    bool stray = true;
    bool tf32x3 = false;               // TF32X3 form: tensor-core z transforms (FP32 form only)
    cudaStream_t stream = nullptr;     // caller's stream
    cudaStream_t cap = nullptr;        // private capture stream
    std::vector<Film> films;
    std::vector<Plan> plans;
    std::map<int, int> plan_of;
    long long ncell = 0, nspec = 0, nktab = 0;
    size_t tsz = 4;
    // device
    Film* d_films = nullptr;
    Plan* d_plans = nullptr;
    void* d_tw = nullptr;
    void* d_lam = nullptr;
    void* d_lam_lo = nullptr;          // low parts of the eigenvalues (FP32 form)
    void* d_dtab = nullptr;
    void* d_ktab = nullptr;
    void* d_field[kMaxSlots] = {};
    void* d_flo[kMaxSlots] = {};       // low parts of the double-float state slots (FP32 form)
    void* d_spec[kMaxSpec] = {};
    void* d_ycache = nullptr;          // y transforms of M_1..3 for the register stray pass
    long long nycache = 0;             // complex elements per component
    void** d_tab = nullptr;            // device copies of the three pointer tables
    void** d_tab_lo = nullptr;
    void** d_tab_spec = nullptr;
    // recorded forward (adjoint)
    bool rec_alloc = false;
    long long rec_nsteps = 0;
    int rec_K = 0;
    void* d_ckpt = nullptr;            // checkpoints: [seg][hi/lo][3][ncell]
    void* d_seg = nullptr;             // states of one segment: [K][hi/lo][3][ncell]
    void* d_rec = nullptr;             // recorded slots of one segment: [K][kRecSlots][ncell] (hi), or null
    void* d_final = nullptr;           // m(T) while the reverse sweep runs
    double* d_apart = nullptr;         // alpha gradient block partials
    double* d_alpha_b = nullptr;       // alpha gradient per film
    std::vector<Launch> rec_prog, adj_prog;
    void* d_he = nullptr;
    bool he_cell = false;
    int* d_status = nullptr;
    int* h_status = nullptr;   // page-locked host copy of d_status (read by check_status)
    int* d_tc_test = nullptr;          // tensor-core wait test switches (TF32X3 form; see sgspm_test_tc_timeout)
    long long* d_step = nullptr;
    void* d_stage = nullptr;
    // launches are split by size class: one instantiation of a pass per class of films
    struct KClass {
        int key;
        int4* work;
        int n;
        size_t smem;
        int rows = 1;                  // slab pass: y rows per CTA (batch packing)
        int threads = kThreads;        // slab pass: threads per packed CTA (below kThreads: packed even at one row)
        bool nz8 = true;               // slab pass: every film of the class has nz = kZReg
    };
    std::vector<KClass> xz_cls, yh_cls, yw_cls;
    int4* d_work_xz = nullptr;
    int n_xz = 0;
    int4* d_work_yh = nullptr;
    int n_yh = 0;
    int tx_h = 8;
    int heat_threads = 256;            // y heat CTA size (128 or 256; the autotuner may change it)
    int4* d_work_ys[4] = {};
    int n_ys[4] = {};
    int tx_s[4] = {};
    size_t smem_xz = 0, smem_yh = 0, smem_ys[4] = {};
    size_t smem_max = 0;               // opt-in shared memory per block of the device
    bool warp_stray = false;           // register-resident stray line pass (all Py in 64..512)
    int4* d_work_yw = nullptr;
    int n_yw = 0;
    size_t smem_yw = 0;
    int4* d_work_e = nullptr;
    int n_e = 0;
    int* d_first_e = nullptr;
    double* d_epart = nullptr;
    double* d_eout = nullptr;
    std::vector<Launch> step_prog, hs_prog, fwd_prog;
    std::vector<double> dtab_host;     // dense short-axis DCT tables, built with the plans
    // persistent ensemble step (SGSPM_PERSISTENT)
    bool persist = false;
    PPhase* d_pph = nullptr;
    PItem* d_pit = nullptr;
    int* d_pfi = nullptr;
    unsigned* d_pctl = nullptr;        // ticket, abandon flag, per-film completed items
    bool p_stale = true;               // the persistent item tables predate a packing or program change
    int p_nphase = 0, p_items = 0, p_grid = 0;
    size_t p_smem = 0;
    long long p_wait_limit = 4000000000LL;   // clock cycles (about 2 s at 2 GHz)
    int p_withhold = -1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t adj_graph = nullptr;       // reverse step: forward transform, recording step, adjoint step
    cudaGraphExec_t adj_gexec = nullptr;
    cudaGraph_t radj_graph = nullptr;      // reverse step from restored recordings: adjoint step only
    cudaGraphExec_t radj_gexec = nullptr;
    cudaGraph_t rrec_graph = nullptr;      // segment replay: recording step
    cudaGraphExec_t rrec_gexec = nullptr;
    bool have_m = false;
    bool forcing = false;
    long long steps = 0;
    std::string err;
};

static thread_local std::string g_create_err;

#define CK(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
            return e_ == cudaErrorMemoryAllocation ? SGSPM_ERR_OOM : SGSPM_ERR_CUDA;           \
        }                                                                                      \
    } while (0)

static int fail(sgspm_ctx* ctx, int code, const std::string& msg) {
    ctx->err = msg;
    return code;
}

// ---------------------------------------------------------------------------------------------
// host numerics: twiddles (long double), Gauss-Legendre rules, radix plans
// ---------------------------------------------------------------------------------------------
static void cis(long long m, long long P, double* c, double* s) {
    // cos, sin of 2 pi m / P, evaluated in long double and rounded once
    long long r = ((m % P) + P) % P;
    long double th = 2.0L * 3.14159265358979323846264338327950288L * (long double)r / (long double)P;
    *c = (double)cosl(th);
    *s = (double)sinl(th);
}

static bool factor(int P, std::vector<int>& rs) {
    rs.clear();
    int p = P;
    const int order[5] = {8, 4, 2, 3, 5};
    for (int r : order)
        while (p % r == 0) {
            rs.push_back(r);
            p /= r;
        }
    return p == 1 && (int)rs.size() <= kMaxStages;
}

static void gauss_legendre(int q, double* x, double* w) {
    for (int i = 0; i < q; ++i) {
        long double z = cosl(3.14159265358979323846264338327950288L * (i + 0.75L) / (q + 0.5L));
        long double pp = 0;
        for (int it = 0; it < 100; ++it) {
            long double p1 = 1, p2 = 0;
            for (int j = 1; j <= q; ++j) {
                long double p3 = p2;
                p2 = p1;
                p1 = ((2.0L * j - 1.0L) * z * p2 - (j - 1.0L) * p3) / j;
            }
            pp = q * (z * p1 - p2) / (z * z - 1.0L);
            long double z1 = z;
            z = z1 - p1 / pp;
            if (fabsl(z - z1) < 1e-19L) break;
        }
        x[i] = (double)(-z);
        w[i] = (double)(2.0L / ((1.0L - z * z) * pp * pp));
    }
}

// ---------------------------------------------------------------------------------------------
template <typename T>
static Dev<T> dev_view(sgspm_ctx* ctx) {
    Dev<T> d;
    d.films = ctx->d_films;
    d.plans = ctx->d_plans;
    d.tw = (const tw_t<T>*)ctx->d_tw;
    d.lam = (const T*)ctx->d_lam;
    d.lam_lo = (const T*)ctx->d_lam_lo;
    d.dtab = (const T*)ctx->d_dtab;
    d.ktab = (const T*)ctx->d_ktab;
    d.field = (T* const*)ctx->d_tab;
    d.flo = (T* const*)ctx->d_tab_lo;
    d.spec = (cplx<T>* const*)ctx->d_tab_spec;
    d.he_cell = ctx->he_cell ? (const T*)ctx->d_he : nullptr;
    d.ycache = (cplx<T>*)ctx->d_ycache;
    d.ycache_n = ctx->nycache;
    d.status = ctx->d_status;
    d.step_ctr = ctx->d_step;
    d.tc_test = ctx->d_tc_test;
    return d;
}

// ---- size-class dispatch ---------------------------------------------------------------------
static int pow2_key(int n, int lo, int hi) { return (n >= lo && n <= hi && (n & (n - 1)) == 0) ? n : 0; }

// slab-pass size class of a film: its x length when that is a power of two in 8..512 and the
// film starts at a pool offset that is a multiple of four cells (the compile-time kernels move
// four cells per access), else 0 (runtime x length); the FP64 form uses the runtime kernel only
static int xz_key(bool fp64, const Film& F) {
    if (fp64 || F.off_cell % 4 != 0) return 0;
    return pow2_key(F.nx, 8, 512);
}

// size classes whose slab pass runs the tensor-core z transforms in the TF32X3 form
static bool ztc_class(bool tf32x3, int key) { return tf32x3 && (key == 128 || key == 256 || key == 512); }

constexpr int kMaxRowsPerCTA = 8;   // slab pass packing: y rows of one film per CTA

// size classes whose slab pass may pack several y rows per CTA (FP32 form; small slabs)
static bool packable_class(bool fp64, bool tf32x3, int key) {
    return !fp64 && !ztc_class(tf32x3, key) && key <= 256;
}

// launch type of a slab program: 1 right-hand sides only, 2 Gauss-Seidel update, 3 damping update
// and projection (the step's programs), 0 anything else (energy, set-up and adjoint programs)
static int xz_mode(const XZProg& p) {
    if (p.n_rhs > 0 && p.n_inv == 0 && p.op == 0 && p.n_fwd == 0 && p.rhs_dct) {
        for (int i = 0; i < p.n_rhs; ++i)
            if (p.rhs_copy[i] >= 0 || p.rhs_hs_store[i] >= 0) return 0;
        return 1;
    }
    if (p.n_rhs == 0 && p.op == 1) return 2;
    if (p.n_rhs == 0 && p.op == 2) return 3;
    return 0;
}

// compile-time x lengths with launch-type kernels (single row per CTA, FP32, no tensor cores)
static bool mode_class(int key) { return key == 64 || key == 128 || key == 256 || key == 512; }

template <typename T, int K>
static void launch_xz_mode(int mode, int nb, size_t smem, cudaStream_t st, const Dev<T>& d, const int4* w, const XZProg& pg,
                           int stray) {
    switch (mode) {
        case 1: xz_go<T, K, false, false, 1>(nb, smem, st, d, w, pg, stray); break;
        case 2: xz_go<T, K, false, false, 2>(nb, smem, st, d, w, pg, stray); break;
        case 3: xz_go<T, K, false, false, 3>(nb, smem, st, d, w, pg, stray); break;
        default: xz_go<T, K, false, false, 0>(nb, smem, st, d, w, pg, stray); break;
    }
}

template <typename T>
static void launch_xz(int key, int nb, size_t smem, cudaStream_t st, const Dev<T>& d, const int4* w, const XZProg& pg, int stray,
                      bool tf32x3, int rows, bool nz8, int threads) {
    if constexpr (sizeof(T) == 8) {   // the FP64 form uses the runtime-length kernel only
        xz_go<T, 0, false, false>(nb, smem, st, d, w, pg, stray);
        return;
    } else {
        // the packed-row kernel: several rows per CTA, or one row with fewer threads than kThreads
        if (rows > 1 || threads < kThreads) {
            switch (key) {
                case 64: xz_go<T, 64, false, true>(nb, smem, st, d, w, pg, stray, threads); return;
                case 128: xz_go<T, 128, false, true>(nb, smem, st, d, w, pg, stray, threads); return;
                case 256: xz_go<T, 256, false, true>(nb, smem, st, d, w, pg, stray, threads); return;
                default: xz_go<T, 0, false, true>(nb, smem, st, d, w, pg, stray, threads); return;
            }
        }
        if (ztc_class(tf32x3, key)) {
            switch (key) {
                case 128: xz_go<T, 128, true, false>(nb, smem, st, d, w, pg, stray); return;
                case 256: xz_go<T, 256, true, false>(nb, smem, st, d, w, pg, stray); return;
                default: xz_go<T, 512, true, false>(nb, smem, st, d, w, pg, stray); return;
            }
        }
        // the 512-thread launch types of the 256-wide class run slabs of nz = kZReg only
        const int mode = (key == 256 && !nz8) ? 0 : xz_mode(pg);
        switch (key) {
            case 64: launch_xz_mode<T, 64>(mode, nb, smem, st, d, w, pg, stray); return;
            case 128: launch_xz_mode<T, 128>(mode, nb, smem, st, d, w, pg, stray); return;
            case 256: launch_xz_mode<T, 256>(mode, nb, smem, st, d, w, pg, stray); return;
            case 512: launch_xz_mode<T, 512>(mode, nb, smem, st, d, w, pg, stray); return;
            default: break;
        }
        switch (key) {
#define SGSPM_XZ(K) case K: xz_go<T, K, false, false>(nb, smem, st, d, w, pg, stray); break;
            SGSPM_XZ(8) SGSPM_XZ(16) SGSPM_XZ(32)
#undef SGSPM_XZ
            default: xz_go<T, 0, false, false>(nb, smem, st, d, w, pg, stray);
        }
    }
}
template <typename T>
static cudaError_t attr_xz(int key, size_t smem, bool tf32x3) {
    if constexpr (sizeof(T) == 8) {
        return xz_attr<T, 0, false, false>(smem);
    } else {
        if (packable_class(false, tf32x3, key)) {
            cudaError_t e;
            if (key == 64) {
                e = xz_attr<T, 64, false, true>(smem);
            } else if (key == 128) {
                e = xz_attr<T, 128, false, true>(smem);
            } else if (key == 256) {
                e = xz_attr<T, 256, false, true>(smem);
            } else {
                // shared by several classes (runtime x length): allow the most dynamic shared
                // memory the device gives this kernel (opt-in maximum less its static part)
                int dev = 0, mx = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
                const long long st = xz_static_smem<T, 0, false, true>();
                if (st < 0) return (cudaError_t)(-st);
                e = xz_attr<T, 0, false, true>(std::max(mx - (int)st, (int)smem));
            }
            if (e != cudaSuccess) return e;
        }
        if (ztc_class(tf32x3, key)) {
            switch (key) {
                case 128: return xz_attr<T, 128, true, false>(smem);
                case 256: return xz_attr<T, 256, true, false>(smem);
                default: return xz_attr<T, 512, true, false>(smem);
            }
        }
        if (mode_class(key)) {
            cudaError_t e = cudaSuccess;
            switch (key) {
#define SGSPM_XZM(K)                                                                                         \
    case K:                                                                                                  \
        e = xz_attr<T, K, false, false, 1>(smem);                                                            \
        if (e == cudaSuccess) e = xz_attr<T, K, false, false, 2>(smem);                                      \
        if (e == cudaSuccess) e = xz_attr<T, K, false, false, 3>(smem);                                      \
        break;
                SGSPM_XZM(64) SGSPM_XZM(128) SGSPM_XZM(256) SGSPM_XZM(512)
#undef SGSPM_XZM
            }
            if (e != cudaSuccess) return e;
        }
        switch (key) {
#define SGSPM_XZ(K) case K: return xz_attr<T, K, false, false>(smem);
            SGSPM_XZ(8) SGSPM_XZ(16) SGSPM_XZ(32) SGSPM_XZ(64) SGSPM_XZ(128) SGSPM_XZ(256) SGSPM_XZ(512)
#undef SGSPM_XZ
            default: return xz_attr<T, 0, false, false>(smem);
        }
    }
}
template <typename T>
static void launch_yh(int key, int nb, size_t smem, cudaStream_t st, const Dev<T>& d, const int4* w, const YProg& pg,
                      int threads) {
    if constexpr (sizeof(T) == 8) {
        yh_go<T, 0>(nb, (unsigned)threads, smem, st, d, w, pg);
    } else {
        switch (key) {
#define SGSPM_YH(K) case K: yh_go<T, K>(nb, (unsigned)threads, smem, st, d, w, pg); break;
            SGSPM_YH(8) SGSPM_YH(16) SGSPM_YH(32) SGSPM_YH(64) SGSPM_YH(128) SGSPM_YH(256) SGSPM_YH(512)
#undef SGSPM_YH
            default: yh_go<T, 0>(nb, (unsigned)threads, smem, st, d, w, pg);
        }
    }
}
template <typename T>
static cudaError_t attr_yh(int key, size_t smem) {
    if constexpr (sizeof(T) == 8) {
        return yh_attr<T, 0>(smem);
    } else {
        switch (key) {
#define SGSPM_YH(K) case K: return yh_attr<T, K>(smem);
            SGSPM_YH(8) SGSPM_YH(16) SGSPM_YH(32) SGSPM_YH(64) SGSPM_YH(128) SGSPM_YH(256) SGSPM_YH(512)
#undef SGSPM_YH
            default: return yh_attr<T, 0>(smem);
        }
    }
}
// key = E = Py / 32
template <typename T, int NOUT>
static void launch_yw_n(int key, int nb, cudaStream_t st, const Dev<T>& d, const int4* w, const YProg& pg) {
    switch (key) {
        case 2: yw_go<T, NOUT, 2>(nb, st, d, w, pg); break;
        case 4: yw_go<T, NOUT, 4>(nb, st, d, w, pg); break;
        case 8: yw_go<T, NOUT, 8>(nb, st, d, w, pg); break;
        default: yw_go<T, NOUT, 16>(nb, st, d, w, pg); break;
    }
}
template <typename T>
static void launch_yw(int key, int nout, int nb, cudaStream_t st, const Dev<T>& d, const int4* w, const YProg& pg) {
    if (nout == 1) launch_yw_n<T, 1>(key, nb, st, d, w, pg);
    else if (nout == 2) launch_yw_n<T, 2>(key, nb, st, d, w, pg);
    else launch_yw_n<T, 3>(key, nb, st, d, w, pg);
}
template <typename T, int NOUT>
static cudaError_t attr_yw_n(int key, size_t smem) {
    switch (key) {
        case 2: return yw_attr<T, NOUT, 2>(smem);
        case 4: return yw_attr<T, NOUT, 4>(smem);
        case 8: return yw_attr<T, NOUT, 8>(smem);
        default: return yw_attr<T, NOUT, 16>(smem);
    }
}

template <typename T>
static int enqueue_t(sgspm_ctx* ctx, const Launch& L, cudaStream_t st) {
    Dev<T> d = dev_view<T>(ctx);
    switch (L.kind) {
        case 0:
            for (const auto& c : ctx->xz_cls)
                launch_xz<T>(c.key, c.n, c.smem, st, d, c.work, L.xz, ctx->stray ? 1 : 0, ctx->tf32x3, c.rows, c.nz8, c.threads);
            break;
        case 1:
            for (const auto& c : ctx->yh_cls) launch_yh<T>(c.key, c.n, c.smem, st, d, c.work, L.y, ctx->heat_threads);
            break;
        case 2: {
            int n = L.y.n;
            if (ctx->warp_stray) {
                for (const auto& c : ctx->yw_cls) launch_yw<T>(c.key, n, c.n, st, d, c.work, L.y);
            } else {
                ys_go<T>(ctx->n_ys[n], ctx->smem_ys[n], st, d, ctx->d_work_ys[n], L.y, ctx->tx_s[n]);
            }
            break;
        }
        case 3:
            step_counter_kernel<<<1, 1, 0, st>>>(ctx->d_step);
            break;
        case 4:
            adj_gs_kernel<T><<<ctx->n_e, kThreads, 0, st>>>(d, ctx->d_work_e, L.gs);
            break;
        case 5:
            adj_f_kernel<T><<<ctx->n_e, kThreads, 0, st>>>(d, ctx->d_work_e, L.af);
            break;
        case 6:
            adj_ew_kernel<T><<<ctx->n_e, kThreads, 0, st>>>(d, ctx->d_work_e, L.ew);
            break;
        case 7:
            adj_proj_kernel<T><<<ctx->n_e, kThreads, 0, st>>>(d, ctx->d_work_e, L.pj);
            break;
        default:
            adj_alpha_partial_kernel<T><<<ctx->n_e, kThreads, 0, st>>>(d, ctx->d_work_e, L.al, ctx->d_apart);
            adj_alpha_final_kernel<<<(ctx->nfilm + 127) / 128, 128, 0, st>>>(ctx->nfilm, ctx->d_first_e, ctx->d_apart,
                                                                              ctx->d_alpha_b);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SGSPM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SGSPM_OK;
}

static int enqueue(sgspm_ctx* ctx, const Launch& L, cudaStream_t st) {
    return ctx->fp64 ? enqueue_t<double>(ctx, L, st) : enqueue_t<float>(ctx, L, st);
}

static int run_prog(sgspm_ctx* ctx, const std::vector<Launch>& prog, cudaStream_t st) {
    for (const Launch& L : prog) {
        int rc = enqueue(ctx, L, st);
        if (rc) return rc;
    }
    return SGSPM_OK;
}

// ---- program builders --------------------------------------------------------------------------
static XZProg xz_empty() {
    XZProg p;
    memset(&p, 0, sizeof(p));
    for (int i = 0; i < 3; ++i) {
        p.rhs_h[i] = -1;
        p.rhs_hs_store[i] = -1;
        p.inv_store[i] = -1;
        p.rhs_copy[i] = -1;
        p.fin_v[i] = -1;
    }
    p.rhs_dct = 1;
    return p;
}

// fresh: components whose x,z spectrum changed since the cache was written (transformed along
// y, and stored when in `store`); the others are read from the y-transform cache.  The cache is
// only used by the register stray pass; the fallback pass always transforms all three.
static Launch mk_ystray(const std::vector<int>& outs, int fresh = 7, int store = 0) {
    Launch L;
    memset(&L, 0, sizeof(L));
    L.kind = 2;
    L.y.kind = 1;
    L.y.n = (int)outs.size();
    L.y.in_mask = 7;
    L.y.fresh_mask = fresh;
    L.y.store_mask = store;
    for (int i = 0; i < 3; ++i) L.y.in_spec[i] = S1 + i;
    for (size_t o = 0; o < outs.size(); ++o) {
        L.y.slot[o] = outs[o];
        L.y.out_spec[o] = H1 + outs[o];
    }
    return L;
}

static Launch mk_rhs(const sgspm_ctx* ctx, const std::vector<int>& comps, int s0, int s1, int s2, int damp) {
    Launch L;
    memset(&L, 0, sizeof(L));
    L.kind = 0;
    L.xz = xz_empty();
    L.xz.n_rhs = (int)comps.size();
    for (size_t i = 0; i < comps.size(); ++i) {
        L.xz.rhs_comp[i] = comps[i];
        L.xz.rhs_h[i] = ctx->stray ? H1 + comps[i] : -1;
        L.xz.rhs_out[i] = D1 + comps[i];
    }
    L.xz.state[0] = s0;
    L.xz.state[1] = s1;
    L.xz.state[2] = s2;
    L.xz.damp = damp;
    return L;
}

static Launch mk_yheat(const std::vector<int>& comps, int damp) {
    Launch L;
    memset(&L, 0, sizeof(L));
    L.kind = 1;
    L.y.kind = 0;
    L.y.n = (int)comps.size();
    for (size_t i = 0; i < comps.size(); ++i) L.y.slot[i] = D1 + comps[i];
    L.y.damp = damp;
    return L;
}

static int slab(int i) { return -1 - i; }

// Gauss-Seidel update pass: inverse-DCT of D_{comp} (delta in slab 0, optionally stored),
// out = base + p*q - r*s, then the forward padded FFT of `out` into S_{fwd_comp}.
static Launch mk_gs(const sgspm_ctx* ctx, int comp, int store, int out, int base, int p, int q, int r, int s, int fwd_comp) {
    Launch L;
    memset(&L, 0, sizeof(L));
    L.kind = 0;
    L.xz = xz_empty();
    L.xz.n_inv = 1;
    L.xz.inv_in[0] = D1 + comp;
    L.xz.inv_store[0] = store;
    L.xz.op = 1;
    L.xz.gs_out = out;
    L.xz.gs_base = base;
    L.xz.gs_p = p;
    L.xz.gs_q = q;
    L.xz.gs_r = r;
    L.xz.gs_s = s;
    if (ctx->stray && fwd_comp >= 0) {
        L.xz.n_fwd = 1;
        L.xz.fwd_src[0] = slab(2);
        L.xz.fwd_dst[0] = S1 + fwd_comp;
    }
    return L;
}

static Launch mk_final(const sgspm_ctx* ctx, int i0, int i1, int i2) {
    Launch L;
    memset(&L, 0, sizeof(L));
    L.kind = 0;
    L.xz = xz_empty();
    L.xz.n_inv = 3;
    for (int i = 0; i < 3; ++i) {
        L.xz.inv_in[i] = D1 + i;
        L.xz.fin_out[i] = M1 + i;
    }
    L.xz.fin_in[0] = i0;
    L.xz.fin_in[1] = i1;
    L.xz.fin_in[2] = i2;
    L.xz.op = 2;
    if (ctx->stray) {
        L.xz.n_fwd = 3;
        for (int i = 0; i < 3; ++i) {
            L.xz.fwd_src[i] = slab(i);
            L.xz.fwd_dst[i] = S1 + i;
        }
    }
    return L;
}

// One SGSPM step (R1) that also stores every intermediate the reverse step needs: all six
// deltas, h_s(m**), m*** and the new state in MN1..3 (M1..3 keep m^n).
static void build_record(sgspm_ctx* ctx) {
    const bool st = ctx->stray;
    std::vector<Launch>& P = ctx->rec_prog;
    P.clear();
    const bool yc = st && ctx->warp_stray;
    auto ys = [&](const std::vector<int>& outs, int fresh, int store) {
        return yc ? mk_ystray(outs, fresh, store) : mk_ystray(outs);
    };
    if (st) P.push_back(ys({1, 2}, 7, 7));
    P.push_back(mk_rhs(ctx, {1, 2}, M1, M2, M3, 0));
    P.push_back(mk_yheat({1, 2}, 0));
    {
        Launch L = mk_gs(ctx, 1, -1, A1, M1, slab(0), M3, slab(1), M2, 0);
        L.xz.n_inv = 2;
        L.xz.inv_in[0] = D2;
        L.xz.inv_in[1] = D3;
        L.xz.inv_store[0] = D2N;
        L.xz.inv_store[1] = E3N;
        P.push_back(L);
    }
    if (st) P.push_back(ys({0}, 1, 1));
    P.push_back(mk_rhs(ctx, {0}, A1, M2, M3, 0));
    P.push_back(mk_yheat({0}, 0));
    P.push_back(mk_gs(ctx, 0, E1S, A2, M2, E3N, A1, slab(0), M3, 1));
    if (st) P.push_back(ys({1}, 2, 2));
    P.push_back(mk_rhs(ctx, {1}, A1, A2, M3, 0));
    P.push_back(mk_yheat({1}, 0));
    P.push_back(mk_gs(ctx, 1, D2S, A3, M3, E1S, A2, slab(0), A1, 2));
    if (st) P.push_back(ys({2}, 4, 4));
    P.push_back(mk_rhs(ctx, {2}, A1, A2, A3, 0));
    P.push_back(mk_yheat({2}, 0));
    P.push_back(mk_gs(ctx, 2, E3SS, B2, M2, slab(0), A1, E1S, A3, 1));
    if (st) P.push_back(ys({1}, 2, 2));
    P.push_back(mk_rhs(ctx, {1}, A1, B2, A3, 0));
    P.push_back(mk_yheat({1}, 0));
    P.push_back(mk_gs(ctx, 1, D2SS, B1, M1, slab(0), A3, E3SS, B2, 0));
    if (st) P.push_back(ys({0, 1, 2}, 1, 0));
    {
        Launch L = mk_rhs(ctx, {0, 1, 2}, B1, B2, A3, 1);
        if (st)
            for (int i = 0; i < 3; ++i) L.xz.rhs_hs_store[i] = ERS1 + i;
        P.push_back(L);
    }
    P.push_back(mk_yheat({0, 1, 2}, 1));
    {
        Launch L = mk_final(ctx, B1, B2, A3);
        for (int i = 0; i < 3; ++i) {
            L.xz.fin_out[i] = MN1 + i;
            L.xz.fin_v[i] = V1 + i;
        }
        L.xz.n_fwd = 0;
        P.push_back(L);
    }
}

// The reverse of one recorded step: G1..3 holds dL/dm^{n+1} on entry and dL/dm^n on exit;
// dL/dh_e accumulates in bHE1..3 and dL/dalpha per film in d_alpha_b.
static void build_adjoint(sgspm_ctx* ctx) {
    const bool st = ctx->stray;
    std::vector<Launch>& P = ctx->adj_prog;
    P.clear();
    auto blank = [](int kind) {
        Launch L;
        memset(&L, 0, sizeof(L));
        L.kind = kind;
        L.xz = xz_empty();
        return L;
    };
    auto ew = [&](int mode, const std::vector<int>& dst, const std::vector<int>& src) {
        for (size_t i0 = 0; i0 < dst.size(); i0 += 16) {
            Launch L = blank(6);
            L.ew.mode = mode;
            L.ew.n = (int)std::min<size_t>(16, dst.size() - i0);
            for (int k = 0; k < L.ew.n; ++k) {
                L.ew.dst[k] = dst[i0 + k];
                L.ew.src[k] = src.empty() ? 0 : src[i0 + k];
            }
            P.push_back(L);
        }
    };
    auto solve = [&](const std::vector<int>& src, const std::vector<int>& dst, int damp) {
        const int k = (int)src.size();
        Launch X = blank(0);
        X.xz.n_rhs = k;
        for (int i = 0; i < k; ++i) {
            X.xz.rhs_comp[i] = i;
            X.xz.rhs_copy[i] = src[i];
            X.xz.rhs_out[i] = D1 + i;
        }
        X.xz.state[0] = M1;
        X.xz.state[1] = M2;
        X.xz.state[2] = M3;
        P.push_back(X);
        std::vector<int> comps;
        for (int i = 0; i < k; ++i) comps.push_back(i);
        P.push_back(mk_yheat(comps, damp));
        Launch I = blank(0);
        I.xz.n_inv = k;
        for (int i = 0; i < k; ++i) {
            I.xz.inv_in[i] = D1 + i;
            I.xz.inv_store[i] = dst[i];
        }
        P.push_back(I);
    };
    auto fadj = [&](const std::vector<int>& comps, const std::vector<int>& rho, const std::vector<int>& fb,
                    const int sb[3], int damp) {
        Launch L = blank(5);
        L.af.n = (int)comps.size();
        for (int k = 0; k < L.af.n; ++k) {
            L.af.comp[k] = comps[k];
            L.af.rho[k] = rho[k];
            L.af.fb[k] = fb[k];
        }
        for (int k = 0; k < 3; ++k) L.af.sb[k] = sb[k];
        L.af.heb = bHE1;
        L.af.damp = damp;
        P.push_back(L);
    };
    auto stray = [&](const std::vector<int>& comps, const std::vector<int>& fb, const int sb[3]) {
        if (!st) return;
        Launch F = blank(0);
        F.xz.n_fwd = (int)comps.size();
        int mask = 0;
        for (size_t k = 0; k < comps.size(); ++k) {
            F.xz.fwd_src[k] = fb[k];
            F.xz.fwd_dst[k] = SA1 + comps[k];
            mask |= 1 << comps[k];
        }
        P.push_back(F);
        Launch Y = mk_ystray({0, 1, 2});
        Y.y.in_mask = mask;
        for (int i = 0; i < 3; ++i) Y.y.in_spec[i] = SA1 + i;
        P.push_back(Y);
        // the inverse transforms add h_s of the adjoint input straight into the state adjoints
        Launch Hs = blank(0);
        Hs.xz.n_rhs = 3;
        Hs.xz.rhs_dct = 0;
        Hs.xz.rhs_hs_add = 1;
        for (int i = 0; i < 3; ++i) {
            Hs.xz.rhs_comp[i] = i;
            Hs.xz.rhs_h[i] = H1 + i;
            Hs.xz.rhs_hs_store[i] = sb[i];
        }
        Hs.xz.state[0] = M1;
        Hs.xz.state[1] = M2;
        Hs.xz.state[2] = M3;
        P.push_back(Hs);
    };
    auto gs = [&](int ub, int base_b, int p, int p_b, int q, int q_b, int r, int r_b, int s_, int s_b) {
        Launch L = blank(4);
        L.gs = AdjGS{ub, base_b, p, p_b, q, q_b, r, r_b, s_, s_b};
        P.push_back(L);
    };
    ew(1, {bM1, bM2, bM3, bA1, bA2, bA3, bB1, bB2, bD2N, bE3N, bE1S, bD2S, bE3SS, bD2SS}, {});
    // projection and damping heat flow (Steps 3 and 2)
    {
        Launch L = blank(7);
        for (int k = 0; k < 3; ++k) {
            L.pj.g[k] = G1 + k;
            L.pj.mn[k] = MN1 + k;
            L.pj.v[k] = V1 + k;
            L.pj.vb[k] = RB1 + k;
        }
        L.pj.eb[0] = bB1;
        L.pj.eb[1] = bB2;
        L.pj.eb[2] = bA3;
        P.push_back(L);
    }
    solve({RB1, RB2, RB3}, {RB1, RB2, RB3}, 1);
    {
        Launch L = blank(8);
        for (int k = 0; k < 3; ++k) {
            L.al.rho[k] = RB1 + k;
            L.al.hs[k] = ERS1 + k;
            L.al.v[k] = V1 + k;
        }
        L.al.e[0] = B1;
        L.al.e[1] = B2;
        L.al.e[2] = A3;
        L.al.have_hs = st ? 1 : 0;
        P.push_back(L);
    }
    const int sE[3] = {bB1, bB2, bA3};
    fadj({0, 1, 2}, {RB1, RB2, RB3}, {FB1, FB2, FB3}, sE, 1);
    stray({0, 1, 2}, {FB1, FB2, FB3}, sE);
    // m1** = m1 + d2** m3** - d3** m2**;  d2** at D = (m1*, m2**, m3**)
    gs(bB1, bM1, D2SS, bD2SS, A3, bA3, E3SS, bE3SS, B2, bB2);
    const int sD[3] = {bA1, bB2, bA3};
    solve({bD2SS}, {RB2}, 0);
    fadj({1}, {RB2}, {FB2}, sD, 0);
    stray({1}, {FB2}, sD);
    // m2** = m2 + d3** m1* - d1* m3**;  d3** at C = (m1*, m2*, m3*)
    gs(bB2, bM2, E3SS, bE3SS, A1, bA1, E1S, bE1S, A3, bA3);
    const int sC[3] = {bA1, bA2, bA3};
    solve({bE3SS}, {RB3}, 0);
    fadj({2}, {RB3}, {FB3}, sC, 0);
    stray({2}, {FB3}, sC);
    // m3* = m3 + d1* m2* - d2* m1*;  d2* at B = (m1*, m2*, m3)
    gs(bA3, bM3, E1S, bE1S, A2, bA2, D2S, bD2S, A1, bA1);
    const int sB[3] = {bA1, bA2, bM3};
    solve({bD2S}, {RB2}, 0);
    fadj({1}, {RB2}, {FB2}, sB, 0);
    stray({1}, {FB2}, sB);
    // m2* = m2 + d3n m1* - d1* m3;  d1* at A = (m1*, m2, m3)
    gs(bA2, bM2, E3N, bE3N, A1, bA1, E1S, bE1S, M3, bM3);
    const int sA[3] = {bA1, bM2, bM3};
    solve({bE1S}, {RB1}, 0);
    fadj({0}, {RB1}, {FB1}, sA, 0);
    stray({0}, {FB1}, sA);
    // m1* = m1 + d2n m3 - d3n m2;  d2n, d3n at m^n
    gs(bA1, bM1, D2N, bD2N, M3, bM3, E3N, bE3N, M2, bM2);
    const int sM[3] = {bM1, bM2, bM3};
    solve({bD2N, bE3N}, {RB2, RB3}, 0);
    fadj({1, 2}, {RB2, RB3}, {FB2, FB3}, sM, 0);
    stray({1, 2}, {FB2, FB3}, sM);
    ew(2, {G1, G2, G3}, {bM1, bM2, bM3});
}

static void build_programs(sgspm_ctx* ctx) {
    const bool R2 = (ctx->flags & SGSPM_FROZEN_STRAY) && ctx->stray;
    const bool gspm = (ctx->flags & SGSPM_GSPM) != 0;
    const bool st = ctx->stray;
    std::vector<Launch>& P = ctx->step_prog;
    P.clear();
    // components: 0 = paper's m1, 1 = m2, 2 = m3.  delta_i = g_i - m_i (see DESIGN: delta form)
    // h_s at m^n, then g2^n, g3^n
    const bool yc = st && !R2 && ctx->warp_stray;   // y-transform cache: refresh only what changed
    auto cached = [&](const std::vector<int>& outs, int fresh, int store) {
        return yc ? mk_ystray(outs, fresh, store) : mk_ystray(outs);
    };
    if (st) P.push_back(R2 ? mk_ystray({0, 1, 2}) : cached({1, 2}, 7, 7));
    P.push_back(mk_rhs(ctx, {1, 2}, M1, M2, M3, 0));
    P.push_back(mk_yheat({1, 2}, 0));
    {
        // m1* = m1 + d2n m3 - d3n m2   (d2n in slab 0, d3n in slab 1, stored)
        Launch L = mk_gs(ctx, 1, -1, A1, M1, slab(0), M3, slab(1), M2, R2 ? -1 : 0);
        L.xz.n_inv = 2;
        L.xz.inv_in[0] = D2;
        L.xz.inv_in[1] = D3;
        L.xz.inv_store[0] = -1;
        L.xz.inv_store[1] = E3N;
        P.push_back(L);
    }
    auto refresh = [&](int comp) {
        if (st && !R2) P.push_back(cached({comp}, 1 << comp, 1 << comp));
    };
    // g1* at (m1*, m2, m3) -> m2* = m2 + d3n m1* - d1* m3
    refresh(0);
    P.push_back(mk_rhs(ctx, {0}, A1, M2, M3, 0));
    P.push_back(mk_yheat({0}, 0));
    P.push_back(mk_gs(ctx, 0, E1S, A2, M2, E3N, A1, slab(0), M3, R2 ? -1 : 1));
    // g2* at (m1*, m2*, m3) -> m3* = m3 + d1* m2* - d2* m1*
    refresh(1);
    P.push_back(mk_rhs(ctx, {1}, A1, A2, M3, 0));
    P.push_back(mk_yheat({1}, 0));
    int m1f = A1, m2f = A2, m3f = A3;
    if (!gspm) {
        P.push_back(mk_gs(ctx, 1, -1, A3, M3, E1S, A2, slab(0), A1, R2 ? -1 : 2));
        // backward sweep: g3** at (m1*, m2*, m3**) -> m2** = m2 + d3** m1* - d1* m3**
        refresh(2);
        P.push_back(mk_rhs(ctx, {2}, A1, A2, A3, 0));
        P.push_back(mk_yheat({2}, 0));
        P.push_back(mk_gs(ctx, 2, E3SS, B2, M2, slab(0), A1, E1S, A3, R2 ? -1 : 1));
        // g2** at (m1*, m2**, m3**) -> m1** = m1 + d2** m3** - d3** m2**
        refresh(1);
        P.push_back(mk_rhs(ctx, {1}, A1, B2, A3, 0));
        P.push_back(mk_yheat({1}, 0));
        Launch L = mk_gs(ctx, 1, -1, B1, M1, slab(0), A3, E3SS, B2, R2 ? -1 : 0);
        if (R2) {
            L.xz.n_fwd = 3;
            L.xz.fwd_src[0] = slab(2);
            L.xz.fwd_dst[0] = S1;
            L.xz.fwd_src[1] = B2;
            L.xz.fwd_dst[1] = S2;
            L.xz.fwd_src[2] = A3;
            L.xz.fwd_dst[2] = S3;
        }
        P.push_back(L);
        m1f = B1;
        m2f = B2;
        m3f = A3;
    } else {
        Launch L = mk_gs(ctx, 1, -1, A3, M3, E1S, A2, slab(0), A1, R2 ? -1 : 2);
        if (R2) {
            L.xz.n_fwd = 3;
            L.xz.fwd_src[0] = A1;
            L.xz.fwd_dst[0] = S1;
            L.xz.fwd_src[1] = A2;
            L.xz.fwd_dst[1] = S2;
            L.xz.fwd_src[2] = slab(2);
            L.xz.fwd_dst[2] = S3;
            // slab 2 must be consumed before the global loads reuse slab 0: order it first
            std::swap(L.xz.fwd_src[0], L.xz.fwd_src[2]);
            std::swap(L.xz.fwd_dst[0], L.xz.fwd_dst[2]);
        }
        P.push_back(L);
    }
    // Step 2: damping heat flow at m**, Step 3: projection (only the component the last
    // Gauss-Seidel update changed is new: m1 for SGSPM, m3 for GSPM)
    if (st) P.push_back(R2 ? mk_ystray({0, 1, 2}) : cached({0, 1, 2}, gspm ? 4 : 1, 0));
    P.push_back(mk_rhs(ctx, {0, 1, 2}, m1f, m2f, m3f, 1));
    P.push_back(mk_yheat({0, 1, 2}, 1));
    P.push_back(mk_final(ctx, m1f, m2f, m3f));
    if (ctx->forcing) {
        Launch L;
        memset(&L, 0, sizeof(L));
        L.kind = 3;
        P.push_back(L);
    }

    // h_s of the current m into HS1..3
    ctx->hs_prog.clear();
    if (st) {
        ctx->hs_prog.push_back(mk_ystray({0, 1, 2}));
        Launch L;
        memset(&L, 0, sizeof(L));
        L.kind = 0;
        L.xz = xz_empty();
        L.xz.n_rhs = 3;
        L.xz.rhs_dct = 0;
        for (int i = 0; i < 3; ++i) {
            L.xz.rhs_comp[i] = i;
            L.xz.rhs_h[i] = H1 + i;
            L.xz.rhs_hs_store[i] = HS1 + i;
        }
        L.xz.state[0] = M1;
        L.xz.state[1] = M2;
        L.xz.state[2] = M3;
        ctx->hs_prog.push_back(L);
    }
    // forward padded FFT of M1..3 into S1..3 (after set_field)
    ctx->fwd_prog.clear();
    if (st) {
        Launch L;
        memset(&L, 0, sizeof(L));
        L.kind = 0;
        L.xz = xz_empty();
        L.xz.n_fwd = 3;
        for (int i = 0; i < 3; ++i) {
            L.xz.fwd_src[i] = M1 + i;
            L.xz.fwd_dst[i] = S1 + i;
        }
        ctx->fwd_prog.push_back(L);
    }
}

static int upload_tables(sgspm_ctx* ctx) {
    if (!ctx->d_tab) {
        CK(cudaMalloc(&ctx->d_tab, kMaxSlots * sizeof(void*)));
        CK(cudaMalloc(&ctx->d_tab_lo, kMaxSlots * sizeof(void*)));
        CK(cudaMalloc(&ctx->d_tab_spec, kMaxSpec * sizeof(void*)));
    }
    CK(cudaMemcpy(ctx->d_tab, ctx->d_field, kMaxSlots * sizeof(void*), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_tab_lo, ctx->d_flo, kMaxSlots * sizeof(void*), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_tab_spec, ctx->d_spec, kMaxSpec * sizeof(void*), cudaMemcpyHostToDevice));
    return SGSPM_OK;
}

static int drop_graph(sgspm_ctx* ctx) {
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->graph) cudaGraphDestroy(ctx->graph);
    if (ctx->adj_gexec) cudaGraphExecDestroy(ctx->adj_gexec);
    if (ctx->adj_graph) cudaGraphDestroy(ctx->adj_graph);
    for (cudaGraphExec_t* e : {&ctx->radj_gexec, &ctx->rrec_gexec})
        if (*e) cudaGraphExecDestroy(*e);
    for (cudaGraph_t* g : {&ctx->radj_graph, &ctx->rrec_graph})
        if (*g) cudaGraphDestroy(*g);
    ctx->gexec = nullptr;
    ctx->graph = nullptr;
    ctx->adj_gexec = nullptr;
    ctx->adj_graph = nullptr;
    ctx->radj_gexec = ctx->rrec_gexec = nullptr;
    ctx->radj_graph = ctx->rrec_graph = nullptr;
    ctx->p_stale = true;
    return SGSPM_OK;
}

// The launches of one reverse step (the state's forward transform, the recording step and the
// adjoint step) captured once into a CUDA graph; the caller loads the step's state before each
// launch of it.
static int capture_reverse(sgspm_ctx* ctx) {
    if (ctx->adj_gexec) return SGSPM_OK;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    int rc = run_prog(ctx, ctx->fwd_prog, ctx->cap);
    if (!rc) rc = run_prog(ctx, ctx->rec_prog, ctx->cap);
    if (!rc) rc = run_prog(ctx, ctx->adj_prog, ctx->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(ctx, SGSPM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    ctx->adj_graph = g;
    CK(cudaGraphInstantiate(&ctx->adj_gexec, g, 0));
    return SGSPM_OK;
}

// One program captured into a graph (the reverse sweep's recording and adjoint steps).
static int capture_prog(sgspm_ctx* ctx, const std::vector<Launch>& prog, cudaGraph_t* graph, cudaGraphExec_t* exec) {
    if (*exec) return SGSPM_OK;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    int rc = run_prog(ctx, prog, ctx->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(ctx, SGSPM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    *graph = g;
    CK(cudaGraphInstantiate(exec, g, 0));
    return SGSPM_OK;
}

template <typename T>
static size_t heat_smem(int ny, int tx);

// ---- persistent ensemble step -------------------------------------------------------------------
// Whether every film of the handle can run in the persistent kernel: FP32 form, register stray
// pass with padded y lengths 64..256 (E = 2, 4, 8), no manufactured forcing.
static bool persist_ok(const sgspm_ctx* ctx, std::string* why) {
    if (ctx->fp64 || ctx->tf32x3) {
        *why = "the persistent step runs the FP32 form only (not FP64, not TF32X3)";
        return false;
    }
    if (ctx->stray && !ctx->warp_stray) {
        *why = "the persistent step needs the register stray pass (padded y lengths 64..512)";
        return false;
    }
    for (const Film& F : ctx->films)
        if (ctx->stray && F.Py > 256) {
            *why = "the persistent step supports films with ny <= 128 (padded y length <= 256)";
            return false;
        }
    return true;
}

// Item tables of one step from the step program: phases in program order, films in order within a
// phase, the work items of each film as the per-pass launches cut them (slab rows packed as the
// class's packing says, heat tiles of tx_h lines, stray groups of kPersistLines lines).
static int build_persist(sgspm_ctx* ctx) {
    std::vector<PPhase> ph;
    std::vector<PItem> items;
    std::vector<int> per_film(ctx->nfilm, 0);
    size_t smem = 0;
    std::map<int, int> rows_of;   // slab class key -> rows per item
    for (const auto& c : ctx->xz_cls) rows_of[c.key] = c.rows;
    for (const Launch& L : ctx->step_prog) {
        if (L.kind > 2) return fail(ctx, SGSPM_ERR_UNSUPPORTED, "the persistent step has no manufactured forcing");
        PPhase P;
        memset(&P, 0, sizeof(P));
        P.kind = L.kind;
        P.first = (int)items.size();
        P.xz = L.xz;
        P.y = L.y;
        // films grouped by size class within the phase, so that CTAs run one class's code for long
        // stretches (an item depends only on its own film's earlier phases)
        std::vector<std::pair<int, int>> order;   // (class key, film)
        for (int f = 0; f < ctx->nfilm; ++f) {
            const Film& F = ctx->films[f];
            const int key = L.kind == 0 ? xz_key(false, F) : L.kind == 1 ? pow2_key(F.ny, 8, 512) : F.Py;
            order.push_back({key, f});
        }
        std::stable_sort(order.begin(), order.end(), [](const std::pair<int, int>& x, const std::pair<int, int>& y) { return x.first < y.first; });
        for (const auto& kf : order) {
            const int f = kf.second;
            const Film& F = ctx->films[f];
            auto add = [&](int4 wi, int key) {
                PItem it;
                memset(&it, 0, sizeof(it));
                it.wi = wi;
                it.key = key;
                it.target = per_film[f];
                it.phase = (int)ph.size();
                items.push_back(it);
            };
            int nf = 0;
            if (L.kind == 0) {
                const int key = xz_key(false, F);
                const int pkey = (key == 64 || key == 128 || key == 256) ? key : 0;
                const int rows = rows_of.count(key) ? rows_of[key] : 1;
                for (int y = 0; y < F.ny; y += rows, ++nf) add(make_int4(f, y, std::min(rows, F.ny - y), 0), pkey);
                smem = std::max(smem, xz_smem_bytes<float>(xz_layout(F.nx, F.nz, F.Px, F.Pz, F.Kx, ctx->stray, false)));
            } else if (L.kind == 1) {
                const int key = pow2_key(F.ny, 8, 512);
                const int pkey = (key == 64 || key == 128 || key == 256) ? key : 0;
                // about 8 cells per thread (at least the tuned tile): short lines get wide tiles
                const int tx = std::max(ctx->tx_h, std::min(32, std::max(1, 8 * kPersistThreads / F.ny)));
                for (int kz = 0; kz < F.nz; ++kz)
                    for (int x0 = 0; x0 < F.nx; x0 += tx, ++nf) add(make_int4(f, kz, x0, std::min(tx, F.nx - x0)), pkey);
                smem = std::max(smem, heat_smem<float>(F.ny, tx));
            } else {
                for (int kz = 0; kz < F.Pz; ++kz)
                    for (int x0 = 0; x0 < F.Kx; x0 += kPersistLines, ++nf)
                        add(make_int4(f, kz, x0, std::min(kPersistLines, F.Kx - x0)), F.Py / 32);
                smem = std::max(smem, yw_smem_bytes<float>(F.Py, L.y.n, kPersistLines));
            }
            per_film[f] += nf;
        }
        P.n = (int)items.size() - P.first;
        ph.push_back(P);
    }
    if (ctx->stream) CK(cudaStreamSynchronize(ctx->stream));
    for (void* p : {(void*)ctx->d_pph, (void*)ctx->d_pit, (void*)ctx->d_pfi, (void*)ctx->d_pctl})
        if (p) cudaFree(p);
    ctx->d_pph = nullptr;
    ctx->d_pit = nullptr;
    ctx->d_pfi = nullptr;
    ctx->d_pctl = nullptr;
    CK(cudaMalloc(&ctx->d_pph, ph.size() * sizeof(PPhase)));
    CK(cudaMemcpy(ctx->d_pph, ph.data(), ph.size() * sizeof(PPhase), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_pit, std::max<size_t>(1, items.size()) * sizeof(PItem)));
    CK(cudaMemcpy(ctx->d_pit, items.data(), items.size() * sizeof(PItem), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_pfi, per_film.size() * sizeof(int)));
    CK(cudaMemcpy(ctx->d_pfi, per_film.data(), per_film.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_pctl, (2 + ctx->nfilm) * sizeof(unsigned)));
    ctx->p_stale = false;
    CK(persist_attr(smem));
    const int per_sm = persist_blocks_per_sm(smem);
    int dev = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) return fail(ctx, SGSPM_ERR_UNSUPPORTED, "the persistent step does not fit on a multiprocessor");
    ctx->p_nphase = (int)ph.size();
    ctx->p_items = (int)items.size();
    ctx->p_smem = smem;
    ctx->p_grid = per_sm * nsm;
    return SGSPM_OK;
}

// One step: reset the ticket, the abandon flag and the film counters, then the persistent launch.
static int enqueue_persist(sgspm_ctx* ctx, cudaStream_t st) {
    CK(cudaMemsetAsync(ctx->d_pctl, 0, (2 + ctx->nfilm) * sizeof(unsigned), st));
    PersistArgs a;
    a.phases = ctx->d_pph;
    a.items = ctx->d_pit;
    a.film_items = ctx->d_pfi;
    a.ctl = ctx->d_pctl;
    a.nphase = ctx->p_nphase;
    a.items_per_step = ctx->p_items;
    a.nsteps = 1;
    a.stray = ctx->stray ? 1 : 0;
    a.wait_limit = ctx->p_wait_limit;
    a.withhold = ctx->p_withhold;
    persist_go((unsigned)ctx->p_grid, ctx->p_smem, st, dev_view<float>(ctx), a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SGSPM_ERR_CUDA, std::string("persistent launch: ") + cudaGetErrorString(e));
    return SGSPM_OK;
}

static int capture_step(sgspm_ctx* ctx) {
    drop_graph(ctx);
    if (ctx->persist) {
        int rc = build_persist(ctx);
        if (rc) return rc;
    }
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    int rc = ctx->persist ? enqueue_persist(ctx, ctx->cap) : run_prog(ctx, ctx->step_prog, ctx->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(ctx, SGSPM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    ctx->graph = g;
    CK(cudaGraphInstantiate(&ctx->gexec, g, 0));
    return SGSPM_OK;
}

// ---------------------------------------------------------------------------------------------
// set-up
// ---------------------------------------------------------------------------------------------
static int get_plan(sgspm_ctx* ctx, int P, std::vector<double2>& tw) {
    auto it = ctx->plan_of.find(P);
    if (it != ctx->plan_of.end()) return it->second;
    Plan pl;
    memset(&pl, 0, sizeof(pl));
    std::vector<int> rs;
    if (!factor(P, rs)) return -1;
    pl.P = P;
    pl.nst = (int)rs.size();
    for (size_t i = 0; i < rs.size(); ++i) pl.radix[i] = rs[i];
    pl.tw = (int)tw.size();
    for (int m = 0; m < P; ++m) {
        double c, s;
        cis(m, P, &c, &s);
        tw.push_back(make_double2(c, -s));
    }
    pl.tw4 = (int)tw.size();
    for (int k = 0; k < P; ++k) {
        double c, s;
        cis(k, 4LL * P, &c, &s);
        tw.push_back(make_double2(c, -s));
    }
    pl.dtab = -1;
    if (P <= 16) {
        // C[k][n] = cos(pi k (2n+1) / (2P));  Ci[n][k] = (k ? 2 : 1) C[k][n]
        pl.dtab = (int)ctx->dtab_host.size();
        for (int k = 0; k < P; ++k)
            for (int n = 0; n < P; ++n) {
                double c, s;
                cis((long long)k * (2 * n + 1), 4LL * P, &c, &s);
                ctx->dtab_host.push_back(c);
            }
        for (int n = 0; n < P; ++n)
            for (int k = 0; k < P; ++k) {
                double c, s;
                cis((long long)k * (2 * n + 1), 4LL * P, &c, &s);
                ctx->dtab_host.push_back(k ? 2.0 * c : c);
            }
    }
    int id = (int)ctx->plans.size();
    ctx->plans.push_back(pl);
    ctx->plan_of[P] = id;
    return id;
}

template <typename T>
static int upload_tw(sgspm_ctx* ctx, const std::vector<double2>& tw) {
    std::vector<tw_t<T>> v(tw.size());
    for (size_t i = 0; i < tw.size(); ++i) v[i] = tw_make(tw[i].x, tw[i].y, (T*)nullptr);
    CK(cudaMalloc(&ctx->d_tw, v.size() * sizeof(tw_t<T>)));
    CK(cudaMemcpy(ctx->d_tw, v.data(), v.size() * sizeof(tw_t<T>), cudaMemcpyHostToDevice));
    return SGSPM_OK;
}

template <typename T>
static int upload_vec(sgspm_ctx* ctx, void** dst, const std::vector<double>& src) {
    std::vector<T> v(src.begin(), src.end());
    CK(cudaMalloc(dst, v.size() * sizeof(T) + 16));
    CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SGSPM_OK;
}

// Newell spectrum of one film into ktab (+ off_ktab), FP64 on the device.
template <typename T>
static int newell_setup(sgspm_ctx* ctx, const Film& F) {
    const int nx = F.nx, ny = F.ny, nz = F.nz, Kx = F.Kx;
    const int Hy = F.Py / 2 + 1, Hz = F.Pz / 2 + 1;
    const long long noct = (long long)nx * ny * nz;
    GLTable gl;
    memset(&gl, 0, sizeof(gl));
    int off = 0;
    for (int q : {4, 5, 6, 7, 8, 14}) {
        gl.off[q] = off;
        gauss_legendre(q, gl.x + off, gl.w + off);
        off += q;
    }
    double *oct = nullptr, *A = nullptr, *B = nullptr, *C = nullptr, *tabs = nullptr;
    const long long nA = 6LL * nz * ny * Kx, nB = 6LL * nz * Hy * Kx, nC = 6LL * Hz * Hy * Kx;
    std::vector<double> h_tab;
    int Ps[3] = {F.Px, F.Py, F.Pz};
    long long toff[3];
    for (int a = 0; a < 3; ++a) {
        toff[a] = (long long)h_tab.size();
        for (int m = 0; m < Ps[a]; ++m) {
            double c, s;
            cis(m, Ps[a], &c, &s);
            h_tab.push_back(c);
        }
        for (int m = 0; m < Ps[a]; ++m) {
            double c, s;
            cis(m, Ps[a], &c, &s);
            h_tab.push_back(s);
        }
    }
    cudaError_t e = cudaSuccess;
    auto al = [&](double** p, long long n) {
        if (e == cudaSuccess) e = cudaMalloc(p, (size_t)n * sizeof(double));
    };
    al(&oct, 6 * noct);
    al(&A, nA);
    al(&B, nB);
    al(&C, nC);
    al(&tabs, (long long)h_tab.size());
    if (e == cudaSuccess) e = cudaMemcpy(tabs, h_tab.data(), h_tab.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        newell_octant_kernel<<<(unsigned)((noct + 127) / 128), 128>>>(oct, nx, ny, nz, F.hx, F.hy, F.hz, gl);
        e = cudaGetLastError();
    }
    auto cs = [&](int a) { return tabs + toff[a]; };
    auto sn = [&](int a) { return tabs + toff[a] + Ps[a]; };
    if (e == cudaSuccess) {
        newell_axis_kernel<<<(unsigned)((nA + 255) / 256), 256>>>(oct, A, 0, nx, Kx, F.Px, ny, nz, 1, nx, (long long)ny * nx,
                                                                 noct, 1, Kx, (long long)ny * Kx, (long long)nz * ny * Kx, cs(0), sn(0));
        newell_axis_kernel<<<(unsigned)((nB + 255) / 256), 256>>>(A, B, 1, ny, Hy, F.Py, Kx, nz, Kx, 1, (long long)ny * Kx,
                                                                 (long long)nz * ny * Kx, Kx, 1, (long long)Hy * Kx,
                                                                 (long long)nz * Hy * Kx, cs(1), sn(1));
        newell_axis_kernel<<<(unsigned)((nC + 255) / 256), 256>>>(B, C, 2, nz, Hz, F.Pz, Hy * Kx, 1, (long long)Hy * Kx, 1, 0,
                                                                 (long long)nz * Hy * Kx, (long long)Hy * Kx, 1, 0,
                                                                 (long long)Hz * Hy * Kx, cs(2), sn(2));
        newell_finish_kernel<T><<<(unsigned)((nC + 255) / 256), 256>>>(C, (T*)ctx->d_ktab + F.off_ktab, Kx, Hy, ktab_row(F.Py), Hz,
                                                                       1.0 / ((double)F.Px * F.Py * F.Pz));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(oct);
    cudaFree(A);
    cudaFree(B);
    cudaFree(C);
    cudaFree(tabs);
    if (e != cudaSuccess) return fail(ctx, SGSPM_ERR_CUDA, std::string("Newell set-up: ") + cudaGetErrorString(e));
    return SGSPM_OK;
}

// y heat pass: shared memory of a CTA of tx lines of length ny
template <typename T>
static size_t heat_smem(int ny, int tx) {
    const size_t V = sizeof(cplx<T>);
    return (size_t)2 * ny * sizeof(tw_t<T>) + (size_t)2 * ((tx + 1) / 2) * ny * V + (size_t)tx * (ny + 8) * sizeof(T);
}

// (Re)build the y heat pass's size classes with tx x lines per CTA (a tuning knob).
template <typename T>
static int build_heat_classes(sgspm_ctx* ctx, int tx) {
    std::map<int, std::vector<int4>> wy;
    std::map<int, size_t> syk;
    for (int f = 0; f < ctx->nfilm; ++f) {
        const Film& F = ctx->films[f];
        const int ky = sizeof(T) == 8 ? 0 : pow2_key(F.ny, 8, 512);
        for (int kz = 0; kz < F.nz; ++kz)
            for (int x0 = 0; x0 < F.nx; x0 += tx) wy[ky].push_back(make_int4(f, kz, x0, std::min(tx, F.nx - x0)));
        syk[ky] = std::max(syk[ky], heat_smem<T>(F.ny, tx));
    }
    if (ctx->stream) CK(cudaStreamSynchronize(ctx->stream));
    for (auto& c : ctx->yh_cls) cudaFree(c.work);
    ctx->yh_cls.clear();
    for (auto& kv : wy) {
        sgspm_ctx::KClass c{kv.first, nullptr, (int)kv.second.size(), syk[kv.first]};
        CK(cudaMalloc(&c.work, std::max<size_t>(1, kv.second.size()) * sizeof(int4)));
        CK(cudaMemcpy(c.work, kv.second.data(), kv.second.size() * sizeof(int4), cudaMemcpyHostToDevice));
        CK(attr_yh<T>(c.key, c.smem));
        ctx->yh_cls.push_back(c);
    }
    ctx->tx_h = tx;
    drop_graph(ctx);
    return SGSPM_OK;
}

template <typename T>
static int setup_t(sgspm_ctx* ctx) {
    const size_t V = sizeof(cplx<T>);
    std::vector<double2> tw;
    std::vector<double> lam;
    ctx->dtab_host.clear();
    // plans, offsets
    long long oc = 0, os = 0, ok = 0, oyc = 0;
    std::map<std::vector<double>, long long> ktab_of;
    std::vector<int> ktab_owner;   // film that computes each unique table (or -1)
    for (int f = 0; f < ctx->nfilm; ++f) {
        Film& F = ctx->films[f];
        F.Px = F.nx > 1 ? 2 * F.nx : 1;
        F.Py = F.ny > 1 ? 2 * F.ny : 1;
        F.Pz = F.nz > 1 ? 2 * F.nz : 1;
        F.Kx = F.Px / 2 + 1;
        int ids[6] = {get_plan(ctx, F.nx, tw), get_plan(ctx, F.ny, tw), get_plan(ctx, F.nz, tw),
                      get_plan(ctx, F.Px, tw), get_plan(ctx, F.Py, tw), get_plan(ctx, F.Pz, tw)};
        for (int i = 0; i < 6; ++i)
            if (ids[i] < 0)
                return fail(ctx, SGSPM_ERR_UNSUPPORTED, "axis length has a prime factor other than 2, 3, 5 (film " + std::to_string(f) + ")");
        F.plan_dx = ids[0];
        F.plan_dy = ids[1];
        F.plan_dz = ids[2];
        F.plan_px = ids[3];
        F.plan_py = ids[4];
        F.plan_pz = ids[5];
        {
            // copies: staged() below grows ctx->plans
            const Plan dx = ctx->plans[ids[0]], dy = ctx->plans[ids[1]], dz = ctx->plans[ids[2]];
            const Plan px = ctx->plans[ids[3]], py = ctx->plans[ids[4]], pz = ctx->plans[ids[5]];
            F.gtw_dx = dx.tw;
            F.gtw4_dx = dx.tw4;
            F.gtw_dz = dz.tw;
            F.gtw4_dz = dz.tw4;
            F.gtw_px = px.tw;
            F.gtw_pz = pz.tw;
            F.gtw_dy = dy.tw;
            F.gtw4_dy = dy.tw4;
            F.gtw_py = py.tw;
            F.gdtab_z = dz.dtab >= 0 ? dz.dtab : 0;
            auto staged = [&](const Plan& src, int tw, int tw4) {
                Plan q = src;
                q.tw = tw;
                q.tw4 = tw4;
                ctx->plans.push_back(q);
                return (int)ctx->plans.size() - 1;
            };
            const int nx = F.nx, nz = F.nz;
            F.splan_dx = staged(dx, 0, nx);
            F.splan_dz = staged(dz, 2 * nx, 2 * nx + nz);
            F.splan_px = staged(px, 2 * nx + 2 * nz, 0);
            F.splan_pz = staged(pz, 2 * nx + 2 * nz + F.Px, 0);
            F.splan_dy = staged(dy, 0, F.ny);
        }
        F.off_cell = oc;
        oc += (long long)F.nx * F.ny * F.nz;
        F.off_spec = os;
        os += (long long)F.Kx * F.ny * F.Pz;
        F.off_ycache = oyc;
        oyc += (long long)F.Pz * F.Kx * F.Py;
        F.lam = (int)lam.size();
        const int ns[3] = {F.nx, F.ny, F.nz};
        const double hs[3] = {F.hx, F.hy, F.hz};
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < ns[a]; ++k) {
                double c, s;
                cis(k, 4LL * ns[a], &c, &s);   // sin(pi k / (2 n))
                lam.push_back(4.0 / (hs[a] * hs[a]) * s * s);
            }
        if (ctx->stray) {
            std::vector<double> key = {(double)F.nx, (double)F.ny, (double)F.nz, F.hx, F.hy, F.hz};
            auto it = ktab_of.find(key);
            if (it == ktab_of.end()) {
                F.off_ktab = ok;
                ktab_of[key] = ok;
                ok += 6LL * (F.Pz / 2 + 1) * ktab_row(F.Py) * F.Kx;
                ktab_owner.push_back(f);
            } else {
                F.off_ktab = it->second;
            }
        }
    }
    ctx->ncell = oc;
    ctx->nspec = os;
    ctx->nycache = oyc;
    ctx->nktab = ok;
    // shared-memory budgets
    int dev = 0;
    CK(cudaGetDevice(&dev));
    int smem_max = 0;
    CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    ctx->smem_max = (size_t)smem_max;
    size_t sx = 0, sy = 0;
    int maxPy = 1, maxny = 1;
    for (const Film& F : ctx->films) {
        const int key = xz_key(sizeof(T) == 8, F);
        XZLayout L = xz_layout(F.nx, F.nz, F.Px, F.Pz, F.Kx, ctx->stray, ztc_class(ctx->tf32x3, key));
        size_t b = xz_smem_bytes<T>(L);
        if (b > sx) sx = b;
        if (F.Py > maxPy) maxPy = F.Py;
        if (F.ny > maxny) maxny = F.ny;
    }
    ctx->tx_h = 8;
    sy = heat_smem<T>(maxny, ctx->tx_h);
    if (sx > (size_t)smem_max || sy > (size_t)smem_max)
        return fail(ctx, SGSPM_ERR_UNSUPPORTED, "slab of " + std::to_string(sx) + " B does not fit in shared memory");
    ctx->smem_xz = sx;
    ctx->smem_yh = sy;
    for (int n = 1; n <= 3; ++n) {
        const size_t budget = 100 * 1024;
        int tx = (int)(budget / ((2 + n) * (size_t)(maxPy + 4) * V));
        if (tx > 16) tx = 16;
        if (tx < 1) tx = 1;
        ctx->tx_s[n] = tx;
        ctx->smem_ys[n] = (size_t)maxPy * sizeof(tw_t<T>) + (size_t)(2 + n) * tx * (maxPy + 4) * V;
        if (ctx->smem_ys[n] > (size_t)smem_max)
            return fail(ctx, SGSPM_ERR_UNSUPPORTED, "y line of length " + std::to_string(maxPy) + " does not fit in shared memory");
    }
    CK(ys_attr<T>(std::max(ctx->smem_ys[1], std::max(ctx->smem_ys[2], ctx->smem_ys[3]))));
    // work lists: slab and heat passes per size class (films of one x / y length share a launch)
    std::vector<int4> we;
    // pointwise and reduction kernels (energy, adjoint): one kThreads CTA per item of `ecell`
    // cells; 1024 (four cells per thread) where that still gives every SM four CTAs, smaller
    // items on small grids, which 1024-cell items would leave on a fraction of the SMs
    int nsm = 0;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    long long ecell = 4 * kThreads;
    while (ecell > kThreads && ctx->ncell / ecell < 4LL * nsm) ecell -= kThreads;
    std::vector<int> first_e;
    auto up4 = [&](int4** d, const std::vector<int4>& h) -> int {
        CK(cudaMalloc(d, std::max<size_t>(1, h.size()) * sizeof(int4)));
        if (!h.empty()) CK(cudaMemcpy(*d, h.data(), h.size() * sizeof(int4), cudaMemcpyHostToDevice));
        return SGSPM_OK;
    };
    int rc;
    {
        std::map<int, std::vector<int4>> wx;
        std::map<int, size_t> sxk;
        for (int f = 0; f < ctx->nfilm; ++f) {
            const Film& F = ctx->films[f];
            const int kx = xz_key(sizeof(T) == 8, F);
            for (int y = 0; y < F.ny; ++y) wx[kx].push_back(make_int4(f, y, 0, 0));
            XZLayout L = xz_layout(F.nx, F.nz, F.Px, F.Pz, F.Kx, ctx->stray, ztc_class(ctx->tf32x3, kx));
            sxk[kx] = std::max(sxk[kx], xz_smem_bytes<T>(L));
            first_e.push_back((int)we.size());
            long long nc = (long long)F.nx * F.ny * F.nz;
            for (long long c0 = 0; c0 < nc; c0 += ecell) we.push_back(make_int4(f, (int)c0, (int)std::min(ecell, nc - c0), 0));
        }
        for (auto& kv : wx) {
            sgspm_ctx::KClass c{kv.first, nullptr, (int)kv.second.size(), sxk[kv.first]};
            for (const Film& F : ctx->films)
                if (xz_key(sizeof(T) == 8, F) == c.key && F.nz != kZReg) c.nz8 = false;
            if ((rc = up4(&c.work, kv.second))) return rc;
            CK(attr_xz<T>(c.key, c.smem, ctx->tf32x3));
            ctx->xz_cls.push_back(c);
        }
    }
    if ((rc = build_heat_classes<T>(ctx, ctx->tx_h))) return rc;
    first_e.push_back((int)we.size());
    if ((rc = up4(&ctx->d_work_e, we))) return rc;
    ctx->n_e = (int)we.size();
    for (int n = 1; n <= 3; ++n) {
        std::vector<int4> ws;
        for (int f = 0; f < ctx->nfilm; ++f) {
            const Film& F = ctx->films[f];
            for (int kz = 0; kz < F.Pz; ++kz)
                for (int x0 = 0; x0 < F.Kx; x0 += ctx->tx_s[n]) ws.push_back(make_int4(f, kz, x0, std::min(ctx->tx_s[n], F.Kx - x0)));
        }
        if ((rc = up4(&ctx->d_work_ys[n], ws))) return rc;
        ctx->n_ys[n] = (int)ws.size();
    }
    // register-resident stray pass when every film's padded y length is 64..512, per length class
    ctx->warp_stray = ctx->stray;
    for (const Film& F : ctx->films)
        if (!(F.Py == 64 || F.Py == 128 || F.Py == 256 || F.Py == 512) || yw_smem_bytes<T>(F.Py, 3) > (size_t)smem_max)
            ctx->warp_stray = false;
    if (ctx->warp_stray) {
        std::map<int, std::vector<int4>> ws;
        for (int f = 0; f < ctx->nfilm; ++f) {
            const Film& F = ctx->films[f];
            for (int kz = 0; kz < F.Pz; ++kz)
                for (int x0 = 0; x0 < F.Kx; x0 += kWarpLines)
                    ws[F.Py / 32].push_back(make_int4(f, kz, x0, std::min(kWarpLines, F.Kx - x0)));
        }
        for (auto& kv : ws) {
            const int Py = 32 * kv.first;
            sgspm_ctx::KClass c{kv.first, nullptr, (int)kv.second.size(), yw_smem_bytes<T>(Py, 3)};
            if ((rc = up4(&c.work, kv.second))) return rc;
            cudaError_t e1 = attr_yw_n<T, 1>(c.key, yw_smem_bytes<T>(Py, 1));
            cudaError_t e2 = attr_yw_n<T, 2>(c.key, yw_smem_bytes<T>(Py, 2));
            cudaError_t e3 = attr_yw_n<T, 3>(c.key, yw_smem_bytes<T>(Py, 3));
            CK(e1);
            CK(e2);
            CK(e3);
            ctx->yw_cls.push_back(c);
        }
    }
    CK(cudaMalloc(&ctx->d_first_e, first_e.size() * sizeof(int)));
    CK(cudaMemcpy(ctx->d_first_e, first_e.data(), first_e.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_epart, std::max(1, ctx->n_e) * 4 * sizeof(double)));
    CK(cudaMalloc(&ctx->d_eout, ctx->nfilm * 5 * sizeof(double)));
    // tables
    if ((rc = upload_tw<T>(ctx, tw))) return rc;
    if ((rc = upload_vec<T>(ctx, &ctx->d_lam, lam))) return rc;
    if (sizeof(T) == 4) {
        std::vector<double> lo(lam.size());
        for (size_t i = 0; i < lam.size(); ++i) lo[i] = lam[i] - (double)(T)lam[i];
        if ((rc = upload_vec<T>(ctx, &ctx->d_lam_lo, lo))) return rc;
    }
    if (ctx->dtab_host.empty()) ctx->dtab_host.push_back(0.0);
    if ((rc = upload_vec<T>(ctx, &ctx->d_dtab, ctx->dtab_host))) return rc;
    CK(cudaMalloc(&ctx->d_films, ctx->films.size() * sizeof(Film)));
    for (Film& F : ctx->films) film_consts(F);
    CK(cudaMemcpy(ctx->d_films, ctx->films.data(), ctx->films.size() * sizeof(Film), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&ctx->d_plans, ctx->plans.size() * sizeof(Plan)));
    CK(cudaMemcpy(ctx->d_plans, ctx->plans.data(), ctx->plans.size() * sizeof(Plan), cudaMemcpyHostToDevice));
    // pools
    for (int i = 0; i < NSLOT_FWD; ++i) {
        CK(cudaMalloc(&ctx->d_field[i], (size_t)ctx->ncell * sizeof(T)));
        CK(cudaMemset(ctx->d_field[i], 0, (size_t)ctx->ncell * sizeof(T)));
    }
    if (sizeof(T) == 4) {
        // FP32 form: the magnetisation states are double-float (hi + lo) so that rounding of the
        // O(1) state does not accumulate over many steps; transforms use the hi part only
        for (int i = M1; i <= B2; ++i) {
            CK(cudaMalloc(&ctx->d_flo[i], (size_t)ctx->ncell * sizeof(T)));
            CK(cudaMemset(ctx->d_flo[i], 0, (size_t)ctx->ncell * sizeof(T)));
        }
    }
    if (ctx->stray) {
        for (int i = 0; i < NSPEC_FWD; ++i) {
            CK(cudaMalloc(&ctx->d_spec[i], (size_t)ctx->nspec * V));
            CK(cudaMemset(ctx->d_spec[i], 0, (size_t)ctx->nspec * V));
        }
        CK(cudaMalloc(&ctx->d_ktab, (size_t)ctx->nktab * sizeof(T)));
        CK(cudaMemset(ctx->d_ktab, 0, (size_t)ctx->nktab * sizeof(T)));   // line padding stays zero
        if (ctx->warp_stray) {
            CK(cudaMalloc(&ctx->d_ycache, (size_t)(3 * ctx->nycache) * sizeof(cplx<T>)));
            CK(cudaMemset(ctx->d_ycache, 0, (size_t)(3 * ctx->nycache) * sizeof(cplx<T>)));
        }
        for (int f : ktab_owner)
            if ((rc = newell_setup<T>(ctx, ctx->films[f]))) return rc;
    }
    CK(cudaMalloc(&ctx->d_stage, (size_t)3 * ctx->ncell * sizeof(double)));
    CK(cudaMalloc(&ctx->d_status, sizeof(int)));
    CK(cudaHostAlloc(&ctx->h_status, sizeof(int), cudaHostAllocDefault));
    if (ctx->tf32x3) {
        CK(cudaMalloc(&ctx->d_tc_test, 2 * sizeof(int)));
        CK(cudaMemset(ctx->d_tc_test, 0, 2 * sizeof(int)));
    }
    CK(cudaMemset(ctx->d_status, 0, sizeof(int)));
    CK(cudaMalloc(&ctx->d_step, sizeof(long long)));
    CK(cudaMemset(ctx->d_step, 0, sizeof(long long)));
    CK(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
    ctx->tsz = sizeof(T);
    if ((rc = upload_tables(ctx))) return rc;
    build_programs(ctx);
    CK(cudaDeviceSynchronize());
    return SGSPM_OK;
}

static void release(sgspm_ctx* ctx) {
    drop_graph(ctx);
    void* ptrs[] = {ctx->d_films, ctx->d_plans, ctx->d_tw, ctx->d_lam, ctx->d_lam_lo, ctx->d_dtab, ctx->d_ktab, ctx->d_he, ctx->d_status, ctx->d_step,
                    ctx->d_stage, ctx->d_work_xz, ctx->d_work_yh, ctx->d_work_e, ctx->d_first_e, ctx->d_epart, ctx->d_eout,
                    ctx->d_work_yw};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < kMaxSlots; ++i) {
        if (ctx->d_field[i]) cudaFree(ctx->d_field[i]);
        if (ctx->d_flo[i]) cudaFree(ctx->d_flo[i]);
    }
    for (int i = 0; i < kMaxSpec; ++i)
        if (ctx->d_spec[i]) cudaFree(ctx->d_spec[i]);
    void* more[] = {ctx->d_tab, ctx->d_tab_lo, ctx->d_tab_spec, ctx->d_ckpt, ctx->d_seg, ctx->d_rec, ctx->d_final, ctx->d_apart,
                    ctx->d_alpha_b, ctx->d_ycache, ctx->d_tc_test, ctx->d_pph, ctx->d_pit, ctx->d_pfi, ctx->d_pctl};
    for (void* p : more)
        if (p) cudaFree(p);
    for (int n = 0; n < 4; ++n)
        if (ctx->d_work_ys[n]) cudaFree(ctx->d_work_ys[n]);
    for (auto* v : {&ctx->xz_cls, &ctx->yh_cls, &ctx->yw_cls})
        for (auto& c : *v)
            if (c.work) cudaFree(c.work);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
}

static int check_status(sgspm_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int st = *ctx->h_status;
    if (st & 1) return fail(ctx, SGSPM_ERR_NONFINITE, "non-finite value or zero vector before projection");
    if (st & 2) return fail(ctx, SGSPM_ERR_NONFINITE, "set_field: zero-length or non-finite magnetisation vector");
    if (st & 4) return fail(ctx, SGSPM_ERR_TIMEOUT, "a tensor-core transform of the slab pass did not complete in time");
    if (st & 8) return fail(ctx, SGSPM_ERR_TIMEOUT, "a work item of the persistent step waited too long for its film's previous pass");
    return SGSPM_OK;
}

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
// The address at which the copy kernels can use the caller's buffer in place, or nullptr: device
// memory of the current device, or page-locked host memory mapped into the device's address space
// (the kernel's own loads and stores cross the bus, with far more requests in flight than one
// copy-engine transfer).  Pageable and managed memory go through the staging buffer.
static const void* direct_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    if (a.type == cudaMemoryTypeDevice && a.device == dev) return a.devicePointer;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

template <typename T>
static int set_field_t(sgspm_t ctx, int which, const void* ptr, int dtype) {
    const long long n = ctx->ncell;
    const size_t bytes = (size_t)3 * n * (dtype == SGSPM_F64_DATA ? 8 : 4);
    const void* src = direct_ptr(ptr);
    if (!src) {
        CK(cudaMemcpyAsync(ctx->d_stage, ptr, bytes, cudaMemcpyDefault, ctx->stream));
        src = ctx->d_stage;
    }
    const unsigned nb = (unsigned)((n + 255) / 256);
    T *d0, *d1, *d2, *l0 = nullptr, *l1 = nullptr, *l2 = nullptr;
    if (which == SGSPM_M) {
        d0 = (T*)ctx->d_field[M1];
        d1 = (T*)ctx->d_field[M2];
        d2 = (T*)ctx->d_field[M3];
        l0 = (T*)ctx->d_flo[M1];
        l1 = (T*)ctx->d_flo[M2];
        l2 = (T*)ctx->d_flo[M3];
    } else {
        // per-cell h_e is kept interleaved [cell][3]; stage through three scratch slots
        d0 = (T*)ctx->d_field[HS1];
        d1 = (T*)ctx->d_field[HS2];
        d2 = (T*)ctx->d_field[HS3];
    }
    // m is normalised by the copy kernel itself (status: bit 2 for a zero-length or non-finite vector)
    int* status = which == SGSPM_M ? ctx->d_status : nullptr;
    if (status) CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    if (dtype == SGSPM_F64_DATA)
        copy_in_kernel<T, double><<<nb, 256, 0, ctx->stream>>>(d0, d1, d2, l0, l1, l2, (const double*)src,
                                                               ctx->d_films, ctx->nfilm, n, status);
    else
        copy_in_kernel<T, float><<<nb, 256, 0, ctx->stream>>>(d0, d1, d2, l0, l1, l2, (const float*)src,
                                                              ctx->d_films, ctx->nfilm, n, status);
    CK(cudaGetLastError());
    if (which == SGSPM_M) {
        int rc = check_status(ctx);
        if (rc) return fail(ctx, SGSPM_ERR_ARG, "set_field: zero-length or non-finite magnetisation vector");
        rc = run_prog(ctx, ctx->fwd_prog, ctx->stream);
        if (rc) return rc;
        ctx->have_m = true;
        // the status check above synchronised after the copy-in: the caller's buffer is no longer
        // read, and the forward transform stays ordered on the stream
        return SGSPM_OK;
    } else {
        if (!ctx->d_he) CK(cudaMalloc(&ctx->d_he, (size_t)3 * n * sizeof(T)));
        he_interleave_kernel<T><<<nb, 256, 0, ctx->stream>>>((T*)ctx->d_he, d0, d1, d2, n);
        CK(cudaGetLastError());
        if (!ctx->he_cell) {
            ctx->he_cell = true;
            drop_graph(ctx);
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return SGSPM_OK;
}

template <typename T>
static int get_field_t(sgspm_t ctx, int which, void* ptr, int dtype) {
    const long long n = ctx->ncell;
    const unsigned nb = (unsigned)((n + 255) / 256);
    int base = M1;
    if (which == SGSPM_HS) {
        if (ctx->stray) {
            int rc = run_prog(ctx, ctx->hs_prog, ctx->stream);
            if (rc) return rc;
        } else {
            for (int i = 0; i < 3; ++i) CK(cudaMemsetAsync(ctx->d_field[HS1 + i], 0, (size_t)n * sizeof(T), ctx->stream));
        }
        base = HS1;
    }
    const T* s0 = (const T*)ctx->d_field[base];
    const T* s1 = (const T*)ctx->d_field[base + 1];
    const T* s2 = (const T*)ctx->d_field[base + 2];
    const T* q0 = (const T*)ctx->d_flo[base];
    const T* q1 = (const T*)ctx->d_flo[base + 1];
    const T* q2 = (const T*)ctx->d_flo[base + 2];
    void* dst = const_cast<void*>(direct_ptr(ptr));
    void* out = dst ? dst : ctx->d_stage;
    if (dtype == SGSPM_F64_DATA)
        copy_out_kernel<T, double><<<nb, 256, 0, ctx->stream>>>((double*)out, s0, s1, s2, q0, q1, q2, ctx->d_films,
                                                                ctx->nfilm, n);
    else
        copy_out_kernel<T, float><<<nb, 256, 0, ctx->stream>>>((float*)out, s0, s1, s2, q0, q1, q2, ctx->d_films,
                                                               ctx->nfilm, n);
    CK(cudaGetLastError());
    if (!dst) {
        const size_t bytes = (size_t)3 * n * (dtype == SGSPM_F64_DATA ? 8 : 4);
        CK(cudaMemcpyAsync(ptr, ctx->d_stage, bytes, cudaMemcpyDefault, ctx->stream));
    }
    return check_status(ctx);
}

// Allocate the slots, spectra and buffers a recorded forward and its reverse need.
template <typename T>
static int rec_alloc_t(sgspm_ctx* ctx, long long nseg, int K) {
    const size_t cell = (size_t)ctx->ncell * sizeof(T);
    if (!ctx->rec_alloc) {
        for (int i = NSLOT_FWD; i < NSLOT; ++i) {
            CK(cudaMalloc(&ctx->d_field[i], cell));
            CK(cudaMemset(ctx->d_field[i], 0, cell));
        }
        if (sizeof(T) == 4)
            for (int i = MN1; i <= MN3; ++i) {
                CK(cudaMalloc(&ctx->d_flo[i], cell));
                CK(cudaMemset(ctx->d_flo[i], 0, cell));
            }
        if (ctx->stray)
            for (int i = NSPEC_FWD; i < NSPEC; ++i) {
                CK(cudaMalloc(&ctx->d_spec[i], (size_t)ctx->nspec * sizeof(cplx<T>)));
                CK(cudaMemset(ctx->d_spec[i], 0, (size_t)ctx->nspec * sizeof(cplx<T>)));
            }
        CK(cudaMalloc(&ctx->d_apart, std::max(1, ctx->n_e) * sizeof(double)));
        CK(cudaMalloc(&ctx->d_alpha_b, ctx->nfilm * sizeof(double)));
        CK(cudaMalloc(&ctx->d_final, 6 * cell));
        ctx->rec_alloc = true;
        int rc = upload_tables(ctx);
        if (rc) return rc;
        build_record(ctx);
        build_adjoint(ctx);
    }
    if (ctx->d_ckpt) cudaFree(ctx->d_ckpt);
    if (ctx->d_seg) cudaFree(ctx->d_seg);
    if (ctx->d_rec) cudaFree(ctx->d_rec);
    ctx->d_ckpt = ctx->d_seg = ctx->d_rec = nullptr;
    CK(cudaMalloc(&ctx->d_ckpt, (size_t)nseg * 6 * cell));
    CK(cudaMalloc(&ctx->d_seg, (size_t)K * 6 * cell));
    // the recorded slots of every step of a segment, so that the reverse sweep need not run each
    // step's recording again; without the memory it falls back to recomputing them
    if (cudaMalloc(&ctx->d_rec, (size_t)K * kRecSlots * cell) != cudaSuccess) {
        cudaGetLastError();
        ctx->d_rec = nullptr;
    }
    return SGSPM_OK;
}

// state (M1..3 hi/lo) <-> buf [hi 3][lo 3] of ncell each
template <typename T>
static int state_io(sgspm_ctx* ctx, T* buf, bool save) {
    const long long n = ctx->ncell;
    const unsigned nb = (unsigned)((n + 255) / 256);
    for (int a = 0; a < 3; ++a) {
        T* hi = buf + a * n;
        T* lo = buf + (3 + a) * n;
        T* mh = (T*)ctx->d_field[M1 + a];
        T* ml = (T*)ctx->d_flo[M1 + a];
        if (save) state_copy_kernel<T><<<nb, 256, 0, ctx->stream>>>(hi, lo, mh, ml, n);
        else state_copy_kernel<T><<<nb, 256, 0, ctx->stream>>>(mh, ml, hi, ml ? lo : nullptr, n);
    }
    CK(cudaGetLastError());
    return SGSPM_OK;
}

template <typename T>
static int record_t(sgspm_ctx* ctx, long long nsteps, int K) {
    const long long nseg = (nsteps + K - 1) / K;
    int rc = rec_alloc_t<T>(ctx, nseg, K);
    if (rc) return rc;
    T* ck = (T*)ctx->d_ckpt;
    const long long per = 6 * ctx->ncell;
    for (long long sgi = 0; sgi < nseg; ++sgi) {
        if ((rc = state_io<T>(ctx, ck + sgi * per, true))) return rc;
        const long long n = std::min<long long>(K, nsteps - sgi * K);
        if ((rc = sgspm_step(ctx, n))) return rc;
    }
    ctx->rec_nsteps = nsteps;
    ctx->rec_K = K;
    return check_status(ctx);
}

template <typename T>
static int grad_t(sgspm_ctx* ctx, const void* dL_dmT, int dtype, void* dL_dhe, double* dL_dalpha) {
    const long long n = ctx->ncell;
    const unsigned nb = (unsigned)((n + 255) / 256);
    const long long nsteps = ctx->rec_nsteps;
    const int K = ctx->rec_K;
    const long long nseg = (nsteps + K - 1) / K;
    const long long per = 6 * n;
    int rc;
    // dL/dm(T) -> G1..3 ; m(T) saved for the end
    const size_t bytes = (size_t)3 * n * (dtype == SGSPM_F64_DATA ? 8 : 4);
    CK(cudaMemcpyAsync(ctx->d_stage, dL_dmT, bytes, cudaMemcpyDefault, ctx->stream));
    T* g0 = (T*)ctx->d_field[G1];
    T* g1 = (T*)ctx->d_field[G2];
    T* g2 = (T*)ctx->d_field[G3];
    if (dtype == SGSPM_F64_DATA)
        copy_in_kernel<T, double><<<nb, 256, 0, ctx->stream>>>(g0, g1, g2, nullptr, nullptr, nullptr,
                                                               (const double*)ctx->d_stage, ctx->d_films, ctx->nfilm, n,
                                                               nullptr);
    else
        copy_in_kernel<T, float><<<nb, 256, 0, ctx->stream>>>(g0, g1, g2, nullptr, nullptr, nullptr,
                                                              (const float*)ctx->d_stage, ctx->d_films, ctx->nfilm, n,
                                                              nullptr);
    CK(cudaGetLastError());
    if ((rc = state_io<T>(ctx, (T*)ctx->d_final, true))) return rc;
    for (int a = 0; a < 3; ++a) CK(cudaMemsetAsync(ctx->d_field[bHE1 + a], 0, (size_t)n * sizeof(T), ctx->stream));
    CK(cudaMemsetAsync(ctx->d_alpha_b, 0, ctx->nfilm * sizeof(double), ctx->stream));
    T* ck = (T*)ctx->d_ckpt;
    T* sg = (T*)ctx->d_seg;
    for (long long sgi = nseg - 1; sgi >= 0; --sgi) {
        const long long L = std::min<long long>(K, nsteps - sgi * K);
        // recompute the segment's step states
        if ((rc = state_io<T>(ctx, ck + sgi * per, false))) return rc;
        if ((rc = run_prog(ctx, ctx->fwd_prog, ctx->stream))) return rc;
        const bool graphs = !(ctx->flags & SGSPM_NO_GRAPH);
        if (ctx->d_rec) {
            // replay the segment with the recording step and keep every step's recorded slots;
            // the reverse of a step then restores them and runs the adjoint step alone
            T* rb = (T*)ctx->d_rec;
            const long long rper = (long long)kRecSlots * n;
            const dim3 sgrid(nb, kRecSlots);
            if (graphs && (rc = capture_prog(ctx, ctx->rec_prog, &ctx->rrec_graph, &ctx->rrec_gexec))) return rc;
            if (graphs && (rc = capture_prog(ctx, ctx->adj_prog, &ctx->radj_graph, &ctx->radj_gexec))) return rc;
            for (long long j = 0; j < L; ++j) {
                if (graphs) CK(cudaGraphLaunch(ctx->rrec_gexec, ctx->stream));
                else if ((rc = run_prog(ctx, ctx->rec_prog, ctx->stream))) return rc;
                slots_io_kernel<T><<<sgrid, 256, 0, ctx->stream>>>(rb + j * rper, ctx->d_tab, n, 1);
                CK(cudaGetLastError());
                if (j + 1 == L) break;
                // the next state is m^{n+1} (MN1..3, hi and lo), with its forward transform
                for (int a = 0; a < 3; ++a)
                    state_copy_kernel<T><<<nb, 256, 0, ctx->stream>>>((T*)ctx->d_field[M1 + a], (T*)ctx->d_flo[M1 + a],
                                                                      (const T*)ctx->d_field[MN1 + a],
                                                                      (const T*)ctx->d_flo[MN1 + a], n);
                CK(cudaGetLastError());
                if ((rc = run_prog(ctx, ctx->fwd_prog, ctx->stream))) return rc;
            }
            for (long long j = L - 1; j >= 0; --j) {
                slots_io_kernel<T><<<sgrid, 256, 0, ctx->stream>>>(rb + j * rper, ctx->d_tab, n, 0);
                CK(cudaGetLastError());
                if (graphs) CK(cudaGraphLaunch(ctx->radj_gexec, ctx->stream));
                else if ((rc = run_prog(ctx, ctx->adj_prog, ctx->stream))) return rc;
            }
            continue;
        }
        if (graphs && !ctx->gexec && (rc = capture_step(ctx))) return rc;
        for (long long j = 0; j < L; ++j) {
            if ((rc = state_io<T>(ctx, sg + j * per, true))) return rc;
            if (j + 1 == L) break;
            if (graphs) CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
            else if ((rc = run_prog(ctx, ctx->step_prog, ctx->stream))) return rc;
        }
        // reverse through the segment
        if (graphs && (rc = capture_reverse(ctx))) return rc;
        for (long long j = L - 1; j >= 0; --j) {
            if ((rc = state_io<T>(ctx, sg + j * per, false))) return rc;
            if (graphs) {
                CK(cudaGraphLaunch(ctx->adj_gexec, ctx->stream));
                continue;
            }
            if ((rc = run_prog(ctx, ctx->fwd_prog, ctx->stream))) return rc;
            if ((rc = run_prog(ctx, ctx->rec_prog, ctx->stream))) return rc;
            if ((rc = run_prog(ctx, ctx->adj_prog, ctx->stream))) return rc;
        }
    }
    // outputs
    const T* h0 = (const T*)ctx->d_field[bHE1];
    const T* h1 = (const T*)ctx->d_field[bHE2];
    const T* h2 = (const T*)ctx->d_field[bHE3];
    if (dtype == SGSPM_F64_DATA)
        copy_out_kernel<T, double><<<nb, 256, 0, ctx->stream>>>((double*)ctx->d_stage, h0, h1, h2, nullptr, nullptr, nullptr,
                                                                ctx->d_films, ctx->nfilm, n);
    else
        copy_out_kernel<T, float><<<nb, 256, 0, ctx->stream>>>((float*)ctx->d_stage, h0, h1, h2, nullptr, nullptr, nullptr,
                                                               ctx->d_films, ctx->nfilm, n);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(dL_dhe, ctx->d_stage, bytes, cudaMemcpyDefault, ctx->stream));
    CK(cudaMemcpyAsync(dL_dalpha, ctx->d_alpha_b, ctx->nfilm * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    // back to m(T)
    if ((rc = state_io<T>(ctx, (T*)ctx->d_final, false))) return rc;
    if ((rc = run_prog(ctx, ctx->fwd_prog, ctx->stream))) return rc;
    return check_status(ctx);
}

extern "C" {

int sgspm_version(void) { return 102; }

const char* sgspm_last_error(sgspm_t h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int sgspm_create_batch(int nfilm, const sgspm_grid* grids, const double* eps, const double* Q, const double* alpha,
                       const double* dt, const double* easy_axis, int flags, void* cuda_stream, sgspm_t* out) {
    if (!out) {
        g_create_err = "out is NULL";
        return SGSPM_ERR_ARG;
    }
    *out = nullptr;
    if (nfilm < 1 || !grids || !eps || !Q || !alpha || !dt || !easy_axis) {
        g_create_err = "nfilm < 1 or a NULL parameter array";
        return SGSPM_ERR_ARG;
    }
    sgspm_ctx* ctx = new sgspm_ctx();
    ctx->nfilm = nfilm;
    ctx->flags = flags;
    ctx->fp64 = (flags & SGSPM_FP64) != 0;
    ctx->stray = !(flags & SGSPM_NO_STRAY);
    ctx->tf32x3 = (flags & SGSPM_TF32X3) && !ctx->fp64;
    ctx->stream = (cudaStream_t)cuda_stream;
    for (int f = 0; f < nfilm; ++f) {
        const sgspm_grid& g = grids[f];
        const double* u = easy_axis + 3 * f;
        double un = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        std::string why;
        if (g.nx < 1 || g.ny < 1 || g.nz < 1) why = "cell counts must be >= 1";
        else if (!(g.hx > 0 && g.hy > 0 && g.hz > 0)) why = "cell sizes must be > 0";
        else if (!(eps[f] >= 0 && Q[f] >= 0 && alpha[f] >= 0)) why = "eps, Q, alpha must be >= 0";
        else if (!(dt[f] > 0)) why = "dt must be > 0";
        else if (!(un > 0) || !std::isfinite(un)) why = "easy axis must be a finite non-zero vector";
        else if ((long long)g.nx * g.ny * g.nz > (1LL << 31) / 4) why = "film too large";
        if (!why.empty()) {
            g_create_err = "film " + std::to_string(f) + ": " + why;
            delete ctx;
            return SGSPM_ERR_ARG;
        }
        Film F;
        memset(&F, 0, sizeof(F));
        F.nx = g.nx;
        F.ny = g.ny;
        F.nz = g.nz;
        F.hx = g.hx;
        F.hy = g.hy;
        F.hz = g.hz;
        F.eps = eps[f];
        F.Q = Q[f];
        F.alpha = alpha[f];
        F.dt = dt[f];
        for (int a = 0; a < 3; ++a) F.u[a] = u[a] / un;
        ctx->films.push_back(F);
    }
    int rc = ctx->fp64 ? setup_t<double>(ctx) : setup_t<float>(ctx);
    if (rc == SGSPM_OK && (flags & SGSPM_PERSISTENT)) {
        std::string why;
        if (persist_ok(ctx, &why)) ctx->persist = true;
        else rc = fail(ctx, SGSPM_ERR_UNSUPPORTED, why);
    }
    if (rc) {
        g_create_err = ctx->err;
        release(ctx);
        delete ctx;
        return rc;
    }
    *out = ctx;
    return SGSPM_OK;
}

int sgspm_create(const sgspm_grid* grid, double eps, double Q, double alpha, double dt, const double easy_axis[3], int flags,
                 void* cuda_stream, sgspm_t* out) {
    if (!grid || !easy_axis) {
        g_create_err = "grid or easy_axis is NULL";
        if (out) *out = nullptr;
        return SGSPM_ERR_ARG;
    }
    return sgspm_create_batch(1, grid, &eps, &Q, &alpha, &dt, easy_axis, flags, cuda_stream, out);
}

int sgspm_destroy(sgspm_t h) {
    if (!h) return SGSPM_OK;
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
    return SGSPM_OK;
}

int sgspm_set_applied_field(sgspm_t ctx, const double* he) {
    if (!ctx || !he) return ctx ? fail(ctx, SGSPM_ERR_ARG, "he is NULL") : SGSPM_ERR_ARG;
    for (int f = 0; f < ctx->nfilm; ++f)
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(he[3 * f + a])) return fail(ctx, SGSPM_ERR_ARG, "applied field must be finite");
            ctx->films[f].he[a] = he[3 * f + a];
        }
    ctx->he_cell = false;
    CK(cudaStreamSynchronize(ctx->stream));
    for (Film& F : ctx->films) film_consts(F);
    CK(cudaMemcpy(ctx->d_films, ctx->films.data(), ctx->films.size() * sizeof(Film), cudaMemcpyHostToDevice));
    drop_graph(ctx);
    return SGSPM_OK;
}

int sgspm_set_alpha(sgspm_t ctx, const double* alpha) {
    if (!ctx || !alpha) return ctx ? fail(ctx, SGSPM_ERR_ARG, "alpha is NULL") : SGSPM_ERR_ARG;
    for (int f = 0; f < ctx->nfilm; ++f)
        if (!(std::isfinite(alpha[f]) && alpha[f] >= 0)) return fail(ctx, SGSPM_ERR_ARG, "alpha must be finite and >= 0");
    for (int f = 0; f < ctx->nfilm; ++f) ctx->films[f].alpha = alpha[f];
    CK(cudaStreamSynchronize(ctx->stream));
    for (Film& F : ctx->films) film_consts(F);
    CK(cudaMemcpy(ctx->d_films, ctx->films.data(), ctx->films.size() * sizeof(Film), cudaMemcpyHostToDevice));
    return SGSPM_OK;
}

int sgspm_set_field(sgspm_t ctx, int which, const void* ptr, int dtype) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (!ptr) return fail(ctx, SGSPM_ERR_ARG, "ptr is NULL");
    if (which != SGSPM_M && which != SGSPM_HE) return fail(ctx, SGSPM_ERR_ARG, "set_field: which must be SGSPM_M or SGSPM_HE");
    if (dtype != SGSPM_F32 && dtype != SGSPM_F64_DATA) return fail(ctx, SGSPM_ERR_ARG, "dtype must be SGSPM_F32 or SGSPM_F64_DATA");
    return ctx->fp64 ? set_field_t<double>(ctx, which, ptr, dtype) : set_field_t<float>(ctx, which, ptr, dtype);
}

int sgspm_get_field(sgspm_t ctx, int which, void* ptr, int dtype) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (!ptr) return fail(ctx, SGSPM_ERR_ARG, "ptr is NULL");
    if (which != SGSPM_M && which != SGSPM_HS) return fail(ctx, SGSPM_ERR_ARG, "get_field: which must be SGSPM_M or SGSPM_HS");
    if (dtype != SGSPM_F32 && dtype != SGSPM_F64_DATA) return fail(ctx, SGSPM_ERR_ARG, "dtype must be SGSPM_F32 or SGSPM_F64_DATA");
    if (!ctx->have_m) return fail(ctx, SGSPM_ERR_STATE, "m has not been set");
    return ctx->fp64 ? get_field_t<double>(ctx, which, ptr, dtype) : get_field_t<float>(ctx, which, ptr, dtype);
}

int sgspm_step(sgspm_t ctx, long long n) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (n < 1) return fail(ctx, SGSPM_ERR_ARG, "n must be >= 1");
    if (!ctx->have_m) return fail(ctx, SGSPM_ERR_STATE, "m has not been set");
    if (ctx->flags & SGSPM_NO_GRAPH) {
        if (ctx->persist && (ctx->p_stale || !ctx->d_pctl)) {
            int rc = build_persist(ctx);
            if (rc) return rc;
        }
        for (long long i = 0; i < n; ++i) {
            int rc = ctx->persist ? enqueue_persist(ctx, ctx->stream) : run_prog(ctx, ctx->step_prog, ctx->stream);
            if (rc) return rc;
        }
    } else {
        if (!ctx->gexec) {
            int rc = capture_step(ctx);
            if (rc) return rc;
        }
        for (long long i = 0; i < n; ++i) CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
    }
    ctx->steps += n;
    return SGSPM_OK;
}

// ---- batch packing and its autotuner ----------------------------------------------------------
static int xz_class_key(const sgspm_ctx* ctx, const Film& F) { return xz_key(ctx->fp64, F); }

// Rebuild the slab-pass work list of class c with `rows` y rows per CTA.
static int set_class_rows(sgspm_ctx* ctx, size_t c, int rows, int threads) {
    auto& K = ctx->xz_cls[c];
    if (K.rows == rows && K.work) {
        if (K.threads != threads) drop_graph(ctx);
        K.threads = threads;
        return SGSPM_OK;
    }
    std::vector<int4> w;
    for (int f = 0; f < ctx->nfilm; ++f) {
        const Film& F = ctx->films[f];
        if (xz_class_key(ctx, F) != K.key) continue;
        for (int y = 0; y < F.ny; y += rows) w.push_back(make_int4(f, y, std::min(rows, F.ny - y), 0));
    }
    int4* d = nullptr;
    CK(cudaMalloc(&d, std::max<size_t>(1, w.size()) * sizeof(int4)));
    CK(cudaMemcpy(d, w.data(), w.size() * sizeof(int4), cudaMemcpyHostToDevice));
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(K.work);
    K.work = d;
    K.n = (int)w.size();
    K.rows = rows;
    K.threads = threads;
    drop_graph(ctx);
    return SGSPM_OK;
}

int sgspm_heat_tile(sgspm_t ctx) { return ctx ? ctx->tx_h : SGSPM_ERR_ARG; }

int sgspm_set_heat_tile(sgspm_t ctx, int tx) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (tx < 1 || tx > 16) return fail(ctx, SGSPM_ERR_ARG, "x lines per heat CTA must be in 1..16");
    int maxny = 1;
    for (const Film& F : ctx->films) maxny = std::max(maxny, F.ny);
    if ((ctx->fp64 ? heat_smem<double>(maxny, tx) : heat_smem<float>(maxny, tx)) > ctx->smem_max)
        return fail(ctx, SGSPM_ERR_UNSUPPORTED, "heat tile does not fit in shared memory");
    return ctx->fp64 ? build_heat_classes<double>(ctx, tx) : build_heat_classes<float>(ctx, tx);
}

int sgspm_xz_classes(sgspm_t ctx, int* keys, int* rows, int cap) {
    if (!ctx) return SGSPM_ERR_ARG;
    const int n = (int)ctx->xz_cls.size();
    if ((keys || rows) && cap < n) return fail(ctx, SGSPM_ERR_ARG, "cap is below the number of size classes");
    for (int c = 0; c < n; ++c) {
        if (keys) keys[c] = ctx->xz_cls[c].key;
        if (rows) rows[c] = ctx->xz_cls[c].rows;
    }
    return n;
}

int sgspm_set_packing(sgspm_t ctx, const int* rows, int n) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (!rows || n != (int)ctx->xz_cls.size()) return fail(ctx, SGSPM_ERR_ARG, "rows must have one entry per size class");
    for (int c = 0; c < n; ++c) {
        if (rows[c] < 1 || rows[c] > kMaxRowsPerCTA) return fail(ctx, SGSPM_ERR_ARG, "rows per CTA must be in 1..8");
        if (rows[c] > 1 && !packable_class(ctx->fp64, ctx->tf32x3, ctx->xz_cls[c].key))
            return fail(ctx, SGSPM_ERR_UNSUPPORTED, "this size class runs one row per CTA");
    }
    for (int c = 0; c < n; ++c)
        if (rows[c] != ctx->xz_cls[c].rows) {
            int rc = set_class_rows(ctx, (size_t)c, rows[c], ctx->xz_cls[c].threads);
            if (rc) return rc;
        }
    return SGSPM_OK;
}

int sgspm_xz_threads(sgspm_t ctx, int* threads, int cap) {
    if (!ctx) return SGSPM_ERR_ARG;
    const int n = (int)ctx->xz_cls.size();
    if (threads && cap < n) return fail(ctx, SGSPM_ERR_ARG, "cap is below the number of size classes");
    for (int c = 0; threads && c < n; ++c) threads[c] = ctx->xz_cls[c].threads;
    return n;
}

int sgspm_set_packing_threads(sgspm_t ctx, const int* threads, int n) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (!threads || n != (int)ctx->xz_cls.size()) return fail(ctx, SGSPM_ERR_ARG, "threads must have one entry per size class");
    for (int c = 0; c < n; ++c) {
        if (threads[c] != 32 && threads[c] != 64 && threads[c] != 128 && threads[c] != kThreads)
            return fail(ctx, SGSPM_ERR_ARG, "threads per packed CTA must be 32, 64, 128 or 256");
        if (threads[c] != kThreads && !packable_class(ctx->fp64, ctx->tf32x3, ctx->xz_cls[c].key))
            return fail(ctx, SGSPM_ERR_UNSUPPORTED, "this size class runs its own kernels only");
    }
    for (int c = 0; c < n; ++c) {
        int rc = set_class_rows(ctx, (size_t)c, ctx->xz_cls[c].rows, threads[c]);
        if (rc) return rc;
    }
    return SGSPM_OK;
}

int sgspm_autotune(sgspm_t ctx, int steps, int* rows_out, int cap) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (steps < 1) return fail(ctx, SGSPM_ERR_ARG, "steps must be >= 1");
    if (!ctx->have_m) return fail(ctx, SGSPM_ERR_STATE, "m has not been set");
    const int ncls = (int)ctx->xz_cls.size();
    if (rows_out && cap < ncls) return fail(ctx, SGSPM_ERR_ARG, "cap is below the number of size classes");
    // keep the state: m (hi and lo parts) and the step counters; restored at the end
    const size_t es = ctx->fp64 ? sizeof(double) : sizeof(float);
    const size_t fb = (size_t)ctx->ncell * es;
    void* keep = nullptr;
    CK(cudaMalloc(&keep, 6 * fb + sizeof(long long)));
    char* kp = (char*)keep;
    // every CUDA error below is recorded and the state restored before returning
    cudaError_t ce = cudaSuccess;
    auto ok = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && ce == cudaSuccess) {
            ce = e;
            ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
        }
        return e == cudaSuccess;
    };
    for (int i = 0; i < 3; ++i) {
        ok(cudaMemcpyAsync(kp + i * fb, ctx->d_field[M1 + i], fb, cudaMemcpyDeviceToDevice, ctx->stream), "autotune: save m");
        if (ctx->d_flo[M1 + i])
            ok(cudaMemcpyAsync(kp + (3 + i) * fb, ctx->d_flo[M1 + i], fb, cudaMemcpyDeviceToDevice, ctx->stream), "autotune: save m");
    }
    ok(cudaMemcpyAsync(kp + 6 * fb, ctx->d_step, sizeof(long long), cudaMemcpyDeviceToDevice, ctx->stream), "autotune: save step");
    const long long steps0 = ctx->steps;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ok(cudaEventCreate(&e0), "autotune: event");
    ok(cudaEventCreate(&e1), "autotune: event");
    int rc = ce == cudaSuccess ? SGSPM_OK : SGSPM_ERR_CUDA;
    for (int c = 0; c < ncls && !rc; ++c) {
        if (!packable_class(ctx->fp64, ctx->tf32x3, ctx->xz_cls[c].key)) continue;
        int maxny = 1;
        for (const Film& F : ctx->films)
            if (xz_class_key(ctx, F) == ctx->xz_cls[c].key) maxny = std::max(maxny, F.ny);
        float best = 1e30f;
        int best_rows = 1, best_th = kThreads;
        // 1, 2, 4, 8 rows per CTA with 256, 128, 64 or 32 threads (one row with 256: the class's
        // own kernels)
        for (int cand = 0; cand < 16 && !rc; ++cand) {
            const int r = 1 << (cand / 4), th = kThreads >> (cand % 4);
            if (r > kMaxRowsPerCTA || r > maxny) continue;
            if ((rc = set_class_rows(ctx, (size_t)c, r, th))) break;
            if ((rc = sgspm_step(ctx, 1))) break;   // captures the graph of this packing
            if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { rc = SGSPM_ERR_CUDA; break; }
            if ((rc = sgspm_step(ctx, steps))) break;
            if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = SGSPM_ERR_CUDA;
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_rows = r;
                best_th = th;
            }
        }
        if (!rc) rc = set_class_rows(ctx, (size_t)c, best_rows, best_th);
    }
    // y heat pass: x lines per CTA
    if (!rc) {
        int maxny = 1;
        for (const Film& F : ctx->films) maxny = std::max(maxny, F.ny);
        float best = 1e30f;
        int best_tx = ctx->tx_h, best_th = ctx->heat_threads;
        // even tiles only: every tile then pairs x lines (2i, 2i+1) the same way, so the choice
        // cannot change results
        for (int cand = 0; cand < 12 && !rc; ++cand) {
            const int tx = std::array<int, 6>{2, 4, 6, 8, 12, 16}[cand % 6], th = cand < 6 ? 256 : 128;
            const size_t sm = ctx->fp64 ? heat_smem<double>(maxny, tx) : heat_smem<float>(maxny, tx);
            if (sm > ctx->smem_max) continue;
            ctx->heat_threads = th;
            if ((rc = ctx->fp64 ? build_heat_classes<double>(ctx, tx) : build_heat_classes<float>(ctx, tx))) break;
            if ((rc = sgspm_step(ctx, 1))) break;
            if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { rc = SGSPM_ERR_CUDA; break; }
            if ((rc = sgspm_step(ctx, steps))) break;
            if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                rc = SGSPM_ERR_CUDA;
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_tx = tx;
                best_th = th;
            }
        }
        ctx->heat_threads = best_th;
        if (!rc) rc = ctx->fp64 ? build_heat_classes<double>(ctx, best_tx) : build_heat_classes<float>(ctx, best_tx);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int i = 0; i < 3; ++i) {
        ok(cudaMemcpyAsync(ctx->d_field[M1 + i], kp + i * fb, fb, cudaMemcpyDeviceToDevice, ctx->stream), "autotune: restore m");
        if (ctx->d_flo[M1 + i])
            ok(cudaMemcpyAsync(ctx->d_flo[M1 + i], kp + (3 + i) * fb, fb, cudaMemcpyDeviceToDevice, ctx->stream), "autotune: restore m");
    }
    ok(cudaMemcpyAsync(ctx->d_step, kp + 6 * fb, sizeof(long long), cudaMemcpyDeviceToDevice, ctx->stream), "autotune: restore step");
    ctx->steps = steps0;
    int rc2 = run_prog(ctx, ctx->fwd_prog, ctx->stream);   // spectra of the restored state
    ok(cudaStreamSynchronize(ctx->stream), "autotune: sync");
    cudaFree(keep);
    if (rc) return rc;
    if (rc2) return rc2;
    if (ce != cudaSuccess) return ce == cudaErrorMemoryAllocation ? SGSPM_ERR_OOM : SGSPM_ERR_CUDA;
    rc = check_status(ctx);
    if (rc) return rc;
    for (int c = 0; rows_out && c < ncls; ++c) rows_out[c] = ctx->xz_cls[c].rows;
    return ncls;
}

int sgspm_energy(sgspm_t ctx, double* out) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (!out) return fail(ctx, SGSPM_ERR_ARG, "out is NULL");
    if (!ctx->have_m) return fail(ctx, SGSPM_ERR_STATE, "m has not been set");
    if (ctx->stray) {
        int rc = run_prog(ctx, ctx->hs_prog, ctx->stream);
        if (rc) return rc;
    }
    if (ctx->fp64)
        energy_partial_kernel<double><<<ctx->n_e, kThreads, 0, ctx->stream>>>(dev_view<double>(ctx), ctx->d_work_e, M1, HS1,
                                                                              ctx->stray ? 1 : 0, ctx->d_epart);
    else
        energy_partial_kernel<float><<<ctx->n_e, kThreads, 0, ctx->stream>>>(dev_view<float>(ctx), ctx->d_work_e, M1, HS1,
                                                                             ctx->stray ? 1 : 0, ctx->d_epart);
    CK(cudaGetLastError());
    energy_final_kernel<<<(ctx->nfilm + 127) / 128, 128, 0, ctx->stream>>>(ctx->d_films, ctx->nfilm, ctx->d_first_e, ctx->d_epart,
                                                                           ctx->d_eout);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, ctx->d_eout, (size_t)5 * ctx->nfilm * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return check_status(ctx);
}

int sgspm_set_forcing(sgspm_t ctx, int kind) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (kind != SGSPM_FORCE_NONE && kind != SGSPM_FORCE_MMS_1D && kind != SGSPM_FORCE_MMS_3D)
        return fail(ctx, SGSPM_ERR_ARG, "unknown forcing kind");
    if (ctx->persist && kind != SGSPM_FORCE_NONE)
        return fail(ctx, SGSPM_ERR_UNSUPPORTED, "the persistent step has no manufactured forcing");
    CK(cudaStreamSynchronize(ctx->stream));
    for (Film& F : ctx->films) F.forcing = kind;
    ctx->forcing = kind != SGSPM_FORCE_NONE;
    for (Film& F : ctx->films) film_consts(F);
    CK(cudaMemcpy(ctx->d_films, ctx->films.data(), ctx->films.size() * sizeof(Film), cudaMemcpyHostToDevice));
    build_programs(ctx);
    drop_graph(ctx);
    return SGSPM_OK;
}

int sgspm_set_time(sgspm_t ctx, double t) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (!std::isfinite(t)) return fail(ctx, SGSPM_ERR_ARG, "t must be finite");
    CK(cudaStreamSynchronize(ctx->stream));
    for (Film& F : ctx->films) F.t0 = t;
    ctx->steps = 0;
    for (Film& F : ctx->films) film_consts(F);
    CK(cudaMemcpy(ctx->d_films, ctx->films.data(), ctx->films.size() * sizeof(Film), cudaMemcpyHostToDevice));
    CK(cudaMemset(ctx->d_step, 0, sizeof(long long)));
    return SGSPM_OK;
}

int sgspm_get_time(sgspm_t ctx, double* t) {
    if (!ctx || !t) return SGSPM_ERR_ARG;
    *t = ctx->films[0].t0 + (double)ctx->steps * ctx->films[0].dt;
    return SGSPM_OK;
}

int sgspm_sync(sgspm_t ctx) {
    if (!ctx) return SGSPM_ERR_ARG;
    return check_status(ctx);
}

int sgspm_profile_step(sgspm_t ctx, float* ms, int* kind, int cap) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (!ms || !kind || cap < (int)ctx->step_prog.size()) return fail(ctx, SGSPM_ERR_ARG, "profile buffers too small");
    if (!ctx->have_m) return fail(ctx, SGSPM_ERR_STATE, "m has not been set");
    const int n = (int)ctx->step_prog.size();
    std::vector<cudaEvent_t> ev(n + 1);
    for (auto& e : ev) CK(cudaEventCreate(&e));
    CK(cudaEventRecord(ev[0], ctx->stream));
    for (int i = 0; i < n; ++i) {
        int rc = enqueue(ctx, ctx->step_prog[i], ctx->stream);
        if (rc) return rc;
        CK(cudaEventRecord(ev[i + 1], ctx->stream));
    }
    CK(cudaEventSynchronize(ev[n]));
    for (int i = 0; i < n; ++i) {
        CK(cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]));
        const Launch& L = ctx->step_prog[i];
        kind[i] = L.kind * 10 + (L.kind == 0 ? (L.xz.n_rhs ? 1 : L.xz.op == 2 ? 3 : 2) : L.y.n);
    }
    for (auto& e : ev) cudaEventDestroy(e);
    ctx->steps += 1;
    return n;
}

static thread_local std::string g_noalloc_err;

int sgspm_energy_noalloc(const sgspm_grid* grid, double eps, double Q, const double easy_axis[3], const double he[3],
                         const void* m, const void* hs, int dtype, double* out, void* cuda_stream) {
    g_noalloc_err.clear();
    if (!grid || !easy_axis || !he || !m || !out) {
        g_noalloc_err = "grid, easy_axis, he, m and out must be non-NULL";
        return SGSPM_ERR_ARG;
    }
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->hx > 0 && grid->hy > 0 && grid->hz > 0)) {
        g_noalloc_err = "cell counts must be >= 1 and cell sizes > 0";
        return SGSPM_ERR_ARG;
    }
    if (dtype != SGSPM_F32 && dtype != SGSPM_F64_DATA) {
        g_noalloc_err = "dtype must be SGSPM_F32 or SGSPM_F64_DATA";
        return SGSPM_ERR_ARG;
    }
    const long long n = (long long)grid->nx * grid->ny * grid->nz;
    const long long nblocks = (n + kNoallocCellsPerBlock - 1) / kNoallocCellsPerBlock;
    if (nblocks > kNoallocMaxBlocks) {
        g_noalloc_err = "grid has " + std::to_string(n) + " cells; the allocation-free energy handles at most " +
                        std::to_string((long long)kNoallocMaxBlocks * kNoallocCellsPerBlock);
        return SGSPM_ERR_UNSUPPORTED;
    }
    double un = std::sqrt(easy_axis[0] * easy_axis[0] + easy_axis[1] * easy_axis[1] + easy_axis[2] * easy_axis[2]);
    if (!(un > 0) || !std::isfinite(un)) {
        g_noalloc_err = "easy axis must be a finite non-zero vector";
        return SGSPM_ERR_ARG;
    }
    double* part = noalloc_scratch(&g_noalloc_err);
    if (!part) return SGSPM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const double u0 = easy_axis[0] / un, u1 = easy_axis[1] / un, u2 = easy_axis[2] / un;
    if (dtype == SGSPM_F64_DATA)
        energy_noalloc_partial_kernel<double><<<(unsigned)nblocks, kThreads, 0, st>>>(
            (const double*)m, (const double*)hs, grid->nx, grid->ny, grid->nz, grid->hx, grid->hy, grid->hz, u0, u1, u2,
            he[0], he[1], he[2], part);
    else
        energy_noalloc_partial_kernel<float><<<(unsigned)nblocks, kThreads, 0, st>>>(
            (const float*)m, (const float*)hs, grid->nx, grid->ny, grid->nz, grid->hx, grid->hy, grid->hz, u0, u1, u2,
            he[0], he[1], he[2], part);
    energy_noalloc_final_kernel<<<1, 32, 0, st>>>(part, (int)nblocks, eps, Q, grid->hx * grid->hy * grid->hz, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("kernel launch: ") + cudaGetErrorString(e);
        return SGSPM_ERR_CUDA;
    }
    return SGSPM_OK;
}

const char* sgspm_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

int sgspm_record(sgspm_t ctx, long long nsteps, int K) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (nsteps < 1 || K < 1) return fail(ctx, SGSPM_ERR_ARG, "nsteps and K must be >= 1");
    if (!ctx->have_m) return fail(ctx, SGSPM_ERR_STATE, "m has not been set");
    if (ctx->forcing) return fail(ctx, SGSPM_ERR_UNSUPPORTED, "recording with a manufactured forcing is not supported");
    if (ctx->flags & (SGSPM_GSPM | SGSPM_FROZEN_STRAY))
        return fail(ctx, SGSPM_ERR_UNSUPPORTED, "the adjoint covers SGSPM with f refreshed at every state");
    if (K > nsteps) K = (int)nsteps;
    return ctx->fp64 ? record_t<double>(ctx, nsteps, K) : record_t<float>(ctx, nsteps, K);
}

int sgspm_grad(sgspm_t ctx, const void* dL_dmT, int dtype, void* dL_dhe, double* dL_dalpha) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (!dL_dmT || !dL_dhe || !dL_dalpha) return fail(ctx, SGSPM_ERR_ARG, "NULL argument");
    if (dtype != SGSPM_F32 && dtype != SGSPM_F64_DATA) return fail(ctx, SGSPM_ERR_ARG, "dtype must be SGSPM_F32 or SGSPM_F64_DATA");
    if (ctx->rec_nsteps < 1) return fail(ctx, SGSPM_ERR_STATE, "no recorded forward: call sgspm_record first");
    return ctx->fp64 ? grad_t<double>(ctx, dL_dmT, dtype, dL_dhe, dL_dalpha)
                     : grad_t<float>(ctx, dL_dmT, dtype, dL_dhe, dL_dalpha);
}


int sgspm_fp64_fma_peak(double* gflops) {
    if (!gflops) return SGSPM_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SGSPM_ERR_CUDA;
    const int blocks = nsm * 8, threads = 256, iters = 1 << 14;
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SGSPM_OK;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return SGSPM_ERR_OOM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SGSPM_ERR_CUDA;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && rc == SGSPM_OK; ++rep) {
        cudaEventRecord(e0, 0);
        fp64_fma_probe_kernel<<<blocks, threads>>>(iters, out);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = SGSPM_ERR_CUDA;
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;   // the first launch is a warm-up
    }
    if (rc == SGSPM_OK) *gflops = 2.0 * kFmaChains * (double)iters * blocks * threads / (best * 1e-3) / 1e9;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

int sgspm_test_tc_timeout(sgspm_t ctx, int skip_mma, int wait_limit) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (!ctx->d_tc_test) return fail(ctx, SGSPM_ERR_STATE, "the handle has no tensor-core transforms (TF32X3 form only)");
    if (wait_limit < 0) return fail(ctx, SGSPM_ERR_ARG, "wait_limit must be >= 0");
    const int v[2] = {skip_mma ? 1 : 0, wait_limit};
    CK(cudaMemcpyAsync(ctx->d_tc_test, v, sizeof(v), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return SGSPM_OK;
}

int sgspm_launches_per_step(sgspm_t ctx) {
    if (!ctx) return SGSPM_ERR_ARG;
    return ctx->persist ? 1 : (int)ctx->step_prog.size();
}

int sgspm_test_persist_wait(sgspm_t ctx, int withhold, long long wait_limit) {
    if (!ctx) return SGSPM_ERR_ARG;
    if (!ctx->persist) return fail(ctx, SGSPM_ERR_STATE, "the handle was not created with SGSPM_PERSISTENT");
    if (wait_limit <= 0) return fail(ctx, SGSPM_ERR_ARG, "wait_limit must be > 0");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->p_withhold = withhold;
    ctx->p_wait_limit = wait_limit;
    drop_graph(ctx);
    return SGSPM_OK;
}

}  // extern "C"
