// Shared device-side types of the SGSPM library: complex arithmetic, FFT plans,
// per-film descriptors and the per-pass programs that the host builds once.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sgspm {

template <typename T> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename T> using cplx = typename CplxOf<T>::type;

template <typename V> __device__ __forceinline__ V cmk(decltype(V::x) a, decltype(V::x) b) { V r; r.x = a; r.y = b; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) { return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename V> __device__ __forceinline__ V cconj(V a) { return cmk<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return cmk<V>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename V> __device__ __forceinline__ V cmul_mi(V a) { return cmk<V>(a.y, -a.x); }
template <typename V> __device__ __forceinline__ V cmul_pi(V a) { return cmk<V>(-a.y, a.x); }

// ---- twiddle factors ---------------------------------------------------------------------------
// A twiddle table entry.  FP64: the complex value.  FP32: the value split into hi = fl(w) and
// lo = fl(w - hi) (x, y = hi; z, w = lo), so that a multiplication by a table entry carries the
// table's own rounding (a fixed relative error of ~3e-8 per entry, identical in every time step,
// which would otherwise act like a perturbed operator and add up coherently over many steps)
// down to ~1e-15; only the rounding of the products themselves remains.
template <typename T> struct TwOf;
template <> struct TwOf<float> { using type = float4; };
template <> struct TwOf<double> { using type = double2; };
template <typename T> using tw_t = typename TwOf<T>::type;

__host__ __device__ __forceinline__ float4 tw_make(double re, double im, float*) {
    const float hr = (float)re, hi = (float)im;
    return make_float4(hr, hi, (float)(re - (double)hr), (float)(im - (double)hi));
}
__host__ __device__ __forceinline__ double2 tw_make(double re, double im, double*) { return make_double2(re, im); }

// a * w, or a * conj(w) when CONJ
template <bool CONJ = false>
__device__ __forceinline__ float2 twmul(float2 a, float4 w) {
    const float wy = CONJ ? -w.y : w.y, ww = CONJ ? -w.w : w.w;
    return make_float2(fmaf(a.x, w.x, fmaf(-a.y, wy, fmaf(a.x, w.z, -a.y * ww))),
                       fmaf(a.x, wy, fmaf(a.y, w.x, fmaf(a.x, ww, a.y * w.z))));
}
template <bool CONJ = false>
__device__ __forceinline__ double2 twmul(double2 a, double2 w) {
    return CONJ ? cmul(a, cconj(w)) : cmul(a, w);
}
// a * w (or a * conj(w)) with the full double-float twiddle when LO, else with its hi part only
template <bool CONJ, bool LO, typename V, typename W>
__device__ __forceinline__ V twmul_p(V a, W w) {
    if constexpr (LO) {
        return twmul<CONJ>(a, w);
    } else {
        const V h = cmk<V>(w.x, CONJ ? -w.y : w.y);
        return cmul(a, h);
    }
}
// the hi part of a twiddle as a plain complex number (for the few places that need one)
__device__ __forceinline__ float2 tw_hi(float4 w) { return make_float2(w.x, w.y); }
__device__ __forceinline__ double2 tw_hi(double2 w) { return w; }

// x * k for a constant k given in FP64: FP32 multiplies by fl(k) and adds x * fl(k - fl(k))
template <typename T> __device__ __forceinline__ T kmul(T x, double k);
template <> __device__ __forceinline__ double kmul<double>(double x, double k) { return x * k; }
template <> __device__ __forceinline__ float kmul<float>(float x, double k) {
    const float hi = (float)k, lo = (float)(k - (double)hi);
    return fmaf(x, hi, x * lo);
}
// a * (c + i s) for FP64 constants c, s
template <typename V> __device__ __forceinline__ V cmulk(V a, double c, double s) {
    using T = decltype(V::x);
    if constexpr (sizeof(T) == 8) {
        return cmk<V>(a.x * c - a.y * s, a.x * s + a.y * c);
    } else {
        const float ch = (float)c, cl = (float)(c - (double)ch), sh = (float)s, sl = (float)(s - (double)sh);
        return cmk<V>(fmaf(a.x, ch, fmaf(-a.y, sh, fmaf(a.x, cl, -a.y * sl))),
                      fmaf(a.x, sh, fmaf(a.y, ch, fmaf(a.x, sl, a.y * cl))));
    }
}

constexpr int kMaxStages = 16;
constexpr int kThreads = 256;

// Mixed-radix (8, 4, 2, 3, 5) Stockham plan of one transform length P.
// tw: offset of W_P^m = exp(-2 pi i m / P), m in [0, P), in the twiddle pool.
// tw4: offset of exp(-i pi k / (2P)), k in [0, P) (DCT post/pre twiddles).
struct Plan {
    int P;
    int nst;
    int radix[kMaxStages];
    int tw;
    int tw4;
    int dtab;   // offset of the dense DCT tables (P <= 16): C[k][n] then Ci[n][k]; -1 if none
};

// One film of a (possibly batched) handle.
struct Film {
    int nx, ny, nz;          // cells
    int Px, Py, Pz;          // zero-padded stray-field lengths (2n, or 1 for n = 1)
    int Kx;                  // Px/2 + 1 half-spectrum length along x
    int pad_;
    long long off_cell;      // offset into every real field pool
    long long off_spec;      // offset into every spectral pool: Kx * ny * Pz per film
    long long off_ycache;    // offset into the y-transform cache: Pz * Kx * Py per film
    long long off_ktab;      // kernel-table offset: 6 * (Pz/2+1) * (Py/2+1) * Kx
    int lam;                 // offset of lambda_x[nx], lambda_y[ny], lambda_z[nz] in the eigen pool
    int plan_dx, plan_dy, plan_dz;   // DCT lengths nx, ny, nz
    int plan_px, plan_py, plan_pz;   // padded lengths Px, Py, Pz
    int forcing;             // 0 none, 1 MMS 1D, 3 MMS 3D
    // plans whose twiddle offsets refer to the shared-memory staging layout of the passes:
    // slab pass [W_nx | W4_nx | W_nz | W4_nz | W_Px | W_Pz], heat line pass [W_ny | W4_ny]
    int splan_dx, splan_dz, splan_px, splan_pz, splan_dy;
    // global offsets of the same tables in the twiddle pool, and of the short-axis DCT table
    int gtw_dx, gtw4_dx, gtw_dz, gtw4_dz, gtw_px, gtw_pz, gtw_dy, gtw4_dy, gtw_py, gdtab_z;
    double hx, hy, hz;
    double eps, Q, alpha, dt;
    double u[3];
    double he[3];
    double t0;               // time at step counter 0
    // The same parameters for the FP32 form, split hi + lo (lo = fl(v - hi)) where the kernels
    // need the full double value, set on the host (film_consts) whenever a parameter changes:
    // the pass kernels then run no FP64 arithmetic, which is slow on this GPU.
    float fs_dt[2][2];       // [damp][hi, lo]: dt (Step 1), alpha dt (Step 2)
    float fs_c[2][2];        // [damp][hi, lo]: eps dt, alpha eps dt (heat-solve coefficient)
    float fs_eps[2];         // eps: hi, lo
    float fs_he[3][2];       // uniform applied field: hi, lo
    float fs_n[2];           // 1 / (nx ny nz): hi, lo
    float fs_Q;              // Q
    float fs_u[3];           // easy axis
    float fs_ih[3];          // 1 / h_a^2
    double ih2[3];           // 1 / h_a^2 (FP64)
};

// Fill the FP32 parameter fields of a film from its FP64 parameters (host).
inline void film_consts(Film& F) {
    auto split = [](double v, float* o) {
        o[0] = (float)v;
        o[1] = (float)(v - (double)o[0]);
    };
    split(F.dt, F.fs_dt[0]);
    split(F.alpha * F.dt, F.fs_dt[1]);
    split(F.eps * F.dt, F.fs_c[0]);
    split(F.alpha * F.eps * F.dt, F.fs_c[1]);
    split(F.eps, F.fs_eps);
    for (int a = 0; a < 3; ++a) split(F.he[a], F.fs_he[a]);
    split(1.0 / ((double)F.nx * F.ny * F.nz), F.fs_n);
    F.fs_Q = (float)F.Q;
    for (int a = 0; a < 3; ++a) F.fs_u[a] = (float)F.u[a];
    F.ih2[0] = 1.0 / (F.hx * F.hx);
    F.ih2[1] = 1.0 / (F.hy * F.hy);
    F.ih2[2] = 1.0 / (F.hz * F.hz);
    F.fs_ih[0] = (float)(1.0 / (F.hx * F.hx));
    F.fs_ih[1] = (float)(1.0 / (F.hy * F.hy));
    F.fs_ih[2] = (float)(1.0 / (F.hz * F.hz));
}

// Operand reference of a pointwise update: >= 0 real field slot, < 0 shared-memory slab (-1 - idx).
constexpr int kMaxSlots = 64;
constexpr int kMaxSpec = 12;

// Slab (XZ) pass program.  Phases run in order; unused phases have count 0 / op 0.
struct XZProg {
    // phase R: right-hand sides r_a = scale * (f_a + eps Delta_h m_a) and their forward DCT
    int n_rhs;
    int rhs_comp[3];       // component a of each rhs
    int rhs_h[3];          // spectral slot of H_a to invert for h_s,a (-1: no stray term)
    int rhs_out[3];        // real slot receiving DCT_xz(r_a)
    int rhs_hs_store[3];   // real slot receiving h_s,a (-1: none)
    int rhs_hs_add;        // 1: h_s,a is added to that slot instead of stored (adjoint accumulators)
    int state[3];          // real slots of the state (m1, m2, m3) at which f is evaluated
    int damp;              // 0: scale = dt; 1: scale = alpha dt
    int rhs_dct;           // 0: only invert h_s (energy), no rhs / DCT
    int rhs_copy[3];       // >= 0: the right-hand side is this slot as given (adjoint solves)
    // phase I: inverse DCT_xz of spectral-solved slots -> delta slabs in shared memory
    int n_inv;
    int inv_in[3];
    int inv_store[3];      // real slot receiving delta (-1: none)
    // phase U: pointwise update
    int op;                // 0 none, 1 Gauss-Seidel cross product, 2 damping + projection
    int gs_out, gs_base, gs_p, gs_q, gs_r, gs_s;   // out = base + p*q - r*s (operand refs)
    int fin_in[3];         // m** slots; delta slabs 0..2; m^{n+1} -> fin_out
    int fin_out[3];
    int fin_v[3];          // >= 0: also store m*** (before projection) here (recorded steps)
    // phase F: forward zero-padded FFT (x R2C, z C2C) of real fields -> spectral slots
    int n_fwd;
    int fwd_src[3];        // operand refs (slab -1-idx means the phase-U result slab idx)
    int fwd_dst[3];
};

// Line (Y) pass program.
struct YProg {
    int kind;              // 0 heat solve, 1 stray field
    int n;                 // heat: fields to solve; stray: outputs
    int slot[3];           // heat: real slots (in place); stray: output component a
    int damp;              // heat: 0 -> c = eps, 1 -> c = alpha eps
    int in_spec[3];        // stray: spectral slots of M_1, M_2, M_3
    int in_mask;           // stray: bit b set if input component b is non-zero (others skipped)
    int out_spec[3];       // stray: spectral slot of H_a for each output
    int fresh_mask;        // stray: bit b set: transform M_b along y (else read its cached transform)
    int store_mask;        // stray: bit b set: store the new y transform of M_b in the cache
};

// Gauss-Legendre rules on [-1, 1] used by the Newell set-up, packed: order q at off[q].
struct GLTable {
    double x[64];
    double w[64];
    int off[16];
};

// Device-side view of a handle (pointers valid on the device).
template <typename T>
struct Dev {
    const Film* films;
    const Plan* plans;
    const tw_t<T>* tw;     // twiddle pool (hi + lo parts in the FP32 form)
    const T* lam;          // eigenvalue pool
    const T* lam_lo;       // low parts of the eigenvalues (FP32 form), else null
    const T* dtab;         // dense DCT tables of short axes
    const T* ktab;         // -N_hat / (Px Py Pz), reduced real table
    T* const* field;       // device table: real field slot -> pool pointer
    T* const* flo;         // device table: low parts of double-float state slots (FP32 form), else null
    cplx<T>* const* spec;  // device table: spectral slot -> pool pointer
    const T* he_cell;      // per-cell applied field [3][ncell_total] or null
    cplx<T>* ycache;       // y transforms of M_1..3 (register order), component stride ycache_n
    long long ycache_n;
    int* status;
    const long long* step_ctr;
    // test support of the tensor-core form: [0] != 0 skips the MMA issue and commit (so that the
    // bounded completion wait runs out with nothing in flight), [1] > 0 replaces the wait's
    // iteration limit; null outside that form.  Only sgspm_test_tc_timeout writes it.
    const int* tc_test;
};

// ---- programmatic dependent launch ------------------------------------------------------------
// Every pass kernel lets the next launch start at once; that launch runs its set-up (work item,
// film record, twiddle staging: data no kernel writes) and then waits for this grid to finish.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- asynchronous global -> shared copies (cp.async; completion per thread by commit group) ----
__device__ __forceinline__ void cp_async_8(void* sdst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc) {
    static_assert(BYTES == 8 || BYTES == 16, "cp.async piece of 8 or 16 bytes");
    if constexpr (BYTES == 8) cp_async_8(sdst, gsrc);
    else cp_async_16(sdst, gsrc);
}
__device__ __forceinline__ void cp_async_4(void* sdst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
}
// The whole CTA copies n elements of 4, 8 or 16 bytes from global to shared memory with
// asynchronous copies (all in flight together; the caller commits and waits)
template <typename E>
__device__ __forceinline__ void stage_async(E* sdst, const E* gsrc, int n) {
    static_assert(sizeof(E) == 4 || sizeof(E) == 8 || sizeof(E) == 16, "element of 4, 8 or 16 bytes");
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        if constexpr (sizeof(E) == 16) cp_async_16(sdst + i, gsrc + i);
        else if constexpr (sizeof(E) == 8) cp_async_8(sdst + i, gsrc + i);
        else cp_async_4(sdst + i, gsrc + i);
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most `pending` (0, 1 or 2) of this thread's committed groups are still in flight
__device__ __forceinline__ void cp_async_wait(int pending) {
    if (pending >= 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else if (pending == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---- error-free transformations (FP32 double-float arithmetic of the state) -----------------
// Knuth's two-sum, Dekker's fast two-sum and the FMA two-product.
template <typename T> __device__ __forceinline__ void two_sum(T a, T b, T& s, T& e) {
    s = a + b;
    T bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
template <typename T> __device__ __forceinline__ void fast_two_sum(T a, T b, T& s, T& e) {
    s = a + b;
    e = b - (s - a);
}
template <typename T> __device__ __forceinline__ void two_prod(T a, T b, T& p, T& e) {
    p = a * b;
    e = fma(a, b, -p);
}

}  // namespace sgspm
