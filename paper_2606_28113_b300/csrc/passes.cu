// XZ slab pass and Y line passes (FP32 and FP64).  Included by the kernel translation units
// (k_*.cu), which instantiate each size class once.
#pragma once
#include "passes.cuh"

// Global reads of fields that a pass does not write are marked restrict (read-only path) in the
// per-pass kernels.  The persistent ensemble kernel runs every pass inside one launch, where a
// field read in one pass is written in another: its translation unit defines SGSPM_FIELD_RO empty.
#ifndef SGSPM_FIELD_RO
#define SGSPM_FIELD_RO __restrict__
#endif

namespace sgspm {

template <typename T>
__device__ __forceinline__ T load_ref(const Dev<T>& d, int ref, long long cell, const T* slabs, int slabsz, int sidx) {
    return ref >= 0 ? d.field[ref][cell] : slabs[(-1 - ref) * slabsz + sidx];
}

// Manufactured forcing f_e(x, t) of Sec. 5.1 (exact Laplacian of m_e), component a.
__device__ inline void mms_forcing(int dim, double x, double y, double z, double t, double alpha, double fe[3]) {
    auto X = [](double s) { return s * s * (1 - s) * (1 - s); };
    auto dX = [](double s) { return 2 * s * (1 - s) * (1 - 2 * s); };
    auto d2X = [](double s) { return 2 * (1 - 6 * s + 6 * s * s); };
    double phi, g2, lp;
    if (dim == 1) {
        phi = X(x);
        g2 = dX(x) * dX(x);
        lp = d2X(x);
    } else {
        double a = X(x), b = X(y), c = X(z);
        double da = dX(x), db = dX(y), dc = dX(z);
        phi = a * b * c;
        g2 = (da * b * c) * (da * b * c) + (a * db * c) * (a * db * c) + (a * b * dc) * (a * b * dc);
        lp = d2X(x) * b * c + a * d2X(y) * c + a * b * d2X(z);
    }
    double cp = cos(phi), sp = sin(phi), st = sin(t), ct = cos(t);
    double me[3] = {cp * st, sp * st, ct};
    double dtm[3] = {cp * ct, sp * ct, -st};
    double L[3] = {(-sp * lp - cp * g2) * st, (cp * lp - sp * g2) * st, 0.0};
    double mxl[3] = {me[1] * L[2] - me[2] * L[1], me[2] * L[0] - me[0] * L[2], me[0] * L[1] - me[1] * L[0]};
    double mmxl[3] = {me[1] * mxl[2] - me[2] * mxl[1], me[2] * mxl[0] - me[0] * mxl[2], me[0] * mxl[1] - me[1] * mxl[0]};
    for (int i = 0; i < 3; ++i) fe[i] = dtm[i] + mxl[i] + alpha * mmxl[i];
}

// Length-P DFT of a column held in registers (P a power of two <= 2 kZReg); false otherwise.
template <typename T, bool INV>
__device__ __forceinline__ bool zfft_reg(cplx<T> (&v)[2 * kZReg], int P) {
    using V = cplx<T>;
    switch (P) {
        case 16: Bfly<16, INV, V>::run(v); return true;
        case 8: Bfly<8, INV, V>::run(v); return true;
        case 4: Bfly<4, INV, V>::run(v); return true;
        case 2: Bfly<2, INV, V>::run(v); return true;
        case 1: return true;
        default: return false;
    }
}

// m^{n+1} = m*** / |m***| for a double-float m*** = h + l (Step 3): |m***|^2 in double-float, its
// inverse square root by one double-float Newton step from rsqrt.  Returns false (and the
// unnormalised m***) if |m***| is zero or not finite.
template <typename T>
__device__ __forceinline__ bool project_df(const T (&h)[3], const T (&l)[3], T (&oh)[3], T (&ol)[3]) {
    T p0, e0, p1, e1, p2, e2;
    two_prod(h[0], h[0], p0, e0);
    two_prod(h[1], h[1], p1, e1);
    two_prod(h[2], h[2], p2, e2);
    T s1, f1, n2h, f2;
    two_sum(p0, p1, s1, f1);
    two_sum(s1, p2, n2h, f2);
    T n2l = f1 + f2 + e0 + e1 + e2 + T(2) * (h[0] * l[0] + h[1] * l[1] + h[2] * l[2]);
    T nh, nl;
    fast_two_sum(n2h, n2l, nh, nl);
    bool ok = true;
    if (!(nh > T(0)) || !isfinite(nh)) {
        ok = false;
        nh = T(1);
        nl = T(0);
    }
    const T r0 = rsqrt(nh);
    T q, qe, a, ae;
    two_prod(r0, r0, q, qe);
    two_prod(nh, q, a, ae);
    const T rho = ((T(1) - a) - ae) - (nh * qe + nl * q);
    const T cc = T(0.5) * r0 * rho;   // 1/|m***| = r0 + cc
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T pp, pe;
        two_prod(h[i], r0, pp, pe);
        fast_two_sum(pp, pe + (h[i] * cc + l[i] * r0), oh[i], ol[i]);
    }
    return ok;
}

// ---- four-cell row access (compile-time x lengths, FP32) ------------------------------------
// A slab is nz lines of NX cells: in shared memory with line stride NX, in a field at row base
// g (the film's cell offset plus y nx, 16-byte aligned: films of these size classes start at
// pool offsets that are multiples of four) with line stride zs.  Each access moves four cells.
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

template <int NX>
__device__ __forceinline__ void slab_load4(float* s, const float* SGSPM_FIELD_RO g, int nz, int zs) {
    constexpr int N4 = NX / 4;
    for (int i = threadIdx.x; i < nz * N4; i += blockDim.x) {
        const int z = i / N4, x4 = i - z * N4;
        st4(s + 4 * i, ld4(g + z * zs + 4 * x4));
    }
}
template <int NX>
__device__ __forceinline__ void slab_store4(float* __restrict__ g, const float* s, int nz, int zs) {
    constexpr int N4 = NX / 4;
    for (int i = threadIdx.x; i < nz * N4; i += blockDim.x) {
        const int z = i / N4, x4 = i - z * N4;
        st4(g + z * zs + 4 * x4, ld4(s + 4 * i));
    }
}

// ------------------------------------------------------------------------------------------
// XZ slab pass
// ------------------------------------------------------------------------------------------
// NX: compile-time x length of the films this launch covers (0: any length, runtime transforms)
// ZTC: TF32X3 form (FP32 only): the z transforms of films with tc_zdct_ok run on the tensor cores
// MULTI: a work item covers rows y0 .. y0 + w - 1 of one film (packing of small slabs); the
//        single-row kernels keep the loop at one compile-time trip
// MODE: 0 runs whatever the program asks for; 1 (right-hand sides), 2 (Gauss-Seidel update) and
//       3 (damping update and projection) compile only the phases of that launch type, so that a
//       launch fetches and caches far less code (the generic kernel's instruction stream is its
//       largest stall)
// One work item of the slab pass (a y row, or rows y0 .. y0 + w - 1 with MULTI) of film wi.x, run
// by the whole CTA (kThreads threads; dynamic shared memory as laid out by xz_layout).
template <typename T, int NX, bool ZTC = false, bool MULTI = false, int MODE = 0>
__device__ __forceinline__ void xz_item(const Dev<T> d, const int4 wi, const XZProg& pg, int stray) {
    using V = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Film F = d.films[wi.x];
    const int y0 = wi.y, nrow = MULTI ? (wi.z > 0 ? wi.z : 1) : 1;
    // compile-time x lengths (NX >= 8) fold every index division by nx into a shift
    // the 512-thread kernels run films with nz = kZReg only (the host dispatches others elsewhere)
    constexpr bool kPairK = xz_nt<NX, MODE, MULTI, ZTC>() == 2 * kThreads;
    const int nx = NX > 0 ? NX : F.nx, ny = F.ny, nz = kPairK ? kZReg : F.nz;
    const int Px = NX > 0 ? 2 * NX : F.Px, Pz = kPairK ? 2 * kZReg : F.Pz, Kx = NX > 0 ? NX + 1 : F.Kx;
    const XZLayout Lo = xz_layout(nx, nz, Px, Pz, Kx, stray != 0, ZTC);
    // the zero-padded x transform (Px = 2 NX) as two NX-point FFTs per line pair
    constexpr bool kHalfX = NX >= 64 && NX <= 512;
    // four-cell loads and stores of the pointwise phases (FP32, compile-time x length)
    constexpr bool kVec = NX >= 8 && sizeof(T) == 4;
    // lane pairs share each column's register z transforms (512-thread kernels): the padded DFTs
    // split into even and odd kz (two 8-point transforms), the dense DCTs into halves of the outputs
    constexpr bool kPair = kPairK;
    const int pr = threadIdx.x & 1;   // lane of the pair
    __shared__ Plan pdx, pdz, ppx, ppz;
    if (threadIdx.x == 0) {
        // pre-staged plan copies (their twiddle offsets refer to the shared layout below)
        pdx = d.plans[F.splan_dx];
        pdz = d.plans[F.splan_dz];
        ppx = d.plans[F.splan_px];
        ppz = d.plans[F.splan_pz];
    }
    // staged twiddles: [W_nx | W4_nx | W_nz | W4_nz | W_Px | W_Pz], then the short-axis DCT tables
    tw_t<T>* stw = reinterpret_cast<tw_t<T>*>(smem_raw);
    {
        const int segs[6] = {F.gtw_dx, F.gtw4_dx, F.gtw_dz, F.gtw4_dz, F.gtw_px, F.gtw_pz};
        const int lens[6] = {nx, nx, nz, nz, stray ? Px : 0, stray ? Pz : 0};
        int off = 0;
        for (int k = 0; k < 6; ++k) {
            stage_async(stw + off, d.tw + segs[k], lens[k]);
            off += lens[k];
        }
    }
    V* xw0 = reinterpret_cast<V*>(stw + Lo.tw);
    V* xw1 = xw0 + Lo.xw;
    V* zw0 = xw1 + Lo.xw;
    V* zw1 = zw0 + Lo.zw;
    T* slabs = reinterpret_cast<T*>(zw1 + Lo.zw);
    T* sdt = slabs + 3 * Lo.slab;
    if (Lo.dt) stage_async(sdt, d.dtab + F.gdtab_z, 2 * nz * nz);
    cp_async_commit();
    cp_async_wait(0);
    __syncthreads();
    // TF32X3 form: B operands (forward hi, lo; inverse hi, lo) after the DCT tables, tensor memory
    const bool tcz = ZTC && tc_zdct_ok(nx, nz);
    unsigned char* tcb =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sdt + Lo.dt) + 15) & ~(uintptr_t)15);
    __shared__ uint64_t tc_bar;
    __shared__ uint32_t tc_slot;
    TcState tcs{};
    if constexpr (ZTC) {
        if (tcz) {
            tc_write_b(sdt, nz, tcb, tcb + kTcBBytes);
            tc_write_b(sdt + nz * nz, nz, tcb + 2 * kTcBBytes, tcb + 3 * kTcBBytes);
        }
        tc_setup(tcs, &tc_slot, &tc_bar, tc_tmem_cols(NX));
    }
    pdl_wait();   // everything above reads constant data; fields of the previous pass from here on
    for (int y = y0; y < y0 + nrow; ++y) {
        const int S = Lo.slab;
        const int KC = Lo.kc;
        const int npx = (nz + 1) / 2;
        const int nxz = nx * nz;
        // in-film offsets are 32-bit; the film's base offsets are 64-bit
        const long long cbase = F.off_cell + (long long)y * nx;
        const long long sbase = F.off_spec;
        const int zstride = ny * nx;
        auto cell_of = [&](int z, int x) -> long long { return cbase + (z * zstride + x); };
        auto spec_of = [&](int kz, int kx) -> int { return (kz * ny + y) * Kx + kx; };
        // slab <-> field row copies
        auto load_slab = [&](T* sl, const T* SGSPM_FIELD_RO f) {
            if constexpr (kVec) {
                slab_load4<NX>(sl, f + cbase, nz, zstride);
            } else {
                for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                    const int z = idx / nx, x = idx - z * nx;
                    sl[idx] = f[cell_of(z, x)];
                }
            }
        };
        auto store_slab = [&](T* __restrict__ f, const T* sl) {
            if constexpr (kVec) {
                slab_store4<NX>(f + cbase, sl, nz, zstride);
            } else {
                for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                    const int z = idx / nx, x = idx - z * nx;
                    f[cell_of(z, x)] = sl[idx];
                }
            }
        };
        auto add_slab = [&](T* __restrict__ f, const T* sl) {   // f += slab (each cell once)
            for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                const int z = idx / nx, x = idx - z * nx;
                f[cell_of(z, x)] += sl[idx];
            }
        };
        const bool zreg = z_in_registers(nz);
        const T* Cz = sdt;                                       // DCT-II  C[k][n]
        const T* Czi = sdt + nz * nz;                            // inverse Ci[n][k]
        const tw_t<T>* twz = stw + ppz.tw;                       // W_Pz^m

        // ---- phase R: right-hand sides and forward DCT ---------------------------------------
        for (int ci = 0; (MODE == 0 || MODE == 1) && ci < pg.n_rhs; ++ci) {
            const int a = pg.rhs_comp[ci];
            T* h = slabs;   // slab 0
            if (MODE == 0 && pg.rhs_copy[ci] >= 0) {
                // the right-hand side is given (adjoint solves): copy it and transform
                load_slab(h, d.field[pg.rhs_copy[ci]]);
                __syncthreads();
            } else if (pg.rhs_h[ci] >= 0 && stray) {
                const V* H = d.spec[pg.rhs_h[ci]] + sbase;
                if (kPair && nz == 8) {
                    // inverse zero-padded DFT along z (Pz = 16), one lane pair per kx column: lane r
                    // transforms the inputs kz = 2j + r (lane 1 then multiplies by W16^-z), the pair
                    // swaps halves, and lane r keeps the outputs z = 4r .. 4r + 3
                    for (int base = 0; base < Kx; base += (int)blockDim.x / 2) {
                        if (base + ((int)threadIdx.x & ~31) / 2 >= Kx) continue;   // whole warp idle
                        const int kx = base + ((int)threadIdx.x >> 1);
                        const bool act = kx < Kx;
                        V v[8];
    #pragma unroll
                        for (int j = 0; j < 8; ++j) v[j] = act ? H[spec_of(2 * j + pr, kx)] : cmk<V>(T(0), T(0));
                        Bfly<8, true, V>::run(v);
                        if (pr) {
    #pragma unroll
                            for (int z = 1; z < 8; ++z) v[z] = twmul<true>(v[z], twz[z]);
                        }
                        V acc[4];
    #pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const V snd = pr ? v[i] : v[4 + i];   // the half the partner keeps
                            V rcv;
                            rcv.x = __shfl_xor_sync(0xffffffffu, snd.x, 1);
                            rcv.y = __shfl_xor_sync(0xffffffffu, snd.y, 1);
                            acc[i] = pr ? cadd(rcv, v[4 + i]) : cadd(v[i], rcv);
                        }
                        if (act) {
    #pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                const int p = 2 * pr + q;
                                if constexpr (kHalfX) c2r_put_h<T>(xw0, p, kx, Px, acc[2 * q], acc[2 * q + 1]);
                                else c2r_put<T>(xw0, p, kx, Px, acc[2 * q], acc[2 * q + 1]);
                            }
                        }
                    }
                    __syncthreads();
                } else if (zreg) {
                    // inverse zero-padded DFT along z in registers, one thread per kx column
                    for (int kx = threadIdx.x; kx < Kx; kx += blockDim.x) {
                        V acc[kZReg];
    #pragma unroll
                        for (int z = 0; z < kZReg; ++z) acc[z] = cmk<V>(T(0), T(0));
                        V hz[2 * kZReg];
    #pragma unroll
                        for (int kz = 0; kz < 2 * kZReg; ++kz)
                            hz[kz] = kz < Pz ? H[spec_of(kz, kx)] : cmk<V>(T(0), T(0));
                        if (zfft_reg<T, true>(hz, Pz)) {
    #pragma unroll
                            for (int z = 0; z < kZReg; ++z) acc[z] = hz[z];
                        } else {
    #pragma unroll
                            for (int kz = 0; kz < 2 * kZReg; ++kz) {
                                if (kz >= Pz) break;
                                const V hv = hz[kz];
                                int m = 0;
    #pragma unroll
                                for (int z = 0; z < kZReg; ++z) {
                                    if (z < nz) acc[z] = cadd(acc[z], twmul<true>(hv, twz[m]));
                                    m += kz;
                                    if (m >= Pz) m -= Pz;
                                }
                            }
                        }
    #pragma unroll
                        for (int p = 0; p < kZReg / 2; ++p)
                            if (2 * p < nz) {
                                const V xb = (2 * p + 1 < nz) ? acc[2 * p + 1] : cmk<V>(T(0), T(0));
                                if constexpr (kHalfX) c2r_put_h<T>(xw0, p, kx, Px, acc[2 * p], xb);
                                else c2r_put<T>(xw0, p, kx, Px, acc[2 * p], xb);
                            }
                    }
                    __syncthreads();
                }
                for (int kc0 = 0; !zreg && kc0 < Kx; kc0 += KC) {
                    const int kcn = min(KC, Kx - kc0);
                    for (int idx = threadIdx.x; idx < Pz * kcn; idx += blockDim.x) {
                        int kz = idx / kcn, kc = idx - kz * kcn;
                        zw0[kz * KC + kc] = H[spec_of(kz, kc0 + kc)];
                    }
                    __syncthreads();
                    V* r = fft_lines<T, true>(zw0, zw1, Lines{kcn, 1, KC}, ppz, stw);
                    for (int idx = threadIdx.x; idx < npx * kcn; idx += blockDim.x) {
                        int p = idx / kcn, kc = idx - p * kcn;
                        V xa = r[(2 * p) * KC + kc];
                        V xb = (2 * p + 1 < nz) ? r[(2 * p + 1) * KC + kc] : cmk<V>(T(0), T(0));
                        if constexpr (kHalfX) c2r_put_h<T>(xw0, p, kc0 + kc, Px, xa, xb);
                        else c2r_put<T>(xw0, p, kc0 + kc, Px, xa, xb);
                    }
                    __syncthreads();
                }
                if constexpr (kHalfX) {
                    // two NX-point inverse FFTs per pair; outputs n < nx only
                    const tw_t<T>* twP = stw + ppx.tw;
                    V* r = fft_lines_t<T, true, NX>(xw0, xw1, Lines{2 * npx, NX, 1}, pdx, stw);
                    for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                        int z = idx / nx, x = idx - z * nx;
                        const int p = z >> 1;
                        const V v = cadd(r[(2 * p) * NX + x], twmul<true>(r[(2 * p + 1) * NX + x], twP[x]));
                        h[idx] = (z & 1) ? v.y : v.x;
                    }
                } else {
                    V* r = fft_lines_t<T, true, 2 * NX>(xw0, xw1, Lines{npx, Px, 1}, ppx, stw);
                    for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                        int z = idx / nx, x = idx - z * nx;
                        V v = r[(z >> 1) * Px + x];
                        h[idx] = (z & 1) ? v.y : v.x;
                    }
                }
            } else {
                for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) h[idx] = T(0);
            }
            __syncthreads();
            if (MODE == 0 && pg.rhs_hs_store[ci] >= 0) {
                if (pg.rhs_hs_add) add_slab(d.field[pg.rhs_hs_store[ci]], h);
                else store_slab(d.field[pg.rhs_hs_store[ci]], h);
            }
            if (MODE == 0 && !pg.rhs_dct) { __syncthreads(); continue; }
            // r_a = scale * (f_a + eps Delta_h m_a),  f_a = -Q (m_a - (m.u) u_a) + h_s,a + h_e,a
            if (MODE != 0 || pg.rhs_copy[ci] < 0) {
                const T* SGSPM_FIELD_RO m1 = d.field[pg.state[0]];
                const T* SGSPM_FIELD_RO m2 = d.field[pg.state[1]];
                const T* SGSPM_FIELD_RO m3 = d.field[pg.state[2]];
                const T* SGSPM_FIELD_RO ma = d.field[pg.state[a]];
                // dt (alpha dt), eps and the uniform applied field are split hi + lo in the FP32
                // form: they set the precession rate in every step, so their FP32 rounding would
                // act as a fixed perturbation of the parameters (lo parts are zero in FP64)
                T sch, scl, eph, epl, Q, ux, uy, uz, ua, ihx, ihy, ihz, hea, heal;
                if constexpr (sizeof(T) == 4) {
                    // precomputed on the host: no FP64 arithmetic in the FP32 kernels
                    const int dm = pg.damp ? 1 : 0;
                    sch = F.fs_dt[dm][0];
                    scl = F.fs_dt[dm][1];
                    eph = F.fs_eps[0];
                    epl = F.fs_eps[1];
                    Q = F.fs_Q;
                    ux = F.fs_u[0];
                    uy = F.fs_u[1];
                    uz = F.fs_u[2];
                    ua = F.fs_u[a];
                    ihx = F.fs_ih[0];
                    ihy = F.fs_ih[1];
                    ihz = F.fs_ih[2];
                    hea = F.fs_he[a][0];
                    heal = F.fs_he[a][1];
                } else {
                    sch = pg.damp ? F.alpha * F.dt : F.dt;
                    scl = T(0);
                    eph = F.eps;
                    epl = T(0);
                    Q = F.Q;
                    ux = F.u[0];
                    uy = F.u[1];
                    uz = F.u[2];
                    ua = F.u[a];
                    ihx = 1.0 / (F.hx * F.hx);
                    ihy = 1.0 / (F.hy * F.hy);
                    ihz = 1.0 / (F.hz * F.hz);
                    hea = F.he[a];
                    heal = T(0);
                }
                const int sz = nx * ny;
                if constexpr (kVec) {
                    // four consecutive x cells per thread: the state, the y and z neighbour rows as
                    // float4, the two outer x neighbours as scalars (mirror ghosts at the ends)
                    constexpr int N4 = NX / 4;
                    const T* r1 = m1 + cbase;
                    const T* r2 = m2 + cbase;
                    const T* r3 = m3 + cbase;
                    const T* ra = ma + cbase;
                    for (int i = threadIdx.x; i < nz * N4; i += blockDim.x) {
                        const int z = i / N4, x4 = i - z * N4;
                        const int o = z * zstride + 4 * x4;
                        const float4 A1 = ld4(r1 + o), A2 = ld4(r2 + o), A3 = ld4(r3 + o);
                        const float4 C = a == 0 ? A1 : (a == 1 ? A2 : A3);
                        const float4 YP = y + 1 < ny ? ld4(ra + o + nx) : C;
                        const float4 YM = y > 0 ? ld4(ra + o - nx) : C;
                        const float4 ZP = z + 1 < nz ? ld4(ra + o + zstride) : C;
                        const float4 ZM = z > 0 ? ld4(ra + o - zstride) : C;
                        const float XM = x4 > 0 ? ra[o - 1] : C.x;
                        const float XP = x4 + 1 < N4 ? ra[o + 4] : C.w;
                        const float4 HV = ld4(h + 4 * i);
                        const float a1[4] = {A1.x, A1.y, A1.z, A1.w}, a2[4] = {A2.x, A2.y, A2.z, A2.w};
                        const float a3[4] = {A3.x, A3.y, A3.z, A3.w}, cc[4] = {C.x, C.y, C.z, C.w};
                        const float yp[4] = {YP.x, YP.y, YP.z, YP.w}, ym[4] = {YM.x, YM.y, YM.z, YM.w};
                        const float zp[4] = {ZP.x, ZP.y, ZP.z, ZP.w}, zm[4] = {ZM.x, ZM.y, ZM.z, ZM.w};
                        const float hv[4] = {HV.x, HV.y, HV.z, HV.w};
                        float rr[4];
    #pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float c0 = cc[k];
                            const float xl = k > 0 ? cc[k - 1] : XM, xr = k < 3 ? cc[k + 1] : XP;
                            const float lap = ihx * ((xr - c0) + (xl - c0)) + ihy * ((yp[k] - c0) + (ym[k] - c0)) +
                                              ihz * ((zp[k] - c0) + (zm[k] - c0));
                            const float mu = a1[k] * ux + a2[k] * uy + a3[k] * uz;
                            const float he = d.he_cell ? d.he_cell[(cbase + o + k) * 3 + a] : hea;
                            const float hel = d.he_cell ? 0.f : heal;
                            const float f = -Q * (c0 - mu * ua) + hv[k] + he;
                            const float xx = f + fmaf(eph, lap, fmaf(epl, lap, hel));
                            rr[k] = fmaf(sch, xx, scl * xx);
                        }
                        st4(h + 4 * i, make_float4(rr[0], rr[1], rr[2], rr[3]));
                    }
                }
                // batches of kB cells per thread: every load of the batch is issued before any use
                constexpr int kB = sizeof(T) == 4 ? 4 : 2;
                for (int i0 = threadIdx.x; !kVec && i0 < nxz; i0 += kB * blockDim.x) {
                    // the stencil reads the hi part of a double-float state: its neighbour differences are
                    // O(h^2 |Delta m|) and the lo parts change them below the FP32 operator rounding
                    T v1[kB], v2[kB], v3[kB], mc[kB], nb[kB][6];
    #pragma unroll
                    for (int u = 0; u < kB; ++u) {
                        const int idx = i0 + u * blockDim.x;
                        if (idx >= nxz) break;
                        const int z = idx / nx, x = idx - z * nx;
                        const long long c = cell_of(z, x);
                        v1[u] = m1[c];
                        v2[u] = m2[c];
                        v3[u] = m3[c];
                        mc[u] = ma[c];
                        // neighbours with mirror ghosts (a missing neighbour repeats the cell)
                        const int o[6] = {x + 1 < nx ? 1 : 0, x > 0 ? -1 : 0, y + 1 < ny ? nx : 0,
                                          y > 0 ? -nx : 0, z + 1 < nz ? sz : 0, z > 0 ? -sz : 0};
    #pragma unroll
                        for (int k = 0; k < 6; ++k) nb[u][k] = ma[c + o[k]];
                    }
    #pragma unroll
                    for (int u = 0; u < kB; ++u) {
                        const int idx = i0 + u * blockDim.x;
                        if (idx >= nxz) break;
                        const long long c = cell_of(idx / nx, idx - (idx / nx) * nx);
                        const T mu = v1[u] * ux + v2[u] * uy + v3[u] * uz;
                        T d6[6];
    #pragma unroll
                        for (int k = 0; k < 6; ++k) d6[k] = nb[u][k] - mc[u];
                        const T lap = ihx * (d6[0] + d6[1]) + ihy * (d6[2] + d6[3]) + ihz * (d6[4] + d6[5]);
                        const T he = d.he_cell ? d.he_cell[c * 3 + a] : hea;
                        const T hel = d.he_cell ? T(0) : heal;
                        const T f = -Q * (mc[u] - mu * ua) + h[idx] + he;
                        if constexpr (sizeof(T) == 8) {
                            h[idx] = sch * (f + eph * lap);
                        } else {
                            const T x = f + fma(eph, lap, fma(epl, lap, hel));
                            h[idx] = fma(sch, x, scl * x);
                        }
                    }
                }
            }
            __syncthreads();
            dct2_lines<T, NX>(h, Lines{nz, nx, 1}, nx, xw0, xw1, pdx, stw);
            bool zdone = false;
            if constexpr (ZTC) {
                if (tcz) {
                    tc_zdct(h, nx, nz, reinterpret_cast<unsigned char*>(xw0), tcb, tcb + kTcBBytes, tcs, d.status, d.tc_test);
                    zdone = true;
                }
            }
            if (zdone) {
            } else if (kPair && zreg) {
                // lane pairs per x column: lane r computes the outputs k = r kh .. of the column
                const int kh = (nz + 1) / 2;
                for (int x = (int)threadIdx.x >> 1; x < nx; x += (int)blockDim.x / 2) {
                    T v[kZReg];
    #pragma unroll
                    for (int z = 0; z < kZReg; ++z) v[z] = z < nz ? h[z * nx + x] : T(0);
                    __syncwarp();
    #pragma unroll
                    for (int kk = 0; kk < kZReg / 2; ++kk) {
                        const int k = pr * kh + kk;
                        if (kk >= kh || k >= nz) break;
                        T acc = T(0);
    #pragma unroll
                        for (int z = 0; z < kZReg; ++z)
                            if (z < nz) acc += Cz[k * nz + z] * v[z];
                        h[k * nx + x] = acc;
                    }
                }
                __syncthreads();
            } else if (zreg) {
                for (int x = threadIdx.x; x < nx; x += blockDim.x) {
                    T v[kZReg];
    #pragma unroll
                    for (int z = 0; z < kZReg; ++z) v[z] = z < nz ? h[z * nx + x] : T(0);
    #pragma unroll
                    for (int k = 0; k < kZReg; ++k) {
                        if (k >= nz) break;
                        T acc = T(0);
    #pragma unroll
                        for (int z = 0; z < kZReg; ++z)
                            if (z < nz) acc += Cz[k * nz + z] * v[z];
                        h[k * nx + x] = acc;
                    }
                }
                __syncthreads();
            } else {
                dct2_lines<T>(h, Lines{nx, 1, nx}, nz, xw0, xw1, pdz, stw);
            }
            store_slab(d.field[pg.rhs_out[ci]], h);
            __syncthreads();
        }

        // ---- phase I: inverse DCT of solved spectra -> delta slabs ------------------------------
        for (int i = 0; MODE != 1 && i < pg.n_inv; ++i) {
            T* s = slabs + i * S;
            load_slab(s, d.field[pg.inv_in[i]]);
            __syncthreads();
            bool zdone = false;
            if constexpr (ZTC) {
                if (tcz) {
                    tc_zdct(s, nx, nz, reinterpret_cast<unsigned char*>(xw0), tcb + 2 * kTcBBytes, tcb + 3 * kTcBBytes, tcs,
                            d.status, d.tc_test);
                    zdone = true;
                }
            }
            if (zdone) {
            } else if (kPair && zreg) {
                // lane pairs per x column: lane r computes the outputs z = r kh .. of the column
                const int kh = (nz + 1) / 2;
                for (int x = (int)threadIdx.x >> 1; x < nx; x += (int)blockDim.x / 2) {
                    T v[kZReg];
    #pragma unroll
                    for (int k = 0; k < kZReg; ++k) v[k] = k < nz ? s[k * nx + x] : T(0);
                    __syncwarp();
    #pragma unroll
                    for (int zz = 0; zz < kZReg / 2; ++zz) {
                        const int z = pr * kh + zz;
                        if (zz >= kh || z >= nz) break;
                        T acc = T(0);
    #pragma unroll
                        for (int k = 0; k < kZReg; ++k)
                            if (k < nz) acc += Czi[z * nz + k] * v[k];
                        s[z * nx + x] = acc;
                    }
                }
                __syncthreads();
            } else if (zreg) {
                for (int x = threadIdx.x; x < nx; x += blockDim.x) {
                    T v[kZReg];
    #pragma unroll
                    for (int k = 0; k < kZReg; ++k) v[k] = k < nz ? s[k * nx + x] : T(0);
    #pragma unroll
                    for (int z = 0; z < kZReg; ++z) {
                        if (z >= nz) break;
                        T acc = T(0);
    #pragma unroll
                        for (int k = 0; k < kZReg; ++k)
                            if (k < nz) acc += Czi[z * nz + k] * v[k];
                        s[z * nx + x] = acc;
                    }
                }
                __syncthreads();
            } else {
                dct3_lines<T>(s, Lines{nx, 1, nx}, nz, xw0, xw1, pdz, stw);
            }
            dct3_lines<T, NX>(s, Lines{nz, nx, 1}, nx, xw0, xw1, pdx, stw);
            if (pg.inv_store[i] >= 0) store_slab(d.field[pg.inv_store[i]], s);
        }

        // ---- phase U: pointwise updates ----------------------------------------------------------
        if ((MODE == 0 || MODE == 2) && pg.op == 1) {
            // Gauss-Seidel cross product: out = base + p*q - r*s  (delta form, see host program)
            T* out = d.field[pg.gs_out];
            T* outl = d.flo[pg.gs_out];
            T* res = slabs + 2 * S;
            const T* bl_ = pg.gs_base >= 0 ? d.flo[pg.gs_base] : nullptr;
            const T* ql_ = pg.gs_q >= 0 ? d.flo[pg.gs_q] : nullptr;
            const T* sl_ = pg.gs_s >= 0 ? d.flo[pg.gs_s] : nullptr;
            if constexpr (kVec) {
                constexpr int N4 = NX / 4;
                const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
                auto ldr = [&](int ref, int o, int i) -> float4 {
                    return ref >= 0 ? ld4(d.field[ref] + cbase + o) : ld4(slabs + (-1 - ref) * S + 4 * i);
                };
                for (int i = threadIdx.x; i < nz * N4; i += blockDim.x) {
                    const int z = i / N4, x4 = i - z * N4;
                    const int o = z * zstride + 4 * x4;
                    const float4 B4 = ldr(pg.gs_base, o, i), P4 = ldr(pg.gs_p, o, i), Q4 = ldr(pg.gs_q, o, i);
                    const float4 R4 = ldr(pg.gs_r, o, i), S4 = ldr(pg.gs_s, o, i);
                    const float4 BL4 = bl_ ? ld4(bl_ + cbase + o) : zero4, QL4 = ql_ ? ld4(ql_ + cbase + o) : zero4;
                    const float4 SL4 = sl_ ? ld4(sl_ + cbase + o) : zero4;
                    const float bb[4] = {B4.x, B4.y, B4.z, B4.w}, pp[4] = {P4.x, P4.y, P4.z, P4.w};
                    const float qq[4] = {Q4.x, Q4.y, Q4.z, Q4.w}, rr[4] = {R4.x, R4.y, R4.z, R4.w};
                    const float ss[4] = {S4.x, S4.y, S4.z, S4.w}, bl[4] = {BL4.x, BL4.y, BL4.z, BL4.w};
                    const float ql[4] = {QL4.x, QL4.y, QL4.z, QL4.w}, sl[4] = {SL4.x, SL4.y, SL4.z, SL4.w};
                    float oh[4], ol[4];
    #pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (outl) {
                            const float rs = fmaf(rr[k], sl[k], rr[k] * ss[k]);
                            const float inc = fmaf(pp[k], qq[k], fmaf(pp[k], ql[k], -rs));
                            float hi, e;
                            two_sum(bb[k], inc, hi, e);
                            fast_two_sum(hi, e + bl[k], oh[k], ol[k]);
                        } else {
                            oh[k] = bb[k] + (pp[k] * qq[k] - rr[k] * ss[k]);
                            ol[k] = 0.f;
                        }
                    }
                    const float4 OH = make_float4(oh[0], oh[1], oh[2], oh[3]);
                    st4(out + cbase + o, OH);
                    if (outl) st4(outl + cbase + o, make_float4(ol[0], ol[1], ol[2], ol[3]));
                    st4(res + 4 * i, OH);
                }
            }
            constexpr int kB = sizeof(T) == 4 ? 4 : 2;
            for (int i0 = threadIdx.x; !kVec && i0 < nxz; i0 += kB * blockDim.x) {
                T bb[kB], pp[kB], qq[kB], rr[kB], ss[kB], bl[kB], ql[kB], sl[kB];
    #pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int idx = i0 + u * blockDim.x;
                    if (idx >= nxz) break;
                    const long long c = cell_of(idx / nx, idx - (idx / nx) * nx);
                    bb[u] = load_ref(d, pg.gs_base, c, slabs, S, idx);
                    pp[u] = load_ref(d, pg.gs_p, c, slabs, S, idx);
                    qq[u] = load_ref(d, pg.gs_q, c, slabs, S, idx);
                    rr[u] = load_ref(d, pg.gs_r, c, slabs, S, idx);
                    ss[u] = load_ref(d, pg.gs_s, c, slabs, S, idx);
                    bl[u] = bl_ ? bl_[c] : T(0);
                    ql[u] = ql_ ? ql_[c] : T(0);
                    sl[u] = sl_ ? sl_[c] : T(0);
                }
    #pragma unroll
                for (int u = 0; u < kB; ++u) {
                    const int idx = i0 + u * blockDim.x;
                    if (idx >= nxz) break;
                    const long long c = cell_of(idx / nx, idx - (idx / nx) * nx);
                    if (outl) {
                        // double-float state: base (hi, lo) + increment p (q_hi + q_lo) - r (s_hi + s_lo)
                        const T rs = fma(rr[u], sl[u], rr[u] * ss[u]);
                        const T inc = fma(pp[u], qq[u], fma(pp[u], ql[u], -rs));
                        T hi, e;
                        two_sum(bb[u], inc, hi, e);
                        T h2, l2;
                        fast_two_sum(hi, e + bl[u], h2, l2);
                        out[c] = h2;
                        outl[c] = l2;
                        res[idx] = h2;
                    } else {
                        const T v = bb[u] + (pp[u] * qq[u] - rr[u] * ss[u]);
                        out[c] = v;
                        res[idx] = v;
                    }
                }
            }
            __syncthreads();
        } else if ((MODE == 0 || MODE == 3) && pg.op == 2) {
            // Step 2 + Step 3: m*** = m** + delta (+ dt f_e), m^{n+1} = m*** / |m***|
            const bool dfl = d.flo[pg.fin_out[0]] != nullptr;
            // forcing of the manufactured solution (Sec. 5.1) added to m*** in FP64
            auto force = [&](T (&h)[3], T (&l)[3], int x, int z) {
                const double tnow = F.t0 + (double)(*d.step_ctr) * F.dt;
                double fe[3];
                mms_forcing(F.forcing, (x + 0.5) * F.hx, (y + 0.5) * F.hy, (z + 0.5) * F.hz, tnow, F.alpha, fe);
    #pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const double v = (double)h[i] + (double)l[i] + F.dt * fe[i];
                    h[i] = (T)v;
                    l[i] = (T)(v - (double)h[i]);
                }
            };
            if constexpr (kVec) {
                // double-float state, four cells per thread
                constexpr int N4 = NX / 4;
                for (int i = threadIdx.x; i < nz * N4; i += blockDim.x) {
                    const int z = i / N4, x4 = i - z * N4;
                    const int o = z * zstride + 4 * x4;
                    float mh[3][4], ml[3][4], dl[3][4];
    #pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        const float4 a = ld4(d.field[pg.fin_in[c3]] + cbase + o);
                        const float4 b = ld4(d.flo[pg.fin_in[c3]] + cbase + o);
                        const float4 e = ld4(slabs + c3 * S + 4 * i);
                        mh[c3][0] = a.x; mh[c3][1] = a.y; mh[c3][2] = a.z; mh[c3][3] = a.w;
                        ml[c3][0] = b.x; ml[c3][1] = b.y; ml[c3][2] = b.z; ml[c3][3] = b.w;
                        dl[c3][0] = e.x; dl[c3][1] = e.y; dl[c3][2] = e.z; dl[c3][3] = e.w;
                    }
                    float oh[3][4], ol[3][4], vv[3][4];
    #pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        float hh[3], ll[3], qh[3], ql[3];
    #pragma unroll
                        for (int c3 = 0; c3 < 3; ++c3) {
                            float s1, e1;
                            two_sum(mh[c3][k], dl[c3][k], s1, e1);
                            fast_two_sum(s1, e1 + ml[c3][k], hh[c3], ll[c3]);
                        }
                        if (F.forcing) force(hh, ll, 4 * x4 + k, z);
                        if (!project_df(hh, ll, qh, ql)) atomicOr(d.status, 1);
    #pragma unroll
                        for (int c3 = 0; c3 < 3; ++c3) {
                            oh[c3][k] = qh[c3];
                            ol[c3][k] = ql[c3];
                            vv[c3][k] = hh[c3] + ll[c3];
                        }
                    }
    #pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        const float4 O = make_float4(oh[c3][0], oh[c3][1], oh[c3][2], oh[c3][3]);
                        st4(d.field[pg.fin_out[c3]] + cbase + o, O);
                        st4(d.flo[pg.fin_out[c3]] + cbase + o, make_float4(ol[c3][0], ol[c3][1], ol[c3][2], ol[c3][3]));
                        st4(slabs + c3 * S + 4 * i, O);
                        if (pg.fin_v[c3] >= 0)
                            st4(d.field[pg.fin_v[c3]] + cbase + o, make_float4(vv[c3][0], vv[c3][1], vv[c3][2], vv[c3][3]));
                    }
                }
            }
            for (int idx = threadIdx.x; !kVec && idx < nxz; idx += blockDim.x) {
                int z = idx / nx, x = idx - z * nx;
                long long c = cell_of(z, x);
                if (dfl) {
                    // m*** = m** + delta in double-float, then |m***|^-1 by one double-float Newton step
                    T h[3], l[3], oh[3], ol[3];
    #pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        T s1, e1;
                        two_sum(d.field[pg.fin_in[i]][c], slabs[i * S + idx], s1, e1);
                        fast_two_sum(s1, e1 + d.flo[pg.fin_in[i]][c], h[i], l[i]);
                    }
                    if (F.forcing) force(h, l, x, z);
                    if (!project_df(h, l, oh, ol)) atomicOr(d.status, 1);
    #pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        d.field[pg.fin_out[i]][c] = oh[i];
                        d.flo[pg.fin_out[i]][c] = ol[i];
                        slabs[i * S + idx] = oh[i];
                        if (pg.fin_v[i] >= 0) d.field[pg.fin_v[i]][c] = h[i] + l[i];
                    }
                    continue;
                }
                T v[3];
    #pragma unroll
                for (int i = 0; i < 3; ++i) v[i] = d.field[pg.fin_in[i]][c] + slabs[i * S + idx];
                if (F.forcing) {
                    const double tnow = F.t0 + (double)(*d.step_ctr) * F.dt;
                    double fe[3];
                    mms_forcing(F.forcing, (x + 0.5) * F.hx, (y + 0.5) * F.hy, (z + 0.5) * F.hz, tnow, F.alpha, fe);
    #pragma unroll
                    for (int i = 0; i < 3; ++i) v[i] += T(F.dt * fe[i]);
                }
                T n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                if (!(n2 > T(0)) || !isfinite(n2)) {
                    atomicOr(d.status, 1);
                    n2 = T(1);
                }
                T inv = T(1) / sqrt(n2);
    #pragma unroll
                for (int i = 0; i < 3; ++i) {
                    T w = v[i] * inv;
                    d.field[pg.fin_out[i]][c] = w;
                    slabs[i * S + idx] = w;
                    if (pg.fin_v[i] >= 0) d.field[pg.fin_v[i]][c] = v[i];
                }
            }
            __syncthreads();
        }

        // ---- phase F: forward zero-padded FFT (x R2C, z C2C) -> spectral slots ---------------------
        if (MODE != 1 && stray) {
            for (int i = 0; i < pg.n_fwd; ++i) {
                const int ref = pg.fwd_src[i];
                const T* src;
                if (ref >= 0) {
                    T* s0 = slabs;
                    load_slab(s0, d.field[ref]);
                    __syncthreads();
                    src = s0;
                } else {
                    src = slabs + (-1 - ref) * S;
                }
                V* r;
                if constexpr (kHalfX) r = r2c_lines_h<T, NX>(src, Lines{nz, nx, 1}, nx, xw0, xw1, pdx, stw, stw + ppx.tw);
                else r = r2c_lines<T, 2 * NX>(src, Lines{nz, nx, 1}, nx, xw0, xw1, ppx, stw);
                auto rget = [&](int line, int k) {
                    if constexpr (kHalfX) return r2c_get_h<T>(r, line, k, Px);
                    else return r2c_get<T>(r, line, k, Px);
                };
                V* out = d.spec[pg.fwd_dst[i]] + sbase;
                if (kPair && nz == 8) {
                    // zero-padded DFT along z (Pz = 16), one lane pair per kx column: lane r computes
                    // the outputs kz = 2j + r as the 8-point DFT of v (r = 0) or of v W16^z (r = 1)
                    for (int kx = (int)threadIdx.x >> 1; kx < Kx; kx += (int)blockDim.x / 2) {
                        V v[8];
    #pragma unroll
                        for (int z = 0; z < 8; ++z) v[z] = rget(z, kx);
                        if (pr) {
    #pragma unroll
                            for (int z = 1; z < 8; ++z) v[z] = twmul(v[z], twz[z]);
                        }
                        Bfly<8, false, V>::run(v);
    #pragma unroll
                        for (int j = 0; j < 8; ++j) out[spec_of(2 * j + pr, kx)] = v[j];
                    }
                    __syncthreads();
                } else if (zreg) {
                    // zero-padded DFT along z in registers, one thread per kx column
                    for (int kx = threadIdx.x; kx < Kx; kx += blockDim.x) {
                        V v[2 * kZReg];
    #pragma unroll
                        for (int z = 0; z < 2 * kZReg; ++z) v[z] = z < nz ? rget(z, kx) : cmk<V>(T(0), T(0));
                        if (zfft_reg<T, false>(v, Pz)) {
    #pragma unroll
                            for (int kz = 0; kz < 2 * kZReg; ++kz)
                                if (kz < Pz) out[spec_of(kz, kx)] = v[kz];
                        } else {
                            for (int kz = 0; kz < Pz; ++kz) {
                                V acc = cmk<V>(T(0), T(0));
                                int m = 0;
    #pragma unroll
                                for (int z = 0; z < kZReg; ++z) {
                                    if (z < nz) acc = cadd(acc, twmul(v[z], twz[m]));
                                    m += kz;
                                    if (m >= Pz) m -= Pz;
                                }
                                out[spec_of(kz, kx)] = acc;
                            }
                        }
                    }
                    __syncthreads();
                }
                for (int kc0 = 0; !zreg && kc0 < Kx; kc0 += KC) {
                    const int kcn = min(KC, Kx - kc0);
                    for (int idx = threadIdx.x; idx < Pz * kcn; idx += blockDim.x) {
                        int z = idx / kcn, kc = idx - z * kcn;
                        zw0[z * KC + kc] = (z < nz) ? rget(z, kc0 + kc) : cmk<V>(T(0), T(0));
                    }
                    __syncthreads();
                    V* q = fft_lines<T, false>(zw0, zw1, Lines{kcn, 1, KC}, ppz, stw);
                    for (int idx = threadIdx.x; idx < Pz * kcn; idx += blockDim.x) {
                        int kz = idx / kcn, kc = idx - kz * kcn;
                        out[spec_of(kz, kc0 + kc)] = q[kz * KC + kc];
                    }
                    __syncthreads();
                }
            }
        }
        if constexpr (MULTI) __syncthreads();   // the next row reuses every shared buffer
    }
    if constexpr (ZTC) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        tc_teardown(tcs, tc_tmem_cols(NX));
    }
}

template <typename T, int NX, bool ZTC = false, bool MULTI = false, int MODE = 0>
__global__ void __launch_bounds__((xz_nt<NX, MODE, MULTI, ZTC>()), 2) xz_kernel(Dev<T> d, const int4* __restrict__ work,
                                                                                const __grid_constant__ XZProg pg, int stray) {
    pdl_launch_dependents();
    xz_item<T, NX, ZTC, MULTI, MODE>(d, work[blockIdx.x], pg, stray);
}

// ------------------------------------------------------------------------------------------
// Y line pass
// ------------------------------------------------------------------------------------------
// NY: compile-time y length of the films this launch covers (0: any length)
// One work item of the heat line pass: x columns kx0 .. kx0 + tn - 1 of plane kz of film wi.x.
template <typename T, int NY>
__device__ __forceinline__ void y_heat_item(const Dev<T> d, const int4 wi, const YProg& pg) {
    using V = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Film F = d.films[wi.x];
    const int kz = wi.y, kx0 = wi.z, tn = wi.w;
    const int nx = F.nx, ny = NY > 0 ? NY : F.ny, nz = F.nz;
    __shared__ Plan pdy;
    if (threadIdx.x == 0) pdy = d.plans[F.splan_dy];   // staged copy: twiddles at 0, quarter-wave at ny
    tw_t<T>* stw = reinterpret_cast<tw_t<T>*>(smem_raw);
    const int npair = (tn + 1) / 2;
    V* c0 = reinterpret_cast<V*>(stw + 2 * ny);
    V* c1 = c0 + npair * ny;
    T* R = reinterpret_cast<T*>(c1 + npair * ny);
    const int LR = ny + 8;   // padded line stride: tile copies hit distinct banks
    stage_async(stw, d.tw + F.gtw_dy, ny);
    stage_async(stw + ny, d.tw + F.gtw4_dy, ny);
    cp_async_commit();
    cp_async_wait(0);
    __syncthreads();
    pdl_wait();
    // tile copies: thread -> column t_ld of rows y_ld, y_ld + rpp, ... (no per-element division)
    const int rpp = (int)blockDim.x / tn;
    const int t_ld = (int)threadIdx.x % tn, y_ld = (int)threadIdx.x / tn;
    const bool ld_on = y_ld < rpp;
    // eigen-scale 1 / (N (1 + c (lx + ly + lz))), c = eps dt (alpha eps dt for Step 2); in the
    // FP32 form c, 1/N and the eigenvalues are double-float so that the scale, which is applied
    // to every mode in every solve, carries no fixed table rounding
    T ch, cl, nh, nl;
    if constexpr (sizeof(T) == 4) {
        // precomputed on the host: no FP64 arithmetic in the FP32 kernels
        const int dm = pg.damp ? 1 : 0;
        ch = F.fs_c[dm][0];
        cl = F.fs_c[dm][1];
        nh = F.fs_n[0];
        nl = F.fs_n[1];
    } else {
        ch = (pg.damp ? F.alpha * F.eps : F.eps) * F.dt;
        nh = 1.0 / ((double)nx * ny * nz);
        cl = nl = T(0);
    }
    const T* lx = d.lam + F.lam;
    const T* ly = lx + nx;
    const T lzh = ly[ny + kz];
    const T* lxl = d.lam_lo ? d.lam_lo + F.lam : nullptr;
    const T lzl = lxl ? lxl[nx + ny + kz] : T(0);
    for (int f = 0; f < pg.n; ++f) {
        T* g = d.field[pg.slot[f]] + F.off_cell + (long long)kz * ny * nx + kx0;
        if (ld_on)
            for (int yy = y_ld; yy < ny; yy += rpp) R[t_ld * LR + yy] = g[yy * nx + t_ld];
        __syncthreads();
        dct2_lines<T, NY>(R, Lines{tn, LR, 1}, ny, c0, c1, pdy, stw);
        for (int idx = threadIdx.x; idx < ny * tn; idx += blockDim.x) {
            const int t = idx / ny, ky = idx - t * ny;
            T& r = R[t * LR + ky];
            if constexpr (sizeof(T) == 8) {
                r *= nh / (T(1) + ch * (lx[kx0 + t] + ly[ky] + lzh));
            } else {
                // Lambda = lx + ly + lz, s = 1 + c Lambda, scale = (1/N) / s, all double-float
                T a, e1, Lh, e2;
                two_sum(lx[kx0 + t], ly[ky], a, e1);
                two_sum(a, lzh, Lh, e2);
                const T Ll = e1 + e2 + (lxl[kx0 + t] + lxl[nx + ky] + lzl);
                T p, pe;
                two_prod(ch, Lh, p, pe);
                const T pl = pe + fma(ch, Ll, cl * Lh);
                T sh, se;
                two_sum(T(1), p, sh, se);
                const T sl = se + pl;
                const T r0 = T(1) / sh;
                const T res = fma(-sh, r0, T(1)) - sl * r0;   // 1 - s r0
                const T ih = r0, il = r0 * res;
                T q, qe;
                two_prod(nh, ih, q, qe);
                const T ql = qe + fma(nh, il, nl * ih);
                r = fma(r, q, r * ql);
            }
        }
        __syncthreads();
        dct3_lines<T, NY>(R, Lines{tn, LR, 1}, ny, c0, c1, pdy, stw);
        if (ld_on)
            for (int yy = y_ld; yy < ny; yy += rpp) g[yy * nx + t_ld] = R[t_ld * LR + yy];
        __syncthreads();
    }
}

template <typename T, int NY>
__global__ void __launch_bounds__(kThreads) y_heat_kernel(Dev<T> d, const int4* __restrict__ work, const __grid_constant__ YProg pg) {
    pdl_launch_dependents();
    y_heat_item<T, NY>(d, work[blockIdx.x], pg);
}

// pair index of (a, b) in the 6-component symmetric tensor: xx yy zz xy xz yz
__device__ __forceinline__ int pair_idx(int a, int b) {
    if (a == b) return a;
    int s = a + b;   // (0,1)->1 -> xy=3, (0,2)->2 -> xz=4, (1,2)->3 -> yz=5
    return s + 2;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) y_stray_kernel(Dev<T> d, const int4* __restrict__ work, YProg pg, int tx) {
    using V = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int4 wi = work[blockIdx.x];
    const Film F = d.films[wi.x];
    const int kz = wi.y, kx0 = wi.z, tn = wi.w;
    const int ny = F.ny, Py = F.Py, Pz = F.Pz, Kx = F.Kx;
    __shared__ Plan ppy;
    if (threadIdx.x == 0) ppy = d.plans[F.plan_py];
    __syncthreads();
    tw_t<T>* stw = reinterpret_cast<tw_t<T>*>(smem_raw);
    stage_plan<T>(ppy, d.tw, stw, 0, false);
    __syncthreads();
    if (threadIdx.x == 0) ppy.tw = 0;
    __syncthreads();
    const int LS = Py + 4;   // padded line stride: tile copies hit distinct banks
    const int B = tx * LS;
    V* w0 = reinterpret_cast<V*>(stw + Py);
    V* w1 = w0 + B;
    V* acc = w1 + B;     // pg.n accumulators
    const int HyP = ktab_row(Py), Hz = Pz / 2 + 1;
    const int kzr = kz <= Pz - kz ? kz : Pz - kz;
    const bool zodd = kz > Pz / 2;
    const T* kt = d.ktab + F.off_ktab;
    for (int o = 0; o < pg.n; ++o)
        for (int idx = threadIdx.x; idx < tn * LS; idx += blockDim.x) acc[o * B + idx] = cmk<V>(T(0), T(0));
    for (int b = 0; b < 3; ++b) {
        if (!(pg.in_mask & (1 << b))) continue;
        const V* Sb = d.spec[pg.in_spec[b]] + F.off_spec + (long long)kz * ny * Kx + kx0;
        for (int idx = threadIdx.x; idx < tn * Py; idx += blockDim.x) {
            int yy = idx / tn, t = idx - yy * tn;
            w0[t * LS + yy] = (yy < ny) ? Sb[(long long)yy * Kx + t] : cmk<V>(T(0), T(0));
        }
        __syncthreads();
        V* M = fft_lines<T, false>(w0, w1, Lines{tn, LS, 1}, ppy, stw);
        // spectral multiply: issue all table loads of a batch before the accumulations
        const int total = tn * Py;
        for (int base = threadIdx.x; base < total; base += 4 * blockDim.x) {
            T kv[4][3];
            int ids[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + u * blockDim.x;
                ids[u] = idx;
                if (idx < total) {
                    const int t = idx / Py, ky = idx - t * Py;
                    const int kyr = ky <= Py - ky ? ky : Py - ky;
                    const bool yodd = ky > Py / 2;
#pragma unroll
                    for (int o = 0; o < 3; ++o) {
                        if (o < pg.n) {
                            const int cc = pair_idx(pg.slot[o], b);
                            T k = kt[ktab_index(cc, kx0 + t, kzr, kyr, Kx, HyP, Hz)];
                            const bool neg = ((cc == 3 || cc == 5) && yodd) != ((cc == 4 || cc == 5) && zodd);
                            kv[u][o] = neg ? -k : k;
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = ids[u];
                if (idx < total) {
                    const int li = (idx / Py) * LS + (idx % Py);
                    const V m = M[li];
#pragma unroll
                    for (int o = 0; o < 3; ++o) {
                        if (o < pg.n) {
                            V& A = acc[o * B + li];
                            A.x += kv[u][o] * m.x;
                            A.y += kv[u][o] * m.y;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    for (int o = 0; o < pg.n; ++o) {
        V* r = fft_lines<T, true>(acc + o * B, w0, Lines{tn, LS, 1}, ppy, stw);
        V* Ho = d.spec[pg.out_spec[o]] + F.off_spec + (long long)kz * ny * Kx + kx0;
        for (int idx = threadIdx.x; idx < tn * ny; idx += blockDim.x) {
            int yy = idx / tn, t = idx - yy * tn;
            Ho[(long long)yy * Kx + t] = r[t * LS + yy];
        }
        __syncthreads();
    }
}

// Twiddle precision of the stray pass's y transforms: the stray field enters each step scaled by
// dt, so the fixed rounding of FP32 twiddles there perturbs the increment far less than in the
// heat solves; hi parts only
constexpr bool kStrayTwLo = false;

// Register-resident stray-field line pass: one warp per kx line (Py = 32 E, E in {2,4,8,16}).
// The CTA first issues asynchronous copies of everything it reads: for each input component b
// the (y < ny, kx0..kx0+lines) tile of the x,z spectrum (fresh components only) and the Newell
// table lines of the pairs (out, b), one commit group per component, so that all loads are in
// flight together.  Then, per component: forward FFT in registers (zero padded) of a fresh
// component, optionally stored to the y-transform cache in register order, or the cached
// transform of an unchanged one; multiply-accumulate with the table in the FFT's own output
// order.  Finally the adjoint FFT of each output and a store of y < ny.  Within one step the
// Gauss-Seidel sweep changes one component between refreshes, so a refresh transforms one
// input instead of three.
// One work item: kx lines kx0 .. kx0 + tn - 1 (tn <= LINES) of plane kz of film wi.x, one warp per
// line; the CTA has 32 LINES threads.
template <typename T, int NOUT, int E, int LINES = kWarpLines>
__device__ __forceinline__ void y_stray_warp_item(const Dev<T> d, const int4 wi, const YProg& pg) {
    using V = cplx<T>;
    constexpr int P = 32 * E, G = 32 / E;
    constexpr int LI = P / 2 + 8;                 // yw_line_stride
    constexpr int HyP = ((P / 2 + 1) + 3) & ~3;   // ktab_row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Film& F = d.films[wi.x];
    const int kz = wi.y, kx0 = wi.z, tn = wi.w;
    const int ny = F.ny, Kx = F.Kx, Pz = F.Pz, Hz = Pz / 2 + 1;
    const int kzr = kz <= Pz - kz ? kz : Pz - kz;
    const bool zodd = kz > Pz / 2;
    tw_t<T>* stw = reinterpret_cast<tw_t<T>*>(smem_raw);
    V* scr0 = reinterpret_cast<V*>(stw + P);
    V* inb = scr0 + LINES * P;                                       // [3][lines][LI]
    T* kbuf = reinterpret_cast<T*>(inb + 3 * LINES * LI);            // [3 NOUT][lines][HyP]
    stage_async(stw, d.tw + d.plans[F.plan_py].tw, P);
    // the Newell table lines of the pairs (o, b) are constant: their copies are issued with the
    // twiddles, before the wait for the previous pass, so that they overlap its tail
    const T* kt = d.ktab + F.off_ktab;
    constexpr int KCH = 16 / (int)sizeof(T);   // table elements per 16-byte piece
    const int nkch = tn * HyP / KCH;
#pragma unroll 1
    for (int b = 0; b < 3; ++b) {
        if (!(pg.in_mask & (1 << b))) continue;
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            const int cc = pair_idx(pg.slot[o], b);
            const T* src = kt + (((long long)cc * Hz + kzr) * Kx + kx0) * HyP;
            T* kd = kbuf + (o * 3 + b) * LINES * HyP;
            for (int i = threadIdx.x; i < nkch; i += blockDim.x) cp_async_16(kd + i * KCH, src + i * KCH);
        }
    }
    cp_async_commit();   // group 0: twiddles and table lines (complete before component 0 is used)
    pdl_wait();
    // ---- asynchronous staging: group 1 + b = the fresh input component b (spectrum tile)
    const long long line0 = F.off_spec + (long long)kz * ny * Kx + kx0;
#pragma unroll 1
    for (int b = 0; b < 3; ++b) {
        if (pg.in_mask & (1 << b)) {
            const V* Sb = d.spec[pg.in_spec[b]] + line0;
            const bool fresh = (pg.fresh_mask >> b) & 1;
            V* dst = inb + b * LINES * LI;
            const int n = fresh ? tn * ny : 0;
            for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
                const int y = idx / tn, t = idx - y * tn;
                cp_async<(int)sizeof(V)>(dst + t * LI + y, Sb + (long long)y * Kx + t);
            }
        }
        cp_async_commit();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool active = warp < tn;
    V* scr = scr0 + warp * P;
    const int q = lane / G, g = lane % G;
    const int s2 = bitrev_lanes(g, G);
    V acc[NOUT][E];
#pragma unroll
    for (int o = 0; o < NOUT; ++o)
#pragma unroll
        for (int s1 = 0; s1 < E; ++s1) acc[o][s1] = cmk<V>(T(0), T(0));
    // cached y transforms: line (kz, kx) of component b, element s1 * 32 + lane = register v[s1]
    const long long cline = F.off_ycache + ((long long)kz * Kx + kx0 + warp) * P + lane;
#pragma unroll 1
    for (int b = 0; b < 3; ++b) {
        cp_async_wait(2 - b);
        __syncthreads();
        if (!active || !(pg.in_mask & (1 << b))) continue;
        V v[E];
        V* cb = d.ycache + b * d.ycache_n + cline;
        if ((pg.fresh_mask >> b) & 1) {
            const V* line = inb + (b * LINES + warp) * LI;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int y = lane + 32 * k;
                v[k] = y < ny ? line[y] : cmk<V>(T(0), T(0));
            }
            wreg_fwd<T, E, kStrayTwLo>(v, scr, stw, lane);
            if ((pg.store_mask >> b) & 1) {
#pragma unroll
                for (int s1 = 0; s1 < E; ++s1) cb[s1 * 32] = v[s1];
            }
        } else {
#pragma unroll
            for (int s1 = 0; s1 < E; ++s1) v[s1] = cb[s1 * 32];
        }
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            const int cc = pair_idx(pg.slot[o], b);
            const bool yflip = (cc == 3 || cc == 5);
            const bool zflip = (cc == 4 || cc == 5) && zodd;
            const T* kb = kbuf + ((o * 3 + b) * LINES + warp) * HyP;
#pragma unroll
            for (int s1 = 0; s1 < E; ++s1) {
                const int ky = q + E * (s1 + E * s2);
                const int kyr = ky <= P / 2 ? ky : P - ky;
                T k = kb[kyr];
                if ((yflip && ky > P / 2) != zflip) k = -k;
                acc[o][s1].x += k * v[s1].x;
                acc[o][s1].y += k * v[s1].y;
            }
        }
    }
    if (!active) return;
    const long long out0 = line0 + warp;
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
        wreg_adj<T, E, kStrayTwLo>(acc[o], scr, stw, lane);
        V* Ho = d.spec[pg.out_spec[o]] + out0;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int y = lane + 32 * k;
            if (y < ny) Ho[(long long)y * Kx] = acc[o][k];
        }
    }
}

template <typename T, int NOUT, int E>
__global__ void __launch_bounds__(32 * kWarpLines) y_stray_warp_kernel(Dev<T> d, const int4* __restrict__ work,
                                                                     const __grid_constant__ YProg pg) {
    pdl_launch_dependents();
    y_stray_warp_item<T, NOUT, E>(d, work[blockIdx.x], pg);
}

}  // namespace sgspm
