// XZ slab pass, Y line pass, energy reduction and small helper kernels (FP32 and FP64).
// Compiled as part of capi.cu (single translation unit).
#pragma once
#include "passes.cuh"

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

// ------------------------------------------------------------------------------------------
// XZ slab pass
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) xz_kernel(Dev<T> d, const int4* __restrict__ work, XZProg pg, int stray) {
    using V = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int4 wi = work[blockIdx.x];
    const Film F = d.films[wi.x];
    const int y = wi.y;
    const int nx = F.nx, ny = F.ny, nz = F.nz, Px = F.Px, Pz = F.Pz, Kx = F.Kx;
    const XZLayout Lo = xz_layout(nx, nz, Px, Pz, Kx, stray != 0);
    V* xw0 = reinterpret_cast<V*>(smem_raw);
    V* xw1 = xw0 + Lo.xw;
    V* zw0 = xw1 + Lo.xw;
    V* zw1 = zw0 + Lo.zw;
    T* slabs = reinterpret_cast<T*>(zw1 + Lo.zw);
    const int S = Lo.slab;
    const int KC = Lo.kc;
    const int npx = (nz + 1) / 2;
    const int nxz = nx * nz;
    const long long cbase = F.off_cell;
    const long long sbase = F.off_spec;
    __shared__ Plan pdx, pdz, ppx, ppz;
    if (threadIdx.x == 0) {
        pdx = d.plans[F.plan_dx];
        pdz = d.plans[F.plan_dz];
        ppx = d.plans[F.plan_px];
        ppz = d.plans[F.plan_pz];
    }
    __syncthreads();
    auto cell_of = [&](int z, int x) -> long long { return cbase + ((long long)z * ny + y) * nx + x; };

    // ---- phase R: right-hand sides and forward DCT ---------------------------------------
    for (int ci = 0; ci < pg.n_rhs; ++ci) {
        const int a = pg.rhs_comp[ci];
        T* h = slabs;   // slab 0
        if (pg.rhs_h[ci] >= 0 && stray) {
            const V* H = d.spec[pg.rhs_h[ci]] + sbase;
            for (int kc0 = 0; kc0 < Kx; kc0 += KC) {
                const int kcn = min(KC, Kx - kc0);
                for (int idx = threadIdx.x; idx < Pz * kcn; idx += blockDim.x) {
                    int kz = idx / kcn, kc = idx - kz * kcn;
                    zw0[kz * KC + kc] = H[((long long)kz * ny + y) * Kx + kc0 + kc];
                }
                __syncthreads();
                V* r = fft_lines<T, true>(zw0, zw1, Lines{kcn, 1, KC}, ppz, d.tw);
                for (int idx = threadIdx.x; idx < npx * kcn; idx += blockDim.x) {
                    int p = idx / kcn, kc = idx - p * kcn;
                    V xa = r[(2 * p) * KC + kc];
                    V xb = (2 * p + 1 < nz) ? r[(2 * p + 1) * KC + kc] : cmk<V>(T(0), T(0));
                    c2r_put<T>(xw0, p, kc0 + kc, Px, xa, xb);
                }
                __syncthreads();
            }
            V* r = fft_lines<T, true>(xw0, xw1, Lines{npx, Px, 1}, ppx, d.tw);
            for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                int z = idx / nx, x = idx - z * nx;
                V v = r[(z >> 1) * Px + x];
                h[idx] = (z & 1) ? v.y : v.x;
            }
        } else {
            for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) h[idx] = T(0);
        }
        __syncthreads();
        if (pg.rhs_hs_store[ci] >= 0) {
            T* out = d.field[pg.rhs_hs_store[ci]];
            for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                int z = idx / nx, x = idx - z * nx;
                out[cell_of(z, x)] = h[idx];
            }
        }
        if (!pg.rhs_dct) { __syncthreads(); continue; }
        // r_a = scale * (f_a + eps Delta_h m_a),  f_a = -Q (m_a - (m.u) u_a) + h_s,a + h_e,a
        {
            const T* m1 = d.field[pg.state[0]];
            const T* m2 = d.field[pg.state[1]];
            const T* m3 = d.field[pg.state[2]];
            const T* ma = d.field[pg.state[a]];
            const T scale = T(pg.damp ? F.alpha * F.dt : F.dt);
            const T eps = T(F.eps), Q = T(F.Q);
            const T ux = T(F.u[0]), uy = T(F.u[1]), uz = T(F.u[2]);
            const T ua = T(F.u[a]);
            const T ihx = T(1.0 / (F.hx * F.hx)), ihy = T(1.0 / (F.hy * F.hy)), ihz = T(1.0 / (F.hz * F.hz));
            const T hea = T(F.he[a]);
            for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                int z = idx / nx, x = idx - z * nx;
                long long c = cell_of(z, x);
                T v1 = m1[c], v2 = m2[c], v3 = m3[c];
                T mc = ma[c];
                T mu = v1 * ux + v2 * uy + v3 * uz;
                T lap = T(0);
                if (nx > 1) lap += ihx * ((x + 1 < nx ? ma[c + 1] : mc) - T(2) * mc + (x > 0 ? ma[c - 1] : mc));
                if (ny > 1) lap += ihy * ((y + 1 < ny ? ma[c + nx] : mc) - T(2) * mc + (y > 0 ? ma[c - nx] : mc));
                if (nz > 1) {
                    long long sz = (long long)nx * ny;
                    lap += ihz * ((z + 1 < nz ? ma[c + sz] : mc) - T(2) * mc + (z > 0 ? ma[c - sz] : mc));
                }
                T he = d.he_cell ? d.he_cell[c * 3 + a] : hea;
                T f = -Q * (mc - mu * ua) + h[idx] + he;
                h[idx] = scale * (f + eps * lap);
            }
        }
        __syncthreads();
        dct2_lines<T>(h, Lines{nz, nx, 1}, nx, xw0, xw1, pdx, d.tw);
        dct2_lines<T>(h, Lines{nx, 1, nx}, nz, xw0, xw1, pdz, d.tw);
        {
            T* out = d.field[pg.rhs_out[ci]];
            for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                int z = idx / nx, x = idx - z * nx;
                out[cell_of(z, x)] = h[idx];
            }
        }
        __syncthreads();
    }

    // ---- phase I: inverse DCT of solved spectra -> delta slabs ------------------------------
    for (int i = 0; i < pg.n_inv; ++i) {
        T* s = slabs + i * S;
        const T* in = d.field[pg.inv_in[i]];
        for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
            int z = idx / nx, x = idx - z * nx;
            s[idx] = in[cell_of(z, x)];
        }
        __syncthreads();
        dct3_lines<T>(s, Lines{nx, 1, nx}, nz, xw0, xw1, pdz, d.tw);
        dct3_lines<T>(s, Lines{nz, nx, 1}, nx, xw0, xw1, pdx, d.tw);
        if (pg.inv_store[i] >= 0) {
            T* out = d.field[pg.inv_store[i]];
            for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                int z = idx / nx, x = idx - z * nx;
                out[cell_of(z, x)] = s[idx];
            }
        }
    }

    // ---- phase U: pointwise updates ----------------------------------------------------------
    if (pg.op == 1) {
        // Gauss-Seidel cross product: out = base + p*q - r*s  (delta form, see host program)
        T* out = d.field[pg.gs_out];
        T* res = slabs + 2 * S;
        for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
            int z = idx / nx, x = idx - z * nx;
            long long c = cell_of(z, x);
            T b = load_ref(d, pg.gs_base, c, slabs, S, idx);
            T p = load_ref(d, pg.gs_p, c, slabs, S, idx);
            T q = load_ref(d, pg.gs_q, c, slabs, S, idx);
            T r = load_ref(d, pg.gs_r, c, slabs, S, idx);
            T s = load_ref(d, pg.gs_s, c, slabs, S, idx);
            T v = b + (p * q - r * s);
            out[c] = v;
            res[idx] = v;
        }
        __syncthreads();
    } else if (pg.op == 2) {
        // Step 2 + Step 3: m*** = m** + delta (+ dt f_e), m^{n+1} = m*** / |m***|
        const double tnow = F.t0 + (double)(*d.step_ctr) * F.dt;
        for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
            int z = idx / nx, x = idx - z * nx;
            long long c = cell_of(z, x);
            T v[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) v[i] = d.field[pg.fin_in[i]][c] + slabs[i * S + idx];
            if (F.forcing) {
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
            }
        }
        __syncthreads();
    }

    // ---- phase F: forward zero-padded FFT (x R2C, z C2C) -> spectral slots ---------------------
    if (stray) {
        for (int i = 0; i < pg.n_fwd; ++i) {
            const int ref = pg.fwd_src[i];
            const T* src;
            if (ref >= 0) {
                T* s0 = slabs;
                const T* in = d.field[ref];
                for (int idx = threadIdx.x; idx < nxz; idx += blockDim.x) {
                    int z = idx / nx, x = idx - z * nx;
                    s0[idx] = in[cell_of(z, x)];
                }
                __syncthreads();
                src = s0;
            } else {
                src = slabs + (-1 - ref) * S;
            }
            V* r = r2c_lines<T>(src, Lines{nz, nx, 1}, nx, xw0, xw1, ppx, d.tw);
            V* out = d.spec[pg.fwd_dst[i]] + sbase;
            for (int kc0 = 0; kc0 < Kx; kc0 += KC) {
                const int kcn = min(KC, Kx - kc0);
                for (int idx = threadIdx.x; idx < Pz * kcn; idx += blockDim.x) {
                    int z = idx / kcn, kc = idx - z * kcn;
                    zw0[z * KC + kc] = (z < nz) ? r2c_get<T>(r, z, kc0 + kc, Px) : cmk<V>(T(0), T(0));
                }
                __syncthreads();
                V* q = fft_lines<T, false>(zw0, zw1, Lines{kcn, 1, KC}, ppz, d.tw);
                for (int idx = threadIdx.x; idx < Pz * kcn; idx += blockDim.x) {
                    int kz = idx / kcn, kc = idx - kz * kcn;
                    out[((long long)kz * ny + y) * Kx + kc0 + kc] = q[kz * KC + kc];
                }
                __syncthreads();
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Y line pass
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) y_heat_kernel(Dev<T> d, const int4* __restrict__ work, YProg pg) {
    using V = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int4 wi = work[blockIdx.x];
    const Film F = d.films[wi.x];
    const int kz = wi.y, kx0 = wi.z, tn = wi.w;
    const int nx = F.nx, ny = F.ny, nz = F.nz;
    __shared__ Plan pdy;
    if (threadIdx.x == 0) pdy = d.plans[F.plan_dy];
    __syncthreads();
    const int npair = (tn + 1) / 2;
    V* c0 = reinterpret_cast<V*>(smem_raw);
    V* c1 = c0 + npair * ny;
    T* R = reinterpret_cast<T*>(c1 + npair * ny);
    const T c = T(pg.damp ? F.alpha * F.eps : F.eps) * T(F.dt);
    const T* lx = d.lam + F.lam;
    const T* ly = lx + nx;
    const T lzv = (lx + nx + ny)[kz];
    const T norm = T(1.0 / ((double)nx * ny * nz));
    for (int f = 0; f < pg.n; ++f) {
        T* g = d.field[pg.slot[f]] + F.off_cell + (long long)kz * ny * nx + kx0;
        for (int idx = threadIdx.x; idx < ny * tn; idx += blockDim.x) {
            int yy = idx / tn, t = idx - yy * tn;
            R[t * ny + yy] = g[(long long)yy * nx + t];
        }
        __syncthreads();
        dct2_lines<T>(R, Lines{tn, ny, 1}, ny, c0, c1, pdy, d.tw);
        for (int idx = threadIdx.x; idx < ny * tn; idx += blockDim.x) {
            int t = idx / ny, ky = idx - t * ny;
            R[idx] *= norm / (T(1) + c * (lx[kx0 + t] + ly[ky] + lzv));
        }
        __syncthreads();
        dct3_lines<T>(R, Lines{tn, ny, 1}, ny, c0, c1, pdy, d.tw);
        for (int idx = threadIdx.x; idx < ny * tn; idx += blockDim.x) {
            int yy = idx / tn, t = idx - yy * tn;
            g[(long long)yy * nx + t] = R[t * ny + yy];
        }
        __syncthreads();
    }
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
    const int B = tx * Py;
    V* w0 = reinterpret_cast<V*>(smem_raw);
    V* w1 = w0 + B;
    V* acc = w1 + B;     // pg.n accumulators
    const int Hy = Py / 2 + 1, Hz = Pz / 2 + 1;
    const int kzr = kz <= Pz - kz ? kz : Pz - kz;
    const bool zodd = kz > Pz / 2;
    const T* kt = d.ktab + F.off_ktab;
    for (int o = 0; o < pg.n; ++o)
        for (int idx = threadIdx.x; idx < tn * Py; idx += blockDim.x) acc[o * B + idx] = cmk<V>(T(0), T(0));
    for (int b = 0; b < 3; ++b) {
        const V* Sb = d.spec[pg.in_spec[b]] + F.off_spec + (long long)kz * ny * Kx + kx0;
        for (int idx = threadIdx.x; idx < tn * Py; idx += blockDim.x) {
            int yy = idx / tn, t = idx - yy * tn;
            w0[t * Py + yy] = (yy < ny) ? Sb[(long long)yy * Kx + t] : cmk<V>(T(0), T(0));
        }
        __syncthreads();
        V* M = fft_lines<T, false>(w0, w1, Lines{tn, Py, 1}, ppy, d.tw);
        for (int idx = threadIdx.x; idx < tn * Py; idx += blockDim.x) {
            int t = idx / Py, ky = idx - t * Py;
            const int kyr = ky <= Py - ky ? ky : Py - ky;
            const bool yodd = ky > Py / 2;
            V m = M[idx];
            for (int o = 0; o < pg.n; ++o) {
                const int a = pg.slot[o];
                const int cc = pair_idx(a, b);
                T k = kt[ktab_index(cc, kx0 + t, kzr, kyr, Kx, Hy, Hz)];
                bool neg = ((cc == 3 || cc == 5) && yodd) != ((cc == 4 || cc == 5) && zodd);
                if (neg) k = -k;
                V& A = acc[o * B + idx];
                A.x += k * m.x;
                A.y += k * m.y;
            }
        }
        __syncthreads();
    }
    for (int o = 0; o < pg.n; ++o) {
        V* r = fft_lines<T, true>(acc + o * B, w0, Lines{tn, Py, 1}, ppy, d.tw);
        V* Ho = d.spec[pg.out_spec[o]] + F.off_spec + (long long)kz * ny * Kx + kx0;
        for (int idx = threadIdx.x; idx < tn * ny; idx += blockDim.x) {
            int yy = idx / tn, t = idx - yy * tn;
            Ho[(long long)yy * Kx + t] = r[t * Py + yy];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// Energy: per-block FP64 partial sums, then an ordered per-film sum (deterministic).
// work: (film, first cell, count, -)
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads) energy_partial_kernel(Dev<T> d, const int4* __restrict__ work, int m0, int hs0,
                                                                  int have_hs, double* __restrict__ part) {
    const int4 wi = work[blockIdx.x];
    const Film F = d.films[wi.x];
    const int nx = F.nx, ny = F.ny, nz = F.nz;
    const long long sxy = (long long)nx * ny;
    const T* m[3] = {d.field[m0], d.field[m0 + 1], d.field[m0 + 2]};
    double ex = 0, an = 0, st = 0, ze = 0;
    for (int i = threadIdx.x; i < wi.z; i += blockDim.x) {
        long long loc = wi.y + i;
        int x = loc % nx;
        int y = (loc / nx) % ny;
        int z = loc / sxy;
        long long c = F.off_cell + loc;
        double v[3] = {(double)m[0][c], (double)m[1][c], (double)m[2][c]};
        for (int a = 0; a < 3; ++a) {
            if (x + 1 < nx) { double q = (double)m[a][c + 1] - v[a]; ex += q * q / (F.hx * F.hx); }
            if (y + 1 < ny) { double q = (double)m[a][c + nx] - v[a]; ex += q * q / (F.hy * F.hy); }
            if (z + 1 < nz) { double q = (double)m[a][c + sxy] - v[a]; ex += q * q / (F.hz * F.hz); }
        }
        double mu = v[0] * F.u[0] + v[1] * F.u[1] + v[2] * F.u[2];
        an += v[0] * v[0] + v[1] * v[1] + v[2] * v[2] - mu * mu;
        if (have_hs)
            for (int a = 0; a < 3; ++a) st += (double)d.field[hs0 + a][c] * v[a];
        for (int a = 0; a < 3; ++a) {
            double he = d.he_cell ? (double)d.he_cell[c * 3 + a] : F.he[a];
            ze += he * v[a];
        }
    }
    __shared__ double red[4][kThreads / 32];
    double vals[4] = {ex, an, st, ze};
    for (int k = 0; k < 4; ++k) {
        double s = vals[k];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        part[blockIdx.x * 4 + threadIdx.x] = s;
    }
}

// one thread per film: sum the film's block partials in order and apply the prefactors
__global__ void energy_final_kernel(const Film* films, int nfilm, const int* __restrict__ first_block,
                                    const double* __restrict__ part, double* __restrict__ out) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfilm) return;
    const Film F = films[f];
    double s[4] = {0, 0, 0, 0};
    for (int b = first_block[f]; b < first_block[f + 1]; ++b)
        for (int k = 0; k < 4; ++k) s[k] += part[b * 4 + k];
    const double V = F.hx * F.hy * F.hz;
    double ex = 0.5 * F.eps * V * s[0];
    double an = 0.5 * F.Q * V * s[1];
    double st = -0.5 * V * s[2];
    double ze = -V * s[3];
    out[5 * f + 0] = ex;
    out[5 * f + 1] = an;
    out[5 * f + 2] = st;
    out[5 * f + 3] = ze;
    out[5 * f + 4] = ex + an + st + ze;
}

// ------------------------------------------------------------------------------------------
// helpers: dtype conversion in/out of the SoA pools, normalisation, step counter
// ------------------------------------------------------------------------------------------
template <typename T, typename S>
__global__ void copy_in_kernel(T* __restrict__ d0, T* __restrict__ d1, T* __restrict__ d2, const S* __restrict__ src,
                               const Film* films, int nfilm, long long ntot) {
    // src: concatenation over films of [3][ncell_f]
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= ntot) return;
    int f = 0;
    while (f + 1 < nfilm && films[f + 1].off_cell <= i) ++f;
    const Film F = films[f];
    long long loc = i - F.off_cell;
    long long nc = (long long)F.nx * F.ny * F.nz;
    const S* s = src + 3 * F.off_cell;
    d0[i] = (T)s[loc];
    d1[i] = (T)s[nc + loc];
    d2[i] = (T)s[2 * nc + loc];
}

template <typename T, typename S>
__global__ void copy_out_kernel(S* __restrict__ dst, const T* __restrict__ d0, const T* __restrict__ d1, const T* __restrict__ d2,
                                const Film* films, int nfilm, long long ntot) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= ntot) return;
    int f = 0;
    while (f + 1 < nfilm && films[f + 1].off_cell <= i) ++f;
    const Film F = films[f];
    long long loc = i - F.off_cell;
    long long nc = (long long)F.nx * F.ny * F.nz;
    S* s = dst + 3 * F.off_cell;
    s[loc] = (S)d0[i];
    s[nc + loc] = (S)d1[i];
    s[2 * nc + loc] = (S)d2[i];
}

template <typename T>
__global__ void normalize_kernel(T* m0, T* m1, T* m2, long long n, int* status) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T a = m0[i], b = m1[i], c = m2[i];
    T n2 = a * a + b * b + c * c;
    if (!(n2 > T(0)) || !isfinite(n2)) {
        atomicOr(status, 2);
        return;
    }
    T inv = T(1) / sqrt(n2);
    m0[i] = a * inv;
    m1[i] = b * inv;
    m2[i] = c * inv;
}

template <typename T>
__global__ void he_interleave_kernel(T* __restrict__ dst, const T* __restrict__ a, const T* __restrict__ b,
                                     const T* __restrict__ c, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst[3 * i] = a[i];
    dst[3 * i + 1] = b[i];
    dst[3 * i + 2] = c[i];
}

__global__ void step_counter_kernel(long long* ctr) { *ctr += 1; }

}  // namespace sgspm
