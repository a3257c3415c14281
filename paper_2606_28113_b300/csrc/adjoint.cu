// Reverse mode of one SGSPM step (Sec. 3.2) in the delta form used by the forward kernels.
// Compiled as part of capi.cu (single translation unit).
//
// Forward (per step): delta_i = S_c(scale (f_i(state) + eps Delta_h state_i)) with the symmetric
// operators S_c = (I - c dt Delta_h)^{-1} and Delta_h, the stray field H = -N* (symmetric), the
// Gauss-Seidel updates u = base + p q - r s, the damping update v = m** + delta and the
// projection m' = v / |v|.  The reverse of each piece is pointwise except for S_c and H, which
// reuse the forward solve and stray-field passes (both operators are their own adjoints).
#pragma once
#include "common.cuh"

namespace sgspm {

// per-cell work list over all films: (film, first cell, count)
struct AdjGS {
    int ub;                 // adjoint of the update's output
    int base_b;             // adjoint accumulators of the operands
    int p, p_b, q, q_b, r, r_b, s, s_b;
};

template <typename T>
__device__ __forceinline__ void film_cell(const Dev<T>& d, const int4& wi, int i, long long& c, int& x, int& y, int& z,
                                          const Film*& F) {
    F = &d.films[wi.x];
    // in-film offsets fit 32 bits (films are limited to 2^29 cells): 32-bit divisions
    const int loc = wi.y + i;
    const int nx = F->nx, sxy = F->nx * F->ny;
    z = loc / sxy;
    const int r = loc - z * sxy;
    y = r / nx;
    x = r - y * nx;
    c = F->off_cell + loc;
}

// u = base + p q - r s:  base_b += u_b, p_b += u_b q, q_b += u_b p, r_b -= u_b s, s_b -= u_b r
template <typename T>
__global__ void __launch_bounds__(kThreads) adj_gs_kernel(Dev<T> d, const int4* __restrict__ work, AdjGS g) {
    const int4 wi = work[blockIdx.x];
    const long long c0 = d.films[wi.x].off_cell + wi.y;
    T* ub = d.field[g.ub];
    T* bb = d.field[g.base_b];
    const T* p = d.field[g.p];
    const T* q = d.field[g.q];
    const T* r = d.field[g.r];
    const T* s = d.field[g.s];
    T* pb = d.field[g.p_b];
    T* qb = d.field[g.q_b];
    T* rb = d.field[g.r_b];
    T* sb = d.field[g.s_b];
    for (int i = threadIdx.x; i < wi.z; i += blockDim.x) {
        const long long c = c0 + i;
        const T u = ub[c];
        bb[c] += u;
        pb[c] += u * q[c];
        qb[c] += u * p[c];
        rb[c] -= u * s[c];
        sb[c] -= u * r[c];
    }
}

// Reverse of delta_a = S(scale (f_a(state) + eps Delta_h state_a)) after rho_b = S(delta_b):
//   fb_a = scale rho_b;  heb_a += fb_a;  state_b[a] += scale eps Delta_h rho_b;
//   state_b[k] += -Q (fb_k - (fb . u) u_k)   (anisotropy; fb is zero outside the listed components)
struct AdjF {
    int n;                  // components in the list
    int comp[3];
    int rho[3];             // rho_b slot of each listed component
    int fb[3];              // f_b output slot of each listed component
    int sb[3];              // adjoint slots of the state components 1, 2, 3
    int heb;                // first of the three h_e adjoint slots (heb, heb+1, heb+2)
    int damp;               // scale = alpha dt (1) or dt (0)
};

template <typename T>
__global__ void __launch_bounds__(kThreads) adj_f_kernel(Dev<T> d, const int4* __restrict__ work, AdjF a) {
    const int4 wi = work[blockIdx.x];
    const Film& F = d.films[wi.x];
    const int nx = F.nx, ny = F.ny, nz = F.nz;
    const T scale = T(a.damp ? F.alpha * F.dt : F.dt);
    const T eps = T(F.eps), Q = T(F.Q);
    const T ihx = T(1.0 / (F.hx * F.hx)), ihy = T(1.0 / (F.hy * F.hy)), ihz = T(1.0 / (F.hz * F.hz));
    const T u[3] = {T(F.u[0]), T(F.u[1]), T(F.u[2])};
    const long long sxy = (long long)nx * ny;
    for (int i = threadIdx.x; i < wi.z; i += blockDim.x) {
        const int loc = wi.y + i;
        const int z = loc / (int)sxy, r = loc - z * (int)sxy, y = r / nx, x = r - y * nx;
        const long long c = F.off_cell + loc;
        T fb[3] = {T(0), T(0), T(0)};
        for (int k = 0; k < a.n; ++k) {
            const int comp = a.comp[k];
            const T* rho = d.field[a.rho[k]];
            const T rc = rho[c];
            T lap = T(0);
            if (nx > 1) lap += ihx * ((x + 1 < nx ? rho[c + 1] - rc : T(0)) + (x > 0 ? rho[c - 1] - rc : T(0)));
            if (ny > 1) lap += ihy * ((y + 1 < ny ? rho[c + nx] - rc : T(0)) + (y > 0 ? rho[c - nx] - rc : T(0)));
            if (nz > 1) lap += ihz * ((z + 1 < nz ? rho[c + sxy] - rc : T(0)) + (z > 0 ? rho[c - sxy] - rc : T(0)));
            fb[comp] = scale * rc;
            d.field[a.fb[k]][c] = fb[comp];
            d.field[a.heb + comp][c] += fb[comp];
            d.field[a.sb[comp]][c] += scale * eps * lap;
        }
        const T fu = fb[0] * u[0] + fb[1] * u[1] + fb[2] * u[2];
        for (int k = 0; k < 3; ++k) d.field[a.sb[k]][c] += -Q * (fb[k] - fu * u[k]);
    }
}

// dst[k] += src[k] (k < n), or dst = 0 (src < 0), or dst = src copy (mode 2)
struct AdjEw {
    int n;
    int mode;               // 0 add, 1 zero, 2 copy
    int dst[16];
    int src[16];
};

template <typename T>
__global__ void __launch_bounds__(kThreads) adj_ew_kernel(Dev<T> d, const int4* __restrict__ work, AdjEw e) {
    const int4 wi = work[blockIdx.x];
    const long long c0 = d.films[wi.x].off_cell + wi.y;
    for (int k = 0; k < e.n; ++k) {
        T* dst = d.field[e.dst[k]];
        const T* src = e.mode == 1 ? nullptr : d.field[e.src[k]];
        for (int i = threadIdx.x; i < wi.z; i += blockDim.x) {
            const long long c = c0 + i;
            if (e.mode == 0) dst[c] += src[c];
            else if (e.mode == 1) dst[c] = T(0);
            else dst[c] = src[c];
        }
    }
}

// Projection m' = v / |v|:  v_b = (g - (m'.g) m') / |v|;  the damping update v = E + delta passes
// v_b on to E's adjoint (eb) and to the damping solve's input (vb).
struct AdjProj {
    int g[3], mn[3], v[3], vb[3], eb[3];
};

template <typename T>
__global__ void __launch_bounds__(kThreads) adj_proj_kernel(Dev<T> d, const int4* __restrict__ work, AdjProj p) {
    const int4 wi = work[blockIdx.x];
    const long long c0 = d.films[wi.x].off_cell + wi.y;
    for (int i = threadIdx.x; i < wi.z; i += blockDim.x) {
        const long long c = c0 + i;
        T g[3], m[3], v[3];
        for (int k = 0; k < 3; ++k) {
            g[k] = d.field[p.g[k]][c];
            m[k] = d.field[p.mn[k]][c];
            v[k] = d.field[p.v[k]][c];
        }
        const T inv = T(1) / sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const T mg = m[0] * g[0] + m[1] * g[1] + m[2] * g[2];
        for (int k = 0; k < 3; ++k) {
            const T vb = (g[k] - mg * m[k]) * inv;
            d.field[p.vb[k]][c] = vb;
            d.field[p.eb[k]][c] += vb;
        }
    }
}

// d L / d alpha of one step: sum_cells sum_i rho_i (dt f_i(E) + eps dt Delta_h v_i), with
// rho = S_{alpha eps}(v_b), E = m** (its h_s recorded), v = m***.  Block partials (FP64).
struct AdjAlpha {
    int rho[3], e[3], hs[3], v[3];
    int have_hs;
};

template <typename T>
__global__ void __launch_bounds__(kThreads) adj_alpha_partial_kernel(Dev<T> d, const int4* __restrict__ work, AdjAlpha a,
                                                                     double* __restrict__ part) {
    const int4 wi = work[blockIdx.x];
    const Film& F = d.films[wi.x];
    const int nx = F.nx, ny = F.ny, nz = F.nz;
    const long long sxy = (long long)nx * ny;
    const double ihx = F.ih2[0], ihy = F.ih2[1], ihz = F.ih2[2];
    double acc = 0.0;
    for (int i = threadIdx.x; i < wi.z; i += blockDim.x) {
        const int loc = wi.y + i;
        const int z = loc / (int)sxy, r = loc - z * (int)sxy, y = r / nx, x = r - y * nx;
        const long long c = F.off_cell + loc;
        double e[3];
        for (int k = 0; k < 3; ++k) e[k] = (double)d.field[a.e[k]][c];
        const double mu = e[0] * F.u[0] + e[1] * F.u[1] + e[2] * F.u[2];
        for (int k = 0; k < 3; ++k) {
            const T* v = d.field[a.v[k]];
            const double vc = (double)v[c];
            double lap = 0.0;
            if (nx > 1) lap += ihx * ((x + 1 < nx ? v[c + 1] - vc : 0.0) + (x > 0 ? v[c - 1] - vc : 0.0));
            if (ny > 1) lap += ihy * ((y + 1 < ny ? v[c + nx] - vc : 0.0) + (y > 0 ? v[c - nx] - vc : 0.0));
            if (nz > 1) lap += ihz * ((z + 1 < nz ? v[c + sxy] - vc : 0.0) + (z > 0 ? v[c - sxy] - vc : 0.0));
            const double he = d.he_cell ? (double)d.he_cell[c * 3 + k] : F.he[k];
            const double hs = a.have_hs ? (double)d.field[a.hs[k]][c] : 0.0;
            const double f = -F.Q * (e[k] - mu * F.u[k]) + hs + he;
            acc += (double)d.field[a.rho[k]][c] * (F.dt * f + F.eps * F.dt * lap);
        }
    }
    __shared__ double red[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void adj_alpha_final_kernel(int nfilm, const int* __restrict__ first_block, const double* __restrict__ part,
                                       double* __restrict__ alpha_b) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfilm) return;
    double s = 0;
    for (int b = first_block[f]; b < first_block[f + 1]; ++b) s += part[b];
    alpha_b[f] += s;
}

// The recorded real slots 0 .. nslot-1 (hi parts) of one step <-> buf [nslot][n]; slot pointers
// from the device slot table; blockIdx.y is the slot
template <typename T>
__global__ void slots_io_kernel(T* __restrict__ buf, void* const* __restrict__ tab, long long n, int save) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    T* f = static_cast<T*>(tab[blockIdx.y]);
    T* b = buf + blockIdx.y * n;
    if (save) b[i] = f[i];
    else f[i] = b[i];
}

// state (hi, lo) <-> a flat buffer; lo may be null (FP64 form)
template <typename T>
__global__ void state_copy_kernel(T* __restrict__ dst_hi, T* __restrict__ dst_lo, const T* __restrict__ src_hi,
                                  const T* __restrict__ src_lo, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst_hi[i] = src_hi[i];
    if (dst_lo) dst_lo[i] = src_lo ? src_lo[i] : T(0);
}

}  // namespace sgspm
