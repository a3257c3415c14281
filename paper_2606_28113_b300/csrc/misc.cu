// Energy reduction and small helper kernels (FP32 and FP64): dtype conversion, normalisation,
// applied-field interleave, step counter.  Included by capi.cu.
#pragma once
#include "common.cuh"

namespace sgspm {

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
        const int loc = wi.y + i;   // in-film offset (32 bits)
        const int z = loc / (int)sxy, r = loc - z * (int)sxy;
        const int y = r / nx, x = r - y * nx;
        long long c = F.off_cell + loc;
        const T* ml[3] = {d.flo[m0], d.flo[m0 + 1], d.flo[m0 + 2]};
        auto val = [&](int a, long long cc) -> double { return (double)m[a][cc] + (ml[a] ? (double)ml[a][cc] : 0.0); };
        double v[3] = {val(0, c), val(1, c), val(2, c)};
        for (int a = 0; a < 3; ++a) {
            if (x + 1 < nx) { double q = val(a, c + 1) - v[a]; ex += q * q * F.ih2[0]; }
            if (y + 1 < ny) { double q = val(a, c + nx) - v[a]; ex += q * q * F.ih2[1]; }
            if (z + 1 < nz) { double q = val(a, c + sxy) - v[a]; ex += q * q * F.ih2[2]; }
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
__global__ void copy_in_kernel(T* __restrict__ d0, T* __restrict__ d1, T* __restrict__ d2, T* __restrict__ l0,
                               T* __restrict__ l1, T* __restrict__ l2, const S* __restrict__ src,
                               const Film* films, int nfilm, long long ntot, int* status) {
    // src: concatenation over films of [3][ncell_f]; with status non-null (magnetisation) the
    // stored vector (hi + lo) is normalised, and a zero-length or non-finite one sets bit 2
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= ntot) return;
    int f = 0;
    while (f + 1 < nfilm && films[f + 1].off_cell <= i) ++f;
    const Film F = films[f];
    long long loc = i - F.off_cell;
    long long nc = (long long)F.nx * F.ny * F.nz;
    const S* s = src + 3 * F.off_cell;
    T* dd[3] = {d0, d1, d2};
    T* ll[3] = {l0, l1, l2};
    double v[3];
    for (int a = 0; a < 3; ++a) {
        const double x = (double)s[a * nc + loc];
        const T hi = (T)x, lo = (T)(x - (double)hi);
        v[a] = (double)hi + (ll[a] ? (double)lo : 0.0);
        if (!status) {
            dd[a][i] = hi;
            if (ll[a]) ll[a][i] = lo;
        }
    }
    if (!status) return;
    const double n2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    if (!(n2 > 0.0) || !isfinite(n2)) {
        atomicOr(status, 2);
        return;
    }
    const double inv = 1.0 / sqrt(n2);
    for (int a = 0; a < 3; ++a) {
        const double w = v[a] * inv;
        dd[a][i] = (T)w;
        if (ll[a]) ll[a][i] = (T)(w - (double)(T)w);
    }
}

template <typename T, typename S>
__global__ void copy_out_kernel(S* __restrict__ dst, const T* __restrict__ d0, const T* __restrict__ d1, const T* __restrict__ d2,
                                const T* __restrict__ l0, const T* __restrict__ l1, const T* __restrict__ l2,
                                const Film* films, int nfilm, long long ntot) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= ntot) return;
    int f = 0;
    while (f + 1 < nfilm && films[f + 1].off_cell <= i) ++f;
    const Film F = films[f];
    long long loc = i - F.off_cell;
    long long nc = (long long)F.nx * F.ny * F.nz;
    S* s = dst + 3 * F.off_cell;
    const T* dd[3] = {d0, d1, d2};
    const T* ll[3] = {l0, l1, l2};
    for (int a = 0; a < 3; ++a) s[a * nc + loc] = (S)((double)dd[a][i] + (ll[a] ? (double)ll[a][i] : 0.0));
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

namespace sgspm {

// FP64 FMA throughput probe: every thread runs kChains independent DFMA chains of `iters` steps
// (a x + b with |a| < 1, so values stay finite) and writes their sum, so nothing is optimised
// away.  2 * kChains * iters flops per thread.
constexpr int kFmaChains = 8;
__global__ void __launch_bounds__(256) fp64_fma_probe_kernel(int iters, double* __restrict__ out) {
    double v[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) v[c] = 1e-3 * (threadIdx.x + c);
    const double a = 0.999999, b = 1e-9;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) v[c] = fma(v[c], a, b);
    }
    double s = 0;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace sgspm
