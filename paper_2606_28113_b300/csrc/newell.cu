// FP64 set-up of the stray-field kernel: the Newell demagnetising tensor of a uniform cell
// grid and its zero-padded spectrum, evaluated once per handle on the device.
//
//   h_s(cell i) = -sum_j N(R_i - R_j) m_j,   N_ab(R) = (1/V) int_{cell i} int_{cell j} D_ab(x - y),
//   D_ab(r) = (delta_ab |r|^2 - 3 r_a r_b) / (4 pi |r|^5)          (Newell, Williams & Dunlop 1993)
//
// Near offsets (the two cells touch or overlap) use Newell's closed form, the triple second
// difference of his auxiliary functions f and g.  Every other offset uses the equivalent
// single integral over the cell-centre difference u, whose density is a product of three
// triangle functions, N_ab(R) = V int T(u) D_ab(R + u) du, by a tensor Gauss-Legendre rule on
// each half of every triangle; the rule's order falls with the cells' separation.  This
// avoids the catastrophic cancellation of the closed form at large |R|.
// Compiled as part of capi.cu (single translation unit).
#pragma once
#include <cmath>
#include "common.cuh"
#include "passes.cuh"

namespace sgspm {

__device__ double asinh_ratio(double num, double den2) { return den2 > 0 ? asinh(num / sqrt(den2)) : 0.0; }
__device__ double atan_ratio(double num, double den) { return den != 0 ? atan(num / den) : 0.0; }

__device__ double newell_f(double x, double y, double z) {
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    double t = 0.5 * y * (z2 - x2) * asinh_ratio(y, x2 + z2);
    t += 0.5 * z * (y2 - x2) * asinh_ratio(z, x2 + y2);
    t -= x * y * z * atan_ratio(y * z, x * R);
    t += (2.0 * x2 - y2 - z2) * R / 6.0;
    return t;
}

__device__ double newell_g(double x, double y, double z) {
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    double t = x * y * z * asinh_ratio(z, x2 + y2);
    t += y / 6.0 * (3.0 * z2 - y2) * asinh_ratio(x, y2 + z2);
    t += x / 6.0 * (3.0 * z2 - x2) * asinh_ratio(y, x2 + z2);
    t -= z2 * z / 6.0 * atan_ratio(x * y, z * R);
    t -= z * y2 / 2.0 * atan_ratio(x * z, y * R);
    t -= z * x2 / 2.0 * atan_ratio(y * z, x * R);
    t -= x * y * R / 3.0;
    return t;
}

// (1/(4 pi V)) prod_axes (2 - S+ - S-) applied to fun at (X, Y, Z)
template <bool G>
__device__ double second_difference(double X, double Y, double Z, double dx, double dy, double dz) {
    const double c[3] = {-1.0, 2.0, -1.0};
    double s = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                double w = c[i] * c[j] * c[k];
                double X1 = X + (i - 1) * dx, Y1 = Y + (j - 1) * dy, Z1 = Z + (k - 1) * dz;
                s += w * (G ? newell_g(X1, Y1, Z1) : newell_f(X1, Y1, Z1));
            }
    return s / (4.0 * M_PI * dx * dy * dz);
}

__device__ int quad_order(double dist) {
    return dist < 2 ? 14 : dist < 3 ? 8 : dist < 6 ? 7 : dist < 10 ? 6 : dist < 40 ? 5 : 4;
}

// out: [6][nz][ny][nx] for non-negative offsets (i dx, j dy, k dz)
__global__ void newell_octant_kernel(double* __restrict__ out, int nx, int ny, int nz, double dx, double dy, double dz, GLTable gl) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long n = (long long)nx * ny * nz;
    if (id >= n) return;
    int i = id % nx, j = (id / nx) % ny, k = id / ((long long)nx * ny);
    double X = i * dx, Y = j * dy, Z = k * dz;
    double gx = fmax(0.0, fabs(X) - dx), gy = fmax(0.0, fabs(Y) - dy), gz = fmax(0.0, fabs(Z) - dz);
    double dist = sqrt(gx * gx + gy * gy + gz * gz) / fmax(dx, fmax(dy, dz));
    double N[6];
    if (dist < 1.0) {
        N[0] = second_difference<false>(X, Y, Z, dx, dy, dz);
        N[1] = second_difference<false>(Y, X, Z, dy, dx, dz);
        N[2] = second_difference<false>(Z, Y, X, dz, dy, dx);
        N[3] = second_difference<true>(X, Y, Z, dx, dy, dz);
        N[4] = second_difference<true>(X, Z, Y, dx, dz, dy);
        N[5] = second_difference<true>(Y, Z, X, dy, dz, dx);
    } else {
        const int q = quad_order(dist);
        const double* gx_ = gl.x + gl.off[q];
        const double* gw_ = gl.w + gl.off[q];
        for (int c = 0; c < 6; ++c) N[c] = 0.0;
        // nodes of the unit-mass tent (h - |u|)/h^2 on [-h, h]: u = +-h (1 + x)/2, weight w h/2 (h - s)/h^2
        for (int a = 0; a < 2 * q; ++a) {
            int ia = a < q ? q - 1 - a : a - q;
            double sa = dx * (1.0 + gx_[ia]) * 0.5;
            double wa = gw_[ia] * 0.5 * (dx - sa) / dx;
            double ua = a < q ? -sa : sa;
            double rx = X + ua;
            for (int b = 0; b < 2 * q; ++b) {
                int ib = b < q ? q - 1 - b : b - q;
                double sb = dy * (1.0 + gx_[ib]) * 0.5;
                double wb = gw_[ib] * 0.5 * (dy - sb) / dy;
                double ry = Y + (b < q ? -sb : sb);
                double acc[6] = {0, 0, 0, 0, 0, 0};
                for (int cc = 0; cc < 2 * q; ++cc) {
                    int ic = cc < q ? q - 1 - cc : cc - q;
                    double sc = dz * (1.0 + gx_[ic]) * 0.5;
                    double wc = gw_[ic] * 0.5 * (dz - sc) / dz;
                    double rz = Z + (cc < q ? -sc : sc);
                    double r2 = rx * rx + ry * ry + rz * rz;
                    double inv5 = wc / (r2 * r2 * sqrt(r2));
                    acc[0] += (r2 - 3.0 * rx * rx) * inv5;
                    acc[1] += (r2 - 3.0 * ry * ry) * inv5;
                    acc[2] += (r2 - 3.0 * rz * rz) * inv5;
                    acc[3] += (-3.0 * rx * ry) * inv5;
                    acc[4] += (-3.0 * rx * rz) * inv5;
                    acc[5] += (-3.0 * ry * rz) * inv5;
                }
                for (int c = 0; c < 6; ++c) N[c] += wa * wb * acc[c];
            }
        }
        const double pref = dx * dy * dz / (4.0 * M_PI);
        for (int c = 0; c < 6; ++c) N[c] *= pref;
    }
    for (int c = 0; c < 6; ++c) out[c * n + id] = N[c];
}

// Parity of component c along axis a (0 x, 1 y, 2 z): true if odd.
__device__ __forceinline__ bool comp_odd(int c, int a) {
    // xx yy zz even everywhere; xy odd in x,y; xz odd in x,z; yz odd in y,z
    if (c < 3) return false;
    if (c == 3) return a != 2;
    if (c == 4) return a != 1;
    return a != 0;
}

// Separable transform of the octant along one axis.
//   even: T(k) = N(0) + 2 sum_{s>=1} N(s) cos(2 pi k s / P)
//   odd : T(k) = 2 sum_{s>=1} N(s) sin(2 pi k s / P)     (the factor (-i) per odd axis is applied at the end)
// in : [6][d2][d1][n]  (transformed axis innermost, length n)  -> out : [6][d2][d1][K]
// For the y and z axes the caller passes strides so that the same kernel walks them.
__global__ void newell_axis_kernel(const double* __restrict__ in, double* __restrict__ out, int axis, int n, int K, int P,
                                   int d1, int d2, long long in_s_elem, long long in_s1, long long in_s2, long long in_sc,
                                   long long out_s_elem, long long out_s1, long long out_s2, long long out_sc,
                                   const double* __restrict__ cs, const double* __restrict__ sn) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = 6LL * d2 * d1 * K;
    if (id >= total) return;
    int k = id % K;
    long long r = id / K;
    int i1 = r % d1;
    r /= d1;
    int i2 = r % d2;
    int c = r / d2;
    const double* src = in + c * in_sc + i2 * in_s2 + i1 * in_s1;
    bool odd = comp_odd(c, axis);
    double s = odd ? 0.0 : src[0];
    for (int t = 1; t < n; ++t) {
        int m = (int)(((long long)k * t) % P);
        s += 2.0 * src[t * in_s_elem] * (odd ? sn[m] : cs[m]);
    }
    out[c * out_sc + i2 * out_s2 + i1 * out_s1 + k * out_s_elem] = s;
}

// ktab[c][kz][kx][ky] = -(+-) N_hat / (Px Py Pz) from nhat[c][kz][ky][kx]: the two odd axes
// of an off-diagonal component contribute (-i)^2 = -1.
template <typename T>
__global__ void newell_finish_kernel(const double* __restrict__ nhat, T* __restrict__ ktab, int Kx, int Hy, int HyP, int Hz,
                                     double scale) {
    long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n6 = (long long)Hz * Hy * Kx;
    if (id >= 6 * n6) return;
    const int c = (int)(id / n6);
    long long r = id - c * n6;
    const int kx = (int)(r % Kx);
    r /= Kx;
    const int ky = (int)(r % Hy);
    const int kz = (int)(r / Hy);
    double v = nhat[id];
    if (c >= 3) v = -v;
    ktab[ktab_index(c, kx, kz, ky, Kx, HyP, Hz)] = (T)(-v * scale);
}

}  // namespace sgspm
