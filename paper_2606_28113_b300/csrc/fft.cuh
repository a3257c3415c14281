// Shared-memory batched 1D transforms used by every pass:
//   * mixed-radix (8, 4, 2, 3, 5) Stockham FFT of many lines at once (out of place,
//     ping-pong between two buffers, one __syncthreads per stage);
//   * DCT-II / its inverse of real lines by Makhoul's permutation, two real lines packed
//     into one complex FFT (J. Makhoul, IEEE Trans. ASSP 28, 1980);
//   * zero-padded real-to-complex and complex-to-real transforms of real lines, again two
//     lines per complex FFT.
// Lines live in shared memory with an arbitrary line stride `ls` and element stride `es`;
// threads are mapped so that consecutive threads touch consecutive addresses.
#pragma once
#include "common.cuh"

namespace sgspm {

struct Lines {
    int n;   // number of lines
    int ls;  // line stride (elements)
    int es;  // element stride (elements)
};

// ---- radix-R butterflies (forward: exp(-2 pi i jk/R), inverse: exp(+2 pi i jk/R)) ------------
template <bool INV, typename V>
__device__ __forceinline__ V rot_i(V a) { return INV ? cmul_pi(a) : cmul_mi(a); }  // * (-i) fwd, (+i) inv

template <int R, bool INV, typename V> struct Bfly;

template <bool INV, typename V> struct Bfly<2, INV, V> {
    static __device__ __forceinline__ void run(V* a) {
        V t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    }
};

template <bool INV, typename V> struct Bfly<4, INV, V> {
    static __device__ __forceinline__ void run(V* a) {
        V t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
        V t2 = cadd(a[1], a[3]), t3 = rot_i<INV>(csub(a[1], a[3]));
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3);
        a[3] = csub(t1, t3);
    }
};

template <bool INV, typename V> struct Bfly<8, INV, V> {
    static __device__ __forceinline__ void run(V* a) {
        using T = decltype(V::x);
        const T h = T(0.70710678118654752440);
        V e[4] = {a[0], a[2], a[4], a[6]};
        V o[4] = {a[1], a[3], a[5], a[7]};
        Bfly<4, INV, V>::run(e);
        Bfly<4, INV, V>::run(o);
        // o[k] *= W8^k, W8 = exp(-+ i pi/4)
        V o1 = INV ? cmk<V>(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                   : cmk<V>(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        V o2 = rot_i<INV>(o[2]);
        V o3 = INV ? cmk<V>(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                   : cmk<V>(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
        a[0] = cadd(e[0], o[0]);
        a[4] = csub(e[0], o[0]);
        a[1] = cadd(e[1], o1);
        a[5] = csub(e[1], o1);
        a[2] = cadd(e[2], o2);
        a[6] = csub(e[2], o2);
        a[3] = cadd(e[3], o3);
        a[7] = csub(e[3], o3);
    }
};

template <bool INV, typename V> struct Bfly<3, INV, V> {
    static __device__ __forceinline__ void run(V* a) {
        using T = decltype(V::x);
        const T s3 = T(0.86602540378443864676);   // sin(2 pi / 3)
        V s = cadd(a[1], a[2]), d = csub(a[1], a[2]);
        V t = cmk<V>(a[0].x - T(0.5) * s.x, a[0].y - T(0.5) * s.y);
        V u = rot_i<INV>(cscale(d, s3));
        a[0] = cadd(a[0], s);
        a[1] = cadd(t, u);
        a[2] = csub(t, u);
    }
};

template <bool INV, typename V> struct Bfly<5, INV, V> {
    static __device__ __forceinline__ void run(V* a) {
        using T = decltype(V::x);
        const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);   // cos(2pi/5), cos(4pi/5)
        const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);    // sin(2pi/5), sin(4pi/5)
        V b1 = cadd(a[1], a[4]), b2 = cadd(a[2], a[3]);
        V d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
        V t1 = cmk<V>(a[0].x + c1 * b1.x + c2 * b2.x, a[0].y + c1 * b1.y + c2 * b2.y);
        V t2 = cmk<V>(a[0].x + c2 * b1.x + c1 * b2.x, a[0].y + c2 * b1.y + c1 * b2.y);
        V u1 = rot_i<INV>(cmk<V>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
        V u2 = rot_i<INV>(cmk<V>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
        a[0] = cadd(a[0], cadd(b1, b2));
        a[1] = cadd(t1, u1);
        a[4] = csub(t1, u1);
        a[2] = cadd(t2, u2);
        a[3] = csub(t2, u2);
    }
};

// One Stockham stage of radix R over all lines: src -> dst.
template <typename T, bool INV, int R>
__device__ __forceinline__ void stockham_stage(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst,
                                               int P, Lines L, int Ns, const cplx<T>* __restrict__ tw) {
    using V = cplx<T>;
    const int nb = P / R;
    const int total = L.n * nb;
    const int twstride = P / (Ns * R);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int line, j;
        if (L.es == 1) { line = idx / nb; j = idx - line * nb; }
        else { j = idx / L.n; line = idx - j * L.n; }
        const V* s = src + (long)line * L.ls;
        V* d = dst + (long)line * L.ls;
        const int k = j % Ns;
        V v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = s[(j + t * nb) * L.es];
        if (Ns > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) {
                V w = tw[k * t * twstride];
                if (INV) w = cconj(w);
                v[t] = cmul(v[t], w);
            }
        }
        Bfly<R, INV, V>::run(v);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) d[(base + t * Ns) * L.es] = v[t];
    }
}

// Full FFT of all lines.  Data starts in `a`; `b` is scratch of the same shape.  Returns the
// buffer holding the result (a or b).  Unnormalised in both directions.
template <typename T, bool INV>
__device__ cplx<T>* fft_lines(cplx<T>* a, cplx<T>* b, Lines L, const Plan& pl, const cplx<T>* __restrict__ twpool) {
    const cplx<T>* tw = twpool + pl.tw;
    int Ns = 1;
    for (int s = 0; s < pl.nst; ++s) {
        const int r = pl.radix[s];
        switch (r) {
            case 8: stockham_stage<T, INV, 8>(a, b, pl.P, L, Ns, tw); break;
            case 4: stockham_stage<T, INV, 4>(a, b, pl.P, L, Ns, tw); break;
            case 2: stockham_stage<T, INV, 2>(a, b, pl.P, L, Ns, tw); break;
            case 3: stockham_stage<T, INV, 3>(a, b, pl.P, L, Ns, tw); break;
            default: stockham_stage<T, INV, 5>(a, b, pl.P, L, Ns, tw); break;
        }
        __syncthreads();
        cplx<T>* t = a; a = b; b = t;
        Ns *= r;
    }
    return a;
}

// Makhoul permutation: position of input sample j in the reordered sequence v.
__device__ __forceinline__ int mk_pos(int j, int N) { return (j & 1) ? N - 1 - (j >> 1) : (j >> 1); }
// inverse: sample index stored at position n of v
__device__ __forceinline__ int mk_src(int n, int N) { return (n < (N + 1) / 2) ? 2 * n : 2 * (N - 1 - n) + 1; }

// Unnormalised DCT-II  X_k = sum_n x_n cos(pi k (2n+1) / (2N))  of L real lines (in place).
// R: real lines (R.ls / R.es strides, length N).  ca, cb: complex scratch of >= ceil(L/2) * N.
template <typename T>
__device__ void dct2_lines(T* R, Lines L, int N, cplx<T>* ca, cplx<T>* cb, const Plan& pl,
                           const cplx<T>* __restrict__ twpool) {
    using V = cplx<T>;
    const int npair = (L.n + 1) / 2;
    Lines C{npair, N, 1};
    for (int idx = threadIdx.x; idx < npair * N; idx += blockDim.x) {
        int p = idx / N, j = idx - p * N;
        T re = R[(2 * p) * L.ls + j * L.es];
        T im = (2 * p + 1 < L.n) ? R[(2 * p + 1) * L.ls + j * L.es] : T(0);
        ca[p * N + mk_pos(j, N)] = cmk<V>(re, im);
    }
    __syncthreads();
    V* res = fft_lines<T, false>(ca, cb, C, pl, twpool);
    const V* w4 = twpool + pl.tw4;
    for (int idx = threadIdx.x; idx < npair * N; idx += blockDim.x) {
        int p = idx / N, k = idx - p * N;
        V Z = res[p * N + k];
        V Zr = cconj(res[p * N + (k == 0 ? 0 : N - k)]);
        V w = w4[k];
        V va = cscale(cadd(Z, Zr), T(0.5));
        V vb = cscale(cmul_mi(csub(Z, Zr)), T(0.5));
        R[(2 * p) * L.ls + k * L.es] = w.x * va.x - w.y * va.y;
        if (2 * p + 1 < L.n) R[(2 * p + 1) * L.ls + k * L.es] = w.x * vb.x - w.y * vb.y;
    }
    __syncthreads();
}

// Inverse of dct2_lines up to a factor N (the caller folds 1/N into its scaling).
template <typename T>
__device__ void dct3_lines(T* R, Lines L, int N, cplx<T>* ca, cplx<T>* cb, const Plan& pl,
                           const cplx<T>* __restrict__ twpool) {
    using V = cplx<T>;
    const int npair = (L.n + 1) / 2;
    Lines C{npair, N, 1};
    const V* w4 = twpool + pl.tw4;
    for (int idx = threadIdx.x; idx < npair * N; idx += blockDim.x) {
        int p = idx / N, k = idx - p * N;
        const bool hasb = (2 * p + 1 < L.n);
        T xa = R[(2 * p) * L.ls + k * L.es];
        T xar = (k == 0) ? T(0) : R[(2 * p) * L.ls + (N - k) * L.es];
        T xb = hasb ? R[(2 * p + 1) * L.ls + k * L.es] : T(0);
        T xbr = (hasb && k != 0) ? R[(2 * p + 1) * L.ls + (N - k) * L.es] : T(0);
        V w = cconj(w4[k]);
        V va = cmul(w, cmk<V>(xa, -xar));
        V vb = cmul(w, cmk<V>(xb, -xbr));
        ca[p * N + k] = cmk<V>(va.x - vb.y, va.y + vb.x);
    }
    __syncthreads();
    V* res = fft_lines<T, true>(ca, cb, C, pl, twpool);
    for (int idx = threadIdx.x; idx < npair * N; idx += blockDim.x) {
        int p = idx / N, n = idx - p * N;
        V z = res[p * N + n];
        int j = mk_src(n, N);
        R[(2 * p) * L.ls + j * L.es] = z.x;
        if (2 * p + 1 < L.n) R[(2 * p + 1) * L.ls + j * L.es] = z.y;
    }
    __syncthreads();
}

// Zero-padded FFT of length P of L real lines of length nlen (P = 2 nlen, or 1).
// Leaves the packed complex transform of line pairs in the returned buffer, layout
// [pair][P]; extract line spectra with r2c_get.
template <typename T>
__device__ cplx<T>* r2c_lines(const T* R, Lines L, int nlen, cplx<T>* ca, cplx<T>* cb, const Plan& pl,
                              const cplx<T>* __restrict__ twpool) {
    using V = cplx<T>;
    const int P = pl.P;
    const int npair = (L.n + 1) / 2;
    for (int idx = threadIdx.x; idx < npair * P; idx += blockDim.x) {
        int p = idx / P, j = idx - p * P;
        V v = cmk<V>(T(0), T(0));
        if (j < nlen) {
            v.x = R[(2 * p) * L.ls + j * L.es];
            if (2 * p + 1 < L.n) v.y = R[(2 * p + 1) * L.ls + j * L.es];
        }
        ca[p * P + j] = v;
    }
    __syncthreads();
    return fft_lines<T, false>(ca, cb, Lines{npair, P, 1}, pl, twpool);
}

// Spectrum X_line[k], k in [0, P/2], of one real line from the packed pair transform.
template <typename T>
__device__ __forceinline__ cplx<T> r2c_get(const cplx<T>* res, int line, int k, int P) {
    using V = cplx<T>;
    const int p = line >> 1;
    V Z = res[p * P + k];
    V Zr = cconj(res[p * P + (k == 0 ? 0 : P - k)]);
    return (line & 1) ? cscale(cmul_mi(csub(Z, Zr)), T(0.5)) : cscale(cadd(Z, Zr), T(0.5));
}

// Pack half spectra (k in [0, P/2]) of a line pair into the full complex sequence whose
// inverse FFT has line 2p in the real part and line 2p+1 in the imaginary part.
// Writes positions k and P-k of pair p.  DC and Nyquist imaginary parts are dropped.
template <typename T>
__device__ __forceinline__ void c2r_put(cplx<T>* ca, int p, int k, int P, cplx<T> xa, cplx<T> xb) {
    using V = cplx<T>;
    if (k == 0 || 2 * k == P) { xa.y = T(0); xb.y = T(0); }
    ca[p * P + k] = cmk<V>(xa.x - xb.y, xa.y + xb.x);
    if (k != 0 && 2 * k != P) ca[p * P + (P - k)] = cmk<V>(xa.x + xb.y, xb.x - xa.y);
}

}  // namespace sgspm
