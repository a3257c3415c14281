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
        constexpr double h = 0.70710678118654752440;
        V e[4] = {a[0], a[2], a[4], a[6]};
        V o[4] = {a[1], a[3], a[5], a[7]};
        Bfly<4, INV, V>::run(e);
        Bfly<4, INV, V>::run(o);
        // o[k] *= W8^k, W8 = exp(-+ i pi/4)
        V o1 = INV ? cmk<V>(kmul<T>(o[1].x - o[1].y, h), kmul<T>(o[1].x + o[1].y, h))
                   : cmk<V>(kmul<T>(o[1].x + o[1].y, h), kmul<T>(o[1].y - o[1].x, h));
        V o2 = rot_i<INV>(o[2]);
        V o3 = INV ? cmk<V>(-kmul<T>(o[3].x + o[3].y, h), kmul<T>(o[3].x - o[3].y, h))
                   : cmk<V>(kmul<T>(o[3].y - o[3].x, h), -kmul<T>(o[3].x + o[3].y, h));
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

template <bool INV, typename V> struct Bfly<16, INV, V> {
    // 16 = 4 x 4: DFT4 over m of a[r + 4m], twiddle W16^{rs}, DFT4 over r; X[s + 4t]
    static __device__ __forceinline__ void run(V* a) {
        constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173, h = 0.70710678118654752440;
        V b[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            V q[4] = {a[r], a[r + 4], a[r + 8], a[r + 12]};
            Bfly<4, INV, V>::run(q);
#pragma unroll
            for (int s = 0; s < 4; ++s) b[r][s] = q[s];
        }
        // W16^k = (cos(2 pi k/16), -+ sin(2 pi k/16)) for k = r*s in {1,2,3,4,6,9}
        constexpr double sg = INV ? 1.0 : -1.0;
        b[1][1] = cmulk(b[1][1], c1, sg * s1);
        b[1][2] = cmulk(b[1][2], h, sg * h);
        b[1][3] = cmulk(b[1][3], s1, sg * c1);
        b[2][1] = cmulk(b[2][1], h, sg * h);
        b[2][2] = rot_i<INV>(b[2][2]);
        b[2][3] = cmulk(b[2][3], -h, sg * h);
        b[3][1] = cmulk(b[3][1], s1, sg * c1);
        b[3][2] = cmulk(b[3][2], -h, sg * h);
        b[3][3] = cmulk(b[3][3], -c1, -sg * s1);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            V q[4] = {b[0][s], b[1][s], b[2][s], b[3][s]};
            Bfly<4, INV, V>::run(q);
#pragma unroll
            for (int t = 0; t < 4; ++t) a[s + 4 * t] = q[t];
        }
    }
};

template <bool INV, typename V> struct Bfly<3, INV, V> {
    static __device__ __forceinline__ void run(V* a) {
        using T = decltype(V::x);
        constexpr double s3 = 0.86602540378443864676;   // sin(2 pi / 3)
        V s = cadd(a[1], a[2]), d = csub(a[1], a[2]);
        V t = cmk<V>(a[0].x - T(0.5) * s.x, a[0].y - T(0.5) * s.y);
        V u = rot_i<INV>(cmk<V>(kmul<T>(d.x, s3), kmul<T>(d.y, s3)));
        a[0] = cadd(a[0], s);
        a[1] = cadd(t, u);
        a[2] = csub(t, u);
    }
};

template <bool INV, typename V> struct Bfly<5, INV, V> {
    static __device__ __forceinline__ void run(V* a) {
        using T = decltype(V::x);
        constexpr double c1 = 0.30901699437494742410, c2 = -0.80901699437494742410;   // cos(2pi/5), cos(4pi/5)
        constexpr double s1 = 0.95105651629515357212, s2 = 0.58778525229247312917;    // sin(2pi/5), sin(4pi/5)
        V b1 = cadd(a[1], a[4]), b2 = cadd(a[2], a[3]);
        V d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
        V t1 = cmk<V>(a[0].x + kmul<T>(b1.x, c1) + kmul<T>(b2.x, c2), a[0].y + kmul<T>(b1.y, c1) + kmul<T>(b2.y, c2));
        V t2 = cmk<V>(a[0].x + kmul<T>(b1.x, c2) + kmul<T>(b2.x, c1), a[0].y + kmul<T>(b1.y, c2) + kmul<T>(b2.y, c1));
        V u1 = rot_i<INV>(cmk<V>(kmul<T>(d1.x, s1) + kmul<T>(d2.x, s2), kmul<T>(d1.y, s1) + kmul<T>(d2.y, s2)));
        V u2 = rot_i<INV>(cmk<V>(kmul<T>(d1.x, s2) - kmul<T>(d2.x, s1), kmul<T>(d1.y, s2) - kmul<T>(d2.y, s1)));
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
                                               int P, Lines L, int Ns, const tw_t<T>* __restrict__ tw) {
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
            for (int t = 1; t < R; ++t) v[t] = twmul<INV>(v[t], tw[k * t * twstride]);
        }
        Bfly<R, INV, V>::run(v);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) d[(base + t * Ns) * L.es] = v[t];
    }
}

// ---- compile-time Stockham for power-of-two lengths: all index arithmetic folds to shifts ----
template <typename T, bool INV, int P, int R, int NS, bool CONTIG>
__device__ __forceinline__ void ct_stage(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst, Lines L,
                                         const tw_t<T>* __restrict__ tw) {
    using V = cplx<T>;
    constexpr int NB = P / R;
    constexpr int TWS = P / (NS * R);
    const int total = L.n * NB;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int line, j;
        if (CONTIG) { line = idx / NB; j = idx % NB; }
        else { j = idx / L.n; line = idx - j * L.n; }
        const int es = CONTIG ? 1 : L.es;
        const V* s = src + (long)line * L.ls;
        V* d = dst + (long)line * L.ls;
        const int k = j % NS;
        V v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = s[(j + t * NB) * es];
        if (NS > 1) {
#pragma unroll
            for (int t = 1; t < R; ++t) v[t] = twmul<INV>(v[t], tw[k * t * TWS]);
        }
        Bfly<R, INV, V>::run(v);
        const int base = (j / NS) * NS * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) d[(base + t * NS) * es] = v[t];
    }
}

__host__ __device__ constexpr int ct_radix(int rem) { return rem % 16 == 0 ? 16 : rem % 8 == 0 ? 8 : rem % 4 == 0 ? 4 : 2; }

template <typename T, bool INV, int P, int NS, bool CONTIG>
struct CtFFT {
    static __device__ __forceinline__ cplx<T>* run(cplx<T>* a, cplx<T>* b, Lines L, const tw_t<T>* tw) {
        constexpr int R = ct_radix(P / NS);
        ct_stage<T, INV, P, R, NS, CONTIG>(a, b, L, tw);
        __syncthreads();
        return CtFFT<T, INV, P, NS * R, CONTIG>::run(b, a, L, tw);
    }
};
template <typename T, bool INV, int P, bool CONTIG>
struct CtFFT<T, INV, P, P, CONTIG> {
    static __device__ __forceinline__ cplx<T>* run(cplx<T>* a, cplx<T>*, Lines, const tw_t<T>*) { return a; }
};

template <typename T, bool INV, int P>
__device__ __forceinline__ cplx<T>* ct_fft(cplx<T>* a, cplx<T>* b, Lines L, const tw_t<T>* tw) {
    if (L.es == 1) return CtFFT<T, INV, P, 1, true>::run(a, b, L, tw);
    return CtFFT<T, INV, P, 1, false>::run(a, b, L, tw);
}

// ---- warp-per-line FFT, P = 32 E (E = 2..16), natural order in and out --------------------------
// Lane j holds x[j + 32k] (k < E): E-point DFT in registers, twiddle W_P^{jq}; one transpose through
// the line's scratch region (XOR swizzle, conflict-free); lane (q, g) (G = 32/E lanes per q) takes
// y_{g + G i}[q], E-point DFT over i, twiddle W_32^{g s1}, then a G-point DIF across the G lanes by
// shuffles, which leaves X[q + E (s1 + E bitrev(g))] in lane (q, g).  Only __syncwarp inside.
// TS: stride into the twiddle table (a table of W_{TS P} serves a P-point FFT with TS > 1)
template <typename T, bool INV, int E, int TS = 1>
__device__ __forceinline__ void warp_fft_line(cplx<T>* __restrict__ a, cplx<T>* __restrict__ scr,
                                              const tw_t<T>* __restrict__ tw, int lane) {
    using V = cplx<T>;
    constexpr int P = 32 * E, G = 32 / E;
    V v[E];
#pragma unroll
    for (int k = 0; k < E; ++k) v[k] = a[lane + 32 * k];
    Bfly<E, INV, V>::run(v);
#pragma unroll
    for (int q = 1; q < E; ++q) v[q] = twmul<INV>(v[q], tw[TS * (lane * q)]);
#pragma unroll
    for (int q = 0; q < E; ++q) scr[q * 32 + (lane ^ ((q * G) & 31))] = v[q];
    __syncwarp();
    const int q = lane / G, g = lane % G;
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = scr[q * 32 + ((g + G * i) ^ ((q * G) & 31))];
    Bfly<E, INV, V>::run(v);
    if (G > 1) {
#pragma unroll
        for (int s1 = 1; s1 < E; ++s1) v[s1] = twmul<INV>(v[s1], tw[TS * (E * g * s1)]);
    }
#pragma unroll
    for (int d = G / 2; d >= 1; d >>= 1) {
        const bool top = (g & d) == 0;
        const tw_t<T> w = tw[TS * ((P / (2 * d)) * (g % d))];
#pragma unroll
        for (int s1 = 0; s1 < E; ++s1) {
            V pv;
            pv.x = __shfl_xor_sync(0xffffffffu, v[s1].x, d);
            pv.y = __shfl_xor_sync(0xffffffffu, v[s1].y, d);
            v[s1] = top ? cadd(v[s1], pv) : twmul<INV>(csub(pv, v[s1]), w);
        }
    }
    const int s2 = G > 1 ? (int)(__brev((unsigned)g) >> (32 - __ffs(G) + 1)) : 0;
#pragma unroll
    for (int s1 = 0; s1 < E; ++s1) a[q + E * (s1 + E * s2)] = v[s1];
}

// Register-resident forward FFT of one line held by a warp: on entry v[k] = x[lane + 32k];
// on exit v[s1] = X[q + E (s1 + E bitrev_G(g))] with q = lane / G, g = lane % G.
template <typename T, int E, bool LO = true>
__device__ __forceinline__ void wreg_fwd(cplx<T> (&v)[E], cplx<T>* __restrict__ scr, const tw_t<T>* __restrict__ tw, int lane) {
    using V = cplx<T>;
    constexpr int P = 32 * E, G = 32 / E;
    Bfly<E, false, V>::run(v);
#pragma unroll
    for (int q = 1; q < E; ++q) v[q] = twmul_p<false, LO>(v[q], tw[lane * q]);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < E; ++q) scr[q * 32 + (lane ^ ((q * G) & 31))] = v[q];
    __syncwarp();
    const int q = lane / G, g = lane % G;
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = scr[q * 32 + ((g + G * i) ^ ((q * G) & 31))];
    Bfly<E, false, V>::run(v);
    if (G > 1) {
#pragma unroll
        for (int s1 = 1; s1 < E; ++s1) v[s1] = twmul_p<false, LO>(v[s1], tw[E * g * s1]);
    }
#pragma unroll
    for (int d = G / 2; d >= 1; d >>= 1) {
        const bool top = (g & d) == 0;
        const tw_t<T> w = tw[(P / (2 * d)) * (g % d)];
#pragma unroll
        for (int s1 = 0; s1 < E; ++s1) {
            V pv;
            pv.x = __shfl_xor_sync(0xffffffffu, v[s1].x, d);
            pv.y = __shfl_xor_sync(0xffffffffu, v[s1].y, d);
            v[s1] = top ? cadd(v[s1], pv) : twmul_p<false, LO>(csub(pv, v[s1]), w);
        }
    }
}

// The adjoint of wreg_fwd: from the scrambled order back to v[k] = P * IDFT(X)[lane + 32k].
template <typename T, int E, bool LO = true>
__device__ __forceinline__ void wreg_adj(cplx<T> (&v)[E], cplx<T>* __restrict__ scr, const tw_t<T>* __restrict__ tw, int lane) {
    using V = cplx<T>;
    constexpr int P = 32 * E, G = 32 / E;
    const int q = lane / G, g = lane % G;
#pragma unroll
    for (int d = 1; d <= G / 2; d <<= 1) {
        const bool top = (g & d) == 0;
        const tw_t<T> w = tw[(P / (2 * d)) * (g % d)];   // used conjugated
#pragma unroll
        for (int s1 = 0; s1 < E; ++s1) {
            V pv;
            pv.x = __shfl_xor_sync(0xffffffffu, v[s1].x, d);
            pv.y = __shfl_xor_sync(0xffffffffu, v[s1].y, d);
            v[s1] = top ? cadd(v[s1], twmul_p<true, LO>(pv, w)) : csub(pv, twmul_p<true, LO>(v[s1], w));
        }
    }
    if (G > 1) {
#pragma unroll
        for (int s1 = 1; s1 < E; ++s1) v[s1] = twmul_p<true, LO>(v[s1], tw[E * g * s1]);
    }
    Bfly<E, true, V>::run(v);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < E; ++i) scr[q * 32 + ((g + G * i) ^ ((q * G) & 31))] = v[i];
    __syncwarp();
#pragma unroll
    for (int qq = 0; qq < E; ++qq) v[qq] = scr[qq * 32 + (lane ^ ((qq * G) & 31))];
#pragma unroll
    for (int qq = 1; qq < E; ++qq) v[qq] = twmul_p<true, LO>(v[qq], tw[lane * qq]);
    Bfly<E, true, V>::run(v);
}

__device__ __forceinline__ int bitrev_lanes(int g, int G) {
    return G > 1 ? (int)(__brev((unsigned)g) >> (33 - __ffs(G))) : 0;
}

template <typename T, bool INV, int E>
__device__ __forceinline__ cplx<T>* warp_fft(cplx<T>* a, cplx<T>* b, Lines L, const tw_t<T>* tw) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int line = threadIdx.x >> 5; line < L.n; line += nw)
        warp_fft_line<T, INV, E>(a + (long)line * L.ls, b + (long)line * L.ls, tw, lane);
    __syncthreads();
    return a;
}

// Full FFT of all lines.  Data starts in `a`; `b` is scratch of the same shape.  Returns the
// buffer holding the result (a or b).  Unnormalised in both directions.  Contiguous lines of
// length 64..512 use the warp-per-line FFT; other power-of-two lengths up to 2048 the
// compile-time Stockham; other lengths the generic mixed-radix Stockham.
template <typename T, bool INV>
__device__ cplx<T>* fft_lines(cplx<T>* a, cplx<T>* b, Lines L, const Plan& pl, const tw_t<T>* __restrict__ twpool) {
    const tw_t<T>* tw = twpool + pl.tw;
    if (L.es == 1 && L.ls >= pl.P) {
        switch (pl.P) {
            case 64: return warp_fft<T, INV, 2>(a, b, L, tw);
            case 128: return warp_fft<T, INV, 4>(a, b, L, tw);
            case 256: return warp_fft<T, INV, 8>(a, b, L, tw);
            case 512: return warp_fft<T, INV, 16>(a, b, L, tw);
            default: break;
        }
    }
    switch (pl.P) {
        case 1: return a;
        case 2: return ct_fft<T, INV, 2>(a, b, L, tw);
        case 4: return ct_fft<T, INV, 4>(a, b, L, tw);
        case 8: return ct_fft<T, INV, 8>(a, b, L, tw);
        case 16: return ct_fft<T, INV, 16>(a, b, L, tw);
        case 32: return ct_fft<T, INV, 32>(a, b, L, tw);
        case 64: return ct_fft<T, INV, 64>(a, b, L, tw);
        case 128: return ct_fft<T, INV, 128>(a, b, L, tw);
        case 256: return ct_fft<T, INV, 256>(a, b, L, tw);
        case 512: return ct_fft<T, INV, 512>(a, b, L, tw);
        case 1024: return ct_fft<T, INV, 1024>(a, b, L, tw);
        case 2048: return ct_fft<T, INV, 2048>(a, b, L, tw);
        default: break;
    }
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

// FFT of all lines with the length known at compile time (PC > 0), or the runtime path (PC = 0).
template <typename T, bool INV, int PC>
__device__ __forceinline__ cplx<T>* fft_lines_t(cplx<T>* a, cplx<T>* b, Lines L, const Plan& pl, const tw_t<T>* __restrict__ twpool) {
    if constexpr (PC == 0) {
        return fft_lines<T, INV>(a, b, L, pl, twpool);
    } else if constexpr (PC == 1) {
        return a;
    } else {
        const tw_t<T>* tw = twpool + pl.tw;
        if constexpr (PC >= 64 && PC <= 512) {
            if (L.es == 1 && L.ls >= PC) return warp_fft<T, INV, PC / 32>(a, b, L, tw);
        }
        return ct_fft<T, INV, PC>(a, b, L, tw);
    }
}

// Makhoul permutation: position of input sample j in the reordered sequence v.
__device__ __forceinline__ int mk_pos(int j, int N) { return (j & 1) ? N - 1 - (j >> 1) : (j >> 1); }
// inverse: sample index stored at position n of v
__device__ __forceinline__ int mk_src(int n, int N) { return (n < (N + 1) / 2) ? 2 * n : 2 * (N - 1 - n) + 1; }
// even/odd split of a packed pair p: position k of the pair's length-2N sequence sits at line
// 2p + (k & 1), index k >> 1, of an [2 pairs][N] layout
__device__ __forceinline__ int half_pos(int p, int k, int N) { return (2 * p + (k & 1)) * N + (k >> 1); }

// Unnormalised DCT-II  X_k = sum_n x_n cos(pi k (2n+1) / (2N))  of L real lines (in place).
// R: real lines (R.ls / R.es strides, length N).  ca, cb: complex scratch of >= ceil(L/2) * N.
template <typename T, int PC = 0>
__device__ void dct2_lines(T* R, Lines L, int N, cplx<T>* ca, cplx<T>* cb, const Plan& pl,
                           const tw_t<T>* __restrict__ twpool) {
    using V = cplx<T>;
    const int npair = (L.n + 1) / 2;
    if constexpr (PC >= 128 && PC <= 1024) {
        // the N-point FFT of each packed pair split by decimation in time into two N/2-point warp
        // FFTs (even and odd positions), so twice as many warps run half as long
        constexpr int H = PC / 2;
        const tw_t<T>* tw = twpool + pl.tw;   // W_N; the half-length FFTs read it with stride 2
        for (int idx = threadIdx.x; idx < npair * PC; idx += blockDim.x) {
            int p = idx / PC, j = idx - p * PC;
            T re = R[(2 * p) * L.ls + j * L.es];
            T im = (2 * p + 1 < L.n) ? R[(2 * p + 1) * L.ls + j * L.es] : T(0);
            ca[half_pos(p, mk_pos(j, PC), H)] = cmk<V>(re, im);
        }
        __syncthreads();
        {
            const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
            for (int line = threadIdx.x >> 5; line < 2 * npair; line += nw)
                warp_fft_line<T, false, H / 32, 2>(ca + line * H, cb + line * H, tw, lane);
            __syncthreads();
        }
        const tw_t<T>* w4 = twpool + pl.tw4;
        auto zat = [&](int p, int k) {   // Z[k] = E[k'] +- W_N^k' O[k'],  k' = k mod H
            const int k2 = k < H ? k : k - H;
            const V e = ca[(2 * p) * H + k2], o = twmul(ca[(2 * p + 1) * H + k2], tw[k2]);
            return k < H ? cadd(e, o) : csub(e, o);
        };
        for (int idx = threadIdx.x; idx < npair * PC; idx += blockDim.x) {
            int p = idx / PC, k = idx - p * PC;
            V Z = zat(p, k);
            V Zr = cconj(zat(p, k == 0 ? 0 : PC - k));
            const tw_t<T> w = w4[k];
            V va = cscale(cadd(Z, Zr), T(0.5));
            V vb = cscale(cmul_mi(csub(Z, Zr)), T(0.5));
            R[(2 * p) * L.ls + k * L.es] = twmul(va, w).x;
            if (2 * p + 1 < L.n) R[(2 * p + 1) * L.ls + k * L.es] = twmul(vb, w).x;
        }
        __syncthreads();
        return;
    }
    Lines C{npair, N, 1};
    for (int idx = threadIdx.x; idx < npair * N; idx += blockDim.x) {
        int p = idx / N, j = idx - p * N;
        T re = R[(2 * p) * L.ls + j * L.es];
        T im = (2 * p + 1 < L.n) ? R[(2 * p + 1) * L.ls + j * L.es] : T(0);
        ca[p * N + mk_pos(j, N)] = cmk<V>(re, im);
    }
    __syncthreads();
    V* res = fft_lines_t<T, false, PC>(ca, cb, C, pl, twpool);
    const tw_t<T>* w4 = twpool + pl.tw4;
    for (int idx = threadIdx.x; idx < npair * N; idx += blockDim.x) {
        int p = idx / N, k = idx - p * N;
        V Z = res[p * N + k];
        V Zr = cconj(res[p * N + (k == 0 ? 0 : N - k)]);
        const tw_t<T> w = w4[k];
        V va = cscale(cadd(Z, Zr), T(0.5));
        V vb = cscale(cmul_mi(csub(Z, Zr)), T(0.5));
        R[(2 * p) * L.ls + k * L.es] = twmul(va, w).x;
        if (2 * p + 1 < L.n) R[(2 * p + 1) * L.ls + k * L.es] = twmul(vb, w).x;
    }
    __syncthreads();
}

// Inverse of dct2_lines up to a factor N (the caller folds 1/N into its scaling).
template <typename T, int PC = 0>
__device__ void dct3_lines(T* R, Lines L, int N, cplx<T>* ca, cplx<T>* cb, const Plan& pl,
                           const tw_t<T>* __restrict__ twpool) {
    using V = cplx<T>;
    const int npair = (L.n + 1) / 2;
    if constexpr (PC >= 128 && PC <= 1024) {
        // inverse N-point FFT split by decimation in frequency into two N/2-point warp FFTs:
        // z[2m] from C[k] + C[k+H], z[2m+1] from (C[k] - C[k+H]) conj(W_N^k)
        constexpr int H = PC / 2;
        const tw_t<T>* tw = twpool + pl.tw;
        const tw_t<T>* w4 = twpool + pl.tw4;
        auto cat = [&](int p, int k) {   // the packed pre-twiddled spectrum C[k] of pair p
            const bool hasb = (2 * p + 1 < L.n);
            T xa = R[(2 * p) * L.ls + k * L.es];
            T xar = (k == 0) ? T(0) : R[(2 * p) * L.ls + (PC - k) * L.es];
            T xb = hasb ? R[(2 * p + 1) * L.ls + k * L.es] : T(0);
            T xbr = (hasb && k != 0) ? R[(2 * p + 1) * L.ls + (PC - k) * L.es] : T(0);
            const tw_t<T> w = w4[k];   // used conjugated
            V va = twmul<true>(cmk<V>(xa, -xar), w);
            V vb = twmul<true>(cmk<V>(xb, -xbr), w);
            return cmk<V>(va.x - vb.y, va.y + vb.x);
        };
        for (int idx = threadIdx.x; idx < npair * H; idx += blockDim.x) {
            int p = idx / H, k = idx - p * H;
            const V c0 = cat(p, k), c1 = cat(p, k + H);
            ca[(2 * p) * H + k] = cadd(c0, c1);
            ca[(2 * p + 1) * H + k] = twmul<true>(csub(c0, c1), tw[k]);
        }
        __syncthreads();
        {
            const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
            for (int line = threadIdx.x >> 5; line < 2 * npair; line += nw)
                warp_fft_line<T, true, H / 32, 2>(ca + line * H, cb + line * H, tw, lane);
            __syncthreads();
        }
        for (int idx = threadIdx.x; idx < npair * PC; idx += blockDim.x) {
            int p = idx / PC, n = idx - p * PC;
            V z = ca[(2 * p + (n & 1)) * H + (n >> 1)];
            int j = mk_src(n, PC);
            R[(2 * p) * L.ls + j * L.es] = z.x;
            if (2 * p + 1 < L.n) R[(2 * p + 1) * L.ls + j * L.es] = z.y;
        }
        __syncthreads();
        return;
    }
    Lines C{npair, N, 1};
    const tw_t<T>* w4 = twpool + pl.tw4;
    for (int idx = threadIdx.x; idx < npair * N; idx += blockDim.x) {
        int p = idx / N, k = idx - p * N;
        const bool hasb = (2 * p + 1 < L.n);
        T xa = R[(2 * p) * L.ls + k * L.es];
        T xar = (k == 0) ? T(0) : R[(2 * p) * L.ls + (N - k) * L.es];
        T xb = hasb ? R[(2 * p + 1) * L.ls + k * L.es] : T(0);
        T xbr = (hasb && k != 0) ? R[(2 * p + 1) * L.ls + (N - k) * L.es] : T(0);
        const tw_t<T> w = w4[k];   // used conjugated
        V va = twmul<true>(cmk<V>(xa, -xar), w);
        V vb = twmul<true>(cmk<V>(xb, -xbr), w);
        ca[p * N + k] = cmk<V>(va.x - vb.y, va.y + vb.x);
    }
    __syncthreads();
    V* res = fft_lines_t<T, true, PC>(ca, cb, C, pl, twpool);
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
template <typename T, int PC = 0>
__device__ cplx<T>* r2c_lines(const T* R, Lines L, int nlen, cplx<T>* ca, cplx<T>* cb, const Plan& pl,
                              const tw_t<T>* __restrict__ twpool) {
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
    return fft_lines_t<T, false, PC>(ca, cb, Lines{npair, P, 1}, pl, twpool);
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

// ---- zero-padded transforms of length P = 2N as two N-point FFTs ------------------------------
// Forward, input zero for n >= N:  X[2j] = FFT_N(v)[j],  X[2j+1] = FFT_N(v W_P^n)[j].
// Inverse, output needed for n < N only:  x[n] = IFFT_N(X_even)[n] + conj(W_P^n) IFFT_N(X_odd)[n].
// A pair p of real lines (packed as v = a + i b) occupies lines 2p (even k) and 2p+1 (odd k),
// N values each: spectral index k of pair p sits at half_pos(p, k, N).

template <typename T>
__device__ __forceinline__ cplx<T> r2c_get_h(const cplx<T>* res, int line, int k, int P) {
    using V = cplx<T>;
    const int p = line >> 1, N = P / 2;
    V Z = res[half_pos(p, k, N)];
    V Zr = cconj(res[half_pos(p, k == 0 ? 0 : P - k, N)]);
    return (line & 1) ? cscale(cmul_mi(csub(Z, Zr)), T(0.5)) : cscale(cadd(Z, Zr), T(0.5));
}

template <typename T>
__device__ __forceinline__ void c2r_put_h(cplx<T>* ca, int p, int k, int P, cplx<T> xa, cplx<T> xb) {
    using V = cplx<T>;
    const int N = P / 2;
    if (k == 0 || 2 * k == P) { xa.y = T(0); xb.y = T(0); }
    ca[half_pos(p, k, N)] = cmk<V>(xa.x - xb.y, xa.y + xb.x);
    if (k != 0 && 2 * k != P) ca[half_pos(p, P - k, N)] = cmk<V>(xa.x + xb.y, xb.x - xa.y);
}

// Forward zero-padded transform (P = 2N) of L.n real lines of length nlen <= N, as pairs, with
// N-point FFTs (plan pN); twP = W_P^m (m < P).  Returns the buffer holding the half layout.
template <typename T, int N>
__device__ cplx<T>* r2c_lines_h(const T* R, Lines L, int nlen, cplx<T>* ca, cplx<T>* cb, const Plan& pN,
                                const tw_t<T>* __restrict__ twpool, const tw_t<T>* __restrict__ twP) {
    using V = cplx<T>;
    const int npair = (L.n + 1) / 2;
    for (int idx = threadIdx.x; idx < npair * N; idx += blockDim.x) {
        const int p = idx / N, n = idx - p * N;
        V v = cmk<V>(T(0), T(0));
        if (n < nlen) {
            v.x = R[(2 * p) * L.ls + n * L.es];
            if (2 * p + 1 < L.n) v.y = R[(2 * p + 1) * L.ls + n * L.es];
        }
        ca[(2 * p) * N + n] = v;
        ca[(2 * p + 1) * N + n] = twmul(v, twP[n]);
    }
    __syncthreads();
    return fft_lines_t<T, false, N>(ca, cb, Lines{2 * npair, N, 1}, pN, twpool);
}

}  // namespace sgspm
