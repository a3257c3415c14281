// Definitions of the per-variant launch functions declared in launch.cuh.  Included only by the
// kernel translation units k_*.cu, each of which instantiates its share of the variants.
#pragma once
#include "launch.cuh"
#include "passes.cu"

namespace sgspm {

template <typename T, int NX, bool ZTC, bool MULTI, int MODE>
void xz_go(unsigned nb, size_t smem, cudaStream_t st, const Dev<T>& d, const int4* w, const XZProg& pg, int stray,
           unsigned nt) {
    launch_pdl(xz_kernel<T, NX, ZTC, MULTI, MODE>, nb, nt ? nt : (unsigned)xz_nt<NX, MODE, MULTI, ZTC>(), smem, st, d, w, pg,
               stray);
}
template <typename T, int NX, bool ZTC, bool MULTI, int MODE>
cudaError_t xz_attr(size_t smem) {
    return cudaFuncSetAttribute(xz_kernel<T, NX, ZTC, MULTI, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <typename T, int NX, bool ZTC, bool MULTI>
long long xz_static_smem() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, xz_kernel<T, NX, ZTC, MULTI>);
    return e == cudaSuccess ? (long long)fa.sharedSizeBytes : -(long long)e;
}

template <typename T, int NY>
void yh_go(unsigned nb, unsigned threads, size_t smem, cudaStream_t st, const Dev<T>& d, const int4* w, const YProg& pg) {
    launch_pdl(y_heat_kernel<T, NY>, nb, threads, smem, st, d, w, pg);
}
template <typename T, int NY>
cudaError_t yh_attr(size_t smem) {
    return cudaFuncSetAttribute(y_heat_kernel<T, NY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, int NOUT, int E>
void yw_go(unsigned nb, cudaStream_t st, const Dev<T>& d, const int4* w, const YProg& pg) {
    launch_pdl(y_stray_warp_kernel<T, NOUT, E>, nb, 32 * kWarpLines, yw_smem_bytes<T>(32 * E, NOUT), st, d, w, pg);
}
template <typename T, int NOUT, int E>
cudaError_t yw_attr(size_t smem) {
    return cudaFuncSetAttribute(y_stray_warp_kernel<T, NOUT, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T>
void ys_go(unsigned nb, size_t smem, cudaStream_t st, const Dev<T>& d, const int4* w, const YProg& pg, int tx) {
    y_stray_kernel<T><<<nb, kThreads, smem, st>>>(d, w, pg, tx);
}
template <typename T>
cudaError_t ys_attr(size_t smem) {
    return cudaFuncSetAttribute(y_stray_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace sgspm

// explicit instantiation of one variant of each family
#define SGSPM_INST_XZ(T, NX, ZTC, MULTI)                                                                        \
    template void sgspm::xz_go<T, NX, ZTC, MULTI, 0>(unsigned, size_t, cudaStream_t, const sgspm::Dev<T>&,     \
                                                     const int4*, const sgspm::XZProg&, int, unsigned);         \
    template cudaError_t sgspm::xz_attr<T, NX, ZTC, MULTI, 0>(size_t);                                          \
    template long long sgspm::xz_static_smem<T, NX, ZTC, MULTI>();
// the three launch-type specialisations of one single-row FP32 size class
#define SGSPM_INST_XZ_MODES(NX)                                                                                  \
    template void sgspm::xz_go<float, NX, false, false, 1>(unsigned, size_t, cudaStream_t,                     \
                                                           const sgspm::Dev<float>&, const int4*,               \
                                                           const sgspm::XZProg&, int, unsigned);                \
    template void sgspm::xz_go<float, NX, false, false, 2>(unsigned, size_t, cudaStream_t,                     \
                                                           const sgspm::Dev<float>&, const int4*,               \
                                                           const sgspm::XZProg&, int, unsigned);                \
    template void sgspm::xz_go<float, NX, false, false, 3>(unsigned, size_t, cudaStream_t,                     \
                                                           const sgspm::Dev<float>&, const int4*,               \
                                                           const sgspm::XZProg&, int, unsigned);                \
    template cudaError_t sgspm::xz_attr<float, NX, false, false, 1>(size_t);                                    \
    template cudaError_t sgspm::xz_attr<float, NX, false, false, 2>(size_t);                                    \
    template cudaError_t sgspm::xz_attr<float, NX, false, false, 3>(size_t);
#define SGSPM_INST_YH(T, NY)                                                                                     \
    template void sgspm::yh_go<T, NY>(unsigned, unsigned, size_t, cudaStream_t, const sgspm::Dev<T>&,          \
                                      const int4*, const sgspm::YProg&);                                        \
    template cudaError_t sgspm::yh_attr<T, NY>(size_t);
#define SGSPM_INST_YW(T, NOUT, E)                                                                                \
    template void sgspm::yw_go<T, NOUT, E>(unsigned, cudaStream_t, const sgspm::Dev<T>&, const int4*,          \
                                           const sgspm::YProg&);                                                \
    template cudaError_t sgspm::yw_attr<T, NOUT, E>(size_t);
#define SGSPM_INST_YS(T)                                                                                         \
    template void sgspm::ys_go<T>(unsigned, size_t, cudaStream_t, const sgspm::Dev<T>&, const int4*,          \
                                  const sgspm::YProg&, int);                                                    \
    template cudaError_t sgspm::ys_attr<T>(size_t);
