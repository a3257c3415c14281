// Host-side entry points of the pass kernels, one per compile-time variant.  The kernels are
// instantiated in the k_*.cu translation units (compiled in parallel); capi.cu sees only these
// declarations and dispatches on the size class at run time.
#pragma once
#include <utility>
#include "common.cuh"
#include "passes.cuh"

namespace sgspm {

// Pass kernels are launched with programmatic stream serialization (see pdl_wait in the kernels).
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// XZ slab pass: NX compile-time x length (0: runtime), ZTC tensor-core z transforms, MULTI
// several y rows per CTA, MODE launch type (0 generic, 1 rhs, 2 Gauss-Seidel, 3 final).
// nt: threads per CTA (0: the variant's own count, xz_nt); the packed-row (MULTI) variants also run
// with 32, 64 or 128, since every loop of the slab pass strides by blockDim.x
template <typename T, int NX, bool ZTC, bool MULTI, int MODE = 0>
void xz_go(unsigned nb, size_t smem, cudaStream_t st, const Dev<T>& d, const int4* w, const XZProg& pg, int stray,
           unsigned nt = 0);
template <typename T, int NX, bool ZTC, bool MULTI, int MODE = 0>
cudaError_t xz_attr(size_t smem);
// static shared memory of the variant's kernel (bytes), or a CUDA error as a negative value
template <typename T, int NX, bool ZTC, bool MULTI>
long long xz_static_smem();

// Y heat line pass: NY compile-time y length (0: runtime).
template <typename T, int NY>
void yh_go(unsigned nb, unsigned threads, size_t smem, cudaStream_t st, const Dev<T>& d, const int4* w, const YProg& pg);
template <typename T, int NY>
cudaError_t yh_attr(size_t smem);

// Register stray line pass: NOUT output components, Py = 32 E.
template <typename T, int NOUT, int E>
void yw_go(unsigned nb, cudaStream_t st, const Dev<T>& d, const int4* w, const YProg& pg);
template <typename T, int NOUT, int E>
cudaError_t yw_attr(size_t smem);

// Shared-memory stray line pass (any padded y length).
template <typename T>
void ys_go(unsigned nb, size_t smem, cudaStream_t st, const Dev<T>& d, const int4* w, const YProg& pg, int tx);
template <typename T>
cudaError_t ys_attr(size_t smem);

// Persistent ensemble step (FP32 form, cooperative launch of `grid` CTAs of kThreads threads).
void persist_go(unsigned grid, size_t smem, cudaStream_t st, const Dev<float>& d, const PersistArgs& a);
cudaError_t persist_attr(size_t smem);
int persist_blocks_per_sm(size_t smem);   // resident CTAs per SM at this shared memory, 0 on error

}  // namespace sgspm
