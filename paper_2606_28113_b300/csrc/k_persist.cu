// Kernel instantiation: the persistent ensemble step (FP32 form).  Every pass runs inside this one
// kernel, so field reads must not take the read-only (non-coherent) path.
#define SGSPM_FIELD_RO
#include "launch.cuh"
#include "persist.cuh"

namespace sgspm {

void persist_go(unsigned grid, size_t smem, cudaStream_t st, const Dev<float>& d, const PersistArgs& a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kPersistThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident at once: waits always end
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, persist_kernel, d, a);
}

cudaError_t persist_attr(size_t smem) {
    return cudaFuncSetAttribute(persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int persist_blocks_per_sm(size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, persist_kernel, kPersistThreads, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace sgspm
