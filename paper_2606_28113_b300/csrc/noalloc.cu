// sgspm_energy_noalloc: the discrete-energy reduction for callers that must not allocate
// device memory.  Included by capi.cu.
//
// Who needs it: code that runs where cudaMalloc / cudaFree are not available or not
// allowed - a plugin inside a host application that owns every device buffer through its
// own fixed pool, a process whose device-memory budget is fixed up front, or a latency-
// critical loop that cannot afford the implicit synchronisation an allocation may cause.
// Such a caller already holds m (and optionally h_s) in its own device buffers and wants
// the five energy terms written to a device buffer it also owns.
//
// The reduction needs scratch for its per-block partial sums.  Here that scratch is the
// file-scope array below, which every GPU that loads the library keeps until the process
// exits.  Consequences:
//   * at most kNoallocMaxBlocks blocks of kNoallocCellsPerBlock cells (16 Mi cells);
//   * every call shares the array; calls whose work overlaps on the GPU (different streams
//     without ordering between them) race on it and must be serialised by the caller;
//   * the array keeps the last call's contents; no element has to start at zero, because
//     each block overwrites its own slot before the final kernel reads it.
#pragma once
#include <mutex>
#include "common.cuh"

namespace sgspm {

constexpr int kNoallocCellsPerBlock = 4096;
constexpr int kNoallocMaxBlocks = 4096;   // 16 Mi cells; scratch = 4096 * 4 doubles = 128 KiB
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[4 * kNoallocMaxBlocks];

// Address of g_noalloc_partials on each device, looked up once per device context: the address
// belongs to the module loaded in that context, so it is looked up again when the device's
// current context differs from the one it was found in (after cudaDeviceReset, say).
static double* g_noalloc_ptr[kNoallocMaxDevices] = {};
static void* g_noalloc_ctx[kNoallocMaxDevices] = {};
static std::mutex g_noalloc_mu;

// the calling thread's current driver context (through the runtime's driver entry point, so that
// the library needs no link to the driver library), or nullptr if it cannot be queried
static void* noalloc_current_context() {
    typedef int (*CtxGetCurrent)(void**);
    static CtxGetCurrent fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrent)f;
    }
    void* c = nullptr;
    if (!fn || fn(&c) != 0) return nullptr;
    return c;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) energy_noalloc_partial_kernel(const T* __restrict__ m, const T* __restrict__ hs,
                                                                          int nx, int ny, int nz, double hx, double hy,
                                                                          double hz, double ux, double uy, double uz,
                                                                          double hex, double hey, double hez,
                                                                          double* __restrict__ part) {
    const long long n = (long long)nx * ny * nz;
    const long long sxy = (long long)nx * ny;
    const long long c0 = (long long)blockIdx.x * kNoallocCellsPerBlock;
    const long long c1 = c0 + kNoallocCellsPerBlock < n ? c0 + kNoallocCellsPerBlock : n;
    double ex = 0, an = 0, st = 0, ze = 0;
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        const int x = (int)(c % nx);
        const int y = (int)((c / nx) % ny);
        const int z = (int)(c / sxy);
        double v[3] = {(double)m[c], (double)m[n + c], (double)m[2 * n + c]};
        for (int a = 0; a < 3; ++a) {
            const T* ma = m + a * n;
            if (x + 1 < nx) { double q = (double)ma[c + 1] - v[a]; ex += q * q / (hx * hx); }
            if (y + 1 < ny) { double q = (double)ma[c + nx] - v[a]; ex += q * q / (hy * hy); }
            if (z + 1 < nz) { double q = (double)ma[c + sxy] - v[a]; ex += q * q / (hz * hz); }
        }
        double mu = v[0] * ux + v[1] * uy + v[2] * uz;
        an += v[0] * v[0] + v[1] * v[1] + v[2] * v[2] - mu * mu;
        if (hs) st += (double)hs[c] * v[0] + (double)hs[n + c] * v[1] + (double)hs[2 * n + c] * v[2];
        ze += hex * v[0] + hey * v[1] + hez * v[2];
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

__global__ void energy_noalloc_final_kernel(const double* __restrict__ part, int nblocks, double eps, double Q, double V,
                                            double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s[4] = {0, 0, 0, 0};
    for (int b = 0; b < nblocks; ++b)
        for (int k = 0; k < 4; ++k) s[k] += part[b * 4 + k];
    const double ex = 0.5 * eps * V * s[0], an = 0.5 * Q * V * s[1], st = -0.5 * V * s[2], ze = -V * s[3];
    out[0] = ex;
    out[1] = an;
    out[2] = st;
    out[3] = ze;
    out[4] = ex + an + st + ze;
}

// Set-up once per device (with that device current): look up the device address of the
// file-scope scratch array.  Returns nullptr and sets *err on failure.
static double* noalloc_scratch(std::string* err) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return nullptr;
    }
    if (dev < 0 || dev >= kNoallocMaxDevices) {
        *err = "device index out of range for the allocation-free entry point";
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    void* ctx = g_noalloc_ptr[dev] ? noalloc_current_context() : nullptr;
    if (!g_noalloc_ptr[dev] || !ctx || ctx != g_noalloc_ctx[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_noalloc_partials);   // makes the device's context current
        if (e != cudaSuccess || !p) {
            *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return nullptr;
        }
        g_noalloc_ptr[dev] = p;
        g_noalloc_ctx[dev] = noalloc_current_context();
    }
    return g_noalloc_ptr[dev];
}

}  // namespace sgspm
