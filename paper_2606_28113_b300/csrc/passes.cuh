// Pass kernels of one SGSPM step.  A step alternates two kinds of launch:
//   XZ slab pass: one CTA per (film, y row) holds the nz x nx slab in shared memory and
//     runs the x and z transforms plus every pointwise operation of the scheme
//     (right-hand sides, Gauss-Seidel cross products, damping update, projection);
//   Y line pass: one CTA per (film, kz, tile of x) transforms along y and applies the
//     spectral diagonal: the heat-solve eigenvalues or the Newell tensor multiply.
// Every launch covers all films of the handle through a work list.
#pragma once
#include "common.cuh"
#include "fft.cuh"

namespace sgspm {

// Shared-memory layout of the XZ pass for one film (host and device agree on it).
struct XZLayout {
    int xw;    // complex elements of each of the two x-work buffers
    int kc;    // kx chunk of the z transforms
    int zw;    // complex elements of each of the two z-work buffers
    int slab;  // real elements of each of the three slabs
};

__host__ __device__ inline XZLayout xz_layout(int nx, int nz, int Px, int Pz, int Kx, bool stray) {
    XZLayout L;
    int a = ((nz + 1) / 2) * nx;
    int b = ((nx + 1) / 2) * nz;
    int c = stray ? ((nz + 1) / 2) * Px : 0;
    L.xw = a > b ? a : b;
    if (c > L.xw) L.xw = c;
    L.kc = Kx < 32 ? Kx : 32;
    L.zw = stray ? Pz * L.kc : 0;
    L.slab = nx * nz;
    return L;
}

template <typename T>
__host__ __device__ inline size_t xz_smem_bytes(const XZLayout& L) {
    return (size_t)(2 * L.xw + 2 * L.zw) * sizeof(cplx<T>) + (size_t)3 * L.slab * sizeof(T);
}

__host__ __device__ inline int ktab_index(int c, int kx, int kzr, int kyr, int Kx, int Hy, int Hz) {
    return ((c * Hz + kzr) * Hy + kyr) * Kx + kx;
}

}  // namespace sgspm
