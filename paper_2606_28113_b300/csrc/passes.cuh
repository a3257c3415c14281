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
#include "tc_dct.cuh"

namespace sgspm {

// Shared-memory layout of the XZ pass for one film (host and device agree on it).
struct XZLayout {
    int tw;    // complex elements of the staged twiddle tables (x DCT, z DCT, x/z padded FFT)
    int dt;    // real elements of the staged short-axis DCT tables
    int xw;    // complex elements of each of the two x-work buffers
    int kc;    // kx chunk of the z transforms
    int zw;    // complex elements of each of the two z-work buffers
    int slab;  // real elements of each of the three slabs
    int tc;    // bytes of the tensor-core B operands (TF32X3 form), 16-byte aligned, else 0
};

// Threads of a slab-pass CTA.  The Gauss-Seidel and right-hand-side launch types of the 256-wide
// slabs run 512 (64 registers each): every pointwise, staging and packing loop of a row is split
// over twice as many threads, and the register z transforms run on lane pairs (see xz_item).
template <int NX, int MODE, bool MULTI, bool ZTC>
__host__ __device__ constexpr int xz_nt() {
    return (NX == 256 && (MODE == 1 || MODE == 2 || MODE == 3) && !MULTI && !ZTC) ? 2 * kThreads : kThreads;
}

// Thin films (nz <= kZReg) transform along z in registers, one thread per column: dense
// DCT-II / DCT-III (nz x nz tables) and the zero-padded DFT of length Pz <= 2 kZReg.
constexpr int kZReg = 8;

__host__ __device__ inline bool z_in_registers(int nz) { return nz <= kZReg; }

// ztc: the TF32X3 form's tensor-core z transforms (operand A reuses the two x-work buffers)
__host__ __device__ inline XZLayout xz_layout(int nx, int nz, int Px, int Pz, int Kx, bool stray, bool ztc = false) {
    XZLayout L;
    const bool zreg = z_in_registers(nz);
    int a = ((nz + 1) / 2) * nx;
    int b = zreg ? 0 : ((nx + 1) / 2) * nz;
    int c = stray ? ((nz + 1) / 2) * Px : 0;
    L.xw = a > b ? a : b;
    if (c > L.xw) L.xw = c;
    L.kc = zreg ? 0 : (Kx < 32 ? Kx : 32);
    L.zw = (stray && !zreg) ? Pz * L.kc : 0;
    L.slab = nx * nz;
    L.tw = 2 * nx + 2 * nz + (stray ? Px + Pz : 0);
    L.dt = zreg ? ((2 * nz * nz + 1) / 2) * 2 : 0;   // even count keeps the complex buffers aligned
    L.tc = 0;
    if (ztc && tc_zdct_ok(nx, nz)) {
        if (L.xw < 4 * nx) L.xw = 4 * nx;   // 2 (hi, lo) x nx/128 tiles of 4 KiB in xw0..xw1
        L.tc = 4 * kTcBBytes + 16;          // forward and inverse tables, hi and lo, + alignment
    }
    return L;
}

template <typename T>
__host__ __device__ inline size_t xz_smem_bytes(const XZLayout& L) {
    return (size_t)L.tw * sizeof(tw_t<T>) + (size_t)(2 * L.xw + 2 * L.zw) * sizeof(cplx<T>) + (size_t)(3 * L.slab + L.dt) * sizeof(T) +
           (size_t)L.tc;
}

// Copy the twiddle tables of `pl` (W_P, and the DCT quarter-wave table when `dct`) from the
// global pool to shared memory at `stw + off`, and point the plan at the staged copy.
template <typename T>
__device__ __forceinline__ void stage_plan(Plan& pl, const tw_t<T>* __restrict__ g, tw_t<T>* stw, int off, bool dct) {
    const int P = pl.P;
    for (int i = threadIdx.x; i < P; i += blockDim.x) stw[off + i] = g[pl.tw + i];
    if (dct)
        for (int i = threadIdx.x; i < P; i += blockDim.x) stw[off + P + i] = g[pl.tw4 + i];
}

// Newell table layout [c][kz'][kx][ky'] (ky' fastest: a y line reads it contiguously).  A line
// holds Py/2 + 1 values and is padded to a multiple of 4 elements (HyP), so that every line
// starts on a 16-byte boundary and can be copied to shared memory in 16-byte pieces.
__host__ __device__ inline int ktab_row(int Py) { return ((Py / 2 + 1) + 3) & ~3; }

__host__ __device__ inline long long ktab_index(int c, int kx, int kzr, int kyr, int Kx, int HyP, int Hz) {
    return (((long long)c * Hz + kzr) * Kx + kx) * HyP + kyr;
}

// Register stray pass (one warp per kx line, Py = 32 E): shared-memory layout of one CTA of
// kWarpLines lines.  Twiddles W_Py; complex: [scratch per warp (Py) | staged input lines 3 x lines x LI];
// real: staged table lines [3 NOUT][lines][HyP].  LI = Py/2 + 8 makes the asynchronous copies of
// a (y, kx) tile land two lanes per bank (the minimum for 8-byte elements).
constexpr int kWarpLines = 4;   // kx lines (warps) per CTA of the register stray pass

__host__ __device__ inline int yw_line_stride(int Py) { return Py / 2 + 8; }

template <typename T>
__host__ __device__ inline size_t yw_smem_bytes(int Py, int nout, int lines = kWarpLines) {
    return (size_t)Py * sizeof(tw_t<T>) + (size_t)(lines * Py + 3 * lines * yw_line_stride(Py)) * sizeof(cplx<T>) +
           (size_t)3 * nout * lines * ktab_row(Py) * sizeof(T);
}

// ---- persistent ensemble step (FP32 form) ------------------------------------------------------
// One launch runs every pass of a step for all films of a batch.  The passes' work items (slab
// rows, heat-line tiles, stray-line groups of kPersistLines lines) form one queue in program order
// (phase by phase, films in order within a phase); CTAs take items from it with a ticket counter.
// An item of phase q of film f may start once all of film f's items of phases < q are complete: a
// per-film counter of completed items, waited on with a bounded acquire-spin.  Films never wait on
// each other, so the tail of one phase of a film overlaps other films' work.
// 64-thread CTAs (eight per SM at 128 registers): the slab items of thin films run one warp per x
// line, so small CTAs leave few warps idle (256-thread CTAs made the 256-film step 16.7 ms, 128
// 12.4 ms, 64 11.7 ms; 64 with 255 registers 15.1 ms, 32 threads 16.8 ms)
constexpr int kPersistThreads = 64;   // threads per CTA of the persistent kernel
constexpr int kPersistLines = kPersistThreads / 32;   // kx lines per stray item (one warp each)

struct PPhase {
    int kind;       // 0 slab pass, 1 heat line pass, 2 stray line pass
    int first;      // index of the phase's first item in the item table
    int n;          // items of the phase
    int pad_;
    XZProg xz;
    YProg y;
};

struct PItem {
    int4 wi;        // work item as the per-pass kernels take it (film, ...)
    int key;        // size class: x length (slab: 0, 64, 128, 256), y length (heat), E = Py / 32 (stray)
    int target;     // completed items of the film (within the step) this item waits for
    int phase;      // index of the item's phase
    int pad_;
};

struct PersistArgs {
    const PPhase* phases;
    const PItem* items;
    const int* film_items;     // items of each film in one step
    unsigned* ctl;             // [0] ticket counter, [1] abandon flag, [2 ..] completed items per film
    int nphase;
    int items_per_step;
    int nsteps;                // steps in this launch
    int stray;
    long long wait_limit;      // clock cycles one dependency wait may take before the launch is abandoned
    int withhold;              // test switch: the ticket whose item is skipped (never completes), or -1
};

}  // namespace sgspm
