// Short-axis (z) DCT of a slab as a dense GEMM on the 5th-generation tensor cores, in 3xTF32
// split precision with FP32 accumulation (the TF32X3 precision form of the FP32 path).
//
// The slab pass holds an nz x nx slab h[z][x] (x fastest).  The z transform with an nz x nz
// table C (forward DCT-II or its inverse) is
//     out[x][k] = sum_z h[z][x] C[k][z],
// i.e. D = A B^T with A[m = x][k = z] (M = 128 rows of x per tile, K = 8: nz <= 8 zero-padded)
// and B[n = k][z] (N = 16: nz outputs zero-padded).  Each operand is split as v = hi + lo with
// hi = tf32(v), lo = tf32(v - hi), and D = A_lo B_hi + A_hi B_lo + A_hi B_hi (the lo*lo term,
// ~2^-22 relative, is dropped).  One thread issues the tcgen05.mma instructions; D lives in
// tensor memory (16 columns per 128-row tile) and is read back with tcgen05.ld.
//
// Operands are stored K-major without swizzling: 8-row x 16-byte core matrices, the two core
// matrices along K 128 bytes apart (leading byte offset), consecutive 8-row groups 256 bytes
// apart (stride byte offset).  Element (r, k) of an operand sits at byte
//     (r / 8) * 256 + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4.
#pragma once
#include <cstdint>

namespace sgspm {

constexpr int kTcK = 8;             // K of one kind::tf32 MMA (32 bytes of 4-byte elements)
constexpr int kTcN = 16;            // N (outputs per row, zero-padded)
constexpr int kTcM = 128;           // rows of x per MMA tile
constexpr int kTcTileBytes = 4096;  // one 128 x 8 operand tile
constexpr int kTcBBytes = 512;      // one 16 x 8 operand

// films whose z transform can run on the tensor cores in this form
__host__ __device__ inline bool tc_zdct_ok(int nx, int nz) { return nz >= 2 && nz <= 8 && nx % kTcM == 0 && nx <= 512; }

// tensor-memory columns a slab of nx rows needs (a power of two >= 32)
__host__ __device__ inline int tc_tmem_cols(int nx) {
    const int c = kTcN * (nx / kTcM);
    return c <= 32 ? 32 : (c <= 64 ? 64 : 128);
}

__device__ __forceinline__ uint32_t tc_off(int r, int k) { return (r >> 3) * 256 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

// shared-memory matrix descriptor: K-major, no swizzle, LBO 128 B, SBO 256 B, fixed 0b001 at 46
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, N = 16, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate));
}

// Tensor-memory and barrier state of one CTA of the slab pass.
struct TcState {
    uint32_t tmem;      // base address of the allocated columns
    uint32_t mbar;      // shared address of the completion barrier
    uint32_t phase;     // parity the next wait expects
};

// Warp 0 allocates `cols` tensor-memory columns; thread 0 initialises the barrier.  All threads
// must call it (it ends with a block barrier).
__device__ __forceinline__ void tc_setup(TcState& s, uint32_t* tmem_slot, uint64_t* mbar, int cols) {
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    s.tmem = *(volatile uint32_t*)tmem_slot;
    s.mbar = smem_u32(mbar);
    s.phase = 0;
}

// Bounded wait on the completion barrier (about a second at most, or `limit` polls when limit > 0);
// false if it expired.
__device__ __forceinline__ bool tc_wait(TcState& s, int limit = 0) {
    const long long t0 = clock64();
    const int maxit = limit > 0 ? limit : (1 << 24);
    uint32_t done = 0;
    for (int it = 0; !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(s.mbar), "r"(s.phase)
            : "memory");
        if (!done && (it > maxit || clock64() - t0 > 2000000000LL)) return false;
    }
    s.phase ^= 1u;
    return true;
}

// Warp 0 frees the columns; call after a block barrier that follows the last tensor-memory read.
__device__ __forceinline__ void tc_teardown(const TcState& s, int cols) {
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem), "r"(cols) : "memory");
}

// Write the hi and lo parts of an nz x nz table C (row k = output, column z = input; C[k * nz + z])
// as B operands (N = 16 rows, K = 8) at bhi / blo (512 bytes each, 16-byte aligned).
__device__ __forceinline__ void tc_write_b(const float* C, int nz, unsigned char* bhi, unsigned char* blo) {
    for (int i = threadIdx.x; i < kTcN * kTcK; i += blockDim.x) {
        const int n = i / kTcK, k = i - n * kTcK;
        const float v = (n < nz && k < nz) ? C[n * nz + k] : 0.0f;
        const uint32_t h = to_tf32(v);
        const uint32_t l = to_tf32(v - __uint_as_float(h));
        *reinterpret_cast<uint32_t*>(bhi + tc_off(n, k)) = h;
        *reinterpret_cast<uint32_t*>(blo + tc_off(n, k)) = l;
    }
}

// In place: h[k][x] <- sum_z h[z][x] B[k][z] for k < nz, on the tensor cores.  abuf: 2 * (nx/128)
// tiles of 4096 bytes (16-byte aligned) of scratch; bhi / blo from tc_write_b.  Ends with a
// block barrier.  A wait that expires sets bit 4 of the status word (the slab is then left as
// it was; the host reports SGSPM_ERR_TIMEOUT).  test: see Dev::tc_test (null in normal use).
__device__ __forceinline__ void tc_zdct(float* h, int nx, int nz, unsigned char* abuf, const unsigned char* bhi,
                                        const unsigned char* blo, TcState& s, int* status, const int* test) {
    const bool skip = test && test[0] != 0;
    const int limit = test ? test[1] : 0;
    const int ntile = nx / kTcM;
    unsigned char* ahi = abuf;
    unsigned char* alo = abuf + ntile * kTcTileBytes;
    for (int i = threadIdx.x; i < kTcK * nx; i += blockDim.x) {
        const int k = i / nx, x = i - k * nx;
        const float v = k < nz ? h[k * nx + x] : 0.0f;
        const uint32_t hv = to_tf32(v);
        const uint32_t lv = to_tf32(v - __uint_as_float(hv));
        const uint32_t o = (x / kTcM) * kTcTileBytes + tc_off(x % kTcM, k);
        *reinterpret_cast<uint32_t*>(ahi + o) = hv;
        *reinterpret_cast<uint32_t*>(alo + o) = lv;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> MMA reads
    __syncthreads();
    if (threadIdx.x == 0 && !skip) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t bh = tc_desc(smem_u32(bhi)), bl = tc_desc(smem_u32(blo));
        for (int t = 0; t < ntile; ++t) {
            const uint32_t d = s.tmem + (uint32_t)(t * kTcN);
            const uint64_t ah = tc_desc(smem_u32(ahi + t * kTcTileBytes)), al = tc_desc(smem_u32(alo + t * kTcTileBytes));
            tc_mma(d, al, bh, 0);
            tc_mma(d, ah, bl, 1);
            tc_mma(d, ah, bh, 1);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s.mbar)
                     : "memory");
    }
    const bool ok = tc_wait(s, limit);
    if (!ok && threadIdx.x == 0) atomicOr(status, 4);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3;            // a warp reads tensor-memory lanes 32 (warp % 4) .. + 31
    const int nwg = (int)(blockDim.x >> 7);  // warpgroups in the block
    for (int t = warp >> 2; ok && t < ntile; t += nwg) {
        const uint32_t taddr = s.tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(t * kTcN);
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
            "[%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int x = t * kTcM + 32 * quarter + lane;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < nz) h[k * nx + x] = __uint_as_float(r[k]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
}

}  // namespace sgspm
