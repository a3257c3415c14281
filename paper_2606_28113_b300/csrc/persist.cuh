// Persistent ensemble step kernel (FP32 form): every pass of a step for every film of a batch in
// one launch, scheduled item by item with per-film completion counters (see PersistArgs).
// Included only by k_persist.cu, which instantiates the pass items it dispatches to.
#pragma once
#include "passes.cu"

namespace sgspm {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until *cnt >= target.  Bounded: if the abandon flag is raised, or the wait exceeds `limit`
// clock cycles (or 2^30 polls), returns false; an expired wait sets status bit 8 and raises the flag
// so that every other CTA stops too.  The acquire load orders this CTA's later reads of the
// producers' data after their release.
__device__ inline bool persist_wait(const unsigned* cnt, unsigned target, unsigned* abandon, long long limit, int* status) {
    const long long t0 = clock64();
    for (unsigned it = 0;; ++it) {
        if (ld_acquire_u32(cnt) >= target) return true;
        if (ld_acquire_u32(abandon) != 0u) return false;
        if (clock64() - t0 > limit || it > (1u << 30)) {
            atomicOr(status, 8);
            atomicExch(abandon, 1u);
            return false;
        }
        __nanosleep(64);
    }
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// the pass item of phase `ph` (staged in shared memory) for work item (wi, key)
__device__ __forceinline__ void persist_item(const Dev<float>& d, const PPhase& ph, const int4 wi, int key, int stray) {
    if (ph.kind == 0) {
        switch (key) {
            case 64: xz_item<float, 64, false, true>(d, wi, ph.xz, stray); break;
            case 128: xz_item<float, 128, false, true>(d, wi, ph.xz, stray); break;
            case 256: xz_item<float, 256, false, true>(d, wi, ph.xz, stray); break;
            default: xz_item<float, 0, false, true>(d, wi, ph.xz, stray); break;
        }
    } else if (ph.kind == 1) {
        switch (key) {
            case 64: y_heat_item<float, 64>(d, wi, ph.y); break;
            case 128: y_heat_item<float, 128>(d, wi, ph.y); break;
            case 256: y_heat_item<float, 256>(d, wi, ph.y); break;
            default: y_heat_item<float, 0>(d, wi, ph.y); break;
        }
    } else {
        const int sel = key * 4 + ph.y.n;   // E (2, 4, 8) and outputs (1..3)
        switch (sel) {
#define SGSPM_PY(E, N) case E * 4 + N: y_stray_warp_item<float, N, E, kPersistLines>(d, wi, ph.y); break;
            SGSPM_PY(2, 1) SGSPM_PY(2, 2) SGSPM_PY(2, 3)
            SGSPM_PY(4, 1) SGSPM_PY(4, 2) SGSPM_PY(4, 3)
            SGSPM_PY(8, 1) SGSPM_PY(8, 2) SGSPM_PY(8, 3)
#undef SGSPM_PY
            default: break;   // not reached: the host accepts only these classes
        }
    }
}

__global__ void __launch_bounds__(kPersistThreads, 512 / kPersistThreads) persist_kernel(const __grid_constant__ Dev<float> d, const __grid_constant__ PersistArgs a) {
    // the current item, decoded by thread 0; the phase program is copied here when it changes
    __shared__ __align__(16) PPhase s_ph;
    __shared__ int4 s_wi;
    __shared__ int s_key, s_q, s_go;
    unsigned* ticket = a.ctl;
    unsigned* abandon = a.ctl + 1;
    unsigned* done = a.ctl + 2;
    const unsigned total = (unsigned)a.items_per_step * (unsigned)a.nsteps;
    int qcur = -1;                                      // phase staged in s_ph
    unsigned t_next = 0;                                // thread 0: the ticket after this one
    if (threadIdx.x == 0) t_next = atomicAdd(ticket, 1u);
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned t = t_next;
            if (t < total) t_next = atomicAdd(ticket, 1u);   // next ticket, in flight during this item
            int go = 0;
            if (t < total) {
                const int step = (int)(t / (unsigned)a.items_per_step);
                const int r = (int)(t - (unsigned)step * (unsigned)a.items_per_step);
                const PItem it = a.items[r];
                const int q = it.phase;
                const unsigned target = (unsigned)step * (unsigned)a.film_items[it.wi.x] + (unsigned)it.target;
                go = persist_wait(done + it.wi.x, target, abandon, a.wait_limit, d.status) ? 1 : 0;
                if (go && (int)t == a.withhold) go = 2;     // run nothing, report nothing
                s_wi = it.wi;
                s_key = it.key;
                s_q = q;
            }
            s_go = go;
        }
        __syncthreads();
        const int go = s_go;
        if (go == 0) break;
        const int q = s_q;
        if (q != qcur) {
            // stage the phase program (all threads copy 4-byte words)
            const int* src = reinterpret_cast<const int*>(a.phases + q);
            int* dst = reinterpret_cast<int*>(&s_ph);
            for (int i = threadIdx.x; i < (int)(sizeof(PPhase) / 4); i += blockDim.x) dst[i] = src[i];
            qcur = q;
            __syncthreads();
        }
        if (go == 1) persist_item(d, s_ph, s_wi, s_key, a.stray);
        // every thread's writes of the item, then one release of the film's counter
        __syncthreads();
        if (threadIdx.x == 0 && go == 1) red_release_add(done + s_wi.x, 1u);
    }
}

}  // namespace sgspm
