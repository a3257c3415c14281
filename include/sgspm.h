/*
 * sgspm.h - C ABI of the B300 (sm_103a) SGSPM library `libsgspm.so`.
 *
 * One time step of the symmetric Gauss-Seidel projection method (SGSPM, Sec. 3.2 of
 * the paper) for the Landau-Lifshitz-Gilbert equation (Sec. 2, Eq. (1)),
 *     m_t = -m x h_eff - alpha m x (m x h_eff),
 *     h_eff = eps Delta m - Q (m - (m.u)u) + h_s + h_e,
 * on a uniform grid of nx*ny*nz rectangular cells with homogeneous Neumann boundaries
 * (Eq. (2)).  Each step:
 *   Step 1 (implicit symmetric Gauss-Seidel, Sec. 3.2): heat solves
 *       g_i = (I - eps dt Delta_h)^{-1} (m_i + dt f_i),  f = -Q(m-(m.u)u) + h_s + h_e,
 *     a forward sweep m1* -> m2* -> m3* and a backward sweep m3** -> m2** -> m1**, each
 *     cross-product update using the newest g;
 *   Step 2 (heat flow without constraint): (I - alpha eps dt Delta_h) m*** = m** + alpha dt f**;
 *   Step 3 (projection): m^{n+1} = m*** / |m***|.
 * With SGSPM_GSPM the one-sided scheme of Sec. 3.1 runs instead (forward sweep only).
 *
 * Discretisation (readings of what the paper leaves open):
 *   - Delta_h is the cell-centred 7-point Laplacian with mirror ghosts, diagonalised by
 *     DCT-II along x, y, z; the solves are done in that basis.
 *   - h_s = -N * m is the zero-padded FFT convolution with the Newell demagnetising
 *     tensor (cell-averaged dipole kernel), evaluated in FP64 once at create time.
 *   - f is re-evaluated (incl. h_s) at the newest state each time a g is formed;
 *     SGSPM_FROZEN_STRAY instead uses h_s(m^n) in Step 1 and h_s(m**) in Step 2.
 *
 * Memory and streams.  Fields are structure-of-arrays [3][nz][ny][nx] with x fastest.
 * For a batch handle the fields of all films are concatenated in film order.  Every
 * call that takes a pointer accepts host or device memory (the copy direction is
 * resolved by unified addressing) and copies the data; the caller keeps ownership.
 * All work is enqueued on the CUDA stream given at create time; calls that return data
 * to the caller (get_field, energy, sync) synchronise that stream.  The library owns all
 * of its device buffers and frees them in sgspm_destroy.  A handle must not be used
 * from two host threads at once.
 *
 * Errors.  Every int-returning call returns SGSPM_OK (0) or a negative status; the text
 * of the last error on the handle is returned by sgspm_last_error.  Device-side
 * problems (a non-finite value or a zero vector before projection) are latched in a
 * device status word and reported as SGSPM_ERR_NONFINITE by the next synchronising call.
 */
#ifndef SGSPM_H
#define SGSPM_H

#ifdef __cplusplus
extern "C" {
#endif

/* Grid: cell counts (>= 1; 1D/2D problems use size-1 axes) and cell sizes (> 0). */
typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
} sgspm_grid;

typedef struct sgspm_ctx* sgspm_t;

enum {
    SGSPM_OK = 0,
    SGSPM_ERR_ARG = -1,          /* invalid argument (checked on the host)                  */
    SGSPM_ERR_OOM = -2,          /* device allocation failed                                */
    SGSPM_ERR_CUDA = -3,         /* a CUDA runtime call failed                              */
    SGSPM_ERR_NONFINITE = -4,    /* device status: non-finite value or |m***| = 0            */
    SGSPM_ERR_TIMEOUT = -5,      /* device status: a bounded wait expired                   */
    SGSPM_ERR_STATE = -6,        /* call not valid in the handle's current state            */
    SGSPM_ERR_UNSUPPORTED = -7   /* size not supported (axis length factors other than 2,3,5,
                                    or a slab that does not fit in shared memory)          */
};

/* create flags */
enum {
    SGSPM_FP64 = 1 << 0,          /* all arithmetic in FP64 (default: FP32 bulk arithmetic)   */
    SGSPM_GSPM = 1 << 1,          /* one-sided GSPM of Sec. 3.1 instead of SGSPM (Sec. 3.2)   */
    SGSPM_NO_STRAY = 1 << 2,      /* h_s = 0                                                 */
    SGSPM_FROZEN_STRAY = 1 << 3,  /* h_s(m^n) for Step 1 and h_s(m**) for Step 2             */
    SGSPM_NO_GRAPH = 1 << 4,      /* launch kernels directly instead of a captured CUDA graph */
    SGSPM_TF32X3 = 1 << 5,        /* FP32 form: short-axis (z) DCTs as 3xTF32 GEMMs on the tensor
                                     cores (films with nx in {128, 256, 512}, 2 <= nz <= 8; other
                                     films keep the FP32 path).  Ignored with SGSPM_FP64.  */
    SGSPM_PERSISTENT = 1 << 6     /* each step is one persistent launch over all films (see
                                     sgspm_create_batch); FP32 form, ny <= 128 with the stray field,
                                     no manufactured forcing; otherwise ERR_UNSUPPORTED at create */
};

/* field selectors */
enum {
    SGSPM_M = 0,      /* magnetisation m (set: normalised on the device; get: current m)      */
    SGSPM_HE = 1,     /* per-cell applied field h_e (set only; replaces the uniform field)    */
    SGSPM_HS = 2      /* stray field h_s(m) of the current m (get only; computed on demand)   */
};

/* dtypes of caller buffers */
enum { SGSPM_F32 = 0, SGSPM_F64_DATA = 1 };

/* forcing kinds for sgspm_set_forcing: the manufactured solutions of Sec. 5.1 on [0,1]^d */
enum { SGSPM_FORCE_NONE = 0, SGSPM_FORCE_MMS_1D = 1, SGSPM_FORCE_MMS_3D = 3 };

/*
 * sgspm_create - one film.  eps (exchange), Q (anisotropy), alpha (damping) >= 0, dt > 0,
 * easy_axis != 0 (normalised internally).  cuda_stream is a cudaStream_t (NULL = legacy
 * default stream).  Allocates the device state, evaluates the Newell tensor and its
 * padded spectrum in FP64 on the device, and builds the FFT plans.  m starts undefined:
 * call sgspm_set_field(SGSPM_M) before stepping.  On error *out is left NULL.
 */
int sgspm_create(const sgspm_grid* grid, double eps, double Q, double alpha, double dt,
                 const double easy_axis[3], int flags, void* cuda_stream, sgspm_t* out);

/*
 * sgspm_create_batch - nfilm independent films (sizes may differ) advanced together:
 * every pass of a step is one kernel launch over all films.  Parameter arrays have
 * nfilm entries (easy_axis: 3*nfilm).  Flags apply to all films.
 */
int sgspm_create_batch(int nfilm, const sgspm_grid* grids, const double* eps, const double* Q,
                       const double* alpha, const double* dt, const double* easy_axis,
                       int flags, void* cuda_stream, sgspm_t* out);

/* Uniform applied field per film (3*nfilm doubles); clears any per-cell h_e. */
int sgspm_set_applied_field(sgspm_t h, const double* he);

/*
 * Batch packing of the slab pass (no counterpart in the paper: a launch-shape choice).  Films are
 * grouped in size classes by nx; a class (FP32 form, nx <= 256 or not a power of two, not
 * TF32X3) may run several consecutive y rows of a film per CTA.
 * sgspm_xz_classes: number of classes (>= 0); with keys/rows non-NULL (cap entries) writes each
 *   class's key (nx, or 0 for the runtime-length kernel) and its current rows per CTA.
 * sgspm_set_packing: rows per CTA (1..8), one entry per class; ERR_UNSUPPORTED for > 1 on a
 *   class that runs one row per CTA.  Results do not depend on the packing (bitwise).
 * sgspm_xz_threads: threads per CTA of each class's packed launches (cap entries when threads is
 *   non-NULL); returns the number of classes.  Default 256.
 * sgspm_set_packing_threads: 32, 64, 128 or 256 threads per packed CTA, one entry per class
 *   (ERR_ARG otherwise; ERR_UNSUPPORTED below 256 on a class that cannot be packed).  A class runs the
 *   packed kernel when it has more than one row per CTA or fewer than 256 threads; one row with
 *   256 runs the class's own kernels.  With fewer threads more CTAs share an SM, and the x
 *   transforms of thin slabs (nz lines per row) leave fewer warps idle.  Results do not depend on
 *   it (bitwise).
 * sgspm_autotune: times `steps` steps of every packable class for 1, 2, 4, 8 rows per CTA with
 *   256, 128, 64 or 32 threads, keeps the fastest, then the heat tile (below) the same way;
 *   m and the step count are restored afterwards (it allocates a copy of m while it runs).  Needs
 *   m set (ERR_STATE).  Writes the chosen rows to rows_out (cap entries) when non-NULL and
 *   returns the number of classes.
 */
int sgspm_xz_classes(sgspm_t h, int* keys, int* rows, int cap);
int sgspm_xz_threads(sgspm_t h, int* threads, int cap);
int sgspm_set_packing_threads(sgspm_t h, const int* threads, int n);
/* y heat pass: x lines per CTA (1..16; default 8).  sgspm_heat_tile returns the current value;
 * sgspm_set_heat_tile: ERR_ARG outside 1..16, ERR_UNSUPPORTED if the tile does not fit in shared
 * memory.  sgspm_autotune also chooses it (from 2, 4, 6, 8, 12, 16), with a CTA of 128 or 256
 * threads.  Lines are transformed in packed pairs (2i, 2i+1): every even tile gives bitwise the
 * same results; an odd tile pairs some lines differently (differences at rounding level). */
int sgspm_heat_tile(sgspm_t h);
int sgspm_set_heat_tile(sgspm_t h, int tx);
int sgspm_set_packing(sgspm_t h, const int* rows, int n);
int sgspm_autotune(sgspm_t h, int steps, int* rows_out, int cap);

/* Damping alpha per film (nfilm doubles, finite, >= 0), e.g. between a recorded forward and the
 * next; the kernels read it at run time, so captured steps pick it up.  ERR_ARG otherwise. */
int sgspm_set_alpha(sgspm_t h, const double* alpha);

/* Copy a field in (SGSPM_M, SGSPM_HE).  ptr: host or device, layout as above, dtype F32/F64.
 * Device memory of the current device and page-locked host memory (cudaHostAlloc, or registered
 * and mapped) are read in place by the copy kernel; pageable and managed memory are first copied
 * to a device staging buffer on the handle's stream.  Either way the work is ordered on the
 * handle's stream only: a device buffer written on another stream must be complete first.
 * The caller's buffer is read completely before the call returns (it may be reused at once).
 * SGSPM_M: m is normalised on the device; a zero-length or non-finite vector returns ERR_ARG (the
 * call waits for that check); the forward transform of the new m is then enqueued on the stream. */
int sgspm_set_field(sgspm_t h, int which, const void* ptr, int dtype);

/* Copy a field out (SGSPM_M, SGSPM_HS) into host or device memory; synchronises.  Device memory
 * of the current device and page-locked host memory are written in place by the copy kernel,
 * pageable and managed memory through the staging buffer; the result is the same. */
int sgspm_get_field(sgspm_t h, int which, void* ptr, int dtype);

/* Enqueue n >= 1 time steps on the handle's stream (asynchronous). */
int sgspm_step(sgspm_t h, long long n);

/*
 * Discrete energy of the current m, FP64, per film: out[5*f + {0..4}] =
 * {exchange, anisotropy, stray, zeeman, total} with
 *   exchange = V eps/2 sum_faces |m_c - m_c'|^2 / h^2,  anisotropy = V Q/2 sum (|m|^2 - (m.u)^2),
 *   stray = -V/2 sum h_s.m,  zeeman = -V sum h_e.m,  V = hx hy hz
 * (the normalisation for which h_eff = -(1/V) dE/dm; Sec. 2 prints E without the 1/2).
 * Synchronises.
 */
int sgspm_energy(sgspm_t h, double* out);

/* Manufactured forcing of Sec. 5.1: m*** += dt f_e(x, t_n) before projection. */
int sgspm_set_forcing(sgspm_t h, int kind);

/* Simulation time t (per film t = t0 + steps*dt); set resets the step counter. */
int sgspm_set_time(sgspm_t h, double t);
int sgspm_get_time(sgspm_t h, double* t);

/*
 * Adjoint (reverse mode) of the SGSPM step, for gradients of a loss L(m(T)) with respect to the
 * per-cell applied field h_e and the damping alpha.  SGSPM with f refreshed at every state
 * (no SGSPM_GSPM, no SGSPM_FROZEN_STRAY), no manufactured forcing.
 *
 * sgspm_record: from the current m (= m(0)), advance nsteps >= 1 steps, keeping a checkpoint of
 *   the state every K >= 1 steps in device memory (nsteps/K checkpoints).  Afterwards m = m(T).
 *   It also reserves, when the device has room, 29 real fields per step of a segment (K x 29 x
 *   ncell values of the form's precision) for the reverse sweep.
 * sgspm_grad: dL_dmT = dL/dm(T) in the field layout (host or device, dtype SGSPM_F32 or
 *   SGSPM_F64_DATA).  Runs the reverse sweep: each segment is recomputed from its checkpoint in
 *   recording form, keeping every step's intermediates in the reserved fields, and the steps are
 *   then reversed with the hand-written reverse step; without the reserved fields every step is
 *   replayed once more in recording form before its reverse (the same results, more time).  Writes dL/dh_e (same layout and dtype as dL_dmT; the
 *   gradient with respect to a per-cell applied field, also when the field is uniform) and
 *   dL/dalpha (nfilm host doubles).  Only the dependence through m(T) is included: a loss term
 *   on h_e or alpha itself is the caller's.  Synchronises; m is m(T) again on return.
 */
int sgspm_record(sgspm_t h, long long nsteps, int K);
int sgspm_grad(sgspm_t h, const void* dL_dmT, int dtype, void* dL_dhe, double* dL_dalpha);

/* Wait for all enqueued work and report the latched device status. */
int sgspm_sync(sgspm_t h);

/* Release every device buffer and the handle (NULL is a no-op). */
int sgspm_destroy(sgspm_t h);

/* Text of the last error on h (or of the last failed create when h is NULL). */
const char* sgspm_last_error(sgspm_t h);

/*
 * Run ONE time step with a CUDA event between consecutive kernel launches (no graph) and
 * report each launch's device time: ms[i] (milliseconds) and kind[i] = 10*k + v, with
 * k = 0 slab (XZ) pass (v = 1 right-hand sides, 2 Gauss-Seidel update, 3 projection),
 * k = 1 heat-solve line pass and k = 2 stray-field line pass (v = fields / outputs).
 * cap is the capacity of both arrays (>= sgspm_launches_per_step).  Returns the number of
 * launches (>= 0) or a negative status.  The step advances the state like sgspm_step(1).
 */
int sgspm_profile_step(sgspm_t h, float* ms, int* kind, int cap);

/* Number of kernel launches one sgspm_step(1) enqueues (for launch accounting). */
int sgspm_launches_per_step(sgspm_t h);

/*
 * Test support for the bounded waits of the tensor-core (SGSPM_TF32X3) form; the paper has no
 * counterpart.  Every slab-pass CTA of that form waits on an mbarrier for its tcgen05.mma
 * results, with a limit of about one second (or 2^24 polls); a wait that runs out sets a status
 * bit, skips the tensor-memory reads and frees its tensor memory, and the next synchronising
 * call returns SGSPM_ERR_TIMEOUT.  With skip_mma != 0 the slab passes issue neither the MMAs
 * nor their commit, so every such wait runs out with nothing in flight; wait_limit > 0
 * replaces the poll limit (0 restores it).  The switches stay until changed; results computed
 * while skip_mma is set are invalid, and the status stays latched on the handle.
 * Errors: SGSPM_ERR_ARG (NULL handle, wait_limit < 0), SGSPM_ERR_STATE (handle without the
 * tensor-core form), SGSPM_ERR_CUDA.  Synchronises the handle's stream.
 */
int sgspm_test_tc_timeout(sgspm_t h, int skip_mma, int wait_limit);

/*
 * Test support for the bounded waits of the persistent step (SGSPM_PERSISTENT); the paper has no
 * counterpart.  In that step a work item waits, spinning on its film's completion counter, until
 * the film's items of the previous passes are complete; the wait is limited to wait_limit clock
 * cycles (default 4e9, about two seconds).  A wait that runs out sets a status bit and an abandon
 * flag that ends the launch on every CTA; the next synchronising call returns SGSPM_ERR_TIMEOUT.
 * withhold >= 0 names one work item (a ticket of the step's queue, 0-based) that is skipped and
 * never reported complete, so that the waits behind it run out; -1 runs every item.  The settings
 * stay until changed; results of a step with a withheld item are invalid, and the status stays
 * latched on the handle.  Errors: SGSPM_ERR_ARG (NULL handle, wait_limit <= 0), SGSPM_ERR_STATE
 * (handle without SGSPM_PERSISTENT), SGSPM_ERR_CUDA.  Synchronises the handle's stream.
 */
int sgspm_test_persist_wait(sgspm_t h, int withhold, long long wait_limit);

/*
 * sgspm_energy_noalloc - the energy of sgspm_energy for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a library-usage variant.
 *
 * Some callers cannot call cudaMalloc: a plugin whose host application owns every device
 * buffer through its own pool, a process with a fixed device-memory budget, or a latency-
 * critical loop that must not risk the synchronisation an allocation can cause.  This entry
 * point allocates nothing and needs no handle: the caller passes m (and h_s) in its own
 * device buffers and receives the result in its own device buffer.
 *
 *   grid, eps, Q, easy_axis (normalised here), he[3]: as for one film of sgspm_create, with a
 *        uniform applied field (host values);
 *   m:   device pointer, SoA [3][nz][ny][nx], dtype SGSPM_F32 or SGSPM_F64_DATA;
 *   hs:  device pointer to h_s(m) in the same layout and dtype, or NULL (stray term 0);
 *        sgspm_get_field(SGSPM_HS) of a handle yields it;
 *   out: device pointer to 5 doubles {exchange, anisotropy, stray, zeeman, total}
 *        (same definitions as sgspm_energy);
 *   cuda_stream: cudaStream_t on which the work is enqueued (asynchronous; out is valid
 *        once the stream reaches this point).
 *
 * Limits and sharing.  The per-block partial sums live in a fixed file-scope device array
 * of 4096 x 4 doubles (128 KiB per GPU that loads the library, held until exit), so the
 * grid may have at most 16,777,216 cells; larger grids return SGSPM_ERR_UNSUPPORTED.  Every
 * call shares that array: calls that overlap on the GPU (unordered streams) race on it and
 * must be serialised by the caller.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is kept with the driver context it was found in and
 * looked up again when the device's current context is a different one (after
 * cudaDeviceReset, for example); a call that has to look it up again must also come before
 * any stream capture.  Errors: SGSPM_ERR_ARG for bad arguments, SGSPM_ERR_CUDA for a
 * failed CUDA call; the text is returned by sgspm_noalloc_last_error (per host thread).
 */
int sgspm_energy_noalloc(const sgspm_grid* grid, double eps, double Q, const double easy_axis[3],
                         const double he[3], const void* m, const void* hs, int dtype, double* out,
                         void* cuda_stream);

/* Text of the last error of sgspm_energy_noalloc on the calling host thread. */
const char* sgspm_noalloc_last_error(void);

/*
 * Diagnostic: FP64 FMA throughput of the current device in GFLOP/s (a plain kernel of
 * independent DFMA chains, 8 CTAs of 256 threads per SM, timed with CUDA events, best of
 * three after a warm-up).  The roofline denominator of the FP64 form's arithmetic.  Allocates
 * and frees a small device buffer; synchronises the device's legacy default stream.
 * Errors: SGSPM_ERR_ARG (NULL), SGSPM_ERR_OOM, SGSPM_ERR_CUDA.
 */
int sgspm_fp64_fma_peak(double* gflops);

/* ABI version (major*100 + minor); 102 added sgspm_xz_threads and sgspm_set_packing_threads. */
int sgspm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SGSPM_H */
