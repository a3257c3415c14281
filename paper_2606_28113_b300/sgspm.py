"""Thin ctypes binding of libsgspm.so (argument marshalling only).

Every step of the method runs in the library's CUDA kernels; this module converts
Python arguments to the C ABI of include/sgspm.h and raises on negative statuses.
There is no CPU fallback: if the library is missing, `lib()` raises.

Fields are [3, nz, ny, nx] (component, z, y, x).  Pointers may be numpy arrays (host)
or torch tensors (host or CUDA); the library copies them.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libsgspm.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
FP64, GSPM, NO_STRAY, FROZEN_STRAY, NO_GRAPH, TF32X3, PERSISTENT = 1, 2, 4, 8, 16, 32, 64
M, HE, HS = 0, 1, 2
F32, F64 = 0, 1
FORCE_NONE, FORCE_MMS_1D, FORCE_MMS_3D = 0, 1, 3

_lib = None


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double)]


class SGSPMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sgspm status {code}: {msg}")
        self.code = code


def lib():
    """Load libsgspm.so (built in-tree by paper_2606_28113_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise RuntimeError(f"{LIBPATH} is missing: build it with `python -m paper_2606_28113_b300.build`")
    L = ctypes.CDLL(LIBPATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    dp = ctypes.POINTER(ctypes.c_double)
    L.sgspm_create.argtypes = [ctypes.POINTER(Grid), d, d, d, d, dp, i, vp, ctypes.POINTER(vp)]
    L.sgspm_create_batch.argtypes = [i, ctypes.POINTER(Grid), dp, dp, dp, dp, dp, i, vp, ctypes.POINTER(vp)]
    L.sgspm_set_applied_field.argtypes = [vp, dp]
    L.sgspm_set_alpha.argtypes = [vp, dp]
    ip = ctypes.POINTER(ctypes.c_int)
    L.sgspm_xz_classes.argtypes = [vp, ip, ip, i]
    L.sgspm_set_packing.argtypes = [vp, ip, i]
    L.sgspm_xz_threads.argtypes = [vp, ip, i]
    L.sgspm_set_packing_threads.argtypes = [vp, ip, i]
    L.sgspm_autotune.argtypes = [vp, i, ip, i]
    L.sgspm_heat_tile.argtypes = [vp]
    L.sgspm_set_heat_tile.argtypes = [vp, i]
    L.sgspm_set_field.argtypes = [vp, i, vp, i]
    L.sgspm_get_field.argtypes = [vp, i, vp, i]
    L.sgspm_step.argtypes = [vp, ll]
    L.sgspm_energy.argtypes = [vp, dp]
    L.sgspm_set_forcing.argtypes = [vp, i]
    L.sgspm_set_time.argtypes = [vp, d]
    L.sgspm_get_time.argtypes = [vp, dp]
    L.sgspm_sync.argtypes = [vp]
    L.sgspm_destroy.argtypes = [vp]
    L.sgspm_last_error.argtypes = [vp]
    L.sgspm_last_error.restype = ctypes.c_char_p
    L.sgspm_launches_per_step.argtypes = [vp]
    L.sgspm_test_tc_timeout.argtypes = [vp, i, i]
    L.sgspm_test_persist_wait.argtypes = [vp, i, ll]
    L.sgspm_fp64_fma_peak.argtypes = [dp]
    L.sgspm_profile_step.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int), i]
    L.sgspm_version.argtypes = []
    L.sgspm_record.argtypes = [vp, ll, i]
    L.sgspm_record.restype = ctypes.c_int
    L.sgspm_grad.argtypes = [vp, vp, i, vp, dp]
    L.sgspm_grad.restype = ctypes.c_int
    L.sgspm_energy_noalloc.argtypes = [ctypes.POINTER(Grid), d, d, dp, dp, vp, vp, i, vp, vp]
    L.sgspm_energy_noalloc.restype = ctypes.c_int
    L.sgspm_noalloc_last_error.argtypes = []
    L.sgspm_noalloc_last_error.restype = ctypes.c_char_p
    for name in ("sgspm_create", "sgspm_create_batch", "sgspm_set_applied_field", "sgspm_set_alpha", "sgspm_xz_classes", "sgspm_set_packing", "sgspm_xz_threads",
                 "sgspm_set_packing_threads", "sgspm_autotune",
                 "sgspm_heat_tile", "sgspm_set_heat_tile",
                 "sgspm_set_field",
                 "sgspm_get_field", "sgspm_step", "sgspm_energy", "sgspm_set_forcing", "sgspm_set_time",
                 "sgspm_get_time", "sgspm_sync", "sgspm_destroy", "sgspm_launches_per_step", "sgspm_version",
                 "sgspm_test_tc_timeout", "sgspm_test_persist_wait", "sgspm_fp64_fma_peak",
                 "sgspm_profile_step"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _buffer(x):
    """(pointer, dtype code, keep-alive) of a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            code = {torch.float32: F32, torch.float64: F64}[x.dtype]
            return ctypes.c_void_p(x.data_ptr()), code, x
    except ImportError:
        pass
    a = np.ascontiguousarray(x)
    if a.dtype not in (np.float32, np.float64):
        a = a.astype(np.float64)
    return ctypes.c_void_p(a.ctypes.data), (F64 if a.dtype == np.float64 else F32), a


def _flags(fp64, scheme, stray, refresh, graph, tf32x3=False, persistent=False):
    f = 0
    if tf32x3:
        f |= TF32X3
    if fp64:
        f |= FP64
    if scheme == "gspm":
        f |= GSPM
    elif scheme != "sgspm":
        raise ValueError(scheme)
    if not stray:
        f |= NO_STRAY
    if refresh == "R2":
        f |= FROZEN_STRAY
    elif refresh != "R1":
        raise ValueError(refresh)
    if not graph:
        f |= NO_GRAPH
    if persistent:
        f |= PERSISTENT
    return f


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(int(stream))


class Handle:
    """A handle of one film or of a batch of films (sgspm_create / sgspm_create_batch)."""

    def __init__(self, films, fp64=False, scheme="sgspm", stray=True, refresh="R1", graph=True, stream=None,
                 tf32x3=False, persistent=False):
        L = lib()
        self.films = [dict(f) for f in films]
        nf = len(self.films)
        grids = (Grid * nf)(*[Grid(*f["n"], *f["h"]) for f in self.films])
        arr = lambda k: np.ascontiguousarray([float(f[k]) for f in self.films], dtype=np.float64)
        self._eps, self._Q, self._alpha, self._dt = arr("eps"), arr("Q"), arr("alpha"), arr("dt")
        self._u = np.ascontiguousarray([f.get("u", (1.0, 0.0, 0.0)) for f in self.films], dtype=np.float64).reshape(-1)
        self.fp64 = fp64
        self.flags = _flags(fp64, scheme, stray, refresh, graph, tf32x3, persistent)
        h = ctypes.c_void_p()
        rc = L.sgspm_create_batch(nf, grids, _dptr(self._eps), _dptr(self._Q), _dptr(self._alpha), _dptr(self._dt),
                                  _dptr(self._u), self.flags, _stream(stream), ctypes.byref(h))
        if rc != OK:
            raise SGSPMError(rc, L.sgspm_last_error(None).decode())
        self.h = h
        self.ncell = [int(np.prod(f["n"])) for f in self.films]
        he = np.ascontiguousarray([f.get("he", (0.0, 0.0, 0.0)) for f in self.films], dtype=np.float64).reshape(-1)
        if np.any(he != 0):
            self.set_applied_field(he)

    # ---- helpers --------------------------------------------------------------------------
    def _check(self, rc):
        if rc != OK:
            raise SGSPMError(rc, lib().sgspm_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().sgspm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def total_cells(self):
        return sum(self.ncell)

    # ---- fields ----------------------------------------------------------------------------
    def set_applied_field(self, he):
        he = np.ascontiguousarray(np.asarray(he, dtype=np.float64).reshape(-1))
        self._check(lib().sgspm_set_applied_field(self.h, _dptr(he)))

    def set_alpha(self, alpha):
        """Damping alpha per film (a scalar sets every film)."""
        a = np.broadcast_to(np.asarray(alpha, dtype=np.float64).reshape(-1), (len(self.films),))
        a = np.ascontiguousarray(a)
        self._check(lib().sgspm_set_alpha(self.h, _dptr(a)))
        for f, v in zip(self.films, a):
            f["alpha"] = float(v)

    # ---- batch packing ------------------------------------------------------------------------
    def xz_classes(self):
        """[(key, rows per CTA)] of the slab-pass size classes (key = nx, or 0: runtime length)."""
        n = lib().sgspm_xz_classes(self.h, None, None, 0)
        if n < 0:
            self._check(n)
        keys, rows = (ctypes.c_int * max(n, 1))(), (ctypes.c_int * max(n, 1))()
        self._check(min(0, lib().sgspm_xz_classes(self.h, keys, rows, n)))
        return [(keys[c], rows[c]) for c in range(n)]

    def set_packing(self, rows):
        r = (ctypes.c_int * len(rows))(*[int(v) for v in rows])
        self._check(lib().sgspm_set_packing(self.h, r, len(rows)))

    def packing_threads(self):
        """Threads per CTA of each size class's packed (rows > 1) slab launches."""
        n = len(self.xz_classes())
        t = (ctypes.c_int * max(n, 1))()
        self._check(min(0, lib().sgspm_xz_threads(self.h, t, n)))
        return [t[c] for c in range(n)]

    def set_packing_threads(self, threads):
        t = (ctypes.c_int * len(threads))(*[int(v) for v in threads])
        self._check(lib().sgspm_set_packing_threads(self.h, t, len(threads)))

    def heat_tile(self):
        """x lines per CTA of the y heat pass."""
        rc = lib().sgspm_heat_tile(self.h)
        if rc < 0:
            self._check(rc)
        return rc

    def set_heat_tile(self, tx):
        self._check(lib().sgspm_set_heat_tile(self.h, int(tx)))

    def autotune(self, steps=3):
        """Choose rows (and threads) per CTA of every packable size class by timing; returns the rows."""
        n = len(self.xz_classes())
        out = (ctypes.c_int * max(n, 1))()
        rc = lib().sgspm_autotune(self.h, int(steps), out, n)
        if rc < 0:
            self._check(rc)
        return [out[c] for c in range(n)]

    def set_field(self, which, x):
        p, code, keep = _buffer(x)
        self._check(lib().sgspm_set_field(self.h, which, p, code))

    def set_m(self, m):
        self.set_field(M, m)

    def set_he(self, he):
        self.set_field(HE, he)

    def get_field(self, which, out=None, dtype=np.float64):
        if out is None:
            out = np.empty(3 * self.total_cells, dtype=dtype)
        p, code, keep = _buffer(out)
        self._check(lib().sgspm_get_field(self.h, which, p, code))
        return out

    def get_m(self, out=None):
        return self.get_field(M, out)

    def get_hs(self, out=None):
        return self.get_field(HS, out)

    def split(self, flat):
        """Per-film [3, nz, ny, nx] views of a concatenated field array."""
        res, o = [], 0
        for f, nc in zip(self.films, self.ncell):
            nx, ny, nz = f["n"]
            res.append(np.asarray(flat[o:o + 3 * nc]).reshape(3, nz, ny, nx))
            o += 3 * nc
        return res

    # ---- time stepping -----------------------------------------------------------------------
    def step(self, n=1):
        self._check(lib().sgspm_step(self.h, int(n)))

    def sync(self):
        self._check(lib().sgspm_sync(self.h))

    def energy(self):
        out = np.zeros(5 * len(self.films))
        self._check(lib().sgspm_energy(self.h, _dptr(out)))
        return out.reshape(len(self.films), 5)

    def set_forcing(self, kind):
        self._check(lib().sgspm_set_forcing(self.h, int(kind)))

    def set_time(self, t):
        self._check(lib().sgspm_set_time(self.h, float(t)))

    def get_time(self):
        t = ctypes.c_double()
        self._check(lib().sgspm_get_time(self.h, ctypes.byref(t)))
        return t.value

    def record(self, nsteps, K):
        """Advance nsteps from the current m with a checkpoint every K steps (for grad)."""
        self._check(lib().sgspm_record(self.h, int(nsteps), int(K)))

    def grad(self, dL_dmT, out=None):
        """Reverse sweep: returns (dL/dh_e, dL/dalpha per film) for dL/dm(T)."""
        p, code, keep = _buffer(dL_dmT)
        if out is None:
            out = np.empty(3 * self.total_cells, dtype=np.float64 if code == F64 else np.float32)
        q, code2, keep2 = _buffer(out)
        if code2 != code:
            raise ValueError("out must have the dtype of dL_dmT")
        da = np.zeros(len(self.films))
        self._check(lib().sgspm_grad(self.h, p, code, q, _dptr(da)))
        return out, da

    def launches_per_step(self):
        return lib().sgspm_launches_per_step(self.h)

    def test_persist_wait(self, withhold=-1, wait_limit=4000000000):
        """Test support (persistent step): skip one work item so that the waits behind it run out."""
        self._check(lib().sgspm_test_persist_wait(self.h, int(withhold), int(wait_limit)))

    def test_tc_timeout(self, skip_mma, wait_limit=0):
        """Test support (TF32X3 form): skip the tensor-core MMAs so that their bounded waits run out."""
        self._check(lib().sgspm_test_tc_timeout(self.h, int(bool(skip_mma)), int(wait_limit)))

    def profile_step(self):
        """One step with per-launch device times: list of (kind, ms)."""
        cap = self.launches_per_step() + 4
        ms = (ctypes.c_float * cap)()
        kind = (ctypes.c_int * cap)()
        n = lib().sgspm_profile_step(self.h, ms, kind, cap)
        if n < 0:
            self._check(n)
        return [(kind[i], ms[i]) for i in range(n)]


def _trajectory_function():
    import torch

    class Trajectory(torch.autograd.Function):
        """m(T) after `steps` SGSPM steps from m0, differentiable in the per-cell applied field and
        alpha: forward = sgspm_record (checkpoints every K steps), backward = sgspm_grad."""

        @staticmethod
        def forward(ctx, he, alpha, handle, m0, steps, K):
            handle.set_alpha(alpha.detach().double().cpu().numpy())
            handle.set_m(m0)
            handle.set_he(he.detach().contiguous())
            handle.record(steps, K)
            mT = torch.empty(3 * handle.total_cells, dtype=he.dtype, device=he.device)
            handle.get_m(mT)
            ctx.handle = handle
            ctx.alpha_meta = (alpha.shape, alpha.dtype, alpha.device)
            return mT

        @staticmethod
        def backward(ctx, g_mT):
            g_he = torch.empty_like(g_mT)
            _, g_alpha = ctx.handle.grad(g_mT.contiguous(), g_he)
            shape, dtype, device = ctx.alpha_meta
            g_a = torch.as_tensor(g_alpha, dtype=dtype, device=device).reshape(shape)
            return g_he, g_a, None, None, None, None

    return Trajectory


_Trajectory = None


def trajectory(handle, m0, he, alpha, steps, K=50):
    """Differentiable m(T) (flat field layout, dtype and device of `he`) of `handle` from m0 under
    the per-cell applied field `he` (torch tensor, 3 x cells) and damping `alpha` (torch tensor: a
    scalar, or one per film).  Gradients flow to `he` and `alpha` through the hand-written adjoint."""
    global _Trajectory
    if _Trajectory is None:
        _Trajectory = _trajectory_function()
    return _Trajectory.apply(he, alpha, handle, m0, int(steps), int(K))


def energy_noalloc(n, h, eps, Q, u, he, m, hs, out, stream=None):
    """sgspm_energy_noalloc: energy of device fields m, hs (torch CUDA tensors, same dtype)
    into the device tensor `out` (5 float64), without any device allocation."""
    import torch
    dtype = {torch.float32: F32, torch.float64: F64}[m.dtype]
    g = Grid(*n, *h)
    ua = np.ascontiguousarray(u, dtype=np.float64)
    ha = np.ascontiguousarray(he, dtype=np.float64)
    rc = lib().sgspm_energy_noalloc(ctypes.byref(g), float(eps), float(Q), _dptr(ua), _dptr(ha),
                                    ctypes.c_void_p(m.data_ptr()),
                                    ctypes.c_void_p(hs.data_ptr() if hs is not None else 0), dtype,
                                    ctypes.c_void_p(out.data_ptr()), _stream(stream))
    if rc != OK:
        raise SGSPMError(rc, lib().sgspm_noalloc_last_error().decode())


def fp64_fma_peak():
    """Measured FP64 FMA throughput of the current device (GFLOP/s)."""
    v = ctypes.c_double(0.0)
    rc = lib().sgspm_fp64_fma_peak(ctypes.byref(v))
    if rc < 0:
        raise SGSPMError(rc, "sgspm_fp64_fma_peak failed")
    return v.value


def film(n, h, eps, Q, alpha, dt, u=(1.0, 0.0, 0.0), he=(0.0, 0.0, 0.0), **kw):
    """One-film handle."""
    return Handle([dict(n=tuple(n), h=tuple(h), eps=eps, Q=Q, alpha=alpha, dt=dt, u=tuple(u), he=tuple(he))], **kw)
