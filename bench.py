"""Benchmark of the SGSPM hot path on B300: one time step of the 256x256x8 film.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

A "step" is one full SGSPM time step (Sec. 3.2: two heat solves at m^n, the forward and
backward Gauss-Seidel sweeps with their four heat solves and stray-field refreshes, the
damping heat flow and the projection) of a 256x256x8-cell film (h = 1/256, eps = 0.016,
Q = 6.2e-4 along x, stray field on, alpha = 1e-3, h_e = (0.02, 0, 0), dt = 0.01) in the
FP32 form, from a seeded smoothed random state.  Metric: cell-steps/s (cells x steps / s).

Default arm: the CUDA library through its C ABI.  Every timed step starts with a cold L2
(a 256 MiB buffer is written between steps, outside the event pair).  Under torchrun each
rank advances its own replica film (replicas only: a film does not shard), so the
whole-job value is the sum over ranks of cells x steps / max-over-ranks time.

Beside the line, "ensemble" reports the batched workload: 256 films of four sizes (64x64x2,
96x64x2, 128x128x4, 128x64x4; per-film alpha and applied field) stepped together in one
handle, FP32 form, aggregate cell-steps/s (--ensemble-steps, 0 to skip); "strip" the
512x64x4 Neel-wall strip (cell-steps/s and the wall's displacement; --strip-steps).

--impl reference: the FP64 CPU oracle (oracle/) on the host cores, same film and metric,
each step one full oracle step; rank 0 only.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_28113_b300 import inputs  # noqa: E402

WORKLOAD = "film256x256x8_fp32"
METRIC = "SGSPM cell-steps/s (256x256x8 film, FP32 form, stray field on)"
UNIT = "cell-steps/s"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms; summary() keeps the samples read
    between mark_start() and mark_end() (the timed region)."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.t0 = self.t1 = None

    def mark_start(self):
        self.t0 = time.monotonic()

    def mark_end(self):
        self.t1 = time.monotonic()

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.monotonic(), [x.strip() for x in line.split(",")]))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # a row is printed when its sample has been taken: keep rows read in the timed region
        # and up to one interval after it
        rows = [r for t, r in self.rows
                if self.t0 is None or (t >= self.t0 and (self.t1 is None or t <= self.t1 + 0.05))]
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax = float(r[1])
                for n, v in zip(names, r[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(w, m0, nsteps=4):
    """The oracle as it stands, on the host cores: FP64 numpy/scipy with all workers."""
    from oracle import scheme
    cores = os.cpu_count()
    o = scheme.Oracle(scheme.Params(n=w["n"], h=w["h"], eps=w["eps"], Q=w["Q"], alpha=w["alpha"], dt=w["dt"],
                                    u=w["u"], he=w["he"], workers=cores))
    m = m0.copy()
    t0 = time.perf_counter()
    for _ in range(nsteps):
        m = o.step(m, 0.0)
    dt = time.perf_counter() - t0
    ncell = int(np.prod(w["n"]))
    return {"value": ncell * nsteps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nsteps} full oracle steps of the 256x256x8 film (FP64, scipy.fft workers={cores}); "
                      f"Newell set-up excluded"}, m


def whole_job(step_ms, ncell, steps, world, device):
    """Replicas: every rank advances its own film.  Returns (max over ranks of the timed ms,
    whole-job cell-steps/s = world x cells x steps / that time)."""
    if world > 1:
        import torch
        import torch.distributed as tdist
        t = torch.tensor([step_ms], dtype=torch.float64, device=device)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        step_ms = float(t.item())
    return step_ms, world * ncell * steps / (step_ms / 1e3)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = inputs.WORKLOADS[WORKLOAD]
    m0 = inputs.initial_state(w)
    nsteps = max(1, args.steps)
    from oracle import scheme
    cores = os.cpu_count()
    o = scheme.Oracle(scheme.Params(n=w["n"], h=w["h"], eps=w["eps"], Q=w["Q"], alpha=w["alpha"], dt=w["dt"],
                                    u=w["u"], he=w["he"], workers=cores))
    m = m0.copy()
    for _ in range(args.warmup):
        m = o.step(m, 0.0)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        m = o.step(m, 0.0)
    dt = time.perf_counter() - t0
    ncell = int(np.prod(w["n"]))
    value = ncell * nsteps / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": nsteps,
            "warmup": args.warmup, "ms_per_step": dt / nsteps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n": list(w["n"]), "stray": True, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{nsteps} full oracle steps after {args.warmup} warm-up steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it stands (cold
# caches, full metric set, 256x256x8 film).  Only valid for the kernel that was captured: set an
# entry back to None when its kernel changes.
# slab pass, right-hand-side launches (kind 1), 256x256x8 FP32, 512-thread kernel: mean over the 6
# launches of a step of the captured 34.47 MB (2 components) and 22.72 MB (1 component), read + write,
# +11.75 MB per component
NCU_TRAFFIC = {1: 28.6e6}


# algorithmic bytes per cell of each launch kind, FP32: every operator reads its real operand
# fields once and writes its real results once (field crossings x 4 B); padded spectra and
# transposes are implementation overhead, not algorithm
def algorithmic_bytes_per_cell(kind, ncomp=1):
    k, v = divmod(kind, 10)
    if k == 2:            # stray refresh operator: changed inputs read + outputs written
        reads = 3 if v == 2 else 1
        return 4 * (reads + v)
    if k == 1:            # heat solve: read rhs, write solution, per field
        return 4 * 2 * v
    if k == 0:
        if v == 1:        # right-hand sides: read m_a and h_s,a, write r_a, per component
            return 4 * 3 * ncomp
        if v == 2:        # Gauss-Seidel update: read delta, base, two operands, stored delta; write m
            return 4 * 6
        if v == 3:        # damping update + projection: read m** (3) and delta (3), write m (3)
            return 4 * 9
    return None


def run_ensemble(sgspm, torch, stream, steps, warmup=3):
    """Aggregate throughput of the batched workload: 256 films of four sizes in one handle (FP32),
    stepped by per-pass launches (24 per step, CUDA graph) and by one persistent launch per step;
    the line reports the faster form, the other beside it."""
    films = inputs.ensemble(seed=0, nfilm=256)
    m0 = np.concatenate([inputs.random_unit(f["seed"], f["n"]).reshape(-1) for f in films])
    ncell = sum(int(np.prod(f["n"])) for f in films)
    res = {}
    for form, persistent in (("persistent", True), ("per_pass", False)):
        H = sgspm.Handle(films, fp64=False, stream=stream.cuda_stream, persistent=persistent)
        H.set_m(torch.from_numpy(m0.astype(np.float32)).cuda())
        H.step(warmup)
        H.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def timed():
            torch.cuda.synchronize()
            a.record(stream)
            H.step(steps)
            b.record(stream)
            H.sync()
            return a.elapsed_time(b)

        ms_untuned = timed()
        packing = H.autotune(3)     # batch packing of the slab pass chosen by timing
        H.step(1)
        ms = timed()
        r = {"ms_per_step": ms / steps, "value": ncell * steps / (ms / 1e3), "unit": UNIT,
             "launches_per_step": H.launches_per_step(), "ms_per_step_untuned": ms_untuned / steps,
             "autotuned_packing": {f"nx class {k}": p for (k, _), p in zip(H.xz_classes(), packing)},
             "autotuned_packed_threads": {f"nx class {k}": t for (k, p), t in zip(H.xz_classes(), H.packing_threads())
                                          if p > 1}}
        if not persistent:
            prof = {}
            for kind, t in H.profile_step():
                prof[kind] = prof.get(kind, 0.0) + t
            tot = sum(prof.values())
            r["launch_shares"] = {str(k): v / tot for k, v in sorted(prof.items())}
        H.close()
        res[form] = r
    sizes = " | ".join("x".join(map(str, n)) for n in inputs.ENSEMBLE_SIZES)
    # both forms give bitwise the same films (tests/test_gpu_persist.py); the line reports the faster
    names = {"persistent": "persistent: one launch per step over all films (work-item queue)",
             "per_pass": "per-pass launches (24 per step) under a CUDA graph"}
    best = min(res, key=lambda k: res[k]["ms_per_step"])
    other = "per_pass" if best == "persistent" else "persistent"
    head = res[best]
    return {"workload": f"ensemble256 ({sizes}; per-film alpha, h_e)", "films": len(films), "cells": ncell,
            "form": names[best], "value": head["value"], "unit": UNIT, "ms_per_step": head["ms_per_step"],
            "steps": steps, "warmup": warmup, "dtype": "f32", "l2": "working set larger than L2 (no flush)",
            "launches_per_step": head["launches_per_step"], "autotuned_packing": head["autotuned_packing"],
            "autotuned_packed_threads": head["autotuned_packed_threads"],
            "ms_per_step_untuned": head["ms_per_step_untuned"], "launch_shares": res["per_pass"].get("launch_shares"),
            "other_form": dict(res[other], form=names[other])}


def run_strip(sgspm, torch, stream, steps, tf32x3=True):
    """The 512x64x4 strip with a Neel wall (h = 0.1, Q = 0.1, h_e = 0.005 along +x, alpha = 1e-2,
    dt = 0.005), TF32X3 form (else FP32): cell-steps/s and the wall's displacement (zero of
    <m_x>(x), cells)."""
    w = dict(inputs.WORKLOADS["strip512x64x4_wall"], alpha=1e-2)
    m0 = inputs.initial_state(w)
    H = sgspm.film(w["n"], w["h"], w["eps"], w["Q"], w["alpha"], w["dt"], u=w["u"], he=w["he"], fp64=False,
                   stream=stream.cuda_stream, tf32x3=tf32x3)
    H.set_m(m0)
    H.step(3)
    H.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    H.step(steps)
    b.record(stream)
    H.sync()
    ms = a.elapsed_time(b)

    def wall(m):
        mx = m[0].mean(axis=(0, 1))
        i = int(np.nonzero(np.sign(mx[:-1]) != np.sign(mx[1:]))[0][0])
        return i + 0.5 + mx[i] / (mx[i] - mx[i + 1])

    x1 = wall(H.split(H.get_m())[0])
    H.close()
    ncell = int(np.prod(w["n"]))
    return {"workload": "strip512x64x4_wall (Neel wall, alpha 1e-2)", "cells": ncell,
            "form": "tf32x3 (z DCTs on tcgen05)" if tf32x3 else "fp32", "dtype": "f32",
            "value": ncell * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "wall_displacement_cells": x1 - wall(m0), "after_steps": steps + 3,
            "l2": "not flushed (working set in L2)"}


def run_small_configs(sgspm, torch, stream):
    """The 32x32x4 FP64 film (200 steps, against the oracle) and the 128x128x4 adjoint (500
    recorded steps with checkpoints every 50, then the reverse sweep), timed with CUDA events."""
    out = {}
    ev = lambda: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    w = inputs.WORKLOADS["film32x32x4_fp64"]
    m0 = inputs.initial_state(w)
    H = sgspm.film(w["n"], w["h"], w["eps"], w["Q"], w["alpha"], w["dt"], u=w["u"], he=w["he"], fp64=True,
                   stream=stream.cuda_stream)
    H.set_m(m0)
    H.step(3)
    H.set_m(m0)
    a, b = ev()
    a.record(stream)
    H.step(w["steps"])
    b.record(stream)
    H.sync()
    ms = a.elapsed_time(b)
    got = H.split(H.get_m())[0]
    H.close()
    from oracle import scheme
    o = scheme.Oracle(scheme.Params(n=w["n"], h=w["h"], eps=w["eps"], Q=w["Q"], alpha=w["alpha"], dt=w["dt"],
                                    u=w["u"], he=w["he"]))
    m = m0.copy()
    t0 = time.perf_counter()
    for _ in range(w["steps"]):
        m = o.step(m, 0.0)
    cpu_s = time.perf_counter() - t0
    nc = int(np.prod(w["n"]))
    out["film32x32x4_fp64"] = {"steps": w["steps"], "ms_per_step": ms / w["steps"],
                               "value": nc * w["steps"] / (ms / 1e3), "unit": UNIT,
                               "max_abs_dm_vs_oracle": float(np.abs(got - m).max()),
                               "oracle_cpu_value": nc * w["steps"] / cpu_s, "oracle_cpu_cores": os.cpu_count()}
    w = inputs.WORKLOADS["film128x128x4_adjoint"]
    m0 = inputs.initial_state(w)
    n = w["n"]
    nc = int(np.prod(n))
    he = 0.01 * np.random.default_rng(3).normal(size=3 * nc)
    H = sgspm.film(n, w["h"], w["eps"], w["Q"], w["alpha"], w["dt"], u=w["u"], fp64=False, stream=stream.cuda_stream)
    H.set_m(m0)
    H.set_he(he)
    # launch shapes chosen by timing forward steps (m is restored afterwards)
    tuned = {"slab_rows_per_cta": H.autotune(3), "slab_threads": H.packing_threads(), "heat_lines_per_cta": H.heat_tile()}
    a, b = ev()
    a.record(stream)
    H.record(w["steps"], 50)
    b.record(stream)
    H.sync()
    fwd_ms = a.elapsed_time(b)
    mT = H.get_m().reshape(3, -1)
    g = np.zeros_like(mT)
    g[0] = 2.0 * (mT[0] - 1.0) / nc
    a.record(stream)
    H.grad(g.reshape(-1))
    b.record(stream)
    H.sync()
    bwd_ms = a.elapsed_time(b)
    H.close()
    out["film128x128x4_adjoint"] = {"steps": w["steps"], "checkpoint_every": 50, "dtype": "f32",
                                    "record_ms": fwd_ms, "grad_ms": bwd_ms, "autotuned": tuned,
                                    "value": nc * w["steps"] / ((fwd_ms + bwd_ms) / 1e3), "unit": UNIT + " (forward + reverse)"}
    return out


def run_gpu(args):
    import torch
    import torch.distributed as tdist
    from paper_2606_28113_b300 import sgspm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    w = inputs.WORKLOADS[WORKLOAD]
    ncell = int(np.prod(w["n"]))
    m0 = inputs.initial_state(dict(w, seed=w["seed"] + rank))
    stream = torch.cuda.current_stream()
    H = sgspm.film(w["n"], w["h"], w["eps"], w["Q"], w["alpha"], w["dt"], u=w["u"], he=w["he"], fp64=False,
                   stream=stream.cuda_stream, tf32x3=(args.form == "tf32x3"))
    m0_t = torch.from_numpy(m0.astype(np.float32).reshape(-1)).cuda()
    H.set_m(m0_t)
    tuned = ({"slab_rows_per_cta": H.autotune(3), "slab_threads": H.packing_threads(), "heat_lines_per_cta": H.heat_tile()}
             if args.autotune else None)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    H.step(args.warmup)
    H.sync()

    def barrier():
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()

    # ---- device-timed steps, cold L2 before each step -----------------------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        # untimed steps until the sampler reports (at most 3 s), so that it samples the timed region
        t_wait = time.monotonic()
        while clk.proc is not None and not clk.rows and time.monotonic() - t_wait < 3.0:
            H.step(20)
            H.sync()
        barrier()
        clk.mark_start()
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            H.step(1)
            ev[i][1].record(stream)
        barrier()
        clk.mark_end()
    step_ms, value = whole_job(sum(a.elapsed_time(b) for a, b in ev), ncell, args.steps, world, "cuda")
    H.sync()

    # ---- dominant kernel: per-launch device times of one step, L2 warm (inside a long run) ---
    prof = {}
    for _ in range(3):
        for kind, ms in H.profile_step():
            prof.setdefault(kind, []).append(ms)
    share = {k: sum(v) for k, v in prof.items()}
    total = sum(share.values())
    kinds = {0: "xz_slab", 1: "y_heat", 2: "y_stray"}
    per_type = {}
    for k, t in share.items():
        per_type.setdefault(k // 10, 0.0)
        per_type[k // 10] += t
    dom_type = max(per_type, key=per_type.get)
    # roofline of the dominant launch variant of the dominant kernel
    dom_kind = max((k for k in share if k // 10 == dom_type), key=lambda k: share[k])
    dom_ms = float(np.mean(prof[dom_kind]))
    # the right-hand-side slab pass handles 2 components (start of step) or 1 or 3; weight by launches
    ncomp = 1.0
    if dom_kind == 1:
        ncomp = 8.0 / 6.0     # per step: {2, 1, 1, 1, 1, 3} components over 6 launches (SGSPM, R1)
    bpc = algorithmic_bytes_per_cell(dom_kind, ncomp)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    roof = None
    if bpc is not None and hbm:
        achieved = bpc * ncell / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": f"{kinds[dom_type]} (launch kind {dom_kind})", "achieved": achieved,
                "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": bpc * ncell, "launch_ms": dom_ms,
                "kernel_share_of_step": per_type[dom_type] / total,
                "traffic": NCU_TRAFFIC.get(dom_kind) if args.form == "fp32" else None,
                "traffic_unit": "bytes per launch (ncu dram read + write, cold caches)",
                "traffic_source": ("profiles/passes_film256x256x8_fp32.md: ncu --set full of the right-hand-side "
                                   "launches of the 512-thread slab kernel (one capture, mean over a step's six "
                                   "launches)") if args.form == "fp32" and NCU_TRAFFIC.get(dom_kind) else None}
    # whole-step algorithmic fraction (292 B per cell-step, FP32)
    step_frac = 292.0 * value / world / (hbm * 1e9) if hbm else None

    # ---- accuracy of the FP32 form against the FP64 form on the same GPU --------------------
    tc_form = fp64_ms = max_dm = rel_e = None
    if args.side:
        nacc = min(args.steps, 200)
        Ha = sgspm.film(w["n"], w["h"], w["eps"], w["Q"], w["alpha"], w["dt"], u=w["u"], he=w["he"], fp64=False,
                        stream=stream.cuda_stream)
        Hb = sgspm.film(w["n"], w["h"], w["eps"], w["Q"], w["alpha"], w["dt"], u=w["u"], he=w["he"], fp64=True,
                        stream=stream.cuda_stream)
        Hc = sgspm.film(w["n"], w["h"], w["eps"], w["Q"], w["alpha"], w["dt"], u=w["u"], he=w["he"], fp64=False,
                        stream=stream.cuda_stream, tf32x3=True)
        Ha.set_m(m0)
        Hb.set_m(m0)
        Hc.set_m(m0)
        Ha.step(nacc)
        evc = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        Hc.step(2)
        Hc.sync()
        evc[0].record(stream)
        Hc.step(nacc - 2)
        evc[1].record(stream)
        Hc.sync()
        tc_ms = evc[0].elapsed_time(evc[1]) / (nacc - 2)
        ev64 = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        Hb.step(2)
        Hb.sync()
        ev64[0].record(stream)
        Hb.step(nacc - 2)
        ev64[1].record(stream)
        Hb.sync()
        fp64_ms = ev64[0].elapsed_time(ev64[1]) / (nacc - 2)
        ma, mb, mc = Ha.get_m(), Hb.get_m(), Hc.get_m()
        Ea, Eb, Ec = Ha.energy()[0], Hb.energy()[0], Hc.energy()[0]
        Ha.close()
        Hb.close()
        Hc.close()
        tc_form = {"ms_per_step": tc_ms, "value": ncell / (tc_ms / 1e3), "unit": UNIT,
                   "accuracy_vs_fp64_form": {"steps": nacc, "max_abs_dm": float(np.abs(mc - mb).max()),
                                             "rel_energy_err": float(abs(Ec[4] - Eb[4]) / abs(Eb[4]))},
                   "note": "not L2-flushed; z DCTs as 3xTF32 GEMMs on tcgen05"}
        max_dm = float(np.abs(ma - mb).max())
        rel_e = float(abs(Ea[4] - Eb[4]) / abs(Eb[4]))

    # ---- end to end through the C ABI with host buffers -------------------------------------
    host_in = torch.from_numpy(m0.astype(np.float32).reshape(-1)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    ne = max(3, min(args.steps, 50))
    barrier()
    t0 = time.perf_counter()
    for i in range(ne):
        H.set_m(host_in)
        H.step(1)
        H.get_m(host_out)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_val = world * ncell * ne / e2e_s
    launches = args.steps * H.launches_per_step()
    H.close()
    ens = run_ensemble(sgspm, torch, stream, args.ensemble_steps) if args.ensemble_steps > 0 else None
    small = run_small_configs(sgspm, torch, stream) if args.small_configs else None
    strip = None
    if args.strip_steps > 0:
        # both forms of the strip; the chosen form is the faster (both are parity-tested)
        forms = {"fp32": run_strip(sgspm, torch, stream, args.strip_steps, tf32x3=False),
                 "tf32x3": run_strip(sgspm, torch, stream, args.strip_steps, tf32x3=True)}
        chosen = min(forms, key=lambda k: forms[k]["ms_per_step"])
        strip = dict(forms[chosen], chosen_form=chosen, other_form=forms["tf32x3" if chosen == "fp32" else "fp32"])
    fma64 = sgspm.fp64_fma_peak() if args.side else None

    if rank == 0:
        cpu, _ = cpu_baseline(w, m0, nsteps=args.cpu_steps) if args.cpu_steps > 0 else (None, None)
        metric = METRIC if args.form == "fp32" else METRIC.replace("FP32 form", "TF32X3 form")
        line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": list(w["n"]), "h": w["h"][0], "eps": w["eps"], "Q": w["Q"],
                           "alpha": w["alpha"], "dt": w["dt"], "he": list(w["he"]), "stray": True,
                           "parallelism": f"replicas{world}", "l2": "flushed before every timed step (256 MiB write)",
                           "autotuned": tuned},
                "roofline": roof,
                "step_algorithmic_hbm_frac": step_frac,
                "fp64_form": None if fp64_ms is None else {
                    "ms_per_step": fp64_ms, "value": ncell / (fp64_ms / 1e3), "unit": UNIT,
                    "note": "the same fused slab/line kernels in double (runtime-length variants), L2 not flushed",
                    "step_algorithmic_hbm_frac": (584.0 * ncell / (fp64_ms / 1e3) / (hbm * 1e9)) if hbm else None,
                    "fp64_fma_peak_gflops": fma64},
                "speedup_vs_fp64_form": None if fp64_ms is None else (fp64_ms / (step_ms / args.steps)),
                "tf32x3_form": tc_form,
                "accuracy_vs_fp64_form": None if max_dm is None else {"steps": min(args.steps, 200), "max_abs_dm": max_dm,
                                                                       "rel_energy_err": rel_e},
                "launch_shares": {str(k): v / total for k, v in sorted(share.items())},
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 3 * ncell * 4,
                        "d2h_bytes_per_step": 3 * ncell * 4,
                        "path": "sgspm_set_field(pinned host f32) + sgspm_step(1) + sgspm_get_field(pinned host f32)"},
                "gpu_launches": launches,
                "ensemble": ens,
                "small_configs": small,
                "strip": strip,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--form", default="fp32", choices=["fp32", "tf32x3"],
                    help="form of the timed film: FP32 (default) or TF32X3 (z DCTs on the tensor cores)")
    ap.add_argument("--cpu-steps", type=int, default=4, help="oracle steps for cpu_baseline (0: skip)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="choose launch shapes of the timed film with sgspm_autotune before timing (0: defaults)")
    ap.add_argument("--side", type=int, default=1,
                    help="also run the FP64 and TF32X3 forms of the film (accuracy, speed-up) and the FP64 FMA probe (0: skip)")
    ap.add_argument("--small-configs", type=int, default=1,
                    help="also time the 32x32x4 FP64 film and the 128x128x4 adjoint (0: skip)")
    ap.add_argument("--strip-steps", type=int, default=400,
                    help="timed steps of the 512x64x4 Neel-wall strip, reported beside the line (0: skip)")
    ap.add_argument("--ensemble-steps", type=int, default=20,
                    help="timed steps of the 256-film batched workload, reported beside the line (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
