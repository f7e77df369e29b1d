"""Benchmark of one two-stage step of the compact gas-kinetic scheme.

Workload: the Sod shock tube on [0,1]x[0,0.1]^2, 64 x 8 x 8 hexahedra x 6
Kuhn tetrahedra = 24,576 cells (49,280 faces), jittered 10%, y and z
periodic, two-step multi-resolution WENO, full kinetic flux, CFL 0.5.  A
"step" is one pass of the whole hot path: time-step minimum, two stages of
(reconstruction step 1, reconstruction step 2, face flux, cell update).

Metric: Mcell-stage updates/s = cells x 2 stages x steps / device time.
``value`` is the FP32-bulk path; the FP64 path is reported beside it, both
with their L1 density error against the exact Riemann solution at t = 0.2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gks|reference]

Under torchrun (N > 1) every rank advances its own replica of the Sod tube
(the scheme has no data exchange between independent cases): weak scaling,
max time over ranks; the batched leg splits its cases over the ranks.  ``--impl reference`` times the FP64 CPU oracle on the
host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2102_01366_gb300 import inputs as I  # noqa: E402
from paper_2102_01366_gb300 import replicas  # noqa: E402

METRIC = "Mcell-stage updates/s"
WORKLOAD = "sod_tube_64x8x8_hex_x6_tets_24576_cells_weno3_cfl0.5"
CPU_SAMPLE = dict(nx=16, nyz=4)  # same recipe, 1,536 cells: oracle per-cell cost is size independent
FLUSH_BYTES = 512 << 20  # > 129 MB L2
# work of the dominant kernel (face flux) per Gauss point and stage, FP32 flop
# (fadd + fmul + 2 ffma) counted by ncu on this workload (147,840 Gauss points
# a launch), and its DRAM bytes (read + write) per launch, the mean of the
# stage-1 and stage-2 launches, from the same capture (the flux kernel's
# summary under profiles/)
FLUX_FLOPS_PER_GP = {"fp32": (4546.7, 3874.2)}
FLUX_DRAM_BYTES_PER_LAUNCH = 11827840.0
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# algorithmic HBM traffic of one cell-stage: the minimum of the four passes
# the method's two global dependencies impose (neighbour slopes; both sides'
# reconstructions), with perfect on-chip reuse of neighbour data -- FP64
# path 536 words = 4,288 B; FP32 bulk 180 FP64 words (stencil operators,
# geometric moments, averages) + 356 FP32 words = 2,864 B
BYTES_PER_CELL_STAGE = {"fp32": 2864.0, "fp64": 4288.0}


def step_hbm(value_mcs, precision, peaks):
    """HBM roofline of the whole step: algorithmic bytes per cell-stage x the
    measured cell-stage rate, against the measured copy bandwidth."""
    b = BYTES_PER_CELL_STAGE[precision]
    achieved = value_mcs * 1e6 * b / 1e9
    peak = peaks.get("hbm_gbs")
    return {"bound": "hbm", "bytes_per_cell_stage": b, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if peak else None}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[2:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def time_device(torch, s, steps, warmup, flush):
    """Per-step CUDA-event timing on the state's stream, L2 flushed between steps."""
    for _ in range(warmup):
        s.step(1)
    s.sync()
    ms = 0.0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with torch.cuda.stream(s.stream):
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(s.stream)
            s.step(1)
            ev[i][1].record(s.stream)
    s.sync()
    torch.cuda.synchronize()
    for a, b in ev:
        ms += a.elapsed_time(b)
    return ms / steps


def l1_at(torch, gks, mesh, W0, dW0, precision, t_end):
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=precision))
    s.init(W0, dW0)
    t = s.run(t_end=t_end, chunk=64)
    W, _ = s.get()
    exact = I.riemann_x_exact_density(mesh, t)
    vol = g.geometry()["vol"]
    return float((vol * np.abs(W[0].cpu().numpy() - exact)).sum() / vol.sum()), W.cpu().numpy()


_ORACLE_WORKER = """
import sys, time
sys.path.insert(0, {root!r})
from paper_2102_01366_gb300 import inputs as I
from oracle import oracle as O
mesh, W, dW = I.sod_case(nx={nx}, nyz={nyz})
om = O.Mesh(mesh)
p = O.params(weno=1, cfl=0.5)
t0 = time.perf_counter()
for _ in range({n}):
    W, dW, _ = om.step(p, W, dW)
print(time.perf_counter() - t0)
"""


def cpu_baseline(max_seconds=20.0, max_steps=40):
    """The FP64 oracle as it stands on a bounded sample: one thread, then one
    independent copy of the same sample on every host core at once (separate
    processes; the oracle itself is serial), the aggregate being the line's
    value."""
    from oracle import oracle as O
    mesh, W, dW = I.sod_case(**CPU_SAMPLE)
    om = O.Mesh(mesh)
    p = O.params(weno=1, cfl=0.5)
    t0 = time.perf_counter()
    n = 0
    while n < max_steps and (time.perf_counter() - t0) < max_seconds:
        W, dW, _ = om.step(p, W, dW)
        n += 1
    el = time.perf_counter() - t0
    single = om.nc * 2 * n / el / 1e6
    sample = "%d steps of the Sod tube at 16x4x4 hexes x 6 = %d cells (same recipe, 1/16 size), FP64 C oracle" % (
        n, om.nc)
    out = {"value": single, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample + ", 1 thread"}
    cores = os.cpu_count() or 1
    if cores > 1:
        code = _ORACLE_WORKER.format(root=ROOT, nx=CPU_SAMPLE["nx"], nyz=CPU_SAMPLE["nyz"], n=n)
        procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                  text=True) for _ in range(cores)]
        times = []
        for pr in procs:
            try:
                o, _ = pr.communicate(timeout=20 * max_seconds)
                times.append(float(o.strip().splitlines()[-1]))
            except (subprocess.TimeoutExpired, ValueError, IndexError):
                pr.kill()
        if len(times) == cores:
            out = {"value": cores * om.nc * 2 * n / max(times) / 1e6, "unit": METRIC, "cores": cores,
                   "kind": "oracle", "sample": sample + ", one independent copy per core (%d processes)" % cores,
                   "single_thread": {"value": single, "cores": 1}}
    return out


def batched_leg(torch, gks, args, flush):
    """Many independent periodic cases of uneven size in one mesh (each with
    its own time step), FP32 bulk, one CUDA graph per step for the batch.
    Under torchrun the cases are split over the ranks (largest first onto the
    least loaded rank), with no data-path collective: the job's total work
    is fixed (strong scaling), and the value is all ranks' cells x 2 over the
    slowest rank's step time."""
    t0 = time.perf_counter()
    batch, W, dW, desc, meshes = I.batch_cases(n_cases=args.batch_cases, n_range=(8, 40), seed=5)
    ws, rank, _ = replicas.world()
    total_cells = batch["tet"].shape[0]
    if ws > 1:
        mine, my_meshes, W, dW = replicas.rank_batch(meshes, W, dW, ws, rank)
        batch = I.batch_mesh(my_meshes)
    else:
        mine = list(range(len(meshes)))
    g = gks.Mesh(batch)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=1))
    s.init(W, dW)
    setup_s = time.perf_counter() - t0
    tuned = s.autotune(steps=5, cache=False, orders=True)
    steps = max(5, args.steps // 5)
    ms_mine = time_device(torch, s, steps, args.warmup, flush)
    ms = replicas.max_over_ranks(ms_mine)
    t, dt = s.case_times()
    forms = stage_forms(torch, s, max(3, steps // 2), min(args.warmup, 3), flush, ms)
    # the same batch with FP64 stencil operators (precision 2), fewer steps
    del s
    torch.cuda.empty_cache()
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=2))
    s.init(W, dW)
    s.set_cell_order(tuned["cell_order"])
    s.set_variant(*tuned["variant"])  # precision 2 has no one-launch stage
    ms_ops64 = replicas.max_over_ranks(time_device(torch, s, max(3, steps // 3), min(args.warmup, 3), flush))
    del s
    torch.cuda.empty_cache()
    value = total_cells * 2 / (ms / 1000.0) / 1e6
    peaks, src = _peaks()
    return {"workload": "%d periodic cubes of 8^3..40^3 hexes x 6 tets (seed 5), density waves and "
                        "Riemann slabs at Mach 0.5-3, WENO, FP32 bulk, per-case dt" % args.batch_cases,
            "step_hbm": dict(step_hbm(value, "fp32", peaks), peak_source=src),
            "cells": int(total_cells), "faces_rank0": g.nf, "cases": len(meshes), "steps": steps,
            "ms_per_step": ms, "value": value, "unit": METRIC,
            "fp32_ops64": {"ms_per_step": ms_ops64, "value": total_cells * 2 / (ms_ops64 / 1000.0) / 1e6},
            "scaling": "strong (cases split over ranks)" if ws > 1 else "one GPU",
            "rank0_cases": len(mine), "rank0_cells": g.nc,
            "dt_range": [float(dt.min()), float(dt.max())], "host_setup_s": setup_s,
            "autotuned_variant": tuned["variant"], "cell_order": tuned["cell_order"],
            "stage_forms": forms,
            "ms_per_cell_order": dict(zip(("caller", "rcm", "morton"), tuned["ms_per_order"])),
            "l2": "inputs larger than L2 (plus the flush)"}


def stage_forms(torch, s, steps, warmup, flush, ms_chosen):
    """Step time of both forms of a stage on an FP32-bulk state: separate
    reconstruction / flux / update kernels, and one persistent launch per
    stage (gks_state_set_fused); the autotuned one (timed already: ms_chosen)
    is restored.  Timing changes the state; the caller has taken its numbers."""
    chosen = s.fused()
    s.set_fused(1 - chosen)
    ms_other = replicas.max_over_ranks(time_device(torch, s, steps, warmup, flush))
    s.set_fused(chosen)
    ms = {chosen: ms_chosen, 1 - chosen: ms_other}
    return {"chosen": "one launch per stage" if chosen else "separate kernels",
            "ms_per_step_separate": ms[0], "ms_per_step_fused": ms[1]}


def adjoint_leg(torch, gks, args):
    """Cost of the adjoint step against the forward step it differentiates:
    the isentropic vortex on the periodic 64^3 x 6 box (1,572,864 cells),
    FP64, linear weights, the time step frozen.  Both timed with CUDA events
    on the state's stream; the forward step's initialisation is outside its
    timed region, the adjoint call includes the forward recomputation of the
    step it differentiates.  Then a shortened configuration-4 chain: the
    gradient through 20 frozen steps (gks.checkpointed_gradient, its default
    checkpoint spacing) against the 20-step primal run alone, wall clock with
    the device synchronised on both sides."""
    mesh, W, dW = I.isentropic_vortex_case(n=64, order=2)
    g = gks.Mesh(mesh)
    s = gks.State(g, gks.params(weno=0, cfl=0.5, precision=0))
    s.init(W, dW)
    dt = s.timestep()
    Wt, dWt = torch.tensor(W, device="cuda"), torch.tensor(dW, device="cuda")
    # the adjoint of the total kinetic energy sum |rho U|^2 / (2 rho) after the step
    lam_W = torch.zeros_like(Wt)
    lam_W[1:4] = Wt[1:4] / Wt[0]
    lam_W[0] = -0.5 * (Wt[1:4] ** 2).sum(0) / Wt[0] ** 2
    lam_dW = torch.zeros_like(dWt)
    reps = 3
    for _ in range(max(1, args.warmup // 2)):
        s.step(1, dt, 0.0)
        s.sync()
        s.adjoint_step(Wt, dWt, lam_W, lam_dW, dt)
    torch.cuda.synchronize()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s.stream)
        fn()
        b.record(s.stream)
        b.synchronize()
        return a.elapsed_time(b)
    fwd, adj = 0.0, 0.0
    for _ in range(reps):
        s.init(Wt, dWt)
        s.sync()
        fwd += timed(lambda: s.step(1, dt, 0.0)) / reps
    for _ in range(reps):
        adj += timed(lambda: s.adjoint_step(Wt, dWt, lam_W, lam_dW, dt)) / reps
    out = {"workload": "isentropic vortex (strength 5, Ma 0.5 along the diagonal), periodic [0,10]^3, "
                       "64^3 hexes x 6 tets = %d cells, FP64, linear weights, dt frozen" % g.nc,
           "forward_ms": fwd, "adjoint_ms": adj, "adjoint_over_forward": adj / fwd,
           "timing": "CUDA events on the state's stream, %d each after warm-up (forward: the step alone; "
                     "adjoint: its call, which recomputes the step's forward stages)" % reps}
    # the shortened chain: 20 steps, J = kinetic energy at the end
    vol = torch.tensor(g.geometry()["vol"], device="cuda")
    energy = lambda Wc: (vol * (Wc[1:4] ** 2).sum(0) / (2.0 * Wc[0])).sum()
    nsteps = 20
    every = gks.checkpoint_interval(g.nc, nsteps)
    del s
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = gks.State(g, gks.params(weno=0, cfl=0.5, precision=0))  # as the gradient call creates its state
    s.init(Wt, dWt)
    s.step(nsteps, dt, 0.0)
    s.sync()
    primal_s = time.perf_counter() - t0
    del s
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gks.checkpointed_gradient(g, gks.params(weno=0, cfl=0.5, precision=0), Wt, dWt, nsteps, dt, energy)
    torch.cuda.synchronize()
    grad_s = time.perf_counter() - t0
    out["chain20"] = {"steps": nsteps, "checkpoint_every": every, "primal_s": primal_s, "gradient_s": grad_s,
                      "gradient_over_primal": grad_s / primal_s,
                      "timing": "wall clock, device synchronised; each side includes creating its state "
                                "(workspace upload) and one initialisation"}
    return out


def adjoint_chain_leg(torch, gks, args):
    """Gradients through 200 frozen-dt steps of the isentropic vortex on the
    periodic 64^3 x 6 box (1,572,864 cells, linear weights), checkpointed
    every 20 steps, of J = total kinetic energy at the end: with respect to
    the free-stream Mach number (chain rule through the input generator's
    central difference, exact for its quadratic dependence) and along a
    random direction of the initial density field (velocity and pressure
    held).  The adjoint runs with the FP32 primal (FP64 checkpoints, FP64
    reverse sweep) and with the FP64 primal; central differences of FP64
    forward runs check both."""
    nsteps, every, ma, hm = 200, 20, 0.5, 1e-6
    case = lambda m: I.isentropic_vortex_case(n=64, mach=m, order=2)
    mesh, W, dW = case(ma)
    _, Wp, dWp = case(ma + hm)
    _, Wm, dWm = case(ma - hm)
    dW_dma, ddW_dma = (Wp - Wm) / (2 * hm), (dWp - dWm) / (2 * hm)
    g = gks.Mesh(mesh)
    vol = torch.tensor(g.geometry()["vol"], device="cuda")
    prm = gks.params(weno=0, cfl=0.5, precision=0)
    s = gks.State(g, prm)
    s.init(W, dW)
    dt = s.timestep()

    def energy(Wc):
        return (vol * (Wc[1:4] ** 2).sum(0) / (2.0 * Wc[0])).sum()

    def forward(W0, dW0):
        s.init(W0, dW0)
        s.step(nsteps, dt, 0.0)
        s.sync()
        return float(energy(s.get()[0]))

    rng = np.random.Generator(np.random.PCG64(17))
    d = rng.standard_normal(g.nc)  # O(1): a 1e-6 step then moves J well above its rounding
    U = W[1:4] / W[0]
    gm1 = 0.4  # gamma - 1 of the vortex case
    pres = gm1 * (W[4] - 0.5 * (W[1:4] ** 2).sum(0) / W[0])

    def with_rho(rho):
        return np.concatenate([rho[None], rho[None] * U, (pres / gm1 + 0.5 * rho * (U ** 2).sum(0))[None]])
    dW_drho = with_rho(W[0] + 1.0 * d) - with_rho(W[0])  # linear in rho: the directional change
    out = {"workload": "isentropic vortex, periodic 64^3 hexes x 6 tets = %d cells, linear weights, "
                       "%d steps of dt %.4g frozen, checkpoint every %d" % (g.nc, nsteps, dt, every),
           "loss": "total kinetic energy at the end"}
    t0 = time.perf_counter()
    fd_ma = (forward(Wp, dWp) - forward(Wm, dWm)) / (2 * hm)
    hr = 1e-6
    fd_rho = (forward(W + hr * dW_drho, dW) - forward(W - hr * dW_drho, dW)) / (2 * hr)
    out["fd_seconds"] = time.perf_counter() - t0
    out["fd"] = {"dJ_dMa": fd_ma, "dJ_drho_along_d": fd_rho}
    for name, prec in (("fp32_primal", 1), ("fp64_primal", 0)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, lW, ldW = gks.checkpointed_gradient(g, prm, W, dW, nsteps, dt, energy, checkpoint_every=every,
                                               primal_precision=prec)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        lW, ldW = lW.cpu().numpy(), ldW.cpu().numpy()
        ad_ma = float((lW * dW_dma).sum() + (ldW * ddW_dma).sum())
        ad_rho = float((lW * dW_drho).sum())
        out[name] = {"J": J, "dJ_dMa": ad_ma, "dJ_drho_along_d": ad_rho,
                     "rel_err_dMa": abs(ad_ma - fd_ma) / abs(fd_ma),
                     "rel_err_drho": abs(ad_rho - fd_rho) / abs(fd_rho), "seconds": el}
    # cost against the primal alone
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    forward(W, dW)
    out["fp64_forward_seconds"] = time.perf_counter() - t0
    return out


def sphere_leg(torch, gks, args, flush):
    """Viscous flow past a sphere, Re 100 on the diameter, Ma 0.2, Pr 0.72: the O-type
    shell of 64 radial (ratio 1.08) x 96 polar x 192 azimuthal hexes x 6
    tets (3 on the pole rows) = 7,004,160 cells, far field at r = 20, flat
    faces (the split mirrored in theta on the southern half), WENO,
    started from the free stream.  The first steps are timed
    in FP32 bulk and in FP64 (CUDA events per step, L2 flushed), and the two
    states are compared after the same steps.  The wall cells reconstruct
    their momenta by the constrained least squares of Sec. 4.4."""
    t0 = time.perf_counter()
    mesh, W, dW, mu = I.sphere_case()
    g = gks.Mesh(mesh)
    setup_s = time.perf_counter() - t0
    # the wall cells' momenta by the constrained least squares of Sec. 4.4
    kw = dict(weno=1, cfl=0.5, viscous=1, mu=mu, prandtl=0.72, wall_constraint=1)
    out = {"workload": "sphere Re 100 Ma 0.2, O-type shell 64 x 96 x 192 hexes x 6 tets (3 on pole rows), "
                       "r 0.5..20, radial ratio 1.08, flat faces, WENO, viscous (mu 0.002, Pr 0.72), "
                       "constrained wall reconstruction, from the free stream",
           "cells": g.nc, "faces": g.nf, "boundary_faces": g.n_boundary, "host_setup_s": setup_s}
    states = {}
    for name, prec, steps in (("fp32", 1, max(5, args.steps // 5)), ("fp64", 0, 3)):
        s = gks.State(g, gks.params(precision=prec, **kw))
        s.init(W, dW)
        if prec == 1:
            tuned = s.autotune(steps=3, cache=False, orders=True)
        ms = replicas.max_over_ranks(time_device(torch, s, steps, min(args.warmup, 3), flush))
        t, _ = s.time()
        out[name] = {"ms_per_step": ms, "value": replicas.world()[0] * g.nc * 2 / (ms / 1000.0) / 1e6,
                     "steps_timed": steps, "t": t, "variant": list(s.variant), "cell_order": s.cell_order}
        if prec == 1:
            out[name]["ms_per_cell_order"] = dict(zip(("caller", "rcm", "morton"), tuned["ms_per_order"]))
            out[name]["stage_forms"] = stage_forms(torch, s, steps, min(args.warmup, 3), flush, ms)
        s.init(W, dW)
        s.step(3)
        s.sync()
        states[name] = s.get()[0].cpu().numpy()
        del s
        torch.cuda.empty_cache()
    # differences after the same 3 steps, each component against its free-stream
    # scale (rho, rho |U|, rho |U|, rho |U|, rho E)
    a, b = states["fp32"], states["fp64"]
    scale = [W[0, 0], W[1, 0], W[1, 0], W[1, 0], W[4, 0]]
    out["fp32_vs_fp64_after_3_steps"] = {n: float(np.abs(a[q] - b[q]).max() / scale[q])
                                         for q, n in enumerate(("rho", "rho_u", "rho_v", "rho_w", "rho_E"))}
    out["unit"] = METRIC
    peaks, src = _peaks()
    out["step_hbm"] = {"fp32": step_hbm(out["fp32"]["value"], "fp32", peaks),
                       "fp64": step_hbm(out["fp64"]["value"], "fp64", peaks), "peak_source": src}
    return out


_ORACLE_STEPPER = """
import sys
sys.path.insert(0, {root!r})
from paper_2102_01366_gb300 import inputs as I
from oracle import oracle as O
mesh, W, dW = I.sod_case(nx={nx}, nyz={nyz})
om = O.Mesh(mesh)
p = O.params(weno=1, cfl=0.5)
print("ready", flush=True)
for line in sys.stdin:
    if line.strip() != "s":
        break
    W, dW, _ = om.step(p, W, dW)
    print("done", flush=True)
"""


def run_reference(args):
    """The oracle as it stands on the host cores: one independent copy of the
    bounded sample per core (separate processes, the oracle being serial),
    all advanced one step per timed step."""
    ws, rank, _ = replicas.world()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    mesh, _, _ = I.sod_case(**CPU_SAMPLE)
    nc = mesh["tet"].shape[0]
    cores = os.cpu_count() or 1
    code = _ORACLE_STEPPER.format(root=ROOT, nx=CPU_SAMPLE["nx"], nyz=CPU_SAMPLE["nyz"])
    procs = [subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                              stderr=subprocess.DEVNULL, text=True, bufsize=1) for _ in range(cores)]
    try:
        for pr in procs:
            if pr.stdout.readline().strip() != "ready":
                raise RuntimeError("an oracle worker did not start")

        def one_step():
            for pr in procs:
                pr.stdin.write("s\n")
                pr.stdin.flush()
            for pr in procs:
                if pr.stdout.readline().strip() != "done":
                    raise RuntimeError("an oracle worker failed")
        for _ in range(args.warmup):
            one_step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            one_step()
        el = time.perf_counter() - t0
    finally:
        for pr in procs:
            try:
                pr.stdin.write("q\n")
                pr.stdin.close()
            except OSError:
                pass
            try:
                pr.wait(timeout=30)
            except subprocess.TimeoutExpired:
                pr.kill()
    v = cores * nc * 2 * args.steps / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1000 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_cells": nc, "cells": 24576},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": cores, "kind": "oracle",
                             "sample": "each step one oracle step of the Sod tube at 16x4x4 hexes x 6 = "
                                       "%d cells (same recipe, 1/16 size) on each of %d cores (independent "
                                       "copies, one process each)" % (nc, cores)},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gks", choices=["gks", "reference"])
    ap.add_argument("--profile-case", action="store_true",
                    help="only the FP32 timed steps (for profilers); no accuracy, e2e or CPU legs")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="precision of --profile-case")
    ap.add_argument("--variant", default="auto",
                    help="execution variant of --profile-case: face_order,flux_blocks,slopes_pass "
                         "(e.g. 1,3,1) or auto (tuned as in the full run)")
    ap.add_argument("--fused", type=int, default=-1, choices=[-1, 0, 1],
                    help="stage form of --profile-case: 1 one launch per stage, 0 separate kernels, "
                         "-1 as tuned (auto) or separate (explicit --variant)")
    ap.add_argument("--batch-cases", type=int, default=48,
                    help="independent cases of the batched leg (0: skip it)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-cost leg")
    ap.add_argument("--no-sphere", action="store_true", help="skip the 7M-cell viscous sphere leg")
    ap.add_argument("--adjoint-chain", action="store_true",
                    help="also run the 200-step checkpointed gradient of the 64^3 vortex (minutes)")
    ap.add_argument("--profile-adjoint", action="store_true",
                    help="only two adjoint steps on the periodic 16^3 x 6 density wave (for profilers)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2102_01366_gb300 import _build, gks
    ws, rank, local = replicas.world()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()
    if ws > 1:
        dist.barrier()
    gks.lib()

    mesh, W0, dW0 = I.sod_case()
    g = gks.Mesh(mesh)
    nc = g.nc
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    if args.profile_adjoint:
        mesh_a, Wa, dWa = I.sine_wave_case(n=16)
        ga = gks.Mesh(mesh_a)
        sa = gks.State(ga, gks.params(weno=0, cfl=0.5, precision=0))
        sa.init(Wa, dWa)
        dta = sa.timestep()
        Wt, dWt = torch.tensor(Wa, device="cuda"), torch.tensor(dWa, device="cuda")
        for _ in range(2):
            sa.adjoint_step(Wt, dWt, torch.ones_like(Wt), torch.ones_like(dWt), dta)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_adjoint": "density wave 16^3 x 6 = %d cells, FP64, linear weights" % ga.nc}))
        return

    if args.profile_case:
        prec = 1 if args.precision == "fp32" else 0
        s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=prec))
        s.init(W0, dW0)
        if args.variant == "auto":
            s.autotune(steps=10, cache=False)
        else:
            s.set_variant(*[int(v) for v in args.variant.split(",")])
        if args.fused >= 0:
            s.set_fused(args.fused)
        ms = time_device(torch, s, args.steps, args.warmup, flush)
        if rank == 0:
            print(json.dumps({"profile_case": WORKLOAD, "precision": args.precision, "variant": s.variant,
                              "fused": s.fused(), "ms_per_step": ms}))
        return

    results = {}
    for name, prec in (("fp64", 0), ("fp32", 1), ("fp32_ops64", 2)):
        s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=prec))
        s.init(W0, dW0)
        tuned = s.autotune(steps=10, cache=False, orders=prec != 0)  # restores the state
        if name == "fp32":
            with ClockSampler(local) as clk:
                ms = time_device(torch, s, args.steps, args.warmup, flush)
            clocks = clk.summary()
        else:
            ms = time_device(torch, s, max(3, args.steps // 5), args.warmup, flush)
        ms = replicas.max_over_ranks(ms)
        fused = s.fused()
        forms = stage_forms(torch, s, max(3, args.steps // 5), args.warmup, flush, ms) if prec == 1 else None
        # kernel breakdown: same steps, kernel by kernel, events between launches
        # (the separate kernels, so that the flux launches are timed alone;
        # with the one-launch stage also its two launches)
        nbr = max(3, args.steps // 5 if name != "fp32" else args.steps)
        br = {}
        for f in ((0, 1) if prec == 1 else (0,)):
            if prec == 1:
                s.set_fused(f)
            s.init(W0, dW0)
            for _ in range(args.warmup):
                s.step(1)
            s.sync()
            for k, v in s.step_timed(nbr).items():
                if v[1] > 0:
                    br[k] = v
        if prec == 1:
            s.set_fused(fused)
        results[name] = {"ms": ms, "breakdown": br, "variant": tuned["variant"], "fused": fused, "forms": forms,
                         "cell_order": tuned.get("cell_order", 0)}
    # equal-L1 comparison at t = 0.2 (untimed)
    l1_64, W64 = l1_at(torch, gks, mesh, W0, dW0, 0, 0.2)
    l1_32, W32 = l1_at(torch, gks, mesh, W0, dW0, 1, 0.2)
    l1_32o, W32o = l1_at(torch, gks, mesh, W0, dW0, 2, 0.2)
    fp32_vs_fp64 = max(np.abs(W32[q] - W64[q]).max() / np.abs(W64[q]).max() for q in range(5))
    ops64_vs_fp64 = max(np.abs(W32o[q] - W64[q]).max() / np.abs(W64[q]).max() for q in range(5))

    # end to end through the host-buffer entry point (pinned buffers, copies timed)
    s = gks.State(g, gks.params(weno=1, cfl=0.5, precision=1))
    s.set_cell_order(results["fp32"]["cell_order"])
    s.set_variant(*results["fp32"]["variant"])  # the autotuned variant, as a user's cached autotune() sets it
    s.set_fused(results["fp32"]["fused"])
    Wh = torch.tensor(W0).pin_memory()
    dWh = torch.tensor(dW0).pin_memory()
    for _ in range(args.warmup):
        s.step_host(Wh, dWh, nsteps=1)
    Wh.copy_(torch.tensor(W0))
    dWh.copy_(torch.tensor(dW0))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step_host(Wh, dWh, nsteps=1)
    e2e_s = replicas.max_over_ranks((time.perf_counter() - t0) / args.steps)

    ms32 = results["fp32"]["ms"]
    value = ws * nc * 2 / (ms32 / 1000.0) / 1e6
    value64 = ws * nc * 2 / (results["fp64"]["ms"] / 1000.0) / 1e6
    br = results["fp32"]["breakdown"]
    flux_ms = (br["flux1"][0] + br["flux2"][0]) / max(1, br["flux1"][1] + br["flux2"][1])
    sep = ("slopes", "recon", "flux1", "update1", "flux2", "update2")
    total_ms = sum(br[k][0] for k in sep if k in br)
    nst = max(1, br["flux1"][1])  # steps in the breakdown pass
    # launches per timed step: the control kernel + the chosen form's kernels
    if results["fp32"]["fused"]:
        launches_per_step = 1 + (br["stage1"][1] + br["stage2"][1]) / nst
    else:
        launches_per_step = 1 + sum(br[k][1] for k in sep if k in br) / nst
    gps = 3 * g.nf
    peaks, peak_src = _peaks()
    clk_mhz = SM_MAX_MHZ
    fp32_peak = SM_COUNT * FP32_LANES * 2 * clk_mhz * 1e6 / 1e12
    fpg = FLUX_FLOPS_PER_GP["fp32"]
    if fpg:
        # both stage variants: total flop of the two launches over their total time
        t_flux = (br["flux1"][0] + br["flux2"][0]) / max(1, br["flux1"][1])
        achieved = (fpg[0] + fpg[1]) * gps / (t_flux / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": FLUX_DRAM_BYTES_PER_LAUNCH, "kernel": "k_flux<float>",
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % clk_mhz,
                "flux_ms_per_launch": flux_ms, "flux_share_of_step": sum(
                    br[k][0] for k in ("flux1", "flux2")) / total_ms}
    else:
        roof = {"bound": "alu", "achieved": None, "peak": fp32_peak, "unit": "TFLOP/s", "frac": None,
                "traffic": None, "kernel": "k_flux<float>", "flux_ms_per_launch": flux_ms,
                "flux_share_of_step": sum(br[k][0] for k in ("flux1", "flux2")) / total_ms}
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": nc, "faces": g.nf, "precision": "fp32-bulk",
                   "l2": "flushed between timed steps (512 MB write)", "graph": "one CUDA graph per step",
                   "replicas": ws},
        "fp64": {"value": value64, "ms_per_step": results["fp64"]["ms"], "dtype": "f64",
                 "step_hbm": step_hbm(value64, "fp64", peaks)},
        "step_hbm": dict(step_hbm(value, "fp32", peaks), peak_source=peak_src,
                         note="latency-bound size: the 24,576-cell workspace fits in L2"),
        "autotuned_variant": {"fp32": results["fp32"]["variant"], "fp64": results["fp64"]["variant"],
                              "meaning": "[face_order, flux_blocks_per_SM, slopes_pass]",
                              "fp32_stage_forms": results["fp32"]["forms"],
                              "fp32_cell_order": results["fp32"]["cell_order"],
                              "cell_orders": "0 caller's, 1 reverse Cuthill-McKee, 2 Morton"},
        "accuracy_t0.2": {"l1_rho_fp64": l1_64, "l1_rho_fp32": l1_32, "l1_rho_fp32_ops64": l1_32o,
                          "fp32_vs_fp64_rel": fp32_vs_fp64, "fp32_ops64_vs_fp64_rel": ops64_vs_fp64},
        "fp32_ops64": {"value": ws * nc * 2 / (results["fp32_ops64"]["ms"] / 1000.0) / 1e6,
                       "ms_per_step": results["fp32_ops64"]["ms"],
                       "meaning": "FP32 bulk with the stencil operators, moments and their products in FP64"},
        "fp32_speedup_over_fp64": value / value64,
        "kernel_ms_per_step": {k: v[0] / nst for k, v in br.items() if v[1] > 0},
        "roofline": roof,
        "e2e": {"value": ws * nc * 2 / e2e_s / 1e6, "unit": METRIC,
                "h2d_bytes_per_step": 20 * nc * 8, "d2h_bytes_per_step": 20 * nc * 8},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clocks,
        "peaks": {"source": peak_src, **{k: peaks[k] for k in ("hbm_gbs", "bf16_tflops") if k in peaks}},
    }
    if args.batch_cases > 0:
        line["batched"] = batched_leg(torch, gks, args, flush)
    if not args.no_adjoint:
        line["adjoint"] = adjoint_leg(torch, gks, args)
    if not args.no_sphere:
        line["sphere"] = sphere_leg(torch, gks, args, flush)
    if args.adjoint_chain:
        line["adjoint_chain"] = adjoint_chain_leg(torch, gks, args)
    if rank == 0 and ws == 1:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
