#!/usr/bin/env python
"""Benchmark of the nDGP fifth-force hot path on one GB300 (or N replicas).

One step is one pass of the whole path over the refinement workload:
  coefficients (Eq. beta) -> FP64 FAS solve of the periodic 128^3 domain grid
  (full-multigrid start) to relative residual 1e-10 + force (Sec. 3.1) -> coarse->fine interpolation
  onto the 2x-refined 64^3 patch over the densest 32^3 coarse cells + force
  on it (the truncated fine level, Sec. 3.2) -> relaxation of the same patch
  with the interpolated Dirichlet ghosts + force (the untruncated level) ->
  mixed-precision (FP64 defect correction around FP32 V-cycles) solve of the
  domain grid to 1e-8 + force.
The metric is cell-updates/s over the step (one cell relaxed in one full
red+black sweep, on every grid), with each phase's time-to-tolerance beside it.

Inputs are synthetic (seeded lognormal Gaussian random fields standing in for
the paper's N-body densities); they are resident in HBM before the timed
region.  The L2 cache (129 MB) is flushed between timed steps by writing a
512 MB buffer.  `--impl reference` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "cell-updates/s & V-cycle time-to-tol (FP64 vs mixed/batched), % HBM peak; p50/p99"
UNIT = "cell-updates/s"
L_BOX = 250.0                  # Mpc/h, the paper's box (Sec. 4.1)
N_FINE, SIGMA, SEED, PN = 256, 1.5, 2, 32
N_COARSE = N_FINE // 2
H_COARSE = L_BOX / N_COARSE    # the 128^3 grid of a 256^3-cell field: 1.95 Mpc/h
TOL64, TOLMIX = 1e-10, 1e-8
NU_COARSE_CAP = 4        # coarsest-grid sweeps a visit in the FP64 solves of the step
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12   # 2 FP64 FMA/clk/SM x 152 SMs x 2.07 GHz x 2 flop
FP64_PEAK_SOURCE = ("derived FP64: 2 FMA/clk/SM x 152 SMs x 2.07 GHz x 2 flop = 1.259 TFLOP/s "
                    "(MEASURED_PEAKS.json has no FP64 figure; an 8-chain FMA probe measured 1.195)")
# The smoother's flops a cell update in the hot-path scope table's own count (about 60
# arithmetic operations, one square root and one divide), reported beside the operation-by-
# operation count of WORK for the same kernel.
SURVEY_FLOPS_SWEEP64 = 62.0

# algorithmic work per cell of each kernel class: (bound, bytes, flops)
#   sweep: read phi + f, write phi (the full red+black sweep of one cell);
#   FP64 smoother: 40 flops per cell update, the method's operations counted one by one
#   (FMA = 2; sqrt and divide 1 each): face sums 5, a, b, c 3, a^2 + bc 3, the three mixed
#   differences 9, their squares 5, b = rhs + alpha Sigma 4, the closed-form root 6,
#   S - h^2 L 2, the relaxed update omega v_root + (1 - omega) v 3
WORK = {
    "sweep64": ("alu", 24.0, 40.0),
    "patch_sweep64": ("alu", 24.0, 40.0),
    "resid_restrict64": ("alu", 19.0, 38.0),    # read v, f; write vc, v0c, rc (1/8 each)
    "sweep32": ("hbm", 16.0, 60.0),          # correction form: read e, B, f; write e
    "resid_restrict32": ("hbm", 13.5, 60.0),    # read e, B, f; write vc, v0c, rc
    "resid64_mixed": ("alu", 24.0, 36.0),     # read phi64, f64; write r32, B32
    "update_mixed": ("hbm", 20.0, 1.0),
    "force64": ("hbm", 32.0, 6.0),
    "sweep64_coarse": ("alu", 24.0, 40.0),
    "sweep32_coarse": ("hbm", 16.0, 60.0),
    "patch_sweep64_coarse": ("alu", 24.0, 40.0),
    "refine64": ("hbm", 9.0, 25.0),
    "prolong64": ("hbm", 18.0, 20.0),
    "prolong32": ("hbm", 9.0, 20.0),
}


# DRAM bytes per cell measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum of one
# launch / its cells), for the kernel as it stands; a launch's traffic = this x its cells.
#   sweep32: k_sweep_march, 256^3 finest-grid launch: 204.6 + 50.7 MB / 16.78 M cells
#   resid_restrict32: k_resid_restrict_march, 256^3 finest grid: 203.2 + 18.7 MB / 16.78 M cells
#   sweep64: k_sweep_red + k_sweep_black<double,0>, 128^3 finest grid
TRAFFIC_PER_CELL = {
    "sweep32": 255.2e6 / 256 ** 3,
    "resid_restrict32": 221.9e6 / 256 ** 3,
    "sweep64": 89.6e6 / 128 ** 3,          # red + black launch, cold-cache ncu capture at 128^3
}


def step_params(mg, alpha, s):
    """Parameters of the step's three solves: (FP64 128^3 domain solve, mixed 128^3 solve,
    FP64 64^3 patch relaxation).  V(3,1) for the domain solve: with the over-relaxed smoother it
    reaches 1e-10 in 5 cycles instead of V(2,2)'s 6 (time to tolerance 12% lower at 128^3; the
    paper fixes no cycle shape).  Both FP64 solves cap the 4^3 coarsest-grid solve at 4 sweeps a
    visit: the V-cycle counts stay 5 and 6, and the latency-bound single-CTA sweeps drop from
    ~14 a visit."""
    p64 = mg.default_params(alpha=alpha, s=s, h=H_COARSE, tol=TOL64, nu1=3, nu2=1,
                            nu_coarse=NU_COARSE_CAP)
    pmix = mg.default_params(alpha=alpha, s=s, h=H_COARSE, tol=TOLMIX, precision="mixed")
    ppatch = mg.default_params(alpha=alpha, s=s, h=H_COARSE / 2, tol=TOL64, nu_coarse=NU_COARSE_CAP)
    return p64, pmix, ppatch


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_replicas(ms: float, cells: float, device, world_size: int):
    """Replicas only: every rank solves its own copy of the workload; the job time is
    the slowest rank's and the work is the sum over ranks (no data-path collective)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    c = torch.tensor([float(cells)], dtype=torch.float64, device=device)
    if world_size > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def make_inputs():
    import workload
    coarse, patch, origin = workload.patch_workload(N_FINE, SIGMA, SEED, PN)
    return coarse, patch, origin


# ---------------------------------------------------------------- our arm

class Step:
    """One pass of the path.  The mixed-precision solve of the domain grid does not
    depend on the FP64 chain (solve -> interpolate -> relax), so it runs on a second
    stream with its own context, concurrently: the FP64 chain keeps the FP64 pipes
    busy while the mixed solve's FP32 kernels use the memory system."""

    def __init__(self, mg, torch, coarse, patch, origin, dev):
        self.mg, self.torch = mg, torch
        f64 = torch.float64
        self.ctx = mg.Context(dev.index or 0)
        self.ctx2 = mg.Context(dev.index or 0)
        self.s1 = torch.cuda.Stream(device=dev)
        self.s2 = torch.cuda.Stream(device=dev)
        self.beta, self.alpha, self.s = mg.ndgp_coefficients(1.0, 0.3, 1.0)
        self.origin = origin
        self.d_c = torch.from_numpy(coarse).to(dev)
        self.d_p = torch.from_numpy(patch).to(dev)
        n, pf = N_COARSE, 2 * PN
        self.phi = torch.zeros((n,) * 3, dtype=f64, device=dev)
        self.grad = torch.empty((3,) + (n,) * 3, dtype=f64, device=dev)
        self.phi_m = torch.zeros_like(self.phi)
        self.grad_m = torch.empty_like(self.grad)
        self.box = torch.empty((pf + 2,) * 3, dtype=f64, device=dev)
        self.box_full = torch.empty_like(self.box)
        self.g_tr = torch.empty((3,) + (pf,) * 3, dtype=f64, device=dev)
        self.g_full = torch.empty_like(self.g_tr)
        self.p64, self.pmix, self.ppatch = step_params(mg, self.alpha, self.s)
        self.graph = True
        self.serial = False
        torch.cuda.synchronize()

    def profile(self, on):
        # events around each launch cannot sit inside a graph: the profiled pass runs the same
        # kernels host-driven, the timed pass replays the captured FP64 solve; and it runs the
        # mixed solve after the FP64 chain instead of beside it, so that every kernel's event-timed
        # span is its own (concurrent launches stretch each other's spans)
        self.graph = not on
        self.serial = on
        self.ctx.profile_enable(on)
        self.ctx2.profile_enable(on)

    def profile_read(self):
        a, b = self.ctx.profile_read(), self.ctx2.profile_read()
        return {k: (a[k][0] + b[k][0], a[k][1] + b[k][1], a[k][2] + b[k][2]) for k in a}

    def run(self, host_io=None):
        """One step; returns (cell updates, per-phase ms, infos, step ms on the device)."""
        torch, ctx = self.torch, self.ctx
        s1, s2 = self.s1, self.s2
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        out = {}

        def mixed(after):
            with torch.cuda.stream(s2):
                s2.wait_event(after)
                ev[5].record(s2)
                if host_io is None:
                    _, _, out["im"] = self.ctx2.solve_fifth_force(self.d_c, self.pmix,
                                                                  phi=self.phi_m, grad=self.grad_m,
                                                                  stream=s2)
                else:   # delta in from the host, phi and grad out to it, inside the call
                    _, _, out["im"] = self.ctx2.solve_fifth_force_host(
                        host_io["delta"], self.pmix, phi=host_io["phi_m"], grad=host_io["grad_m"],
                        stream=s2)
                ev[6].record(s2)

        with torch.cuda.stream(s1):
            # a1: coefficients of Eq. (beta) / Eq. (eomvarphi) at a = 1
            self.beta, self.alpha, self.s = self.mg.ndgp_coefficients(1.0, 0.3, 1.0)
            ev[0].record(s1)
            if not self.serial:
                th = threading.Thread(target=mixed, args=(ev[0],))
                th.start()
            if host_io is None:
                _, _, i64 = ctx.solve_fifth_force(self.d_c, self.p64, phi=self.phi, grad=self.grad,
                                                  stream=s1, fmg=True, graph=self.graph)
            else:
                _, _, i64 = ctx.solve_fifth_force_host(host_io["delta"], self.p64,
                                                       phi=host_io["phi"], grad=host_io["grad"],
                                                       stream=s1, fmg=True, graph=self.graph)
                self.phi.copy_(host_io["phi"], non_blocking=True)
                self.d_p.copy_(host_io["patch"], non_blocking=True)
            ev[1].record(s1)
            self.compat_c = i64.compat_c
            ctx.refine_interpolate(self.phi, self.origin, (PN, PN, PN), 1, out=self.box, stream=s1)
            ctx.force(self.box, H_COARSE / 2, ghost=1, periodic=False, grad=self.g_tr, stream=s1)
            ev[2].record(s1)
            self.box_full.copy_(self.box)
            _, ip = ctx.relax_patch(self.d_p, self.ppatch, i64.compat_c, self.box_full, stream=s1,
                                    graph=self.graph)
            ctx.force(self.box_full, H_COARSE / 2, ghost=1, periodic=False, grad=self.g_full,
                      stream=s1)
            ev[3].record(s1)
            if self.serial:
                mixed(ev[3])
            else:
                th.join()
            s1.wait_event(ev[6])
            if host_io is not None:
                host_io["g_tr"].copy_(self.g_tr, non_blocking=True)
                host_io["g_full"].copy_(self.g_full, non_blocking=True)
            ev[4].record(s1)
        ev[4].synchronize()
        im = out["im"]
        ms = {"solve_fp64": ev[0].elapsed_time(ev[1]), "interpolate": ev[1].elapsed_time(ev[2]),
              "relax_patch": ev[2].elapsed_time(ev[3]), "solve_mixed": ev[5].elapsed_time(ev[6])}
        cu = i64.cell_updates + ip.cell_updates + im.cell_updates
        return cu, ms, (i64, ip, im), ev[0].elapsed_time(ev[4])


def run_ours(args):
    import torch
    import paper_1511_08200_gb300 as mg
    ws, rank, local = _dist()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    coarse, patch, origin = make_inputs()
    step = Step(mg, torch, coarse, patch, origin, dev)
    tune = {}
    if not args.no_autotune:
        # sweep schedules of every grid side, timed before the warm-up (not in the timed region)
        t0 = time.perf_counter()
        step.ctx.autotune(N_COARSE, "fp64")
        step.ctx2.autotune(N_COARSE, "mixed")
        tune = {"seconds": time.perf_counter() - t0,
                "fp64": schedules(mg, dev.index or 0, "fp64", N_COARSE),
                "mixed": schedules(mg, dev.index or 0, "mixed", N_COARSE)}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        step.run()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = mg.kernel_launches()
    tot_ms, tot_cu, phase = 0.0, 0, {}
    infos = None
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        cu, ms, infos, step_ms = step.run()
        tot_ms += step_ms
        tot_cu += cu
        for k, v in ms.items():
            phase[k] = phase.get(k, 0.0) + v
    torch.cuda.synchronize()
    launches = mg.kernel_launches() - launches0
    if ws > 1:
        torch.distributed.barrier()
    # the same steps again with the library's event profiler on (per-kernel device time)
    step.profile(True)
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        step.run()
    prof = step.profile_read()
    step.profile(False)
    clk = clocks.stop()
    max_ms, all_cu = aggregate_replicas(tot_ms, tot_cu, dev, ws)

    # e2e: the same step through the C ABI with HOST buffers (pinned), copies inside
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    hio = {"delta": pin(coarse), "patch": pin(patch),
           "phi": torch.zeros(step.phi.shape, dtype=torch.float64).pin_memory(),
           "grad": torch.zeros(step.grad.shape, dtype=torch.float64).pin_memory(),
           "g_tr": torch.zeros(step.g_tr.shape, dtype=torch.float64).pin_memory(),
           "g_full": torch.zeros(step.g_full.shape, dtype=torch.float64).pin_memory(),
           "phi_m": torch.zeros(step.phi.shape, dtype=torch.float64).pin_memory(),
           "grad_m": torch.zeros(step.grad.shape, dtype=torch.float64).pin_memory()}
    e2e_ms, e2e_cu = 0.0, 0
    if not args.no_e2e:
        step.run(hio)
    for _ in range(0 if args.no_e2e else args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cu, _, _, _ = step.run(hio)
        torch.cuda.synchronize()
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_cu += cu
    # delta goes in twice (the FP64 and the mixed solve each copy it from the host)
    h2d = (2 * hio["delta"].numel() + hio["patch"].numel()) * 8
    d2h = (hio["phi"].numel() + hio["grad"].numel() + hio["g_tr"].numel() + hio["g_full"].numel()
           + hio["phi_m"].numel() + hio["grad_m"].numel()) * 8

    if rank != 0:
        return
    i64, ip, im = infos
    # truncation error (Eq. errors2 context): interpolated vs relaxed fine phi and force
    box_tr, box_full = step.box[1:-1, 1:-1, 1:-1], step.box_full[1:-1, 1:-1, 1:-1]
    dphi = float(torch.linalg.vector_norm(box_tr - box_full) / torch.linalg.vector_norm(box_full))
    dg = float(torch.linalg.vector_norm(step.g_tr - step.g_full) / torch.linalg.vector_norm(step.g_full))
    mixed_vs64 = float(torch.linalg.vector_norm(step.phi_m - step.phi) / torch.linalg.vector_norm(step.phi))
    peaks = _peaks()
    roof = roofline(prof, peaks, args.steps)
    value = all_cu / (max_ms / 1e3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "refine128: periodic 128^3 nDGP FP64 solve to 1e-10 (lognormal GRF "
                               "sigma=1.5 at 256^3, seed 2, block-mean to 128^3, h=1.95 Mpc/h) + "
                               "64^3 fine patch over the densest 32^3 cells (interpolated vs relaxed "
                               "to 1e-10) + mixed-precision solve of the 128^3 grid to 1e-8 "
                               "(second stream, concurrent)",
                   "n": N_COARSE, "patch": 2 * PN, "tol_fp64": TOL64, "tol_mixed": TOLMIX,
                   "eps_alpha_s": step.alpha * step.s, "l2": "flushed between steps (512 MB write)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "time_to_tol_ms": {k: v / args.steps for k, v in phase.items()},
        "solve": {"fp64_cycles": i64.cycles, "fp64_rel_residual": i64.rel_residual,
                  "mixed_outer": im.outer_iters, "mixed_inner_cycles": im.cycles,
                  "mixed_rel_residual": im.rel_residual, "patch_cycles": ip.cycles,
                  "mixed_vs_fp64_rel_l2": mixed_vs64},
        "truncation": {"dphi_rel_l2": dphi, "dgrad_rel_l2": dg,
                       "relax_over_interp_ms": phase.get("relax_patch", 0) / max(phase.get("interpolate", 1e-9), 1e-9)},
        "roofline": roof,
        "kernels": {k: {"ms": v[0] / args.steps, "launches": v[1] // args.steps}
                    for k, v in prof.items() if v[1] > 0},
        "clocks": clk,
        "e2e": ({"value": e2e_cu / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                 "d2h_bytes_per_step": d2h} if e2e_ms > 0 else None),
        "gpu_launches": launches,
        "autotune": tune or None,
    }
    out["geff"] = geff_report(step)
    if not args.no_truncation_levels:
        try:
            out["masked_truncation"] = masked_truncation_report(step)
        except mg.MG5Error as e:   # reported, not fatal to the bench line
            out["masked_truncation"] = {"error": str(e)}
    if not args.no_truncation_levels:
        try:
            out["truncation_levels"] = truncation_levels_report(mg, torch, dev)
        except mg.MG5Error as e:   # reported, not fatal to the bench line
            out["truncation_levels"] = {"error": str(e)}
    if not args.no_batch:
        out["batch"] = run_batch(mg, torch, dev, step.alpha, step.s, autotune=not args.no_autotune)
    if not args.no_sizes:
        out.update(size_records(mg, torch, dev, step.alpha, step.s, autotune=not args.no_autotune))
    if args.serve_seconds > 0:
        out["serving"] = run_serving(mg, torch, dev, step.alpha, step.s, args.serve_seconds,
                                     slots=args.serve_slots, autotune=not args.no_autotune)
    if args.serve_seconds > 0 and args.serve_compare_seconds > 0:
        out["serving_vs_fp64"] = serving_vs_fp64(mg, torch, dev, step.alpha, step.s,
                                                 args.serve_compare_seconds, args.serve_slots,
                                                 autotune=not args.no_autotune)
    if not args.no_cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(coarse, patch, origin, budget_s=args.cpu_seconds)
    print(json.dumps(out), flush=True)


def geff_fields(mg, torch, ctx, d_c, d_p, phi, grad, origin, pn, h, beta, s, tol=TOL64):
    """Device fields of Eq. (errors2) on one refinement (once, outside the timed region): the
    GR potential from the same engine at alpha = 0 with source (3 beta / 2) s delta
    (Eq. modpoisson), its force on the periodic domain grid and, relaxed on the patch like the
    fifth force, on the refinement; and the truncated level's interpolation variants -- the
    tricubic phi (an extension) and the coarse force interpolated directly (the Fig. amr
    caption's wording) instead of differencing the interpolated phi.  d_c: domain delta (n^3),
    d_p: patch delta ((2 pn)^3), phi / grad: the fifth-force solution and its gradient on the
    domain grid of cell size h."""
    pn = tuple(int(x) for x in pn)
    s_gr = 1.5 * beta * s
    p_gr = mg.default_params(alpha=0.0, s=s_gr, h=h, tol=tol)
    p_grp = mg.default_params(alpha=0.0, s=s_gr, h=h / 2, tol=tol, max_cycles=1000)
    psi = torch.zeros_like(phi)
    g_psi = torch.empty_like(grad)
    _, _, ig = ctx.solve_fifth_force(d_c, p_gr, phi=psi, grad=g_psi)
    box = ctx.refine_interpolate(psi, origin, pn, 1)
    ctx.relax_patch(d_p, p_grp, ig.compat_c, box)
    g_gr = ctx.force(box, h / 2, ghost=1, periodic=False)
    box_c = ctx.refine_interpolate_cubic(phi, origin, pn, 1)
    g_cub = ctx.force(box_c, h / 2, ghost=1, periodic=False)
    g_fi = torch.stack([ctx.refine_interpolate(grad[a].contiguous(), origin, pn, 0)
                        for a in range(3)])
    torch.cuda.synchronize()
    return {"g_psi": g_psi, "g_gr": g_gr, "g_cub": g_cub, "g_fi": g_fi, "gr_cycles": ig.cycles}


def geff_numbers(torch, beta, grad, g_psi, g_tr, g_full, g_gr, g_cub, g_fi):
    """Eq. (errors2) quantities from the forces (FP64, every cell; quantiles by linear
    interpolation): F5 = grad(phi) / 2 against F_GR = grad(Psi_GR) on the domain and on the
    patch (screening lowers F5/F_GR below the linear value 1/(3 beta)), eps_trunc =
    |F5_trunc - F5_full| / |F5_full| and the G_eff error it causes,
    |F5_trunc - F5_full| / |F_GR| = (F5_full / F_GR) eps_trunc; g_tr: the truncated level's
    force (trilinear phi), g_full: the relaxed level's."""
    mag = lambda g: torch.linalg.vector_norm(g, dim=0)   # noqa: E731
    qs = torch.tensor([0.5, 0.99], dtype=torch.float64, device=grad.device)
    q = lambda t: [float(x) for x in torch.quantile(t.flatten(), qs)]   # noqa: E731
    rl2 = lambda a, b: float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))  # noqa: E731
    d5 = 0.5 * mag(g_tr - g_full)
    return {"linear_ratio_1_over_3beta": 1.0 / (3.0 * beta),
            "eps_trunc_rel_l2_by_interpolant": {"phi_trilinear": rl2(g_tr, g_full),
                                                "phi_tricubic": rl2(g_cub, g_full),
                                                "force_trilinear": rl2(g_fi, g_full)},
            "f5_over_fgr_domain_p50_p99": q(0.5 * mag(grad) / mag(g_psi)),
            "f5_over_fgr_patch_p50_p99": q(0.5 * mag(g_full) / mag(g_gr)),
            "f5_over_fgr_patch_trunc_p50_p99": q(0.5 * mag(g_tr) / mag(g_gr)),
            "eps_trunc_rel_l2": rl2(g_tr, g_full),
            "eps_trunc_p50_p99": q(d5 / (0.5 * mag(g_full))),
            "geff_error_p50_p99": q(d5 / mag(g_gr))}


def geff_report(step):
    """Eq. (errors2) on the refinement workload (once, outside the timed region)."""
    f = geff_fields(step.mg, step.torch, step.ctx, step.d_c, step.d_p, step.phi, step.grad,
                    step.origin, (PN, PN, PN), H_COARSE, step.beta, step.s)
    step.g_gr_dom, step.g_gr_patch = f["g_psi"], f["g_gr"]   # reused by masked_truncation_report
    out = geff_numbers(step.torch, step.beta, step.grad, f["g_psi"], step.g_tr, step.g_full,
                       f["g_gr"], f["g_cub"], f["g_fi"])
    out["gr_cycles"] = f["gr_cycles"]
    return out


def masked_truncation_report(step, quantiles=(0.25, 0.5, 0.75, 0.9), reps=3):
    """Position-dependent truncation (Sec. 3.3) on the refinement workload (once, outside
    the timed region): the 64^3 patch iterates a fine cell only where its parent's
    F5/F_GR (domain grid, F5 = grad(phi)/2, F_GR from the alpha = 0 solve of geff_report)
    exceeds theta; the other cells keep the interpolated phi.  Per theta (quantiles of the
    ratio over the patch's parents): masked fraction, V-cycles, device time of the masked
    relaxation (library events, best of `reps`) against the full relaxation, and the force
    error against the fully relaxed patch: eps_trunc = |F5 - F5_full| / |F5_full| and the
    G_eff error |F5 - F5_full| / |F_GR| (Eq. errors2)."""
    mg, torch, ctx = step.mg, step.torch, step.ctx
    pn = (PN, PN, PN)
    hf = H_COARSE / 2
    mag = lambda g: torch.linalg.vector_norm(g, dim=0)
    ratio = 0.5 * mag(step.grad) / mag(step.g_gr_dom)
    n = ratio.shape[0]
    idx = [torch.arange(step.origin[a], step.origin[a] + PN, device=ratio.device) % n for a in range(3)]
    par = ratio[idx[0]][:, idx[1]][:, :, idx[2]].flatten()
    box0 = torch.empty_like(step.box)
    ctx.refine_interpolate(step.phi, step.origin, pn, 1, out=box0)
    g_full, g_gr = step.g_full, step.g_gr_patch
    nf = float(torch.linalg.vector_norm(g_full))

    def run(mask):
        best, info, out = float("inf"), None, None
        for _ in range(reps):
            out = box0.clone()
            if mask is None:
                _, info = ctx.relax_patch(step.d_p, step.ppatch, step.compat_c, out)
            else:
                _, info = ctx.relax_patch_masked(step.d_p, mask, step.ppatch, step.compat_c, out)
            best = min(best, info.ms_total)
        return out, info, best

    _, ifull, ms_full = run(None)
    rows = []
    for q in quantiles:
        theta = float(torch.quantile(par.float(), q))
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        mask, cnt = ctx.parent_force_mask(step.grad, step.g_gr_dom, step.origin, pn, theta,
                                          count=True)
        t1.record()
        torch.cuda.synchronize()
        out, info, ms = run(mask)
        g = ctx.force(out, hf, ghost=1, periodic=False)
        d5 = 0.5 * mag(g - g_full)
        dge = (d5 / mag(g_gr)).flatten()
        qq = torch.quantile(dge[::7].float(), torch.tensor([0.5, 0.99], device=dge.device))
        rows.append({"theta": theta, "theta_over_linear": theta * 3.0 * step.beta,
                     "masked_fraction": cnt / float((2 * PN) ** 3), "cycles": info.cycles,
                     "ms": ms, "mask_ms": t0.elapsed_time(t1),
                     "eps_trunc_rel_l2": float(torch.linalg.vector_norm(g - g_full)) / nf,
                     "geff_error_p50_p99_max": [float(qq[0]), float(qq[1]), float(dge.max())]})
    eps_tr = float(torch.linalg.vector_norm(step.g_tr - g_full)) / nf
    return {"patch": [2 * PN] * 3, "full_ms": ms_full, "full_cycles": ifull.cycles,
            "all_truncated_eps_rel_l2": eps_tr, "by_theta": rows}


def nested_chain(ctx, mg, torch, d_levels, origins, spacings, phi_dom, alpha, s, compat_c, T, tol):
    """phi on every refinement of a nested hierarchy: relaxed (mg5_relax_patch) on levels
    < T, the coarse-to-fine interpolant of its parent (mg5_refine_interpolate[_box]) on levels
    >= T (the truncation of Sec. 3.2 at l_trunc = l_d + T).  Returns the level boxes."""
    boxes = [None]
    for lev in range(1, len(d_levels)):
        pn = (int(d_levels[lev].shape[0]) // 2,) * 3
        if lev == 1:
            box = ctx.refine_interpolate(phi_dom, origins[1], pn, 1)
        else:
            box = ctx.refine_interpolate_box(boxes[lev - 1], 1, origins[lev], pn, 1)
        if lev < T:
            p = mg.default_params(alpha=alpha, s=s, h=spacings[lev], tol=tol, max_cycles=200)
            ctx.relax_patch(d_levels[lev], p, compat_c, box)
        boxes.append(box)
    return boxes


def masked_chain(ctx, mg, torch, d_levels, origins, spacings, phi_dom, g5_dom, ggr, alpha, s,
                 compat_c, theta, tol):
    """The position-dependent truncation of Sec. 3.3 on a nested hierarchy: on every level
    l >= 1 a fine cell is relaxed only where its parent's F5/F_GR exceeds theta
    (mg5_parent_force_mask on the parent's forces: the periodic domain for l = 1, the
    parent refinement's interior below; ggr[l] the GR force vectors per level), the other
    cells keep the interpolated parent phi (mg5_relax_patch_masked; an empty mask skips the
    relaxation, a full one runs the unmasked one).  Returns (boxes, masked fraction per level)."""
    boxes, fracs = [None], []
    g_par = g5_dom
    for lev in range(1, len(d_levels)):
        pn = (int(d_levels[lev].shape[0]) // 2,) * 3
        if lev == 1:
            box = ctx.refine_interpolate(phi_dom, origins[1], pn, 1)
        else:
            box = ctx.refine_interpolate_box(boxes[lev - 1], 1, origins[lev], pn, 1)
        mask, cnt = ctx.parent_force_mask(g_par, ggr[lev - 1], origins[lev], pn, theta,
                                          periodic=(lev == 1), count=True)
        ncell = 8 * pn[0] * pn[1] * pn[2]
        p = mg.default_params(alpha=alpha, s=s, h=spacings[lev], tol=tol, max_cycles=200)
        if cnt == ncell:
            ctx.relax_patch(d_levels[lev], p, compat_c, box)
        elif cnt > 0:
            ctx.relax_patch_masked(d_levels[lev], mask, p, compat_c, box)
        fracs.append(cnt / float(ncell))
        boxes.append(box)
        g_par = ctx.force(box, spacings[lev], ghost=1, periodic=False)
    return boxes, fracs


def truncation_levels_report(mg, torch, dev, n_dom=128, levels=4, pn=16):
    """The multi-level truncation analogue of the paper's Table 1 / Fig. ratio (once, not
    timed in the step): a 128^3 domain plus 4 nested 2x refinements (32^3 each) around an
    NFW halo (M200 = 1e14 M_sun/h, c = 5) on the lognormal background; phi relaxed on every
    level (full) or truncated at l_trunc = l_d + T (levels >= T interpolated), T = 1, 2, 4;
    the GR force relaxed on every level.  Per level: median F5/F_GR (full), eps_trunc and
    the G_eff error of Eq. errors2; GPU time of each chain."""
    import workload
    deltas, origins, spacings = workload.nested_halo_workload(n_dom, 250.0, levels, pn)
    beta, alpha, s = mg.ndgp_coefficients(1.0, 0.3, 1.0)
    d = [torch.from_numpy(x).to(dev) for x in deltas]
    ctx = mg.Context(dev.index or 0)
    tol = 1e-8
    p = mg.default_params(alpha=alpha, s=s, h=spacings[0], tol=tol)
    phi, _, i5 = ctx.solve_fifth_force(d[0], p)
    s_gr = 1.5 * beta * s
    pg = mg.default_params(alpha=0.0, s=s_gr, h=spacings[0], tol=tol)
    psi, _, ig = ctx.solve_fifth_force(d[0], pg)
    mag = lambda g: torch.linalg.vector_norm(g, dim=0)
    force = lambda b, h: ctx.force(b, h, ghost=1, periodic=False)
    gr = nested_chain(ctx, mg, torch, d, origins, spacings, psi, 0.0, s_gr, ig.compat_c,
                      levels + 1, tol)
    ggr = [ctx.force(psi, spacings[0])] + [force(gr[l], spacings[l]) for l in range(1, levels + 1)]
    f_gr = [None] + [mag(ggr[l]) for l in range(1, levels + 1)]
    chains, ms = {}, {}
    for T in (levels + 1, 1, 2, 4):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        boxes = nested_chain(ctx, mg, torch, d, origins, spacings, phi, alpha, s, i5.compat_c, T, tol)
        g5 = [None] + [0.5 * force(boxes[l], spacings[l]) for l in range(1, levels + 1)]
        e1.record()
        e1.synchronize()
        chains[T], ms[T] = g5, e0.elapsed_time(e1)
    full = chains[levels + 1]
    q = lambda t: [float(x) for x in torch.quantile(t.flatten().float(),
                                                    torch.tensor([0.5, 0.99], device=t.device))]
    out = {"levels": levels, "spacing_mpc_h": spacings, "box_cells": 2 * pn,
           "f5_over_fgr_p50_by_level": [float(torch.median(mag(full[l]) / f_gr[l]))
                                        for l in range(1, levels + 1)],
           "linear_ratio": 1.0 / (3.0 * beta), "chain_ms": {}, "eps_trunc_rel_l2": {},
           "geff_error_p50_p99": {}}
    for T in (1, 2, 4):
        key = "l_trunc=l_d+%d" % T
        out["chain_ms"][key] = ms[T]
        out["eps_trunc_rel_l2"][key] = [
            float(torch.linalg.vector_norm(chains[T][l] - full[l]) / torch.linalg.vector_norm(full[l]))
            for l in range(1, levels + 1)]
        out["geff_error_p50_p99"][key] = [q(mag(chains[T][l] - full[l]) / f_gr[l])
                                         for l in range(1, levels + 1)]
    out["chain_ms"]["full"] = ms[levels + 1]
    # position-dependent truncation (Sec. 3.3): thresholds as fractions of the linear ratio
    g5_dom = ctx.force(phi, spacings[0])
    out["masked"] = {}
    for frac in (0.97, 0.93, 0.85):
        theta = frac / (3.0 * beta)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        boxes, fr = masked_chain(ctx, mg, torch, d, origins, spacings, phi, g5_dom, ggr, alpha, s,
                                 i5.compat_c, theta, tol)
        g5 = [None] + [0.5 * force(boxes[l], spacings[l]) for l in range(1, levels + 1)]
        e1.record()
        e1.synchronize()
        out["masked"]["theta=%.2f/(3beta)" % frac] = {
            "chain_ms": e0.elapsed_time(e1), "masked_fraction_by_level": fr,
            "eps_trunc_rel_l2": [float(torch.linalg.vector_norm(g5[l] - full[l])
                                       / torch.linalg.vector_norm(full[l]))
                                 for l in range(1, levels + 1)],
            "geff_error_p50_p99": [q(mag(g5[l] - full[l]) / f_gr[l]) for l in range(1, levels + 1)]}
    ctx.close()
    return out


def schedules(mg, device, prec, n):
    """The sweep schedule of every non-coarsest grid side of n's hierarchy, as text."""
    out = {}
    while n % 2 == 0 and n // 2 >= 4:
        sch, tuned = mg.schedule_get(device, prec, n)
        txt = {mg.SWEEP_FUSED: "fused/%d" % sch.chunk, mg.SWEEP_MARCH: "march/%d" % sch.chunk}.get(
            sch.form, "two-pass/%d" % sch.block)
        out[str(n)] = txt + ("" if tuned else " (default)")
        n //= 2
    return out


def batch_boxes(mg, dev, alpha, s):
    """The 96 boxes of the batched workload: sizes uniform from {32,48,64,96,128}, lognormal
    sigma = 1 with seeds 1000 + b, alpha log-uniform in [0.1, 10] x nominal, mixed precision to
    1e-8.  Returns (sizes, alpha scales, device deltas, params)."""
    import workload
    rng = np.random.Generator(np.random.PCG64(4))
    sizes = rng.choice(np.asarray([32, 48, 64, 96, 128]), size=96)
    scales = 10.0 ** rng.uniform(-1.0, 1.0, size=96)
    deltas = [workload.lognormal_delta_torch(int(n), 1.0, 1000 + b, dev) for b, n in enumerate(sizes)]
    params = [mg.default_params(alpha=alpha * float(a), s=s, h=L_BOX / 512, tol=TOLMIX,
                                precision="mixed") for a in scales]
    return sizes, scales, deltas, params


def run_batch(mg, torch, dev, alpha, s, reps=5, autotune=True):
    """The batched workload: 96 boxes, sizes uniform from {32,48,64,96,128}, seeds 1000 + b,
    alpha log-uniform in [0.1, 10] x nominal, mixed precision to 1e-8, solved as ONE
    CUDA-graph launch; compared with the same boxes solved one after another."""
    sizes, scales, deltas, params = batch_boxes(mg, dev, alpha, s)
    phis = [torch.zeros_like(d) for d in deltas]
    grads = [torch.empty((3,) + d.shape, dtype=torch.float64, device=dev) for d in deltas]
    ctx = mg.Context(dev.index or 0)
    t0 = time.perf_counter()
    if autotune:
        for n in sorted(set(int(x) for x in sizes)):
            ctx.autotune(n, "mixed")
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctx.solve_batch(deltas, params, phis=phis, grads=grads)          # capture + first launch
    build_s = time.perf_counter() - t0
    ms, cu = [], 0
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, infos = ctx.solve_batch(deltas, params, phis=phis, grads=grads)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        cu = sum(i.cell_updates for i in infos)
    seq_ms = []
    for _ in range(2):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for d, p, x, g in zip(deltas, params, phis, grads):
            ctx.solve_fifth_force(d, p, phi=x, grad=g)
        e1.record()
        e1.synchronize()
        seq_ms.append(e0.elapsed_time(e1))
    t = float(np.median(ms))
    cells = int(sum(int(n) ** 3 for n in sizes))
    worst = max(i.rel_residual for i in infos)
    ctx.close()
    return {"boxes": 96, "cells": cells, "ms_per_batch": t, "cell_updates_per_s": cu / (t / 1e3),
            "time_to_tol_ms": t, "sequential_ms": float(np.median(seq_ms)),
            "graph_build_s": build_s, "autotune_s": tune_s, "max_rel_residual": worst,
            "outer_iters": [i.outer_iters for i in infos][:8], "dtype": "f32+f64"}


SERVE_SEED0 = 50000   # request i draws its field from seed SERVE_SEED0 + i


def serving_stream(count, rate=200.0):
    """The serving stream's requests: exponential gaps at `rate`, sides
    16 round(10^U(log 32, log 256)/16), sigma ~ U(0.5, 2), tol 1e-6 or 1e-8 with p = 1/2.
    Returns (gaps, sizes, sigmas, tols); request i's field is serving_field(i, ...)."""
    import workload
    rng = np.random.Generator(np.random.PCG64(5))
    gaps = rng.exponential(1.0 / rate, size=count)
    sizes = workload.serving_sizes(rng, count)
    sigmas = rng.uniform(0.5, 2.0, size=count)
    tols = np.where(rng.uniform(size=count) < 0.5, 1e-6, 1e-8)
    return gaps, sizes, sigmas, tols


def serving_field(i, sizes, sigmas, dev):
    """Request i's own lognormal field (its own seed: no two requests share an input)."""
    import workload
    return workload.lognormal_delta_torch(int(sizes[i]), float(sigmas[i]), SERVE_SEED0 + i, dev)


class FieldFeeder:
    """Generates each request's field on a side stream ahead of its arrival time (outside
    the server's path; the server measures latency from the submission at arrival)."""

    def __init__(self, torch, dev, sizes, sigmas, count, ahead=96):
        self.torch, self.dev = torch, dev
        self.sizes, self.sigmas, self.count = sizes, sigmas, count
        self.ready = {}
        self.cv = threading.Condition()
        self.next_needed = 0
        self.ahead = ahead
        self.stop = False
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    def _run(self):
        torch = self.torch
        st = torch.cuda.Stream(device=self.dev)
        for i in range(self.count):
            with self.cv:
                while not self.stop and i >= self.next_needed + self.ahead:
                    self.cv.wait(0.05)
                if self.stop:
                    return
            with torch.cuda.stream(st):
                d = serving_field(i, self.sizes, self.sigmas, self.dev)
            st.synchronize()
            with self.cv:
                self.ready[i] = d
                self.cv.notify_all()

    def take(self, i):
        with self.cv:
            while i not in self.ready:
                self.cv.wait(0.05)
            self.next_needed = i + 1
            self.cv.notify_all()
            return self.ready.pop(i)

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        self.th.join(timeout=30)


def run_serving(mg, torch, dev, alpha, s, seconds, rate=200.0, slots=16, warm_s=5.0,
                autotune=True, precision="mixed", max_backlog=1024):
    """Poisson arrivals at `rate` req/s for `seconds`: sides 16 round(10^U(log 32, log 256)/16),
    sigma ~ U(0.5, 2), tol 1e-6 or 1e-8 with p = 1/2, every request its own field (generated
    ahead of its arrival on a side stream), all in one `precision` ("mixed": captured graphs
    from the server's pool; "fp64": host-driven solves on the workers' contexts); admitted by
    HBM footprint.  Latency = completion - arrival (server clock); the first `warm_s` seconds
    are discarded (a fifth of the run if that is shorter).  A server that falls behind (more
    than `max_backlog` requests submitted and not done) ends the run early: saturated."""
    count = int(rate * seconds * 1.2) + 8
    gaps, sizes, sigmas, tols = serving_stream(count, rate)
    budget = int(torch.cuda.get_device_properties(dev).total_memory * 0.5)
    if autotune:   # the schedule table is process-wide: the server's solves read it
        tctx = mg.Context(dev.index or 0)
        for n in sorted(set(int(x) for x in sizes)):
            tctx.autotune(n, precision)
        tctx.close()
    srv = mg.Server(dev.index or 0, slots=slots, hbm_budget_bytes=budget)
    # warm the server's graph pool (two entries per (size, tolerance): its cap) before timing
    for i, n in enumerate(sorted(set(int(x) for x in sizes))):
        dw = workload_field(torch, dev, n)
        for j, tol in enumerate((1e-6, 1e-8)):
            p = mg.default_params(alpha=alpha, s=s, h=L_BOX / 512, tol=tol, precision=precision)
            for r in range(2):
                srv.submit(dw, p, torch.zeros_like(dw), tag=10 ** 9 + 4 * i + 2 * j + r)
        while srv.pending() != (0, 0):
            srv.poll(wait_ms=50)
    srv.poll(max_n=1000)
    feeder = FieldFeeder(torch, dev, sizes, sigmas, count)
    while len(feeder.ready) < min(32, count):   # a head start before the clock starts
        time.sleep(0.01)
    done = {}
    t_start = srv.clock()
    t_next = t_start
    i = 0
    saturated = False
    while True:
        now = srv.clock()
        if now - t_start >= seconds:
            break
        if i - len(done) > max_backlog:
            saturated = True
            break
        if now >= t_next and i < count:
            p = mg.default_params(alpha=alpha, s=s, h=L_BOX / 512, tol=float(tols[i]),
                                  precision=precision)
            d = feeder.take(i)
            srv.submit(d, p, torch.empty_like(d), tag=i)
            t_next += gaps[i]
            i += 1
            continue
        for c in srv.poll(wait_ms=0):
            done[c.tag] = c
        time.sleep(max(0.0, min(t_next - srv.clock(), 0.0005)))
    submitted = i
    srv_end = srv.clock()
    feeder.close()
    while len(done) < submitted:
        for c in srv.poll(wait_ms=100):
            done[c.tag] = c
    stats = srv.stats()
    srv.close()
    warm = min(warm_s, (srv_end - t_start) / 5.0)
    rows = [c for c in done.values() if c.t_submit - t_start >= warm]
    lat = np.array([(c.t_done - c.t_submit) * 1e3 for c in rows])
    t_first = min(c.t_submit for c in rows)
    t_last = max(c.t_done for c in rows)
    cu = sum(c.info.cell_updates for c in rows)
    ok = sum(1 for c in rows if c.status in (0, 1))
    lag = [(c.t_submit - t_start) - float(np.sum(gaps[:c.tag])) for c in rows]
    return {"precision": precision, "offered_req_per_s": rate, "seconds": seconds,
            "ran_s": float(srv_end - t_start), "saturated": saturated,
            "discarded_s": warm, "slots": slots,
            "requests": len(rows), "submitted": submitted, "completed_ok": ok,
            "distinct_inputs": len(rows),
            "throughput_req_per_s": len(rows) / (t_last - t_first),
            "cell_updates_per_s": cu / (t_last - t_first),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "mean": float(lat.mean()), "max": float(lat.max())},
            "submit_lag_ms_max": float(max(lag) * 1e3) if lag else 0.0,
            "mean_cells_per_request": float(np.mean([int(sizes[c.tag]) ** 3 for c in rows])),
            "sigma_range": [float(sigmas[:submitted].min()), float(sigmas[:submitted].max())],
            "hbm_budget_bytes": budget, "server": stats}


def serving_vs_fp64(mg, torch, dev, alpha, s, seconds, slots, rate=100.0, autotune=True):
    """The serving stream in mixed precision and in plain FP64 on the same server, at `rate`
    req/s (half the main run's) for `seconds` each, and FP64 at the main run's 200 req/s until
    it falls behind (more than 512 requests outstanding): its capacity."""
    keys = ("saturated", "ran_s", "requests", "throughput_req_per_s", "cell_updates_per_s",
            "latency_ms", "completed_ok")
    out = {"offered_req_per_s": rate, "seconds": seconds, "slots": slots}
    for prec in ("mixed", "fp64"):
        r = run_serving(mg, torch, dev, alpha, s, seconds, rate=rate, slots=slots,
                        autotune=autotune, precision=prec, max_backlog=512)
        out[prec] = {k: r[k] for k in keys}
    r = run_serving(mg, torch, dev, alpha, s, seconds, rate=200.0, slots=slots,
                    autotune=autotune, precision="fp64", max_backlog=512)
    out["fp64_at_200"] = {k: r[k] for k in keys}
    out["p99_fp64_over_mixed"] = out["fp64"]["latency_ms"]["p99"] / out["mixed"]["latency_ms"]["p99"]
    return out


def workload_field(torch, dev, n):
    """A field of side n for warming the server's graph pool (not one of the requests)."""
    import workload
    return workload.lognormal_delta_torch(n, 1.0, 4999, dev)


def roofline(prof: dict, peaks: dict, steps: int) -> dict:
    """The dominant kernel: of the classes that are one kernel on one grid (the *_coarse classes
    gather the launches of every coarser level), the one with the most device time;
    algorithmic work / its event-timed duration."""
    top = max(((k, v) for k, v in prof.items()
               if k in WORK and not k.endswith("_coarse") and v[1] > 0), key=lambda kv: kv[1][0])
    name, (ms, calls, cells) = top
    bound, bpc, fpc = WORK[name]
    sec = ms / 1e3
    if bound == "hbm":
        achieved = bpc * cells / sec / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        unit = "GB/s"
    else:
        achieved = fpc * cells / sec / 1e12
        peak = FP64_PEAK_TFLOPS
        unit = "TFLOP/s"
    tpc = TRAFFIC_PER_CELL.get(name)
    traffic = tpc * cells / max(calls, 1) if tpc is not None else None
    out = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
           "frac": achieved / peak, "traffic": traffic,
           "avg_launch_ms": ms / max(calls, 1), "launches_per_step": calls / steps,
           "alg_bytes_per_cell": bpc, "alg_flops_per_cell": fpc,
           "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json)" if bound == "hbm"
           else FP64_PEAK_SOURCE}
    if name.startswith("sweep64") or name.startswith("patch_sweep64"):
        a2 = SURVEY_FLOPS_SWEEP64 * cells / sec / 1e12
        out.update({"achieved_survey_count": a2, "frac_survey_count": a2 / peak,
                    "flops_per_cell_survey_count": SURVEY_FLOPS_SWEEP64})
    return out


# ---------------------------------------------------------------- the oracle on host cores

def cpu_baseline(coarse, patch, origin, budget_s=20.0) -> dict:
    """The FP64 CPU oracle, as it stands, on a bounded sample of the same step."""
    import oracle
    beta, alpha, s = oracle.ndgp_coefficients(1.0, 0.3, 1.0)
    oracle.build()
    cores = os.cpu_count()
    t0 = time.perf_counter()
    phi, info = oracle.solve(coarse, alpha, s, H_COARSE, tol=TOL64)
    t_solve = time.perf_counter() - t0
    box = oracle.refine_interpolate(phi, origin, (PN, PN, PN), 1)
    left = max(budget_s - t_solve, 1.0)
    # bounded patch relaxation: sweeps in batches of 10 until the budget is used
    t1 = time.perf_counter()
    sweeps = 0
    while time.perf_counter() - t1 < left and sweeps < 100000:
        box, nsw, rel = oracle.relax_patch(patch, box, alpha, s, H_COARSE / 2, info.compat_c,
                                           tol=TOL64, max_sweeps=10, check=10)
        sweeps += nsw
        if rel <= TOL64 or nsw == 0:
            break
    t_patch = time.perf_counter() - t1
    cu = info.cell_updates + sweeps * (2 * PN) ** 3
    return {"value": cu / (t_solve + t_patch), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "FP64 oracle solve of the 128^3 grid to 1e-10 (%d cycles, %.1f s) + %d "
                      "Dirichlet sweeps of the 64^3 patch (%.1f s); OpenMP over %d threads"
                      % (info.cycles, t_solve, sweeps, t_patch, cores)}


def time_solve(torch, ctx, d, p, reps=3, warm=1, **kw):
    """Median device time (CUDA events on the current stream, first kernel to the last
    result on the device) of `reps` solves after `warm` untimed ones; returns (ms, info)."""
    for _ in range(warm):
        _, _, info = ctx.solve_fifth_force(d, p, **kw)
    ms = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, info = ctx.solve_fifth_force(d, p, **kw)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return float(np.median(ms)), info


def class_roofline(prof: dict, name: str, peaks: dict) -> dict:
    """Algorithmic bytes (or flops) of one kernel class / its event-timed device time."""
    ms, calls, cells = prof.get(name, (0.0, 0, 0.0))
    if calls == 0 or ms <= 0:
        return None
    bound, bpc, fpc = WORK[name]
    sec = ms / 1e3
    if bound == "hbm":
        achieved, peak, unit = bpc * cells / sec / 1e9, peaks.get("hbm_gbs", 6800.0), "GB/s"
    else:
        achieved, peak, unit = fpc * cells / sec / 1e12, FP64_PEAK_TFLOPS, "TFLOP/s"
    return {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "avg_launch_ms": ms / calls, "launches": calls,
            "alg_bytes_per_cell": bpc, "alg_flops_per_cell": fpc,
            "peak_source": "measured hbm_gbs (MEASURED_PEAKS.json)" if bound == "hbm"
            else FP64_PEAK_SOURCE}


def size_records(mg, torch, dev, alpha, s, autotune=True):
    """The single-grid configurations beside the step (once, after its timed region), each
    to its stated tolerance with inputs resident on the device:
      fp64_32   the 32^3 sigma = 1 grid (seed 1, numpy generator), FP64 to 1e-10, median of
                10 after 2 warm-ups, host-driven and as a graph replay (L2-resident);
      mixed512  the 512^3 sigma = 2 grid (seed 3), FP32 V-cycles inside the FP64 defect
                correction to 1e-8 (inputs larger than L2), per-class device time and the FP32
                smoother's HBM roofline;
      fp64_512  the same input solved in plain FP64 (FMG start, V(3,1), coarsest capped at 4
                sweeps a visit) to 1e-8 and to 1e-10;
      mixed_over_fp64  FP64 time to 1e-8 / mixed time to 1e-8 on that input (> 1: the mixed
                mode is faster)."""
    import workload
    peaks = _peaks()
    out = {}
    ctx = mg.Context(dev.index or 0)
    # C1: 32^3 FP64 to 1e-10
    h32 = L_BOX / 512
    d32 = torch.from_numpy(workload.lognormal_delta(32, 1.0, 1)).to(dev)
    p32 = mg.default_params(alpha=alpha, s=s, h=h32, tol=TOL64)
    t_host, i_host = time_solve(torch, ctx, d32, p32, reps=10, warm=2)
    t_graph, i_graph = time_solve(torch, ctx, d32, p32, reps=10, warm=2, graph=True)
    out["fp64_32"] = {"n": 32, "tol": TOL64, "time_to_tol_ms": min(t_host, t_graph),
                      "host_driven_ms": t_host, "graph_ms": t_graph, "cycles": i_graph.cycles,
                      "rel_residual": i_graph.rel_residual,
                      "cell_updates_per_s": i_graph.cell_updates / (t_graph / 1e3),
                      "l2": "L2-resident (256 KiB field)"}
    # C3: 512^3, mixed and FP64 on the same input
    n = 512
    d = workload.lognormal_delta_torch(n, 2.0, 3, dev)
    phi = torch.zeros_like(d)
    if autotune:
        ctx.autotune(n, "mixed")
        ctx.autotune(n, "fp64")
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    pm = mg.default_params(alpha=alpha, s=s, h=h32, tol=TOLMIX, precision="mixed")
    tm, im = time_solve(torch, ctx, d, pm, phi=phi)
    tmg, img = time_solve(torch, ctx, d, pm, phi=phi, graph=True)
    ctx.profile_enable(True)
    ctx.solve_fifth_force(d, pm, phi=phi)
    prof_m = ctx.profile_read()
    ctx.profile_enable(False)
    out["mixed512"] = {"n": n, "tol": TOLMIX, "time_to_tol_ms": min(tm, tmg),
                       "host_driven_ms": tm, "graph_ms": tmg,
                       "outer_iters": im.outer_iters, "inner_cycles": im.cycles,
                       "rel_residual": im.rel_residual,
                       "cell_updates_per_s": im.cell_updates / (min(tm, tmg) / 1e3),
                       "roofline_sweep32": class_roofline(prof_m, "sweep32", peaks),
                       "kernels_ms": {k: round(v[0], 3) for k, v in prof_m.items() if v[1] > 0},
                       "l2": "inputs larger than L2"}
    out["fp64_512"] = {}
    for tol in (TOLMIX, TOL64):
        p = mg.default_params(alpha=alpha, s=s, h=h32, tol=tol, nu1=3, nu2=1,
                              nu_coarse=NU_COARSE_CAP)
        t, i = time_solve(torch, ctx, d, p, phi=phi, fmg=True, graph=True)
        out["fp64_512"]["tol_%g" % tol] = {"time_to_tol_ms": t, "cycles": i.cycles,
                                          "rel_residual": i.rel_residual,
                                          "cell_updates_per_s": i.cell_updates / (t / 1e3)}
    p = mg.default_params(alpha=alpha, s=s, h=h32, tol=TOLMIX, nu1=3, nu2=1,
                          nu_coarse=NU_COARSE_CAP)
    ctx.profile_enable(True)
    ctx.solve_fifth_force(d, p, phi=phi, fmg=True)
    prof_64 = ctx.profile_read()
    ctx.profile_enable(False)
    out["fp64_512"]["kernels_ms_tol_1e-08"] = {k: round(v[0], 3) for k, v in prof_64.items()
                                               if v[1] > 0}
    out["fp64_512"]["roofline_sweep64"] = class_roofline(prof_64, "sweep64", peaks)
    out["mixed_over_fp64"] = (out["fp64_512"]["tol_%g" % TOLMIX]["time_to_tol_ms"]
                              / out["mixed512"]["time_to_tol_ms"])
    out["clocks"] = clocks.stop()
    ctx.close()
    del d, phi
    torch.cuda.empty_cache()
    return out


def run_mixed_workload(args):
    """The large mixed-precision workload on its own: one periodic N^3 grid (default 512^3),
    lognormal sigma = 2, seed 3, FP32 V-cycles inside an FP64 defect-correction loop to
    relative residual 1e-8.  Inputs are larger than L2."""
    import torch
    import paper_1511_08200_gb300 as mg
    import workload
    ws, rank, local = _dist()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n = args.n
    beta, alpha, s = mg.ndgp_coefficients(1.0, 0.3, 1.0)
    d = workload.lognormal_delta_torch(n, 2.0, 3, dev)
    phi = torch.zeros_like(d)
    grad = torch.empty((3,) + d.shape, dtype=torch.float64, device=dev)
    ctx = mg.Context(local)
    p = mg.default_params(alpha=alpha, s=s, h=L_BOX / 512, tol=TOLMIX, precision="mixed")
    tune = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        ctx.autotune(n, "mixed")
        tune = {"seconds": time.perf_counter() - t0, "mixed": schedules(mg, local, "mixed", n)}
    for _ in range(args.warmup):
        ctx.solve_fifth_force(d, p, phi=phi, grad=grad)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, cu = [], 0
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, info = ctx.solve_fifth_force(d, p, phi=phi, grad=grad)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        cu += info.cell_updates
    ctx.profile_enable(True)
    for _ in range(args.steps):
        ctx.solve_fifth_force(d, p, phi=phi, grad=grad)
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    clk = clocks.stop()
    if rank != 0:
        return
    tot = sum(ms)
    out = {"metric": METRIC, "value": cu / (tot / 1e3), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
           "data": "synthetic",
           "config": {"workload": "mixed%d: periodic %d^3 nDGP mixed-precision solve to 1e-8 "
                                  "(lognormal GRF sigma=2, seed 3, h=0.488 Mpc/h)" % (n, n),
                      "n": n, "tol": TOLMIX, "l2": "inputs larger than L2"},
           "time_to_tol_ms": tot / args.steps, "outer_iters": info.outer_iters,
           "inner_cycles": info.cycles, "rel_residual": info.rel_residual,
           "roofline": roofline(prof, _peaks(), args.steps),
           "kernels": {k: {"ms": v[0] / args.steps, "launches": v[1] // args.steps}
                       for k, v in prof.items() if v[1] > 0},
           "clocks": clk, "autotune": tune}
    print(json.dumps(out), flush=True)


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    coarse, patch, origin = make_inputs()
    per_step = max(args.cpu_seconds / 2.0, 5.0)
    for _ in range(args.warmup and 1):
        cpu_baseline(coarse, patch, origin, budget_s=1.0)
    vals, cus = [], 0.0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b = cpu_baseline(coarse, patch, origin, budget_s=per_step)
        vals.append(b)
    wall = time.perf_counter() - t0
    v = float(np.mean([b["value"] for b in vals]))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "refine128 (bounded sample on host cores: the FP64 oracle)",
                      "n": N_COARSE, "patch": 2 * PN},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                            "sample": vals[0]["sample"]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mg5", choices=["mg5", "ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--workload", default="refine128", choices=["refine128", "mixed"])
    ap.add_argument("--n", type=int, default=512, help="grid side of --workload mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer pass (profiling runs)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 96-box batched workload")
    ap.add_argument("--no-sizes", action="store_true",
                    help="skip the 32^3 FP64 and 512^3 mixed / FP64 records")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--no-truncation-levels", action="store_true",
                    help="skip the nested multi-level truncation report")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default sweep schedules instead of the tuned ones")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the serving run (0 skips it)")
    ap.add_argument("--serve-compare-seconds", type=float, default=12.0,
                    help="length of each leg of the mixed-vs-FP64 serving comparison "
                         "(0 skips it, as --serve-seconds 0 does)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "mixed":
        run_mixed_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
