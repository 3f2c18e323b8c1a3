"""Benchmark of the LBGK hot path on GB300 (one JSON line on stdout).

Default workload: the batched ensemble of 4096 independent KdV-Burgers problems
u_t + a u u_x - b u_xx + d u_xxx = 0 (N ~ U{256..8192}, a ~ U[1,6], b ~ U[0,0.1],
d ~ U[0.5,1], single-soliton initial profiles with c ~ U[1,4], seed-fixed), D1Q5 scheme 1,
dx = 0.1, dt = 1e-4, tau = 1.15, 1000 time steps, FP32 deviation storage, one launch.

One benchmark step = one pass of the whole hot path over the batch: initialisation from
the device-resident initial profiles (a1), 1000 collide+stream steps (a2-a6) and the FP64
diagnostics reduction (a7).  The model set-up (a0) happens once, at batch creation.
``value`` is lattice node-updates per second over all ranks.

--workload long_grid: the 2^24-node Kawahara grid (D1Q7, 1000 steps) in temporally blocked
windows; with --kernel stream, on the one-step-per-launch streaming kernel (HBM roofline).
--workload bounded: a tau sweep of Example 4.1 on its bounded grid (non-equilibrium
extrapolation boundary, A_40 left out as for Table I): --sweep-members instances of N = 601,
dx = 0.1, dt = 1e-3, tau spread over [1.989, 2.6], 1000 steps, one shared boundary array;
every instance resident (FP32: 16 nodes a thread, 13 instances a CTA; FP64: one CTA each), 11856
instances by default (78 per SM).
--workload nu_grid: a 2^24-node periodic grid of u_t + u^1.5 u_x + u_xxx = 0 (class (1) with a
real exponent), 1000 steps in on-chip windows (the real-exponent variant evaluates phi^nu once
per node; ALU roofline), or on the streaming kernel with --kernel stream (HBM roofline).
--impl reference: the CPU oracle timed on the host cores on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0907_1720_gb300 import workloads as W  # noqa: E402

METRIC = "lattice-node updates/s (FP32 batched vs FP64 plain) at stated L2 error; p99 solve latency"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# FP32 lanes per SM of GB300 (the SM count is read from the device): the ALU roof of the on-chip
# kernels.
FP32_LANES = 128
FP64_FMA_PER_SM_CLK = 2  # GB300: 152 x 2 x 2 flops x 2070 MHz = 1.26 TFLOP/s, the nominal 1.25
BOUNDED_STEPS = 1000
BOUNDED_TAU = (1.989, 2.6)

# DRAM bytes (read + write) per node of one k_stream<float,7,7,...> launch, from an ncu capture
# on a 2^23-node grid (traffic grows with N); used for the streaming roofline's "traffic".
STREAM_F32_D1Q7_DRAM_BYTES_PER_NODE = (235003648 + 184919808) / 8388608


class ClockSampler:
    """nvidia-smi clock/throttle samples (200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def ensemble_problems(rank=0, members=4096, world=1, nodes=0):
    """Members rank, rank + world, ... of the one seeded ensemble (a partition over the ranks);
    nodes > 0: every member that many nodes (profiling cases)."""
    if nodes > 0:
        return W.kdv_burgers_ensemble(count=members, n_lo=nodes, n_hi=nodes)[rank::world]
    return W.kdv_burgers_ensemble(count=members)[rank::world]


def sm_count(torch, dev):
    """Streaming multiprocessors of the device, as the runtime reports them."""
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def alu_peak(esz, clocks, peaks, sms):
    """ALU roof at the median SM clock under load: FP32 lanes, or GB300's FP64 FMA rate."""
    sm_mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    if esz == 4:
        return (sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12,
                f"derived: {sms} SMs (queried from the device) x {FP32_LANES} FP32 lanes x 2 x median SM clock "
                f"under load ({sm_mhz:.0f} MHz)")
    return (sms * FP64_FMA_PER_SM_CLK * 2 * sm_mhz * 1e6 / 1e12,
            f"derived: {sms} SMs (queried from the device) x {FP64_FMA_PER_SM_CLK} FP64 FMA/clk x 2 x median SM "
            f"clock under load ({sm_mhz:.0f} MHz; 1.26 TFLOP/s at 152 SMs and 2070 MHz, the nominal 1.25)")


def bounded_problems(members):
    """Example 4.1 (Table I, c = 100) with tau spread evenly over BOUNDED_TAU."""
    taus = np.linspace(BOUNDED_TAU[0], BOUNDED_TAU[1], members)
    probs = []
    for t in taus:
        p = W.bounded_config("4.1", 1e-3, float(t), BOUNDED_STEPS * 1e-3, scheme=1 | 0x100)
        p.meta["depth"] = 2
        probs.append(p)
    return probs


def workload_problems(args, rank=0, world=1):
    """(problems, steps per benchmark step, description) of the workload; both arms name the
    workload by this description.  The ensemble is one seeded batch whose members rank,
    rank + world, ... this rank takes; the description names the whole batch."""
    if args.workload == "ensemble":
        nodes = getattr(args, "member_nodes", 0)
        probs = ensemble_problems(rank, args.members, world, nodes)
        nsteps = W.ENSEMBLE_STEPS
        total_n = (sum(p.N for p in ensemble_problems(0, args.members, 1, nodes)) if world > 1
                   else sum(p.N for p in probs))
        sizes = f"N={nodes}" if nodes > 0 else "N~U{256..8192}"
        desc = (f"kdv_burgers_ensemble_{args.members}: {args.members} x {sizes} "
                f"(sum N = {total_n}), "
                f"D1Q5 scheme 1, dx={W.ENSEMBLE_DX}, dt={W.ENSEMBLE_DT}, tau={W.ENSEMBLE_TAU}, "
                f"{nsteps} steps per benchmark step")
    elif args.workload == "bounded":
        probs = bounded_problems(args.sweep_members)
        nsteps = BOUNDED_STEPS
        desc = (f"ks_shock_tau_sweep_{args.sweep_members}: {args.sweep_members} x N=601 (Example 4.1 on "
                f"[-30, 30], bounded grid, non-equilibrium extrapolation depth 2), D1Q5 scheme 1 without "
                f"A_40, dx=0.1, dt=1e-3, tau in [{BOUNDED_TAU[0]}, {BOUNDED_TAU[1]}], {nsteps} steps per "
                f"benchmark step, every instance resident")
    elif args.workload == "nu_grid":
        p = W.gkdv_grid_config(N=args.nodes, nsteps=1000)
        probs, nsteps = [p], p.nsteps
        desc = (f"gkdv_real_exponent_grid: N={args.nodes}, u_t + u^1.5 u_x + u_xxx = 0, D1Q5 scheme 1, "
                f"dx=0.1, dt=1e-4, tau=1.3, {nsteps} steps per benchmark step ("
                f"{'streaming kernel' if args.kernel == 'stream' else 'temporally blocked windows'}, "
                f"phi^nu once per node)")
    else:
        p = W.long_grid_config(N=args.nodes, nsteps=1000)
        probs, nsteps = [p], p.nsteps
        desc = (f"kawahara_long_grid: N={args.nodes}, D1Q7 scheme 1, dx=0.1, dt=1e-4, tau=2.02, "
                f"{nsteps} steps per benchmark step "
                f"({'streaming kernel' if args.kernel == 'stream' else 'temporally blocked windows'})")
    return probs, nsteps, desc


def flops_per_node_update(b, D):
    """Algorithmic FP operations of one node-update in the kernels' formulation: per moving
    population one Horner polynomial of degree D plus the relaxation (D + 1 multiply-adds,
    2 flops each) and the flux-difference update of phi (one subtract, one add)."""
    return (b - 1) * (2 * (D + 1) + 2)


def flops_per_node_update_nu(b, A, Dg):
    """The same for f^eq_j = sum_{a<=A} w^a Q_{j,a}(phi) with rows of degree Dg: per moving
    population (A + 1) Dg multiply-adds within the rows, A across them and one for the
    relaxation, plus the flux-difference update.  w = phi^nu (one per node, special-function
    unit) is not counted."""
    return (b - 1) * (2 * ((A + 1) * Dg + A + 1) + 2)


def nu_shape(L, p):
    """(A, Dg) of a real-exponent problem's model."""
    info = L.lbhpde_model(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau, lattice=p.eq.lattice, scheme=p.scheme,
                          nu=p.eq.nu, pi_nu=p.eq.pi_nu)
    return info.nu_rows - 1, info.nu_deg


def bytes_per_node_update(b, esz):
    """One read and one write of the b stored rows (phi and b-1 populations)."""
    return 2 * b * esz


# ----------------------------------------------------------------------- ours

def aggregate(t_local, units_local, world, device="cpu"):
    """Whole-job throughput over ranks that each process their own units (weak scaling):
    (sum of units over ranks) / (max of the ranks' times), and that max time."""
    if world <= 1:
        return units_local / t_local, t_local
    import torch
    import torch.distributed as dist

    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


def gather_member_records(records, world, device="cpu"):
    """Per-member records (index, sum phi, max |phi|, non-finite count) of every rank, gathered
    to all ranks and ordered by member index: the results of the whole partitioned batch."""
    import numpy as _np
    if world <= 1:
        return sorted(records)
    import torch
    import torch.distributed as dist

    loc = torch.tensor(_np.asarray(records, dtype=_np.float64).reshape(-1, 4), device=device)
    n = torch.tensor([loc.shape[0]], device=device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n)
    m = int(max(int(x.item()) for x in sizes))
    pad = torch.zeros((m, 4), dtype=torch.float64, device=device)
    pad[: loc.shape[0]] = loc
    bufs = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad)
    out = []
    for b, k in zip(bufs, sizes):
        out += [tuple(r) for r in b[: int(k.item())].cpu().numpy().tolist()]
    return sorted((int(r[0]), r[1], r[2], int(r[3])) for r in out)


def run_ours(args, rank, world, cpu=None):
    import torch

    from paper_0907_1720_gb300 import lbhpde as L

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    peaks, peak_src = load_peaks()

    with torch.cuda.stream(stream):
        # the autotuner picks nodes per thread and steps per window for this precision, lattice
        # and degree (outside the timed region); the batch below uses its choice
        tuned = None
        if args.onchip and args.workload in ("ensemble", "long_grid") and args.kernel != "stream":
            # a recorded choice instead of the timed one (profiling runs: ncu's serialised
            # timing would mislead the tuner); the batch then plans exactly as after tuning
            K_f, T_f = (int(v) for v in args.onchip.split(","))
            prec0 = L.FP32_DEV if args.precision == "fp32" else L.FP64
            b0, d0 = (5, 5) if args.workload == "ensemble" else (7, 7)
            L.set_tuning(prec0, b0, d0, K_f, T_f)
            tuned = {"nodes_per_thread": K_f, "steps_per_window": T_f, "recorded": True}
        elif (not args.no_tune and args.workload not in ("bounded", "nu_grid")
                and not (args.workload == "long_grid" and args.kernel == "stream")):
            prec0 = L.FP32_DEV if args.precision == "fp32" else L.FP64
            b0, d0 = (5, 5) if args.workload == "ensemble" else (7, 7)
            K_t, T_t, r_t = L.autotune(prec0, b0, d0)
            tuned = {"nodes_per_thread": K_t, "steps_per_window": T_t, "tuning_rate": r_t}
        probs, nsteps, workload = workload_problems(args, rank, world)
        prec = L.FP32_DEV if args.precision == "fp32" else L.FP64
        solver = L.Batch(probs, precision=prec)
        if args.kernel == "stream" and args.workload in ("nu_grid", "long_grid"):
            solver.set_kernel(L.KERNEL_STREAM)
        total = sum(p.N for p in probs)
        b = 5 if args.workload in ("ensemble", "bounded", "nu_grid") else 7
        bounded = args.workload == "bounded"
        phib_h = W.boundary_values(probs[0], 2, 0, nsteps) if bounded else None
        phib_d = torch.tensor(phib_h, device="cuda", dtype=torch.float64) if bounded else None

        def advance(pb):
            if bounded:
                solver.step_nee(nsteps, pb, 0)
            else:
                solver.step(nsteps)
        esz = 4 if prec == L.FP32_DEV else 8
        D = solver_model_degree(L, probs)
        phi0_h = np.concatenate([p.phi0 for p in probs])
        phi0_d = torch.tensor(phi0_h, device="cuda", dtype=torch.float64)
        pinned_in = torch.empty(total, dtype=torch.float64, pin_memory=True)
        pinned_in.numpy()[:] = phi0_h
        pinned_out = torch.empty(total, dtype=torch.float64, pin_memory=True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

        def one_step(record=None):
            solver.set_phi(phi0_d)
            if record is not None:
                record[0].record(stream)
            advance(phib_d)
            if record is not None:
                record[1].record(stream)
            return solver.diagnostics()

        for _ in range(args.warmup):
            one_step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        kernel_ms = []
        launches0 = solver.kernel_launches()
        with ClockSampler(dev) as clk:
            torch.cuda.synchronize()
            ev[2].record(stream)
            for _ in range(args.steps):
                rec = [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
                diag = one_step(rec)
                kernel_ms.append(rec)
            ev[3].record(stream)
            torch.cuda.synchronize()
        total_ms = ev[2].elapsed_time(ev[3])
        launches_timed = solver.kernel_launches() - launches0  # counted by the library
        kern = [a.elapsed_time(c) for a, c in kernel_ms]
        upd_step = total * nsteps
        value, t_max = aggregate(total_ms / 1e3, upd_step * args.steps, world, device="cuda")

        clocks = clk.summary()
        # the state after the last timed step: sampled members against the oracle (run on the host
        # cores before the GPU work, same inputs, same 1000 steps)
        oracle_cmp = None
        if cpu is not None and cpu.get("oracle_phi"):
            outs = solver.split(solver.read_phi())
            oracle_cmp = compare_members(outs, cpu["oracle_phi"], probs)
        # per-member results of the whole (partitioned) batch, gathered to every rank
        records = [(int(p.meta.get("index", i)), d["sum_phi"], d["max_abs_phi"], int(d["nonfinite"]))
                   for i, (p, d) in enumerate(zip(probs, diag))]
        members_all = gather_member_records(records, world, device="cuda")

        # accuracy beside the number: members against the FP64 path (ensemble) or the exact
        # solution (long grid)
        accuracy = None if args.quick else accuracy_report(L, args, probs, solver, prec, torch)
        if oracle_cmp is not None:
            accuracy = dict(accuracy or {})
            accuracy.update(oracle_cmp)
            accuracy["clocks"] = clocks

        # end to end through the public API, host buffers
        e2e_steps = 0 if args.quick else max(3, args.steps)  # as many steps as the timed region
        if e2e_steps:  # one untimed step through the same calls (first-touch of the host buffers)
            solver.set_phi(pinned_in)
            advance(phib_h)
            solver.read_phi(pinned_out.numpy())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            solver.set_phi(pinned_in)  # host pointer (pinned): copied inside the call
            advance(phib_h)            # boundary values from host memory, copied inside the call
            solver.read_phi(pinned_out.numpy())
        t_e2e = (time.perf_counter() - t0) / max(e2e_steps, 1)
        e2e = None if args.quick else {"value": world * upd_step / t_e2e, "unit": "node-updates/s",
                                       "h2d_bytes_per_step": total * 8 + (phib_h.nbytes if bounded else 0),
                                       "d2h_bytes_per_step": total * 8}

        # FP64 plain path on the same workload (fewer steps: it is ALU bound on GB300); its result
        # against the oracle on the sampled members
        fp64 = None
        if args.workload == "ensemble" and prec == L.FP32_DEV and not args.no_fp64 and not args.quick:
            fp64, outs64 = fp64_plain(L, probs, phi0_d, nsteps, stream, torch, steps=max(1, min(args.steps, 2)))
            if oracle_cmp is not None:
                c64 = compare_members(outs64, cpu["oracle_phi"], probs)
                accuracy["fp64_normwise_vs_oracle"] = c64["normwise_vs_oracle"]

        kern_ms = float(np.mean(kern))
        sms = sm_count(torch, dev)
        if bounded:
            fl = flops_per_node_update(b, D)
            peak_tf, src = alu_peak(esz, clocks, peaks, sms)
            achieved = fl * upd_step / (kern_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": achieved / peak_tf, "traffic": None,
                    "kernel": ("k_ring_nee<float,5,16,512,5,D2> (13 instances a CTA, interior nodes in registers, "
                               "depth-2 inflow rebuilt by its reader at fixed register positions)" if esz == 4 else
                               "k_bounded<double,5,4,512,5> (one resident CTA per instance)"),
                    "flops_per_node_update": fl, "peak_source": src}
        elif args.workload == "nu_grid" and args.kernel != "stream":
            A, Dg = nu_shape(L, probs[0])
            fl = flops_per_node_update_nu(b, A, Dg)
            peak_tf, src = alu_peak(esz, clocks, peaks, sms)
            achieved = fl * upd_step / (kern_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": achieved / peak_tf, "traffic": None,
                    "kernel": f"k_onchip<{'float' if esz == 4 else 'double'},5,K,...,-1> (halo windows, phi^nu)",
                    "flops_per_node_update": fl, "peak_source": src}
        elif args.workload == "nu_grid":
            by = bytes_per_node_update(b, esz)
            achieved = by * upd_step / (kern_ms / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                    "kernel": f"k_stream_rt<{'float' if esz == 4 else 'double'},5,256> (run-time degree, phi^nu)",
                    "bytes_per_node_update": by, "peak_source": peak_src}
        elif args.workload == "ensemble" or args.kernel != "stream":
            fl = flops_per_node_update(b, D)
            peak_tf, src = alu_peak(esz, clocks, peaks, sms)
            achieved = fl * upd_step / (kern_ms / 1e3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                    "frac": achieved / peak_tf, "traffic": None,
                    "kernel": (f"k_ring<float,5,16,512,5> (every member resident: whole waves at 16 nodes a "
                               f"thread, then the tail on k_onchip<float,5,8,512,0,5>)"
                               if args.workload == "ensemble" and esz == 4 else
                               f"k_onchip<{'float' if esz == 4 else 'double'},{b},K> "
                               f"({'resident instances + halo windows' if args.workload == 'ensemble' else 'halo windows'})"),
                    "flops_per_node_update": fl, "peak_source": src}
        else:
            by = bytes_per_node_update(b, esz)
            achieved = by * upd_step / (kern_ms / 1e3) / 1e9
            traffic = STREAM_F32_D1Q7_DRAM_BYTES_PER_NODE * total if esz == 4 else None
            roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                    "traffic_note": "per launch; ncu capture on 2^23 nodes scaled by N",
                    "kernel": "k_stream<float,7,7,256,1>" if esz == 4 else "k_stream<double,7,7,256,1>",
                    "bytes_per_node_update": by, "peak_source": peak_src}
            if esz == 8:
                # FP64 on GB300: the FP64 units bind long before HBM does
                fl = flops_per_node_update(b, D)
                peak_tf, src = alu_peak(esz, clocks, peaks, sms)
                alu = fl * upd_step / (kern_ms / 1e3) / 1e12
                roof = {"bound": "alu", "achieved": alu, "peak": peak_tf, "unit": "TFLOP/s",
                        "frac": alu / peak_tf, "traffic": None, "kernel": roof["kernel"],
                        "flops_per_node_update": fl, "peak_source": src,
                        "hbm": {"achieved_gbs": achieved, "frac": achieved / peaks["hbm_gbs"],
                                "bytes_per_node_update": by}}
        line = {
            "metric": METRIC, "value": value, "unit": "node-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "strong" if args.workload == "ensemble" and world > 1 else "weak", "vs_baseline": None,
            "dtype": "f32" if prec == L.FP32_DEV else "f64", "data": "synthetic (seeded, shaped like the paper's test problems)",
            "config": {"workload": workload, "node_updates_per_step": upd_step, "precision": args.precision,
                       "autotuned": tuned,
                       "l2": (f"inputs larger than L2: state {total * b * esz / 2**20:.0f} MiB, updated in place"
                              if bounded else
                              f"inputs larger than L2: state {2 * total * b * esz / 2**20:.0f} MiB (two buffers)"),
                       "parallelism": (f"members r::{world} of one seeded ensemble on rank r (no collective in the "
                                       f"steps; per-member results gathered once after the timed region)"
                                       if args.workload == "ensemble" and world > 1 else
                                       f"replicas x{world} (independent copies of the workload)")},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches_timed, "clocks": clocks,
            "kernel_ms_per_step": kern_ms, "accuracy": accuracy,
        }
        if fp64 is not None:
            line["fp64_plain"] = fp64
        if world > 1:
            line["members"] = {"gathered": len(members_all),
                               "sum_phi_total": float(sum(r[1] for r in members_all)),
                               "nonfinite": int(sum(r[3] for r in members_all))}
        solver.close()
        # the small configurations and the serving stream, measured in the same run (rank 0, one
        # GPU, default workload)
        if args.workload == "ensemble" and world == 1 and not args.quick and not args.no_legs:
            line["configs_small"] = small_configs_leg(L, torch, stream, cpu.get("small") if cpu else None)
            line["serving"] = serving_leg(args, L, torch)
    return line


def compare_members(outs, want, probs):
    """Sampled members of a batch result against the oracle's phi: normwise, relative L2 and E
    (the paper's L1 ratio), the maximum over the members, and each member's figures."""
    per = []
    for i, w in sorted(want.items()):
        g = np.asarray(outs[i], dtype=np.float64)
        per.append({"member": int(i), "N": int(probs[i].N),
                    "normwise": float(np.abs(g - w).max() / np.abs(w).max()),
                    "l2": float(np.linalg.norm(g - w) / np.linalg.norm(w)),
                    "E": float(np.abs(g - w).sum() / np.abs(w).sum())})
    return {"l2_vs_oracle": max(r["l2"] for r in per), "E_vs_oracle": max(r["E"] for r in per),
            "normwise_vs_oracle": max(r["normwise"] for r in per), "members_vs_oracle": per,
            "reference": "the FP64 CPU oracle on the host cores, same inputs and steps"}


def serving_description(args):
    return (f"serving: Poisson arrivals (mean {args.rate:g} req/s) of mixed KdV / mKdV / K(2,2) / KS / Kawahara "
            f"requests, N log-uniform [128, 65536], steps uniform [1e3, 1e5], FP32 deviation storage, "
            f"memory-admitted")


def serve_rate(L, rate, count, precision, arena_gb, block):
    """One serving run: `count` requests of the seeded Poisson stream at `rate` submitted from a
    host thread at their arrival times while the server runs, then drained; latency = finish -
    submit on the server's clock.  Offered vs achieved node-updates/s, p50/p99 latency, the GPU
    busy fraction and the scheduler's phase times."""
    reqs = W.serving_requests(count, rate=rate, seed=W.SEED + int(rate))
    srv = L.Server(precision=L.FP32_DEV if precision == "fp32" else L.FP64,
                   device_bytes=arena_gb << 30, max_active=4096, steps_per_block=block)
    ids = [None] * count
    t_start = time.perf_counter()

    def submitter():
        for i, (ta, p) in enumerate(reqs):
            dt_ = ta - (time.perf_counter() - t_start)
            if dt_ > 0:
                time.sleep(dt_)
            ids[i] = srv.submit_problem(p)

    th = threading.Thread(target=submitter)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        th.start()
        done = {}
        while len(done) < count:
            for i in range(count):
                if i in done or ids[i] is None:
                    continue
                rc, _, info = srv.poll(ids[i])
                if rc != L.PENDING:
                    done[i] = (rc, info)
            time.sleep(0.002)
        th.join()
    st = srv.stats()
    srv.close()
    lat = np.array([done[i][1]["finish_s"] - done[i][1]["submit_s"] for i in range(count)])
    t0 = min(done[i][1]["submit_s"] for i in range(count))
    t1 = max(done[i][1]["finish_s"] for i in range(count))
    work = sum(p.N * p.nsteps for _, p in reqs)
    ok = sum(1 for i in range(count) if done[i][0] == L.OK)
    return {"rate_req_s": rate, "requests": count, "ok": ok,
            "offered_node_updates_s": work / reqs[-1][0],
            "achieved_node_updates_s": work / (t1 - t0), "makespan_s": t1 - t0,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "launches": st["launches"], "gpu_busy_s": st["gpu_busy_s"],
            "host_s": {k[5:-2]: st[k] for k in ("host_admit_s", "host_setup_s", "host_plan_s",
                                                 "host_launch_s", "host_wait_s", "host_retire_s")},
            "gpu_busy_frac": st["gpu_busy_s"] / (t1 - t0), "clocks": clk.summary()}


def run_serving(args):
    """Continuous batching: Poisson arrivals of mixed requests submitted from a host thread
    while the server runs; latency = finish - submit on the server's clock."""
    import torch

    from paper_0907_1720_gb300 import lbhpde as L

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    out = []
    rates = [args.rate] + ([args.rate / 4, args.rate / 16] if args.sweep else [])
    for rate in rates:
        count = min(args.requests, max(64, int(args.window * rate)))
        out.append(serve_rate(L, rate, count, args.precision, args.arena_gb, args.block))
    head = out[0]
    fp64 = None if args.quick else serving_fp64_plain(L, W.serving_requests(
        min(args.requests, max(64, int(args.window * args.rate))), rate=args.rate, seed=W.SEED + int(args.rate)))
    line = {"metric": METRIC, "value": head["achieved_node_updates_s"], "unit": "node-updates/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": head["makespan_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic (seeded Poisson request stream)",
            "config": {"workload": serving_description(args),
                       "window_requests": head["requests"], "steps_per_block": args.block},
            "p50_latency_s": head["p50_latency_s"], "p99_latency_s": head["p99_latency_s"],
            "gpu_launches": head["launches"],
            "clocks": head["clocks"], "sweep": out}
    if fp64 is not None:
        line["fp64_plain"] = fp64
    return line


SERVING_LEG_RATES = (2000.0, 500.0)  # the configuration's rate, and one below the knee


def serving_leg(args, L, torch):
    """The serving configuration inside the default run: the seeded stream at 2000 requests/s
    (the configuration's mean rate, beyond one GPU's capacity) and at 500/s (below the knee),
    each over 1 s of arrivals, drained; then the plain per-request FP64 path on the first
    requests of the 2000/s stream.  p50/p99 are those of the 2000/s run."""
    torch.cuda.synchronize()
    rates = [serve_rate(L, r, int(r * 1.0), "fp32", args.arena_gb, args.block) for r in SERVING_LEG_RATES]
    fp64 = serving_fp64_plain(L, W.serving_requests(int(SERVING_LEG_RATES[0]), rate=SERVING_LEG_RATES[0],
                                                    seed=W.SEED + int(SERVING_LEG_RATES[0])))
    head = rates[0]
    return {"workload": "Poisson arrivals of mixed KdV / mKdV / K(2,2) / KS / Kawahara requests, N log-uniform "
                        "[128, 65536], steps uniform [1e3, 1e5], FP32 deviation storage, 1 s of arrivals per rate",
            "rate_req_s": head["rate_req_s"], "p50_latency_s": head["p50_latency_s"],
            "p99_latency_s": head["p99_latency_s"], "achieved_node_updates_s": head["achieved_node_updates_s"],
            "offered_node_updates_s": head["offered_node_updates_s"], "gpu_busy_frac": head["gpu_busy_frac"],
            "clocks": head["clocks"], "rates": rates, "fp64_plain": fp64,
            "batched_over_fp64_plain": head["achieved_node_updates_s"] / fp64["value"]}


def small_configs_leg(L, torch, stream, refs):
    """Configurations 1 (KdV soliton, N = 400, t = 1, 100 000 steps) and 2 (Kuramoto-Sivashinsky,
    N = 1024, t = 10, 100 000 steps), each in FP64 and FP32 on the automatic kernel: the whole
    instance resident in one CTA (one SM) for every step, with as many threads as it has node
    pairs, since a grid this small has no more parallel work than one CTA holds and more CTAs
    would need a grid-wide exchange each step (latency-bound: a step is a barrier, an exchange
    and two nodes' arithmetic per thread).
    CUDA-event time of the steps, E and relative L2 against the exact solution (KdV) or the
    ETDRK4 reference (KS), and the oracle's single-thread rate on the host beside it."""
    out = {}
    cases = (("kdv_n400_t1", W.kdv_config()), ("ks_n1024_t10", W.ks_config()))
    with torch.cuda.stream(stream):
        for name, p in cases:
            if name.startswith("kdv"):
                ref, ref_kind = p.exact(p.t_end), "exact soliton"
            else:
                ref = refs[name]["reference"] if refs and name in refs else W.ks_spectral_reference(t_end=p.t_end)
                ref_kind = "Fourier ETDRK4 reference"
            rec = {"N": p.N, "steps": p.nsteps, "dt": p.dt, "tau": p.tau, "error_against": ref_kind,
                   "ctas": 1, "sms": 1}
            for prec, tag in ((L.FP64, "fp64"), (L.FP32_DEV, "fp32")):
                sv = L.Solver.for_problem(p, precision=prec)
                sv.set_phi(p.phi0).step(500)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                sv.set_phi(p.phi0)
                a.record(stream)
                sv.step(p.nsteps)
                b.record(stream)
                b.synchronize()
                sec = a.elapsed_time(b) / 1e3
                phi = sv.read_phi()
                sv.close()
                rec[tag] = {"us_per_step": sec / p.nsteps * 1e6, "solve_s": sec,
                            "node_updates_s": p.N * p.nsteps / sec,
                            "E": float(np.abs(phi - ref).sum() / np.abs(ref).sum()),
                            "l2": float(np.linalg.norm(phi - ref) / np.linalg.norm(ref)),
                            "kernel": (f"k_onchip<{'float' if tag == 'fp32' else 'double'},5,2,1024,false,5>: the "
                                       f"whole instance resident in one CTA, 2 nodes a thread (the automatic "
                                       f"choice for a batch too small to give every SM a warp)")}
            rec["fp32_E_over_fp64_E"] = rec["fp32"]["E"] / rec["fp64"]["E"]
            if refs and name in refs:
                rec["oracle_single_thread"] = refs[name]["oracle"]
            out[name] = rec
    if refs and "kawahara_2^24" in refs:
        out["kawahara_2^24_oracle_single_thread"] = refs["kawahara_2^24"]["oracle"]
    return out


def serving_fp64_plain(L, reqs, max_updates=2e9):
    """The plain per-instance FP64 path on the same request stream: requests taken in arrival
    order until about max_updates node-updates, each solved alone (its own handle, FP64,
    streaming kernel) back to back on one stream; CUDA-event service time per request."""
    import torch

    stream = torch.cuda.Stream()
    times, work = [], 0
    with torch.cuda.stream(stream):
        for _, p in reqs:
            if work > max_updates:
                break
            s = L.Solver.for_problem(p, precision=L.FP64).set_kernel(L.KERNEL_STREAM)
            phi0 = torch.tensor(p.phi0, device="cuda", dtype=torch.float64)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.set_phi(phi0)
            a.record(stream)
            s.step(p.nsteps)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b) / 1e3)
            work += p.N * p.nsteps
            s.close()
    t = np.array(times)
    return {"value": work / t.sum(), "unit": "node-updates/s", "requests": len(t),
            "service_s_p50": float(np.percentile(t, 50)), "service_s_p99": float(np.percentile(t, 99)),
            "path": "one handle per request, FP64, k_stream one launch per step (graph-replayed), back to back"}


def solver_model_degree(L, probs):
    D = 0
    for p in probs[:64]:
        info = L.lbhpde_model(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau, lattice=p.eq.lattice, scheme=p.scheme,
                              nu=p.eq.nu, pi_nu=p.eq.pi_nu)
        D = max(D, info.D)
    return D


def fp64_plain(L, probs, phi0_d, nsteps, stream, torch, steps=2):
    s = L.Batch(probs, precision=L.FP64).set_kernel(L.KERNEL_STREAM)
    s.set_phi(phi0_d)
    s.step(5)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        s.set_phi(phi0_d)
        s.step(nsteps)
        s.diagnostics()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    total = sum(p.N for p in probs)
    outs = s.split(s.read_phi())
    s.close()
    return ({"value": total * nsteps / (ms / 1e3), "unit": "node-updates/s", "ms_per_step": ms,
             "kernel": "k_stream<double,5,5> (one fused collide+stream launch per time step, HBM)"}, outs)


def accuracy_report(L, args, probs, solver, prec, torch):
    out = {}
    if args.workload == "ensemble":
        # FP32 members against the FP64 path on the same inputs (normwise, max over 8 members)
        idx = list(range(0, len(probs), max(1, len(probs) // 8)))[:8]
        sub = [probs[i] for i in idx]
        phi0 = np.concatenate([p.phi0 for p in sub])
        res = {}
        for pr in (L.FP64, prec):
            bt = L.Batch(sub, precision=pr)
            bt.set_phi(phi0).step(W.ENSEMBLE_STEPS)
            res[pr] = bt.split(bt.read_phi())
            bt.close()
        errs = [float(np.abs(a - c).max() / np.abs(c).max()) for a, c in zip(res[prec], res[L.FP64])]
        out["fp32_vs_fp64_normwise_max"] = max(errs)
        out["members_checked"] = len(sub)
    elif args.workload == "nu_grid":
        # FP32 against FP64 on a 2^16-node grid of the same configuration (no exact solution for
        # the soliton train), normwise
        q = W.gkdv_grid_config(N=1 << 16, nsteps=1000)
        res = {}
        for pr in (L.FP64, prec):
            bt = L.Batch([q], precision=pr)
            bt.set_phi(q.phi0).step(q.nsteps)
            res[pr] = bt.read_phi()
            bt.close()
        out["fp32_vs_fp64_normwise_2^16_nodes"] = float(np.abs(res[prec] - res[L.FP64]).max()
                                                       / np.abs(res[L.FP64]).max())
    elif args.workload == "bounded":
        # error E of every member against the exact solution at t = 1: the tau with the smallest
        # error, and the member at the paper's tau_opt = 1.989 against Table I (c = 100, t = 1)
        ex = torch.tensor(np.concatenate([p.exact(p.nsteps * p.dt) for p in probs]), device="cuda",
                          dtype=torch.float64)
        phib = W.boundary_values(probs[0], 2, 0, BOUNDED_STEPS)
        solver.set_phi(torch.tensor(np.concatenate([p.phi0 for p in probs]), device="cuda", dtype=torch.float64))
        solver.step_nee(BOUNDED_STEPS, phib, 0)
        E = np.array([d["err_E"] for d in solver.diagnostics(ex)])
        i = int(np.nanargmin(E))
        out["E_min"] = float(E[i])
        out["tau_at_E_min"] = float(probs[i].tau)
        out["E_at_tau_1.989"] = float(E[0])
        out["table_I_c100_t1"] = 2.9926e-3
    else:
        p = probs[0]
        ex = torch.tensor(p.exact(p.nsteps * p.dt), device="cuda", dtype=torch.float64)
        solver.set_phi(torch.tensor(p.phi0, device="cuda", dtype=torch.float64)).step(p.nsteps)
        d = solver.diagnostics(ex)[0]
        out["E_vs_exact"] = d["err_E"]
        out["L2_vs_exact"] = d["err_L2"]
    return out


# ------------------------------------------------------------ oracle on the CPU

def ensemble_sample(probs, count):
    """Members the oracle runs on the host cores: the smallest, the largest, the first member of each
    resident CTA size class (up to 2048, 4096 and 8192 nodes) and seeded random picks, `count` in
    all."""
    Ns = np.array([p.N for p in probs])
    pick = [int(np.argmin(Ns)), int(np.argmax(Ns))]
    for lo, hi in ((0, 2048), (2048, 4096), (4096, 8192)):
        sel = np.where((Ns > lo) & (Ns <= hi))[0]
        if sel.size:
            pick.append(int(sel[0]))
    rng = np.random.default_rng(W.SEED)
    for i in rng.permutation(len(probs)):
        if len(set(pick)) >= count:
            break
        pick.append(int(i))
    return sorted(set(pick))[:max(count, 5)]


def oracle_members(oracle, probs, idx, steps, threads):
    """phi of members idx after `steps` steps (one member per thread; ctypes releases the GIL) and
    the wall time."""
    from concurrent.futures import ThreadPoolExecutor

    order = sorted(idx, key=lambda i: -probs[i].N)  # largest first: the threads finish together
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        outs = list(ex.map(lambda i: oracle.run_problem(probs[i], nsteps=steps), order))
    return dict(zip(order, outs)), time.perf_counter() - t0


def cpu_oracle_rate(args, sample_s=15.0, keep=False):
    """Oracle node-updates/s on the host cores: one member per thread (ctypes releases the GIL), on a
    bounded sample of the same workload.  Ensemble: 2 members per core (smallest, largest, one per
    resident size class, seeded random picks) at the full 1000 steps; with keep, their phi is
    returned too (the accuracy reference of the GPU result)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle

    cores = os.cpu_count() or 1
    if args.workload == "ensemble":
        probs = ensemble_problems(0, args.members, 1, getattr(args, "member_nodes", 0))
        idx = ensemble_sample(probs, 2 * cores)
        steps = W.ENSEMBLE_STEPS
        outs, el = oracle_members(oracle, probs, idx, steps, min(cores, len(idx)))
        upd = sum(probs[i].N for i in idx) * steps
        sizes = sorted(probs[i].N for i in idx)
        res = {"value": upd / el, "unit": "node-updates/s", "cores": min(cores, len(idx)), "kind": "oracle",
               "sample": f"{len(idx)} ensemble members (N from {sizes[0]} to {sizes[-1]}: the smallest, the largest, "
                         f"one per resident CTA size class, seeded random picks) x {steps} steps, one member per thread",
               "seconds": el}
        if keep:
            res["oracle_phi"] = outs
        return res
    elif args.workload == "bounded":
        p0 = bounded_problems(1)[0]
        pb = W.boundary_values(p0, 2, 0, BOUNDED_STEPS)

        def run(p, steps):
            M = oracle.Model(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau, scheme=p.scheme)
            f = M.init(p.phi0)
            M.step_nee(f, pb[:steps], 2)
            return f

        t0 = time.perf_counter()
        run(p0, 50)
        dt1 = (time.perf_counter() - t0) / 50
        steps = BOUNDED_STEPS
        # members of the full sweep (every tau of the benchmark), as many as fill the sample time
        nmem = int(min(args.sweep_members, max(2 * cores, sample_s * cores / (steps * dt1))))
        probs = bounded_problems(args.sweep_members)[:: max(1, args.sweep_members // nmem)][:nmem]
        t0 = time.perf_counter()
        with ThreadPoolExecutor(cores) as ex:
            list(ex.map(lambda p: run(p, steps), probs))
        el = time.perf_counter() - t0
        upd = sum(p.N for p in probs) * steps
        sample = f"{len(probs)} tau-sweep members x {steps} steps, one member per thread"
    elif args.workload == "serving":
        # the first requests of the same seeded stream, one per thread, each advanced by the
        # same number of steps (a bounded sample of their work)
        count = min(args.requests, max(64, int(args.window * args.rate)))
        probs = [q for _, q in W.serving_requests(count, rate=args.rate, seed=W.SEED + int(args.rate))][: 2 * cores]
        t0 = time.perf_counter()
        oracle.run_problem(probs[0], nsteps=5)
        dt1 = max((time.perf_counter() - t0) / 5 / max(probs[0].N, 1), 1e-12)  # seconds per node-update
        # one request per thread: the largest one sets the wall time of the sample
        steps = int(max(5, min(1000, sample_s / (dt1 * max(p.N for p in probs)))))
        t0 = time.perf_counter()
        with ThreadPoolExecutor(cores) as ex:
            list(ex.map(lambda p: oracle.run_problem(p, nsteps=steps), probs))
        el = time.perf_counter() - t0
        upd = sum(p.N for p in probs) * steps
        sample = f"the first {len(probs)} requests of the stream x {steps} steps each, one request per thread"
    elif args.workload == "nu_grid":
        p = W.gkdv_grid_config(N=1 << 16, nsteps=1)
        M = oracle.Model(p.eq.alpha, p.eq.pi, p.dx, p.dt, p.tau, nu=p.eq.nu, pi_nu=p.eq.pi_nu)
        f = M.init(p.phi0)
        t0 = time.perf_counter()
        M.step(f, 1)
        dt1 = time.perf_counter() - t0
        steps = int(max(1, min(1000, sample_s / dt1)))
        t0 = time.perf_counter()
        M.step(f, steps)
        el = time.perf_counter() - t0
        upd = p.N * steps
        cores = 1
        sample = f"2^16-node gKdV (n = 1.5) grid x {steps} steps, single thread"
    else:
        p = W.long_grid_config(nsteps=1)
        steps = 1
        t0 = time.perf_counter()
        oracle.run_problem(p, nsteps=steps)
        el = time.perf_counter() - t0
        upd = p.N * steps
        cores = 1
        sample = "2^24-node Kawahara grid x 1 step, single thread"
    return {"value": upd / el, "unit": "node-updates/s", "cores": cores, "kind": "oracle", "sample": sample,
            "seconds": el}


def small_refs():
    """Host side of the small configurations: the oracle's single-thread rate on configurations 1
    (KdV, N = 400) and 2 (KS, N = 1024) over a bounded number of steps, and on configuration 4 (the
    2^24-node Kawahara grid) over one step, each extrapolated to the configuration's full step
    count and labelled so; and the ETDRK4 reference of the KS run."""
    import oracle

    out = {}
    for name, p, steps, full_n in (("kdv_n400_t1", W.kdv_config(), 10000, 400),
                                   ("ks_n1024_t10", W.ks_config(), 4000, 1024),
                                   ("kawahara_2^24", W.long_grid_config(N=1 << 22, nsteps=1), 2, 1 << 24)):
        t0 = time.perf_counter()
        oracle.run_problem(p, nsteps=0)  # set-up and initialisation alone, subtracted below
        t1 = time.perf_counter()
        oracle.run_problem(p, nsteps=steps)
        el = max(time.perf_counter() - t1 - (t1 - t0), 1e-9)
        full = p.nsteps if name != "kawahara_2^24" else 1000
        rate = p.N * steps / el
        out[name] = {"oracle": {"node_updates_s": rate, "threads": 1, "steps_run": steps, "nodes_run": p.N,
                                "seconds": el, "solve_s_extrapolated": full_n * full / rate,
                                "note": f"{p.N} nodes x {steps} steps timed (initialisation excluded); the "
                                        f"{full_n}-node, {full}-step solve time extrapolated from that rate"}}
    out["ks_n1024_t10"]["reference"] = W.ks_spectral_reference(t_end=W.ks_config().t_end)
    return out


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, on the host cores, bounded sample."""
    cores = os.cpu_count() or 1
    vals = []
    for _ in range(args.warmup):
        cpu_oracle_rate(args, sample_s=2.0)
    for _ in range(args.steps):
        vals.append(cpu_oracle_rate(args, sample_s=8.0))
    v = float(np.median([r["value"] for r in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "node-updates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean([r["seconds"] for r in vals])) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": serving_description(args) if args.workload == "serving"
                       else workload_problems(args)[2], "sample": vals[-1]["sample"]},
            "cpu_baseline": {"value": v, "unit": "node-updates/s", "cores": vals[-1]["cores"], "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "node-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ensemble",
                    choices=["ensemble", "long_grid", "serving", "bounded", "nu_grid"])
    ap.add_argument("--sweep-members", type=int, default=11856,
                    help="bounded: tau-sweep instances (11856 = 152 SMs x 6 waves x 13 instances of 38 "
                         "threads a CTA on the 16-node kernel; the state exceeds L2)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: mean arrival rate (requests/s)")
    ap.add_argument("--window", type=float, default=1.0, help="serving: seconds of arrivals per rate")
    ap.add_argument("--requests", type=int, default=2000, help="serving: cap on requests per rate")
    ap.add_argument("--sweep", action="store_true", help="serving: also rates / 4 and / 16")
    ap.add_argument("--block", type=int, default=256, help="serving: steps per scheduling block")
    ap.add_argument("--arena-gb", type=int, default=8, help="serving: device arena (GiB)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "stream"],
                    help="long_grid only: the streaming kernel instead of temporally blocked windows")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--members", type=int, default=4096, help="ensemble members (profiling: smaller)")
    ap.add_argument("--member-nodes", type=int, default=0,
                    help="ensemble: every member this many nodes (profiling cases; 0 = the configuration's sizes)")
    ap.add_argument("--nodes", type=int, default=1 << 24, help="long-grid nodes (profiling: smaller)")
    ap.add_argument("--no-tune", action="store_true", help="skip the on-chip autotuner")
    ap.add_argument("--onchip", default=None, metavar="K,T",
                    help="ensemble/long grid: record this on-chip choice instead of running the autotuner")
    ap.add_argument("--no-legs", action="store_true",
                    help="ensemble: skip the small-configuration and serving legs")
    ap.add_argument("--quick", action="store_true",
                    help="only the timed region: no accuracy check, e2e, FP64 or CPU legs (profiling)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    # the CPU legs run before any GPU work: the oracle baseline (for the ensemble also the accuracy
    # reference of the sampled members) and the host side of the small configurations
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.quick:
        cpu = cpu_oracle_rate(args, keep=True)
        if args.workload == "ensemble" and not args.no_legs:
            cpu["small"] = small_refs()
    from paper_0907_1720_gb300 import build as B

    B.build()
    if args.workload == "serving":
        if rank == 0:
            print(json.dumps(run_serving(args)), flush=True)
        return
    line = run_ours(args, rank, world, cpu)
    if cpu is not None:
        line["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
