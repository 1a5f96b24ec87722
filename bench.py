"""Benchmark: Mcell-updates/s of the multi-material FV step on one GB300.

Default workload: the 256^3 shock-bubble problem with Mie-Grueneisen water and
an air bubble (shock 1e9 Pa at x = 0.2, bubble radius 0.15 at the centre), in
mixed precision (the headline ``value``), with the plain FP64 path timed on
the same grid next to it (``fp64``). A "step" is one full RK2 time step of the
whole grid: both stages (MUSCL + HLLC + FIVER + level set), the phase update,
and every tenth step the reinitialisation. The state (805 MB) is larger than
L2, so no flush is needed between steps.

--impl reference times the CPU oracle (the only reference: the paper ships no
code) on a bounded sample of the same workload.

Under torchrun each rank runs its own replica on its own GPU (the workload is
independent grids: weak scaling, no collective on the data path); rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# the headline metric as stated for this benchmark: `value` is the mixed-precision rate, the FP64
# rate is reported beside it (`fp64`), and the served latencies by `--workload served`
METRIC = "Mcell-updates/s at 256^3 two-phase, FP64 vs mixed; served p50/p99 latency"
UNIT = "Mcell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256, help="grid edge")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-variant", action="store_true", help="skip the FP32-Riemann-start line")
    ap.add_argument("--tile-rows", type=int, default=0, help="bulk-kernel tile rows (0: the library's default)")
    ap.add_argument("--l1-steps", type=int, default=300,
                    help="steps of the mixed-vs-FP64 L1 check after the timed runs (0: skip)")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"], help="precision of the headline run")
    ap.add_argument("--workload", default="grid256", choices=["grid256", "batched", "served"])
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--jobs", type=int, default=200)
    ap.add_argument("--serial-jobs", type=int, default=16)
    ap.add_argument("--slice-steps", type=int, default=25)
    ap.add_argument("--late-steps", type=int, default=50,
                    help="steps timed after the untimed advance of the L1 check (late window; 0: skip)")
    ap.add_argument("--sub-batch-steps", type=int, default=20,
                    help="steps of the batched sub-run of the default line (0: skip)")
    ap.add_argument("--sub-served-jobs", type=int, default=16,
                    help="jobs of the served sub-run of the default line (0: skip)")
    ap.add_argument("--sub-served-light-rate", type=float, default=1.0,
                    help="arrival rate (jobs/s) of the served sub-run's second pass, below the GPU's capacity (0: skip)")
    return ap.parse_args()


def dist_env():
    from paper_2508_16387_gb300 import dist as D
    return D.rank_env()


def setup(n):
    from paper_2508_16387_gb300 import workloads as WL
    return WL.shock_bubble(n=n, water=WL.WATER_MG, steps=500, name=f"shock_bubble_{n}^3_mg_water")


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            t0 = time.time()  # the first sample marks the sampler as running (nvidia-smi starts slowly)
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.02)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm

def make_grid(M, s, precision, stream=None):
    from paper_2508_16387_gb300 import runner as RN
    return RN.grid_for(s, precision, stream=stream)


def launches_per_step(step_index, reinit_every, reinit_iters):
    """Kernels m2c_step launches for step `step_index`: stage kernel, FIVER and finish for each of
    the two stages, phase update and end of step; on a reinitialisation step also one launch per
    iteration and the launch that copies the last iterate back (it exits at once unless there is
    a single iteration)."""
    n = 8
    if reinit_every > 0 and (step_index + 1) % reinit_every == 0 and reinit_iters > 0:
        n += reinit_iters + 1
    return n


def time_steps(torch, g, steps, warmup, barrier=None, breakdown=True):
    """Runs warmup steps, then times exactly `steps` steps with CUDA events on the grid's stream,
    the library recording event pairs around the bulk stage kernel launches only (so that the
    timed steps carry as little measurement as possible). Before that, untimed for the
    headline, the same `steps` steps from the same state run with event pairs around every
    launch for the per-kernel split; the state, time and step count are then put back, so both
    passes cover the same window of the run."""
    stream = torch.cuda.current_stream()
    g.step(warmup)
    t0, k0 = g.sync()
    kern = {}
    if breakdown:
        W0, phi0 = g.W.clone(), g.phi.clone()
        g.profile(True)
        g.step(steps)
        g.sync()
        kern = g.profile_read_kernels()
        g.profile(False)
        g.set_state(W0, phi0, t0, k0)
        del W0, phi0
    if barrier:
        barrier()
    torch.cuda.synchronize()
    g.profile(True, bulk_only=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kms, klaunch = g.profile_read_kernels()["stage"]
    g.profile(False)
    g.sync()
    time_steps.kernels = kern
    return ms, kms, klaunch


def e2e_run(torch, M, s, g, steps):
    """End to end through the C-ABI with host buffers: every step uploads the state from
    pinned host memory, advances one time step and downloads the new state into the same
    host buffers (the next step starts from it), one m2c_step_host call per step (which
    overlaps a call's download with the next call's upload, one state component at a time)."""
    nx, ny, nz = s.n
    Wh = torch.empty((5, nz, ny, nx), dtype=torch.float64, pin_memory=True)
    ph = torch.empty((nz, ny, nx), dtype=torch.float64, pin_memory=True)
    g.download(Wh, ph)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        g.step_host(Wh, ph, 1)
    g.sync()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nbytes = (Wh.numel() + ph.numel()) * 8
    return dt, nbytes


def l1_vs_fp64(torch, M, s, steps, late_steps=0):
    """Mixed against FP64 on the same workload after `steps` steps from the same initial state:
    relative L1 of 4^3-block averages (n^3 -> (n/4)^3) of density and pressure, from the
    library's own FP64 primitive fields. With late_steps, each grid is then timed over that many
    more steps (a late window: the shock is inside the bubble, interface work at its largest),
    mixed and FP64 (a fifth of the steps), with CUDA events on the grid's stream."""
    prims, late = {}, {}
    for prec in (M.MIXED, M.FP64):
        g = make_grid(M, s, prec)
        g.step(steps)
        g.sync()
        prims[prec] = g.prims()
        g.sync()
        k = late_steps if prec == M.MIXED else max(1, late_steps // 5)
        if late_steps > 0:
            with ClockSampler(torch.cuda.current_device()) as clk:
                ms, _, _ = time_steps(torch, g, k, 0, breakdown=prec == M.MIXED)
            late["mixed" if prec == M.MIXED else "fp64"] = {
                "value": round(s.ncells * k / (ms * 1e-3) / 1e6, 2), "unit": UNIT, "steps": k,
                "from_step": steps, "ms_per_step": round(ms / k, 4), "clocks": clk.summary(),
                **({"step_breakdown_ms": {kk: round(v[0] / k, 4) for kk, v in time_steps.kernels.items()},
                    "interface_faces": g.stats().interface_faces} if prec == M.MIXED else {})}
        del g

    def blocks(a):
        nz, ny, nx = a.shape
        return a.reshape(nz // 4, 4, ny // 4, 4, nx // 4, 4).mean(dim=(1, 3, 5))
    res = {"steps": steps, "blocks": f"4^3 ({s.n[0]}^3 -> {s.n[0] // 4}^3)", "tolerance": 1e-4}
    for name, v in (("rho", 0), ("p", 4)):
        a, b = blocks(prims[M.MIXED][v]), blocks(prims[M.FP64][v])
        res[name] = float((a - b).abs().sum() / b.abs().sum())
    del prims
    torch.cuda.empty_cache()
    l1_vs_fp64.late = late
    return res


def batched_run(torch, M, instances, steps, tune=True):
    """The batched workload: `instances` shock-bubble grids (edges from {32, 48, 64, 96, 128},
    radius, centre and shock pressure from seed 3) stepped together `steps` steps in one captured
    CUDA graph, mixed and FP64, after the autotuner has picked the tile shape, schedule and
    persistent grid size; CUDA events around the graph launch."""
    from paper_2508_16387_gb300 import autotune as AT
    from paper_2508_16387_gb300 import workloads as WL
    setups = WL.batched_instances(count=instances, seed=3, steps=steps)
    N = sum(x.ncells for x in setups)
    res = {}
    for name, prec in (("mixed", M.MIXED), ("fp64", M.FP64)):
        grids = [make_grid(M, x, prec) for x in setups]
        cands = AT.DEFAULT_CANDIDATES if prec == M.MIXED else AT.FP64_CANDIDATES
        best, trials = AT.tune_batch(grids, candidates=cands, trial_steps=2) if tune else ((8, 0, 0, 0), [])
        bt = M.Batch(grids, best)
        t0 = time.perf_counter()
        bt.capture(steps)
        cap_s = time.perf_counter() - t0
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(torch.cuda.current_device()) as clk:
            e0.record(torch.cuda.current_stream())
            bt.launch_graph()
            e1.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        for g in grids:
            g.sync()
        res[name] = {"value": round(N * steps / (ms * 1e-3) / 1e6, 2), "unit": UNIT, "ms": round(ms, 2),
                     "tuning": {"tile_rows": best[0], "tile_z": best[1], "schedule": ["stride", "atomic"][best[2]],
                                "blocks_per_sm": best[3]},
                     "autotune_trials": len(trials), "capture_s": round(cap_s, 2), "clocks": clk.summary()}
        del bt, grids
        torch.cuda.empty_cache()
    return {"workload": f"batched_{instances}_grids_seed3", "cells": N, "steps": steps,
            "edges": sorted({x.n[0] for x in setups}), "graph": True, **res}


def served_run(M, jobs, slice_steps):
    """Serving a trace: continuous batching in mixed precision against serving the same jobs one
    at a time in plain FP64 (arrival times honoured); p50/p99 latency (arrival to result on the
    host) and Mcell-updates/s over the wall time of each."""
    from paper_2508_16387_gb300 import serve as S

    def summary(st):
        ok = sum(1 for r in st.results if r.status == 0)
        return {"jobs": len(st.results), "ok": ok, "wall_s": round(st.wall_s, 2),
                "value": round(st.cell_updates / st.wall_s / 1e6, 2), "unit": UNIT,
                "p50_latency_s": round(st.percentile(50), 3), "p99_latency_s": round(st.percentile(99), 3),
                "max_resident": st.max_resident, "slices": st.slices}
    cont = S.Server(precision=M.MIXED, slice_steps=slice_steps).run(jobs, realtime=True)
    ser = S.serve_serial(jobs, precision=M.FP64, realtime=True)
    return {"continuous_mixed": summary(cont), "serial_fp64": summary(ser)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            P = json.load(f)
        return P.get("hbm_gbs", 6800.0), "measured"
    except OSError:
        return 6800.0, "fallback"


def _kernel_source_hash():
    """Identity of the bulk kernel's code: sha256 of its sources with comments and whitespace
    removed (so that a comment edit keeps the counters taken on the same code)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("m2c_stage.cuh", "m2c_stage_fp32.cu", "m2c_stage_fp64.cu", "m2c_device.cuh", "m2c_physics.cuh",
              "m2c_kernels.cuh"):
        with open(os.path.join(ROOT, "paper_2508_16387_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update(re.sub(r"\s+", "", text).encode())
    return h.hexdigest()[:16]


def _ncu_per_launch(key, n):
    """A per-launch counter of the bulk stage kernel from the committed ncu summary, scaled from
    256^3 to n^3 (both grow with the cells); None if the kernel sources changed since the
    counters were taken."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_traffic.txt")
    try:
        vals = {}
        with open(path) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("kernel_source_sha256_16") != _kernel_source_hash():
            return None
        return float(vals[key]) * (n / 256.0) ** 3
    except (OSError, KeyError, ValueError):
        return None


def ncu_traffic(kind, n):
    """DRAM read + write bytes per launch of the bulk stage kernel (dram__bytes_read.sum +
    dram__bytes_write.sum)."""
    return _ncu_per_launch(f"{kind}_bytes_per_launch_256", n)


def fp64_flops_per_cell_update():
    """FP64 operations per cell-update of the 256^3 MG shock-bubble workload, counted by the
    op-counting build of the oracle (committed summary; None if absent)."""
    try:
        with open(os.path.join(ROOT, "profiles", "fp64_flops_per_cell_update.txt")) as f:
            for line in f:
                if line.startswith("flops_per_cell_update_256_mg_shock_bubble"):
                    return float(line.split("=")[1])
    except (OSError, ValueError):
        pass
    return None


# GB300 FP64 rate: 1.89 DFMA per clock per SM (own probe on this machine's GB300), 2 FLOPs each
FP64_DFMA_PER_CLK_SM = 1.89


def issue_roofline(warp_inst, kernel_ms, sms, sm_mhz):
    """Instruction-issue roofline of a launch: warp instructions per launch (smsp__inst_executed.sum
    of the ncu capture, scaled to the launch) over the live mean launch time, against the SMs'
    issue rate, 4 schedulers x 1 warp instruction per clock per SM at the sampled SM clock.
    None without the counter or the clock."""
    if not warp_inst or not kernel_ms or not sm_mhz:
        return None
    achieved = warp_inst / (kernel_ms * 1e-3) / 1e9
    peak = sms * 4 * sm_mhz * 1e6 / 1e9
    return {"achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "G warp-inst/s",
            "frac": round(achieved / peak, 4), "warp_inst_per_launch": round(warp_inst),
            "source": "smsp__inst_executed.sum per launch from the ncu capture, scaled by cells; "
                      "peak = SMs x 4 schedulers x 1/clock x median sampled SM clock"}


def cpu_baseline(n=256, steps=8):
    """The oracle, as it stands, on the same 256^3 workload for a bounded number of steps."""
    from oracle import oracle as O
    s = setup(n)
    g = O.Grid(n=s.n, h=s.h, eos=tuple(O.EOS(*e) for e in s.eos), bc=s.bc, cfl=s.cfl,
               reinit_every=s.reinit_every, reinit_iters=s.reinit_iters)
    amb = s.prims_by_region[s.shock[1]]
    r1, u1, _ = O.shock_state(O.EOS(*s.eos[0]), (amb[0], amb[1], amb[4]), s.shock[0])
    W = O.prims_to_cons(g, s.prims((r1, u1)), s.phi)
    O.run(g, W, s.phi, 1)  # warm-up (page-in, thread start)
    t0 = time.perf_counter()
    O.run(g, W, s.phi, steps)
    dt = time.perf_counter() - t0
    return {"value": s.ncells * steps / dt / 1e6, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{steps} oracle time steps of the {n}^3 MG shock-bubble setup ({dt:.1f} s wall)"}


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    barrier = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        barrier = dist.barrier
    from paper_2508_16387_gb300 import m2c as M
    M.lib()
    s = setup(args.n)
    N = s.ncells
    out = {}

    g = make_grid(M, s, M.MIXED if args.prec == "mixed" else M.FP64)
    if args.tile_rows:
        g.set_tiling(args.tile_rows, 0)
    with ClockSampler(local) as clk:
        ms, kms, kl = time_steps(torch, g, args.steps, args.warmup, barrier)
    from paper_2508_16387_gb300 import dist as D
    t_max = D.max_over_ranks(ms)
    value = ws * N * args.steps / (t_max * 1e-3) / 1e6
    hbm, src = peaks()
    avg = kms / max(kl, 1)
    # tile rows of the bulk kernel: the requested ones, else the library's default rule
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    nx, ny, nz = s.n
    rows = args.tile_rows or (16 if -(-nx // 32) * -(-ny // 16) * -(-nz // 16) >= 8 * sms else 8)
    alg_bytes = 120.0 * N  # mean over stage 1 (96 B/cell) and stage 2 (144 B/cell)
    achieved = alg_bytes / (avg * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": ncu_traffic(args.prec, args.n),
            "kernel": f"k_stage<float,{rows}> (bulk stage)" if args.prec == "mixed"
                      else "k_stage<double,8> (bulk stage)", "peak_source": src,
            "kernel_ms_avg": round(avg, 4), "kernel_share": round(kms / ms, 3) if ms > 0 else None,
            "step_breakdown_ms": {k: round(v[0] / args.steps, 4) for k, v in time_steps.kernels.items()},
            "issue": issue_roofline(_ncu_per_launch(f"{args.prec}_warp_inst_per_launch_256", args.n), avg, sms,
                                    clk.summary()["sm_mhz"])}
    launches = sum(launches_per_step(args.warmup + i, s.reinit_every, s.reinit_iters) for i in range(args.steps))
    e2e = None
    if not args.no_e2e:
        sec, nbytes = e2e_run(torch, M, s, g, max(3, args.steps // 4))
        e2e = {"value": round(N * max(3, args.steps // 4) / sec / 1e6, 2), "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
    fp32_start = None
    if args.prec == "mixed" and not args.no_variant:
        # the same grid with the FIVER Newton iteration started on FP32 wave curves
        # (an option beyond the stated configuration, reported beside it, not as it)
        g.set_riemann_start(True)
        kv = max(5, args.steps // 2)
        msv, _, _ = time_steps(torch, g, kv, args.warmup, barrier)
        fp32_start = {"value": round(ws * N * kv / (D.max_over_ranks(msv) * 1e-3) / 1e6, 2), "unit": UNIT,
                      "steps": kv, "ms_per_step": round(msv / kv, 4),
                      "step_breakdown_ms": {k: round(v[0] / kv, 4) for k, v in time_steps.kernels.items()},
                      "what": "m2c_set_riemann_start(1): FP32 Newton start, FP64 finishing steps"}
        g.set_riemann_start(False)
    del g
    torch.cuda.empty_cache()
    fp64 = None
    if not args.no_fp64:
        g64 = make_grid(M, s, M.FP64)
        k64 = max(5, args.steps // 2)
        with ClockSampler(local) as clk64:
            ms64, kms64, kl64 = time_steps(torch, g64, k64, args.warmup, barrier, breakdown=False)
        avg64 = kms64 / max(kl64, 1)
        fpc = fp64_flops_per_cell_update()
        mhz = clk64.summary()["sm_mhz"] or 2070.0
        peak64 = FP64_DFMA_PER_CLK_SM * 2 * sms * mhz * 1e6 / 1e12
        ach = fpc * N * k64 / (ms64 * 1e-3) / 1e12 if fpc else None
        fp64 = {"value": round(N * k64 / (ms64 * 1e-3) / 1e6, 2), "unit": UNIT, "steps": k64,
                "ms_per_step": round(ms64 / k64, 3), "dtype": "f64", "clocks": clk64.summary(),
                "roofline": {"bound": "alu", "pipe": "fp64",
                             "achieved": round(ach, 4) if ach else None, "peak": round(peak64, 4), "unit": "TFLOP/s",
                             "frac": round(ach / peak64, 4) if ach else None,
                             "flops_per_cell_update": fpc,
                             "flops_source": "op-counting build of the oracle (profiles/fp64_flops_per_cell_update.txt)"
                                             "; add, mul, div, sqrt one FLOP each; achieved over the whole step",
                             "peak_source": "measured 1.89 DFMA/clk/SM x 2 FLOPs x SMs x median sampled SM clock",
                             "fp64_pipe_busy_ncu": 0.72, "kernel": "k_stage<double,8> (bulk stage)",
                             "kernel_ms_avg": round(avg64, 4), "traffic": ncu_traffic("fp64", args.n),
                             "hbm_frac": round(alg_bytes / (avg64 * 1e-3) / 1e9 / hbm, 4)}}
        del g64
    if rank != 0:
        return
    l1, late = None, None
    if args.prec == "mixed" and not args.no_fp64 and args.l1_steps > 0:
        l1 = l1_vs_fp64(torch, M, s, args.l1_steps, args.late_steps if ws == 1 else 0)
        late = l1_vs_fp64.late or None
    # sub-runs of the batched and served workloads (one GPU only: they are not weak-scaling runs)
    batched, served = None, None
    if ws == 1 and args.sub_batch_steps > 0:
        batched = batched_run(torch, M, args.instances, args.sub_batch_steps)
    if ws == 1 and args.sub_served_jobs > 0:
        from paper_2508_16387_gb300 import workloads as WL
        jobs = WL.served_trace(n_jobs=args.jobs, rate=20.0, seed=4)[:args.sub_served_jobs]
        with ClockSampler(local) as sclk:
            served = served_run(M, jobs, args.slice_steps)
        served.update({"workload": f"first_{len(jobs)}_jobs_of_served_200_jobs_poisson20_seed4",
                       "clocks": sclk.summary(),
                       "p50_s": served["continuous_mixed"]["p50_latency_s"],
                       "p99_s": served["continuous_mixed"]["p99_latency_s"]})
        if args.sub_served_light_rate > 0:
            # the same jobs arriving at a rate the GPU keeps up with: latency is service time
            # (the 20 jobs/s trace offers several times the GPU's rate, so its latencies are
            # mostly queueing)
            from paper_2508_16387_gb300 import serve as S
            light = WL.served_trace(n_jobs=args.jobs, rate=args.sub_served_light_rate, seed=4)[:args.sub_served_jobs]
            with ClockSampler(local) as lclk:
                st = S.Server(precision=M.MIXED, slice_steps=args.slice_steps).run(light, realtime=True)
            offered = sum(j.params.edge ** 3 * j.params.steps for j in light) / max(light[-1].arrival, 1e-9)
            served["light_load_mixed"] = {
                "rate_jobs_per_s": args.sub_served_light_rate, "jobs": len(st.results),
                "ok": sum(1 for r in st.results if r.status == 0), "wall_s": round(st.wall_s, 2),
                "offered_Mcell_updates_per_s": round(offered / 1e6, 1),
                "value": round(st.cell_updates / st.wall_s / 1e6, 2), "unit": UNIT,
                "p50_latency_s": round(st.percentile(50), 3), "p99_latency_s": round(st.percentile(99), 3),
                "max_resident": st.max_resident, "clocks": lclk.summary()}
    out = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64 (mixed)" if args.prec == "mixed" else "f64", "data": "synthetic",
           "config": {"workload": s.name, "grid": list(s.n), "precision": args.prec, "cells": N,
                      "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                      "l2": f"state ({48 * N / 1e6:.0f} MB) larger than L2, no flush"
                            if 48 * N > 129e6 else f"state ({48 * N / 1e6:.0f} MB) fits in L2"},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clk.summary(), "fp64": fp64,
           "mixed_fp32_riemann_start": fp32_start, "l1_error_vs_fp64": l1, "late_window": late,
           "batched": batched, "served": served}
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out))


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    import numpy as np  # noqa: F401
    n = 64
    s = setup(n)
    g = O.Grid(n=s.n, h=s.h, eos=tuple(O.EOS(*e) for e in s.eos), bc=s.bc, cfl=s.cfl,
               reinit_every=s.reinit_every, reinit_iters=s.reinit_iters)
    amb = s.prims_by_region[s.shock[1]]
    r1, u1, _ = O.shock_state(O.EOS(*s.eos[0]), (amb[0], amb[1], amb[4]), s.shock[0])
    W = O.prims_to_cons(g, s.prims((r1, u1)), s.phi)
    phi = s.phi
    r = O.run(g, W, phi, args.warmup)
    W, phi = r.W, r.phi
    t0 = time.perf_counter()
    r = O.run(g, W, phi, args.steps, step0=args.warmup)
    dt = time.perf_counter() - t0
    value = s.ncells * args.steps / dt / 1e6
    sample = (f"each step one oracle time step of the {n}^3 version of the 256^3 MG shock-bubble workload "
              f"(same physics, same per-cell work)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": setup(args.n).name, "grid": [args.n] * 3, "precision": "f64 (oracle)",
                   "sample_grid": [n] * 3},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_batched(args):
    """The batched workload alone (--workload batched): 200 steps in one captured CUDA graph."""
    import torch
    from paper_2508_16387_gb300 import m2c as M
    torch.cuda.set_device(dist_env()[2])
    M.lib()
    res = batched_run(torch, M, args.instances, args.batch_steps)
    print(json.dumps({"metric": "Mcell-updates/s, uneven shock-bubble grids stepped in one CUDA graph",
                      "value": res["mixed"]["value"], "unit": UNIT, "n_gpus": 1, "steps": args.batch_steps,
                      "higher_is_better": True, "dtype": "f32+f64 (mixed)", "data": "synthetic",
                      "config": {"workload": res["workload"], "cells": res["cells"], "edges": res["edges"]},
                      "mixed": res["mixed"], "fp64": res["fp64"]}))


def run_served(args):
    """Poisson arrivals at 20 jobs/s of shock-bubble jobs (edge log-uniform on [48, 192], 100-1000
    steps, seed 4) served with continuous batching in mixed precision (--workload served); the
    first `--serial-jobs` jobs of the trace are also served one at a time in plain FP64 and with
    continuous batching, for a same-trace comparison."""
    import torch
    from paper_2508_16387_gb300 import m2c as M
    from paper_2508_16387_gb300 import serve as S
    from paper_2508_16387_gb300 import workloads as WL
    torch.cuda.set_device(dist_env()[2])
    M.lib()
    jobs = WL.served_trace(n_jobs=args.jobs, rate=20.0, seed=4)
    with ClockSampler(dist_env()[2]) as clk:
        full = S.Server(precision=M.MIXED, slice_steps=args.slice_steps).run(jobs, realtime=True)
    ok = sum(1 for r in full.results if r.status == 0)
    full_s = {"jobs": len(full.results), "ok": ok, "wall_s": round(full.wall_s, 2),
              "value": round(full.cell_updates / full.wall_s / 1e6, 2),
              "p50_latency_s": round(full.percentile(50), 3), "p99_latency_s": round(full.percentile(99), 3),
              "max_resident": full.max_resident, "slices": full.slices}
    sub = served_run(M, jobs[:args.serial_jobs], args.slice_steps)
    offered = sum(j.params.edge ** 3 * j.params.steps for j in jobs) / jobs[-1].arrival
    out = {"metric": "served shock-bubble jobs: Mcell-updates/s and p50/p99 job latency",
           "value": full_s["value"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
           "dtype": "f32+f64 (mixed)", "data": "synthetic",
           "config": {"workload": f"served_{args.jobs}_jobs_poisson20_seed4", "slice_steps": args.slice_steps,
                      "offered_Mcell_updates_per_s": round(offered / 1e6, 1)},
           "served_mixed": full_s, "clocks": clk.summary(), f"first_{args.serial_jobs}_jobs": sub}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "batched":
        run_batched(a)
    elif a.workload == "served":
        run_served(a)
    else:
        run_ours(a)
