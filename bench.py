"""Benchmark of the fused explicit phase-field PVD step (cell-updates per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--workload NAME]

One bench step is one whole run of the workload: the default ``paper512`` is
the paper-scale plain DNS, a 512 x 512 FP32 grid advanced 50,000 explicit
midpoint steps from a seeded film, with mass/free-energy diagnostics every
1,000 steps, launched as CUDA-graph replays of 1,000 fused step kernels.
Every run restarts from the same initial state (reset outside the timed
events); L2 is flushed between runs.  Under torchrun each rank runs its own
replica (independent deposition runs: weak scaling, no collective on the data
path) and rank 0 prints one JSON line with the max time over ranks.

On one GPU the default line also carries
- ``secondary``: the same step on HBM-resident grids (4096^2) and the 64-run
  ensemble, each against the HBM roofline;
- ``hybrid``: the hybrid DNS / U-Net solver (16 runs of 256^2 to 100,000 steps,
  committed trained weights) against plain DNS of the same batch, timed in one
  loop, with its field and S2 errors;
- ``cpu_baseline`` (the FP64 oracle, single thread) and ``cpu_baseline_all_cores``
  (its OpenMP build over the host's cores) on a bounded sample.

``--impl reference`` times the FP64 CPU oracle on the host cores instead
(a bounded sample of the same workload), rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2312_05410_gb300 import inputs as I  # noqa: E402
from paper_2312_05410_gb300.dist import aggregate  # noqa: E402

METRIC = "DNS cell-updates/s (%HBM peak)"
UNIT = "cell-updates/s"
BYTES_PER_CELL_UPDATE = 24  # read phi, c, rho + write phi, c, rho, FP32
# FP32 FMA peak of a GB300: a probe of independent packed fma.rn.f32x2 chains on all 152 SMs, CUDA events,
# SM clock sampled at 2070 MHz (the scalar form measured 78.4)
FMA_PEAK_TFLOPS = 79.5


def step_flops(p: dict) -> int:
    """FP32 FLOPs (FMA = 2) of one fused step per cell, counted from the kernel's expression tree: 80 per
    Runge-Kutta stage for the Cahn-Hilliard phi with a uniform mobility; the bulk interpolation of the
    mobility adds 6, the surface term 5 more (and one exp2), the Allen-Cahn phi saves 5."""
    per_stage = 80
    if p.get("MA_surf", 0.0) != 0.0 or p.get("MB_surf", 0.0) != 0.0:
        per_stage += 11
    elif p.get("MA_bulk", 1.0) != p.get("MB_bulk", 1.0):
        per_stage += 6
    if p.get("phi_mode", 0) == 1:
        per_stage -= 5
    return 2 * per_stage


def alu_roofline(flops_per_cell: int, cells: int, per_launch_s: float) -> dict:
    """The fused step against the FP32 FMA peak: algorithmic FLOPs per launch / launch duration."""
    achieved = flops_per_cell * cells / per_launch_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": FMA_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FMA_PEAK_TFLOPS, "flops_per_cell_update": flops_per_cell,
            "peak_source": "measured FP32 FMA probe (packed f32x2, 152 SMs, 2070 MHz)"}

WORKLOADS = {
    "paper512": dict(spec=I.PAPER_512["spec"], params=I.PAPER_512["params"], steps=50000,
                     desc="plain DNS 512x512, 50000 steps, diagnostics every 1000"),
    "small64": dict(spec=I.SMALL_64["spec"], params=dict(I.SMALL_64["params"], diag_every=1000), steps=2000,
                    desc="plain DNS 64x64, 2000 steps"),
    "large4096": dict(spec=I.FilmSpec(4096, 4096, 16.0, seed=1), params=dict(v_mag=0.3, diag_every=1000),
                      steps=2000, desc="plain DNS 4096x4096, 2000 steps, diagnostics every 1000"),
    "large8192": dict(spec=I.FilmSpec(8192, 8192, 16.0, seed=1), params=dict(v_mag=0.3, diag_every=1000),
                      steps=1000, desc="plain DNS 8192x8192, 1000 steps, diagnostics every 1000"),
    "paper512_surface": dict(spec=I.PAPER_512["spec"],
                             params=dict(I.PAPER_512["params"], MA_bulk=2.0, MB_bulk=0.5, MA_surf=10.0, MB_surf=4.0,
                                         sigma_surf=0.5),
                             steps=50000, desc="plain DNS 512x512, 50000 steps, bulk + surface mobility (exp path)"),
    "paper512_angle50": dict(spec=I.PAPER_512["spec"], params=dict(I.PAPER_512["params"], v_angle_deg=50.0),
                             steps=50000, desc="plain DNS 512x512, 50000 steps, oblique incidence at 50 degrees"),
    "paper512_ac": dict(spec=I.PAPER_512["spec"], params=dict(I.PAPER_512["params"], phi_mode=1),
                        steps=50000, desc="plain DNS 512x512, 50000 steps, Allen-Cahn order parameter + source"),
    "adjoint256": dict(kind="adjoint", spec=I.FilmSpec(256, 256, 16.0, seed=4), params=dict(v_mag=0.4), steps=1000,
                       K=50, bytes_per_cell_update=84,
                       desc="adjoint 256x256, 1000 steps, checkpoint every 50, gradient of a final-state loss"),
    "hybrid256": dict(kind="hybrid", n_runs=16, side=256, seed=5, steps=100000, dns_stretch=2000, jump=2000,
                      frame_every=1000, lead_5pct=40000,
                      desc="hybrid DNS / U-Net: 16 runs of 256x256, 2000 DNS steps alternating with one U-Net jump "
                           "of 2000 steps (look-back frames 1000 steps apart), to 100000 steps"),
    "ensemble64": dict(kind="ensemble", n_runs=64, seed=3, steps=10000,
                       desc="batched DNS ensemble: 64 runs, sides in {128,192,256,384,512}, V~U[0.1,0.9], "
                            "c_inc~U[0.3,0.7], 10000 steps"),
}

DEFAULT_WORKLOAD = "paper512"
SECONDARY_WORKLOADS = ("large4096", "ensemble64")

# DRAM bytes (read + write) per step-kernel launch from one ncu capture (cold caches),
# keyed by workload, with the hash of the kernel source it was taken on; reported as
# null once the source changes.  Summaries: profiles/step_kernel_*_full.md.
NCU_TRAFFIC = {
    "paper512": {"bytes": 3175424, "src": "548a0e3871344ffe"},
    "large4096": {"bytes": 356260864, "src": "548a0e3871344ffe"},
}


def kernel_source_hash() -> str:
    with open(os.path.join(ROOT, "paper_2312_05410_gb300", "csrc", "pf_step.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return dict(hbm_gbs=d["hbm_gbs"], bf16_tflops=d.get("bf16_tflops", 1900.0), source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, source="fallback")


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        reasons = sorted({n for r in self.rows for n, v in zip(self.NAMES, r[2:]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class SingleRun:
    """One plain-DNS run through pf.Sim (periodic diagnostics inside the graph)."""

    def __init__(self, pf, W):
        spec = W["spec"]
        p = I.default_params(**W["params"])
        p["dt"] = 0.5 * pf.pf_dt_limit(p)[0]
        self.params = p
        self.sim = pf.Sim(p, *I.film_state(spec, p), history_rows=W["steps"] // max(1, p["diag_every"]) + 2)
        self.stream = self.sim.stream
        self.fields = list(self.sim.fields)
        self.cells = spec.nx * spec.ny
        self.nsteps = W["steps"]
        de = p["diag_every"]
        self.launches = self.nsteps + (2 * ((self.nsteps + de - 1) // de) if de else 0)
        self.config = {"nx": spec.nx, "ny": spec.ny, "timesteps_per_run": self.nsteps, "diag_every": de,
                       "dt": p["dt"], "launch": "CUDA graph replays of fused step kernels"}

    def reset_counters(self):
        self.sim.set_step(0)

    def run(self):
        self.sim.step(self.nsteps)

    def final_diag(self):
        return [float(x) for x in self.sim.diag()]

    def close(self):
        self.sim.close()


class EnsembleRun:
    """Independent runs of uneven sizes, one launch per step for all of them."""

    def __init__(self, pf, W):
        ms = []
        for m in I.ensemble_members(W["n_runs"], seed=W["seed"]):
            p = I.default_params(v_mag=m["v_mag"])
            p["dt"] = 0.5 * pf.pf_dt_limit(p)[0]
            ms.append((p, *I.film_state(m["spec"], p)))
        self.ens = pf.Ensemble(ms)
        self.stream = self.ens.stream
        self.fields = [t for run in self.ens.fields for t in run]
        self.cells = sum(ny * nx for ny, nx in self.ens.shapes)
        self.nsteps = W["steps"]
        self.chosen, self.tune = self.ens.autotune(10)
        per = pf.ENS_STEPS_PER_PERSISTENT_LAUNCH if self.chosen == 4 else 1
        self.launches = -(-self.nsteps // per)
        sides = sorted({nx for _, nx in self.ens.shapes})
        self.config = {"runs": len(ms), "sides": sides, "total_cells": self.cells, "timesteps_per_run": self.nsteps,
                       "tile_kind": f"{self.chosen}: {pf.TILE_KINDS[self.chosen]}", "autotune_s_per_step": self.tune,
                       "launch": "one fused launch per step for all runs, CUDA graph replays"}

    def reset_counters(self):
        pass

    def run(self):
        self.ens.step(self.nsteps)

    def final_diag(self):
        return [float(x) for x in self.ens.diag(0)]

    def close(self):
        self.ens.close()


class AdjointRun:
    """Gradient of a final-microstructure loss through nsteps steps (forward with checkpoints
    every K steps, then the hand-written adjoint backwards), as one pf_adjoint call."""

    def __init__(self, pf, W):
        import torch

        spec = W["spec"]
        p = I.default_params(**W["params"])
        p["dt"] = 0.5 * pf.pf_dt_limit(p)[0]
        self.pf, self.p, self.nx = pf, p, spec.nx
        self.nsteps, self.K = W["steps"], W["K"]
        st = I.film_state(spec, p)
        self.fields = pf.device_fields(st)
        # target: the same film deposited 30 % faster (the gradient points towards its rate)
        tsim = pf.Sim(dict(p, v_mag=1.3 * p["v_mag"]), *st)
        tsim.step(self.nsteps)
        self.target = [t.clone() for t in tsim.fields]
        tsim.close()
        self.stream = torch.cuda.current_stream()
        self.cells = spec.nx * spec.ny
        self.w = [torch.zeros_like(t) for t in self.fields]
        self.launches = self.nsteps * (1 + 1 + 1 + 4) + 1  # forward, recompute, Euler, two (A, B) passes; final sum
        self.config = {"nx": spec.nx, "ny": spec.ny, "timesteps_per_run": self.nsteps, "checkpoint_every": self.K,
                       "loss": "sum (phi_N - phi_T)^2 + (c_N - c_T)^2, target deposited 1.3x faster",
                       "launch": "pf_adjoint: forward with checkpoints, segment recompute, adjoint passes"}
        self.last = None

    def reset_counters(self):
        pass

    def run(self):
        # cotangent of the loss at the final state from the previous evaluation (fixed after warm-up)
        res = self.pf.adjoint(self.p, self.fields, self.nx, self.nsteps, self.K, *self.w)
        for q in range(2):
            self.w[q].copy_(2.0 * (res["final"][q] - self.target[q]))
        self.last = res

    def final_diag(self):
        r = self.last
        return [r["v_mag"], r["m_scale"], r["kappa_c"]]

    def close(self):
        pass


UNET_WEIGHTS = os.path.join(ROOT, "paper_2312_05410_gb300", "weights", "unet_lb3_hybrid256.npz")


class HybridPair:
    """The hybrid solver (pf.Hybrid: DNS stretches with look-back frames, U-Net jumps on the tensor cores,
    the plausibility gate with its DNS fallback) and plain DNS of the same batch, both from the same
    seeded states and with the tile shape the ensemble autotuner picks for the batch (timed on a
    throwaway copy)."""

    def __init__(self, pf, W):
        import torch

        ms = []
        for m in I.hybrid_members(W["n_runs"], W["side"], seed=W["seed"]):
            p = I.default_params(v_mag=m["v_mag"])
            p["dt"] = 0.5 * pf.pf_dt_limit(p)[0]
            ms.append((p, *I.film_state(m["spec"], p)))
        self.pf = pf
        probe = pf.Ensemble(ms)
        self.tile, _ = probe.autotune(20)
        probe.close()
        self.hyb, self.dns = pf.Ensemble(ms), pf.Ensemble(ms)
        for e in (self.hyb, self.dns):
            e.set_tile(self.tile)
        self.stream = self.hyb.stream
        side = W["side"]
        wpath = W.get("unet_weights") or (UNET_WEIGHTS if os.path.exists(UNET_WEIGHTS) else "")
        if wpath:
            with np.load(wpath) as z:
                weights = {k: z[k] for k in z.files}
            self.weights_desc = f"trained on GPU-DNS trajectories ({os.path.basename(wpath)})"
        else:
            weights = I.unet_weights(0)
            self.weights_desc = ("seeded, untrained: jumps that fail the plausibility check fall back to DNS "
                                 "(train with python -m paper_2312_05410_gb300.train_unet, pass --unet-weights)")
        self.trained = bool(wpath)
        self.net = pf.UNet(weights, W["n_runs"], side, side, stream=self.stream)
        self.solver = pf.Hybrid(self.hyb, self.net, dns_stretch=W["dns_stretch"], jump_steps=W["jump"],
                                frame_every=W["frame_every"])
        # the same alternation after a DNS lead-in: the schedule measured to keep phi and c within 5 %
        self.lead = W.get("lead_5pct", 0)
        self.lead_solver = pf.Hybrid(self.hyb, self.net, dns_stretch=W["dns_stretch"], jump_steps=W["jump"],
                                     frame_every=W["frame_every"], dns_lead=self.lead) if self.lead else None
        self.lead_stats = self.lead_errors = None
        self.h_fields = [t for run in self.hyb.fields for t in run]
        self.d_fields = [t for run in self.dns.fields for t in run]
        self.init = [t.clone() for t in self.h_fields]
        self.cells, self.nsteps, self.side = W["n_runs"] * side * side, W["steps"], side
        self.cycles = self.nsteps // (W["dns_stretch"] + W["jump"])
        self.stats = None
        # one jump alone (two frames pushed first), timed; then the state is restored
        self.net.frame(self.hyb.fields)
        self.net.frame(self.hyb.fields)
        self.net.jump(self.hyb.fields, 1.0)
        torch.cuda.synchronize()
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        ev[0].record(self.stream)
        for _ in range(5):
            self.net.jump(self.hyb.fields, 1.0)
        ev[1].record(self.stream)
        torch.cuda.synchronize()
        self.jump_s = ev[0].elapsed_time(ev[1]) / 5e3
        self.net.sync()
        self.reset_hybrid()
        self.reset_dns()
        from paper_2312_05410_gb300.unet_flops import flops_per_sample
        self.jump_flops = W["n_runs"] * flops_per_sample(side, side)
        self.config = {"runs": W["n_runs"], "nx": side, "ny": side, "timesteps_per_run": self.nsteps,
                       "dns_stretch": W["dns_stretch"], "jump_steps": W["jump"],
                       "lookback": "3 frames 1000 steps apart", "cycles": self.cycles,
                       "unet": "32-64-128-256, BF16 tensor-core convolutions, "
                               + ("trained weights" if self.trained else "seeded untrained weights"),
                       "dns_tile": pf.TILE_KINDS[self.tile] + " (autotuned)",
                       "launch": "pf_hybrid_run: fused ensemble step launches (graph replays), 2 frame kernels, "
                                 "28 U-Net launches and one plausibility check per cycle"}

    def reset_hybrid(self):
        for t, s in zip(self.h_fields, self.init):
            t.copy_(s)

    def reset_dns(self):
        for t, s in zip(self.d_fields, self.init):
            t.copy_(s)

    def run_hybrid(self):
        self.stats = self.solver.run(self.nsteps)

    def run_lead(self):
        self.lead_stats = self.lead_solver.run(self.nsteps)

    def run_dns(self):
        self.dns.step(self.nsteps)

    def launches(self):
        """Kernels of one hybrid run: every DNS step, 2 frame kernels + 28 jump kernels + 1 check per cycle."""
        st = self.stats or {"dns_steps": self.nsteps, "jumps": 0, "fallbacks": 0}
        return st["dns_steps"] + self.cycles * (2 + 28 + 1)

    def errors(self) -> dict:
        """Relative L2 of phi, c, rho of the hybrid's final states against plain DNS (model columns,
        all runs), and the mean relative L2 of the S2 maps."""
        self.net.sync()
        n = self.side
        out = {}
        for q, name in enumerate(("phi", "c", "rho")):
            num = sum(float(((a[q][:, :n] - b[q][:, :n]) ** 2).sum()) for a, b in zip(self.hyb.fields, self.dns.fields))
            den = sum(float((b[q][:, :n] ** 2).sum()) for b in self.dns.fields)
            out[name] = (num / den) ** 0.5
        s2 = [self.pf.s2_rel_l2(self.pf.s2_counts(b[0], b[1], n, n, 32, self.stream),
                                self.pf.s2_counts(a[0], a[1], n, n, 32, self.stream))
              for a, b in zip(self.hyb.fields, self.dns.fields)]
        out["s2"] = sum(s2) / len(s2)
        return out

    def close(self):
        self.net.close()
        self.hyb.close()
        self.dns.close()


class HybridRun:
    """Runner view of HybridPair for --workload hybrid256: one bench step is one hybrid run."""

    def __init__(self, pf, W):
        self.pair = HybridPair(pf, W)
        self.stream, self.fields = self.pair.stream, self.pair.h_fields
        self.cells, self.nsteps = self.pair.cells, self.pair.nsteps
        self.launches = self.pair.launches()
        self.config = self.pair.config

    def reset_counters(self):
        pass

    def run(self):
        self.pair.run_hybrid()
        self.launches = self.pair.launches()

    def final_diag(self):
        return self.pair.errors()

    def close(self):
        self.pair.close()


def time_hybrid_against_dns(pair, steps, warmup, flush) -> dict:
    """The hybrid and plain DNS timed in one loop: each repeat restores both batches to the seeded
    state, flushes L2, and brackets each run with CUDA events on the launch stream."""
    import torch

    arms = [(pair.reset_hybrid, pair.run_hybrid, []), (pair.reset_dns, pair.run_dns, [])]
    if pair.lead_solver is not None:  # first in each repeat: its errors use the final DNS state of the last repeat
        arms.insert(0, (pair.reset_hybrid, pair.run_lead, []))
    for _ in range(warmup):
        for reset, run, _ in arms:
            reset()
            run()
    torch.cuda.synchronize()
    for _ in range(steps):
        for reset, run, acc in arms:
            reset()
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(pair.stream)
            run()
            b.record(pair.stream)
            torch.cuda.synchronize()
            acc.append(a.elapsed_time(b) / 1e3)
            if run == pair.run_lead:
                pair.lead_errors = pair.errors()
    th, td = arms[-2][2], arms[-1][2]
    out = {"hybrid_s": statistics.median(th), "plain_dns_s": statistics.median(td), "hybrid_runs_s": th,
           "plain_dns_runs_s": td}
    if pair.lead_solver is not None:
        out["lead_s"] = statistics.median(arms[0][2])
        out["lead_runs_s"] = arms[0][2]
    return out


def hybrid_block(pair, timing: dict, peaks: dict) -> dict:
    err = pair.errors()
    jump_tf = pair.jump_flops / pair.jump_s / 1e12
    st = pair.stats
    return {"hybrid_s": timing["hybrid_s"], "plain_dns_s": timing["plain_dns_s"],
            "speedup_vs_dns": timing["plain_dns_s"] / timing["hybrid_s"],
            "timing": "median of the repeats; hybrid and plain DNS alternate in one loop, each from the seeded "
                      "state after an L2 flush, CUDA events on the launch stream",
            "jumps": st["jumps"], "dns_fallbacks": st["fallbacks"], "dns_steps": st["dns_steps"],
            "rel_l2_vs_dns": {"phi": err["phi"], "c": err["c"], "rho": err["rho"]},
            "s2_rel_l2_vs_dns": err["s2"], "jump_ms": pair.jump_s * 1e3, "jump_tflops": jump_tf,
            "jump_tensor_frac_of_bf16_peak": jump_tf / peaks["bf16_tflops"], "weights": pair.weights_desc,
            "config": pair.config, "with_dns_lead": lead_block(pair, timing)}


def lead_block(pair, timing: dict):
    """The same alternation after a DNS lead-in (the paper starts its hybrid with the solver alone),
    timed in the same loop as plain DNS: speed-up and errors against plain DNS."""
    if pair.lead_solver is None:
        return None
    e, st = pair.lead_errors, pair.lead_stats
    return {"dns_lead": pair.lead, "hybrid_s": timing["lead_s"], "speedup_vs_dns": timing["plain_dns_s"] / timing["lead_s"],
            "jumps": st["jumps"], "dns_fallbacks": st["fallbacks"], "dns_steps": st["dns_steps"],
            "rel_l2_vs_dns": {"phi": e["phi"], "c": e["c"], "rho": e["rho"]}, "s2_rel_l2_vs_dns": e["s2"],
            "phi_and_c_within_5pct": bool(e["phi"] <= 0.05 and e["c"] <= 0.05)}


def measure(R, steps, warmup, flush, local, reset_extra=None):
    """Warm-up, then `steps` whole runs, each restored to the seeded state outside the timed events and
    after an L2 flush; returns (per-run ms, clock summary, wall seconds)."""
    import torch

    init = [t.clone() for t in R.fields]

    def reset():
        for t, s in zip(R.fields, init):
            t.copy_(s)
        R.reset_counters()
        flush.zero_()

    for _ in range(warmup):
        reset()
        R.run()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, b in evs:
            reset()
            a.record(R.stream)
            R.run()
            b.record(R.stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    return [a.elapsed_time(b) for a, b in evs], clk.summary(), wall, init


def secondary_line(pf, name, args, flush, local, peaks) -> dict:
    """A short measurement of another workload (HBM-resident grids, the ensemble) for the default line."""
    W = WORKLOADS[name]
    R = {"ensemble": EnsembleRun}.get(W.get("kind"), SingleRun)(pf, W)
    run_ms, clk, _, _ = measure(R, args.steps, args.warmup, flush, local)
    R.close()
    secs = sum(run_ms) / 1e3
    per_launch = secs / (R.nsteps * args.steps)
    achieved = BYTES_PER_CELL_UPDATE * R.cells / per_launch / 1e9
    return {"workload": W["desc"], "value": R.cells * R.nsteps * args.steps / secs, "unit": UNIT,
            "ms_per_run": secs / args.steps * 1e3, "runs": args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "peak_source": peaks["source"]},
            "alu_roofline": alu_roofline(step_flops(I.default_params(**W.get("params", {}))), R.cells, per_launch),
            "clocks": clk, "config": R.config}


def run_native(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2312_05410_gb300 import build as B

    B.build()
    from paper_2312_05410_gb300 import pf

    W = WORKLOADS[args.workload]
    kind = W.get("kind")
    runners = {"ensemble": EnsembleRun, "adjoint": AdjointRun, "hybrid": HybridRun}
    R = runners.get(kind, SingleRun)(pf, W)
    stream = R.stream
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    cells, nsteps = R.cells, R.nsteps
    peaks = measured_peaks()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: K whole runs, each bracketed by events on the launch stream
    barrier()
    run_ms, clocks, wall, init = measure(R, args.steps, args.warmup, flush, local)
    barrier()
    # max time over ranks and the cell-updates of all ranks (independent replicas)
    total_s, all_units = aggregate(sum(run_ms) / 1e3, cells * nsteps * args.steps, device="cuda")
    launches = R.launches
    hybrid = None
    if kind == "hybrid":  # errors need the plain-DNS run of the same batch, timed in the same loop
        hybrid = hybrid_block(R.pair, time_hybrid_against_dns(R.pair, args.steps, 1, flush), peaks)
        final_diag = dict(hybrid["rel_l2_vs_dns"], s2=hybrid["s2_rel_l2_vs_dns"])
    else:
        final_diag = R.final_diag()

    # ---- end to end through the public API with host buffers (pinned H2D + D2H inside): single runs
    # through the C ABI's host-buffer calls (pf_load_host / pf_step / pf_store_host), the others
    # through stream-ordered copies of the caller's tensors
    via_abi = isinstance(R, SingleRun)
    if via_abi:
        host_in = [torch.from_numpy(np.ascontiguousarray(t[:, :R.sim.nx].cpu().numpy())).pin_memory() for t in init]
    else:
        host_in = [torch.from_numpy(np.ascontiguousarray(t.cpu().numpy())).pin_memory() for t in init]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for a, b in e2e_ev:
        R.reset_counters()
        flush.zero_()
        a.record(stream)
        if via_abi:
            R.sim.load_host(*host_in)
        else:
            with torch.cuda.stream(stream):
                for t, h in zip(R.fields, host_in):
                    t.copy_(h, non_blocking=True)
        R.run()
        if via_abi:
            R.sim.store_host(*host_out)
        else:
            with torch.cuda.stream(stream):
                for t, h in zip(R.fields, host_out):
                    h.copy_(t, non_blocking=True)
        b.record(stream)
    barrier()
    e2e_s, _ = aggregate(sum(a.elapsed_time(b) for a, b in e2e_ev) / 1e3, 0.0, device="cuda")
    io_bytes = sum(h.numel() * h.element_size() for h in host_in)

    R.close()
    extras = {}
    if ws == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_extras:
        # the headline grid is L2-resident: HBM-resident grids and the ensemble show the kernel against
        # the HBM roofline; the hybrid solver is the second half of the metric
        extras["secondary"] = {name: secondary_line(pf, name, args, flush, local, peaks)
                               for name in SECONDARY_WORKLOADS}
        pair = HybridPair(pf, WORKLOADS["hybrid256"])
        hybrid = hybrid_block(pair, time_hybrid_against_dns(pair, args.steps, 1, flush), peaks)
        pair.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    value = all_units / total_s
    # Dominant kernel: the fused step. Its average launch duration is bounded above by
    # the timed region per step launch (it also covers the diagnostic kernels and gaps).
    per_launch_s = total_s / (nsteps * args.steps)
    if kind == "hybrid":  # the DNS launches only: the jumps' time (measured alone) is taken out
        dns_steps = R.pair.stats["dns_steps"]
        per_launch_s = max(total_s / args.steps - R.pair.stats["jumps"] * R.pair.jump_s, 1e-9) / dns_steps
    bpc = W.get("bytes_per_cell_update", BYTES_PER_CELL_UPDATE)
    achieved = bpc * cells / per_launch_s / 1e9
    tr = NCU_TRAFFIC.get(args.workload)
    traffic = tr["bytes"] if tr and tr["src"] == kernel_source_hash() else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict({"workload": W["desc"], "per_rank": "independent replica",
                        "l2": "flushed between timed runs (256 MB write)"}, **R.config),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_source": peaks["source"], "algorithmic_bytes_per_cell_update": bpc},
        "alu_roofline": (alu_roofline(step_flops(I.default_params(**W.get("params", {}))), cells, per_launch_s)
                         if kind != "adjoint" else None),
        "gpu_launches": launches * args.steps,
        "e2e": {"value": all_units / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
                "path": "C ABI pf_load_host / pf_step / pf_store_host" if via_abi else
                        "stream-ordered copies of the caller's tensors around the public API call"},
        "clocks": clocks,
        "wall_s": wall,
        "final_diag": final_diag,
    }
    if hybrid is not None:
        line["hybrid"] = hybrid
    line.update(extras)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, budget_s=args.cpu_budget)
        line["cpu_baseline_all_cores"] = cpu_baseline(args.workload, budget_s=args.cpu_budget, all_cores=True)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def oracle_problem(W):
    """(spec, params, what) of the grid the CPU oracle samples for workload W."""
    import oracle as O

    if W.get("kind") == "ensemble":
        m = I.ensemble_members(W["n_runs"], seed=W["seed"])[0]
        return m["spec"], O.with_dt(I.default_params(v_mag=m["v_mag"])), "run 0 of the ensemble"
    if W.get("kind") == "adjoint":
        return W["spec"], O.with_dt(I.default_params(**W["params"])), "forward steps only, on the"
    if W.get("kind") == "hybrid":
        m = I.hybrid_members(W["n_runs"], W["side"], seed=W["seed"])[0]
        return m["spec"], O.with_dt(I.default_params(v_mag=m["v_mag"])), "plain DNS of run 0 of the hybrid batch, the"
    return W["spec"], O.with_dt(I.default_params(**W["params"])), "the"


def cpu_baseline(workload: str, budget_s: float = 15.0, steps: int | None = None, all_cores: bool = False) -> dict:
    """Time the FP64 oracle on a bounded sample of the workload: as it stands (single thread), or its
    OpenMP build over all host cores (the same loops, identical results)."""
    import oracle as O

    W = WORKLOADS[workload]
    spec, p, what = oracle_problem(W)
    state = I.film_state(spec, p)
    step = O.step_all_cores if all_cores else O.step
    step(p, *state, 1)  # load and warm the library
    if steps is None:
        t = time.perf_counter()
        step(p, *state, 5)
        per = (time.perf_counter() - t) / 5
        steps = max(1, min(W["steps"], int(budget_s / per)))
    t = time.perf_counter()
    step(p, *state, steps)
    dt = time.perf_counter() - t
    host = os.cpu_count() or 1
    cores = int(os.environ.get("OMP_NUM_THREADS", host)) if all_cores else 1
    how = f"FP64, OpenMP over {cores} threads" if all_cores else "FP64, single thread"
    return {"value": spec.nx * spec.ny * steps / dt, "unit": UNIT, "cores": cores, "host_cores": host,
            "kind": "oracle",
            "sample": f"{what} {spec.nx}x{spec.ny} grid, first {steps} of the {W['steps']} steps, {how}",
            "seconds": dt}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    W = WORKLOADS[args.workload]
    import oracle as O

    spec, p, _ = oracle_problem(W)
    state = I.film_state(spec, p)
    # size one sample step so that warmup + timed steps take about a minute in total
    t = time.perf_counter()
    O.step(p, *state, 3)
    per = (time.perf_counter() - t) / 3
    k = max(1, int(60.0 / (args.steps + args.warmup) / per))
    k = min(k, W["steps"])
    for _ in range(args.warmup):
        O.step(p, *state, k)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        O.step(p, *state, k)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = spec.nx * spec.ny * k * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": W["desc"], "nx": spec.nx, "ny": spec.ny, "timesteps_per_sample_step": k},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{spec.nx}x{spec.ny} grid, {k} of the {W['steps']} steps per bench step, "
                                   "FP64 single-thread oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the secondary workloads and the hybrid block")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--unet-weights", default="",
                    help="hybrid: weights .npz written by paper_2312_05410_gb300.train_unet (default: the committed "
                         "weights under paper_2312_05410_gb300/weights/)")
    ap.add_argument("--timesteps", type=int, default=0,
                    help="override the workload's time steps per run (short runs for profiling only)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.timesteps > 0:
        WORKLOADS[args.workload] = dict(WORKLOADS[args.workload], steps=args.timesteps)
    if args.unet_weights:
        WORKLOADS["hybrid256"] = dict(WORKLOADS["hybrid256"], unet_weights=args.unet_weights)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
