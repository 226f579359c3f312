#!/usr/bin/env python
"""Throughput benchmark of the FP64 symplectic tracker on one GB300.

Workload: the LHC-scale synthetic ring (20,000 thin elements: 6,800 exact
drifts, 6,800 order-10 thin multipoles with 1e-4 Gaussian field errors,
8 RF cavities, 6,392 circular apertures of r = 20 mm) with 999,990 protons at
450 GeV on the polar dynamic-aperture grid (22,222 radii in 0-20 sigma x 9
angles x 5 momentum offsets).  A step tracks the whole ensemble for
``--turns-per-step`` turns, continuing from the previous step (loss turns and
losses accumulate as in a long run).  The metric counts particle-element
passes actually made (lost particles stop counting where they were lost).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
on bounded samples of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle·element·turns/s FP64 (1 GB300); DA-scan wall time surrogate vs plain"
UNIT = "particle*element*turns/s"
WORKLOAD = ("LHC-scale synthetic ring, 20,000 thin elements (6800 drifts, 6800 order-10 multipoles "
            "with 1e-4 field errors, 8 RF cavities, 6392 circular apertures r=20 mm), 999,990 protons "
            "at 450 GeV on a polar DA grid (22,222 r in 0-20 sigma x 9 angles x 5 delta offsets), FP64")
# FP64 peak from unit counts and clocks: 2 FP64 fma lanes per SM per clock
# (4 flop/clk/SM), 152 SMs, 2070 MHz maximum SM clock -> 1.2586 TFLOP/s.
FP64_FLOP_PER_CLK_SM = 4.0
N_SM = 152
SM_MAX_MHZ = 2070.0
NOMINAL_FP64 = FP64_FLOP_PER_CLK_SM * N_SM * SM_MAX_MHZ * 1e6
# DRAM bytes (read + write) of a tracking launch per particle and turn: ncu
# capture of the current kernel on a 400,000-particle subset of this workload
# over one turn (34,656,512 B read, 0 B written; all 152 SMs busy).  The
# per-launch traffic is the particle state, so it scales with the particle
# count.
TRACK_DRAM_BYTES_PER_PARTICLE_TURN = 34656512.0 / 400000.0


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------
# clocks sampled with nvidia-smi during the timed region
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                c = [x.strip() for x in line.split(",")]
                if len(c) >= 9:
                    rows.append(c)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(rows), "reasons": reasons}


def gpu_id_for_smi(local_rank: int) -> str | None:
    import torch
    try:
        u = str(torch.cuda.get_device_properties(local_rank).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        if vis:
            return vis.split(",")[local_rank]
        return str(local_rank)


# ----------------------------------------------------------------------------
# CPU oracle timing (worker processes started with spawn)
def _oracle_worker(args):
    seed, idx, turns = args
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2310_00317_gb300 import inputs as I
    el, ref = I.lhc_ring(seed=seed)
    g = I.da_grid(el, ref)
    p = I.subset(g, idx)
    oracle.build()
    t0 = time.perf_counter()
    o = oracle.track(el, ref, p, turns)
    dt = time.perf_counter() - t0
    n_el = len(el)
    st, at, ae = o["state"], o["at_turn"].astype(np.int64), o["at_element"].astype(np.int64)
    units = int((st == 1).sum()) * turns * n_el + int((at[st != 1] * n_el + ae[st != 1] + 1).sum())
    return units, dt


def oracle_sample(seed: int, n_per_proc: int, turns: int, procs: int, rng_seed: int):
    rng = np.random.default_rng(rng_seed)
    N = 22222 * 45
    jobs = [(seed, np.sort(rng.choice(N, n_per_proc, replace=False)), turns) for _ in range(procs)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(procs) as pool:
        res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    units = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return units, busy, wall


def cpu_baseline(seed, n_per_proc, turns):
    procs = os.cpu_count() or 1
    units, busy, wall = oracle_sample(seed, n_per_proc, turns, procs, 12345)
    return {"value": units / busy, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": ("%d DA-grid particles (random, %d per process) x %d turns x 20,000 elements, "
                       "single-threaded oracle in %d processes; %.3g particle-element passes in %.1f s"
                       % (n_per_proc * procs, n_per_proc, turns, procs, units, busy))}


# ----------------------------------------------------------------------------
# Secondary measurements (N = 1 only).
def _passes(before, after, start, T, n_el):
    alive0 = before == 1
    st, at, ae = after["state"], after["at_turn"].astype(np.int64), after["at_element"].astype(np.int64)
    surv = alive0 & (st == 1)
    lost = alive0 & (st != 1)
    return int(surv.sum()) * T * n_el + int(((at[lost] - start) * n_el + ae[lost] + 1).sum())


def measure_batched(T=20, steps=5, plain_steps=1):
    """64 error seeds of the LHC-scale ring, uneven particle counts
    round(10^U(3,5)), one persistent launch per segment: `steps` x T turns
    replayed from a CUDA graph (100 turns by default, so that seeds losing
    particles at different rates show in the (seed, tile) queue's balance),
    then `plain_steps` x T turns without the graph."""
    import torch
    from paper_2310_00317_gb300 import inputs as I
    from paper_2310_00317_gb300 import xtgb
    counts = I.batched_seed_counts(64)
    el0, ref = I.lhc_ring(seed=I.BASE_SEED)
    optics = I.design_optics(el0, ref)  # errors are orders >= 2: the linear optics are shared
    trs, ps = [], []
    for i, n in enumerate(counts):
        scales, _ = I.seed_error_scales(i)
        el, _ = I.lhc_ring(seed=I.BASE_SEED + 100 + i, error_scales=scales)
        p = I.polar_sample(el, ref, int(n), seed=I.BASE_SEED + 200 + i, optics=optics)
        trs.append(xtgb.Tracker(el, ref))
        ps.append(xtgb.Particles.from_numpy(I.subset(p, np.arange(int(n)))))
    n_el = el0.shape[0]
    out = {"seeds": 64, "particles": int(counts.sum()), "count_min": int(counts.min()),
           "count_max": int(counts.max()), "n_elements": int(n_el), "turns_per_step": T}
    # block, lattice-chunk and segment sizes from the autotuner on a probe of
    # 65,536 particles of seed 0 over 2 turns; the batched launch takes tracker
    # 0's options for every seed
    scales0, _ = I.seed_error_scales(0)
    el_p, _ = I.lhc_ring(seed=I.BASE_SEED + 100, error_scales=scales0)
    pr = I.polar_sample(el_p, ref, 65536, seed=I.BASE_SEED + 300, optics=optics)
    probe = xtgb.Particles.from_numpy(I.subset(pr, np.arange(65536)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    opt = trs[0].autotune(probe, 2)
    torch.cuda.synchronize()
    out["autotune"] = {"block": int(opt["block"]), "chunk_bytes": int(opt["chunk_bytes"]),
                       "segment_turns": int(opt["segment_turns"]), "seconds": time.perf_counter() - t0,
                       "probe": "65,536 particles of seed 0, 2 turns, 3 blocks x 4 chunks x 3 segments"}
    turn = 0
    xtgb.track_batched(trs, ps, T, turn, graph=True)  # capture + warm
    turn += T
    for graph in (True, False):
        ms, units = 0.0, 0
        n_steps = steps if graph else plain_steps
        for _ in range(n_steps):
            before = [P.t["state"].cpu().numpy() for P in ps]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            xtgb.track_batched(trs, ps, T, turn, graph=graph)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            for b, P in zip(before, ps):
                units += _passes(b, {k: P.t[k].cpu().numpy() for k in ("state", "at_turn", "at_element")},
                                 turn, T, n_el)
            turn += T
        out["graph" if graph else "no_graph"] = {"value": units / (ms * 1e-3), "ms_per_step": ms / n_steps,
                                                 "turns": [turn - n_steps * T, turn],
                                                 "alive_at_end": int(sum(int((P.t["state"] == 1).sum()) for P in ps))}
    if xtgb.batched_sync_status(trs, ps) != xtgb.XT_OK:
        raise RuntimeError("batched tracking reported an error status")
    xtgb.batched_release()
    for t in trs:
        t.close()
    out["unit"] = UNIT
    return out


def measure_steady(turns=200, window=50, n=0):
    """The headline workload from turn 0 through the DA-boundary losses: a
    fresh copy of the full grid tracked `turns` turns in windows of `window`
    turns (one xt_track call each, the tracker's own segmentation and
    compaction inside), the rate, alive count and FP64 fraction per window."""
    import torch
    from paper_2310_00317_gb300 import inputs as I
    from paper_2310_00317_gb300 import xtgb
    el, ref = I.lhc_ring(seed=I.BASE_SEED)
    n_el = el.shape[0]
    grid = I.da_grid(el, ref)
    N = grid["x"].shape[0]
    sel = np.arange(N) if n <= 0 or n >= N else np.unique(np.linspace(0, N - 1, n).astype(np.int64))
    tr = xtgb.Tracker(el, ref)
    fprefix = np.cumsum(tr.element_flops().astype(np.float64))
    P = xtgb.Particles.from_numpy(I.subset(grid, sel))
    out = {"workload": WORKLOAD if sel.size == N else WORKLOAD + " (evenly spaced subset of %d)" % sel.size,
           "turns": turns, "window_turns": window, "windows": []}
    tr.set_profiling(True)
    tr.kernel_time()
    ms_all, units_all, flops_all = 0.0, 0, 0.0
    for start in range(0, turns, window):
        T = min(window, turns - start)
        before = P.t["state"].cpu().numpy()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        tr.track(P, T, start)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        kms, _ = tr.kernel_time()
        after = {k: P.t[k].cpu().numpy() for k in ("state", "at_turn", "at_element")}
        alive0 = before == 1
        surv = alive0 & (after["state"] == 1)
        lost = alive0 & (after["state"] != 1)
        at, ae = after["at_turn"].astype(np.int64), after["at_element"].astype(np.int64)
        units = int(surv.sum()) * T * n_el + int(((at[lost] - start) * n_el + ae[lost] + 1).sum())
        flops = float(surv.sum()) * T * fprefix[-1] + float(((at[lost] - start) * fprefix[-1] + fprefix[ae[lost]]).sum())
        out["windows"].append({"turns": [start, start + T], "alive_at_end": int(surv.sum()),
                               "value": units / (ms * 1e-3), "frac": flops / (kms * 1e-3) / NOMINAL_FP64,
                               "ms": ms})
        ms_all += ms
        units_all += units
        flops_all += flops
    tr.set_profiling(False)
    if tr.sync_status() != xtgb.XT_OK:
        raise RuntimeError("tracking reported an error status")
    tr.close()
    out.update(value=units_all / (ms_all * 1e-3), unit=UNIT, seconds=ms_all * 1e-3,
               roofline={"bound": "alu", "achieved": flops_all / (ms_all * 1e-3) / 1e12, "peak": NOMINAL_FP64 / 1e12,
                         "unit": "TFLOP/s", "frac": flops_all / (ms_all * 1e-3) / NOMINAL_FP64,
                         "note": "achieved over the windows' whole event-timed duration, compaction included"})
    return out


def measure_fodo(n=1000000, turns=300):
    """A short lattice with many particles: the FODO-10 ring (51 elements)
    with n matched protons.  The tracker's own segmentation (about 1e8
    particle-element passes per launch) reloads the particle state every few
    turns here; the rate shows what that costs next to the 20,000-element
    ring, where a launch covers one turn."""
    import torch
    from paper_2310_00317_gb300 import inputs as I
    from paper_2310_00317_gb300 import xtgb
    el, ref = I.fodo10()
    p = I.matched_gaussian(el, ref, n, 2.5e-6, 3e-4, seed=I.BASE_SEED + 9)
    tr = xtgb.Tracker(el, ref)
    fl = tr.element_flops().astype(np.float64)
    P = xtgb.Particles.from_numpy(p)
    tr.track(P, 3, 0)
    before = P.t["state"].cpu().numpy()
    tr.set_profiling(True)
    tr.kernel_time()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    tr.track(P, turns, 3)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kms, launches = tr.kernel_time()
    tr.set_profiling(False)
    units = _passes(before, {k: P.t[k].cpu().numpy() for k in ("state", "at_turn", "at_element")}, 3, turns,
                    el.shape[0])
    per_pass = float(fl.sum()) / el.shape[0]
    tr.close()
    return {"workload": "FODO-10 ring (51 elements), %d matched protons at 450 GeV" % n, "turns": turns,
            "value": units / (ms * 1e-3), "unit": UNIT, "tracking_launches": launches,
            "turns_per_launch": turns / max(launches, 1), "kernel_ms": kms, "event_ms": ms,
            "roofline": {"bound": "alu", "achieved": units * per_pass / (ms * 1e-3) / 1e12,
                         "peak": NOMINAL_FP64 / 1e12, "unit": "TFLOP/s",
                         "frac": units * per_pass / (ms * 1e-3) / NOMINAL_FP64,
                         "algorithmic_flops_per_pass": per_pass}}


def measure_refinement(tr, host, ds=0.01, n_angles=128, reps=5):
    """Loss-location refinement of the particles the headline run lost at the
    LHC-scale ring's apertures (state 0): CUDA-event time per call."""
    import torch
    from paper_2310_00317_gb300 import inputs as I
    from paper_2310_00317_gb300 import xtgb
    lost = np.flatnonzero(host["state"] == 0)
    if lost.size == 0:
        return {"lost": 0}
    P = xtgb.Particles.from_numpy(I.subset({k: host[k] for k in xtgb.ALL_FIELDS}, lost))
    s = tr.refine_losses(P, ds, n_angles)  # builds the tables
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        s = tr.refine_losses(P, ds, n_angles)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    sv = s.cpu().numpy()
    return {"lost": int(lost.size), "refined": int(np.sum(~np.isnan(sv))), "ds_m": ds, "n_angles": n_angles,
            "ms": ms, "particles_per_s": lost.size / (ms * 1e-3),
            "workload": "particles lost at the 20 mm circular apertures of the LHC-scale ring in the headline run"}


def measure_beambeam(n=1000000, n_lens=1000, turns=2):
    """Throughput of the 4D beam-beam lens: a line of flat lenses (two w(z)
    evaluations per pass), CUDA-event time, FP64 fraction from the library's
    flop count per lens."""
    import torch
    from paper_2310_00317_gb300 import inputs as I
    from paper_2310_00317_gb300 import xtgb
    ref = I.proton_reference(450e9)
    lens = I.beambeam4d(1.5e11, 1.0, 0.8e-3, 0.25e-3)
    el = I.table([lens] * n_lens)
    rng = np.random.default_rng(I.BASE_SEED + 11)
    p = I.make_particles(ref, rng.normal(0, 1e-3, n), rng.normal(0, 1e-6, n), rng.normal(0, 0.4e-3, n),
                         rng.normal(0, 1e-6, n), np.zeros(n), np.zeros(n))
    tr = xtgb.Tracker(el, ref)
    P = xtgb.Particles.from_numpy(p)
    tr.track(P, 1)
    tr.set_profiling(True)
    tr.kernel_time()
    tr.track(P, turns, 1)
    ms, nl = tr.kernel_time()
    per_pass = float(tr.element_flops().sum()) / n_lens
    alive = int((P.t["state"] == 1).sum())
    tr.close()
    passes = alive * n_lens * turns
    achieved = passes * per_pass / (ms * 1e-3)
    return {"workload": "%d particles through %d flat 4D beam-beam lenses (sigma 0.8 x 0.25 mm), %d turns"
                        % (n, n_lens, turns),
            "value": passes / (ms * 1e-3), "unit": "particle*lens passes/s", "kernel_ms": ms,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": NOMINAL_FP64 / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / NOMINAL_FP64, "algorithmic_flops_per_pass": per_pass}}


def measure_thick(n=1000000, turns=4):
    """Throughput of the thick elements: a small ring (bending radius 1.5 m,
    50 cells) of full-model sector bends between non-linear edges, expanded
    combined-function bends between linear edges, thick quadrupoles,
    sextupoles, drifts and apertures; CUDA-event time of the tracking
    kernel, FP64 fraction from the library's flop counts."""
    from paper_2310_00317_gb300 import inputs as I
    from paper_2310_00317_gb300 import xtgb
    ref = I.proton_reference(450e9)
    h = 1 / 1.5
    rows = []
    th = h * 0.9
    for c in range(50):
        rows += [I.quadrupole(0.8, 0.3), I.drift(0.3), I.dipedge(h, th / 2, hgap=0.02, fint=0.5, nonlinear=True),
                 I.bend(h, h, 0.9, full=True), I.dipedge(h, th / 2, hgap=0.02, fint=0.5, nonlinear=True, exit=True),
                 I.drift(0.3), I.multipole(knl=[0.0, 0.0, 0.5]), I.quadrupole(-0.8, 0.3), I.drift(0.3),
                 I.dipedge(h, 0.05), I.bend(h, h, 0.9, k1=-0.05), I.dipedge(h, 0.05), I.drift(0.3),
                 I.aperture(0.02)]
    el = I.table(rows)
    rng = np.random.default_rng(I.BASE_SEED + 13)
    p = I.make_particles(ref, rng.normal(0, 1e-3, n), rng.normal(0, 5e-4, n), rng.normal(0, 1e-3, n),
                         rng.normal(0, 5e-4, n), np.zeros(n), rng.normal(0, 5e-4, n))
    tr = xtgb.Tracker(el, ref)
    P = xtgb.Particles.from_numpy(p)
    tr.track(P, 1)
    tr.set_profiling(True)
    tr.kernel_time()
    alive0 = int((P.t["state"] == 1).sum())
    tr.track(P, turns, 1)
    ms, nl = tr.kernel_time()
    alive1 = int((P.t["state"] == 1).sum())
    per_turn = float(tr.element_flops().sum())
    tr.close()
    units = 0.5 * (alive0 + alive1) * len(rows) * turns
    achieved = 0.5 * (alive0 + alive1) * per_turn * turns / (ms * 1e-3)
    return {"workload": "%d particles, %d turns of a %d-row ring of full thick bends between non-linear edges, "
                        "expanded bends between linear edges, thick quadrupoles, sextupoles and drifts"
                        % (n, turns, len(rows)),
            "value": units / (ms * 1e-3), "unit": "particle*element*turns/s", "kernel_ms": ms,
            "alive": [alive0, alive1],
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": NOMINAL_FP64 / 1e12, "unit": "TFLOP/s",
                         "frac": achieved / NOMINAL_FP64, "algorithmic_flops_per_turn": per_turn}}


def measure_twiss():
    """Wall time of the lattice functions along the LHC-scale ring (closed
    orbit, one-turn Jacobian, eigenvectors carried along 20,000 rows by the
    monitor) and of the energy-loss compensation loop on the 45.6 GeV lepton
    ring with its RF in 4 stations (each pass one monitor launch)."""
    import time
    from paper_2310_00317_gb300 import inputs as I
    from paper_2310_00317_gb300 import twiss as T
    el, ref = I.lhc_ring(seed=I.BASE_SEED)
    T.twiss_along(el, ref)  # warm-up (first-use costs)
    t0 = time.perf_counter()
    tw = T.twiss_along(el, ref)
    t_tw = time.perf_counter() - t0
    rows, lref, info = I.lepton_ring(rf_every=50)
    t0 = time.perf_counter()
    c = T.compensate_energy_loss(I.table(rows), lref)
    t_c = time.perf_counter() - t0
    return {"twiss_along": {"workload": "LHC-scale ring, %d rows" % el.shape[0], "seconds": t_tw,
                            "qx": tw["qx"], "qy": tw["qy"], "betx_max": float(np.max(tw["betx"]))},
            "energy_loss_compensation": {"workload": "45.6 GeV lepton ring, %d rows, 4 RF stations" % len(rows),
                                         "seconds": t_c, "iterations": c["iterations"],
                                         "converged": bool(c["converged"]),
                                         "energy_loss_eV": c["energy_loss"], "design_U0_eV": info["U0"],
                                         "max_abs_x_m": float(np.max(np.abs(c["x"])))}}


def measure_lepton(n=200000, turns=10):
    """Lepton ring (10,000 elements) with mean radiation + quantum excitation."""
    import torch
    from paper_2310_00317_gb300 import inputs as I
    from paper_2310_00317_gb300 import xtgb
    el, ref, _ = I.lepton_ring()
    p = I.matched_gaussian(el, ref, n, 0.0, 1.06e-3, seed=5, emit_x=2 * 3.9e-8, emit_y=2 * 3.9e-10)
    tr = xtgb.Tracker(el, ref, radiation=xtgb.RAD_QUANTUM, seed=1)
    P = xtgb.Particles.from_numpy(p)
    # block, chunk and segment from the autotuner on these particles (2 turns)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    opt = tr.autotune(P, 2)
    torch.cuda.synchronize()
    tune = {"block": int(opt["block"]), "chunk_bytes": int(opt["chunk_bytes"]),
            "segment_turns": int(opt["segment_turns"]), "seconds": time.perf_counter() - t0}
    tr.track(P, 2, 0)
    before = P.t["state"].cpu().numpy()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    tr.track(P, turns, 2)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    units = _passes(before, {k: P.t[k].cpu().numpy() for k in ("state", "at_turn", "at_element")}, 2, turns,
                    el.shape[0])
    # algorithmic FP64 flops per pass with radiation (the survivors traverse every row)
    fl = tr.element_flops()
    per_pass = float(fl.sum()) / el.shape[0]
    tr.close()
    achieved = units * per_pass / (ms * 1e-3)
    return {"workload": "lepton ring 10,000 elements, 45.6 GeV, mean + quantum radiation, %d particles" % n,
            "turns": turns, "value": units / (ms * 1e-3), "unit": UNIT, "autotune": tune,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": NOMINAL_FP64 / 1e12,
                         "unit": "TFLOP/s", "frac": achieved / NOMINAL_FP64,
                         "algorithmic_flops_per_pass": per_pass,
                         "note": "quantum emission adds integer Philox4x64 rounds, a Poisson loop and table "
                                 "look-ups that count no FP64 flops"}}


def measure_lepton_equilibrium(n=200000, turns=2000, every=10, tail=500):
    """The lepton ring with mean radiation and quantum excitation at its
    stated size: 200,000 electrons started at twice the equilibrium
    emittance in both planes and twice the longitudinal one, tracked 2000
    turns.  eps_x, eps_y and sigma_delta are read every `every` turns at
    element 0 (betatron parts about the dispersion), averaged over the last
    `tail` turns and compared with the synchrotron integrals
    eps_x = C_q gamma^2 I5 / (J_x I2) and sigma_delta^2 = C_q gamma^2 I3 / (J_z I2)
    (I2, I3, I5 from the ring's dipole slices and the lattice functions that
    the twiss module computes on the GPU, J_k = 4 alpha_k / sum alpha from
    the one-turn damping decrements).  The damping times come from fits of
    the decays against 1/alpha_k."""
    import torch
    from paper_2310_00317_gb300 import inputs as I
    from paper_2310_00317_gb300 import twiss as TW
    from paper_2310_00317_gb300 import xtgb
    el, ref, info = I.lepton_ring()
    m0, _, p0c = ref
    gamma0 = math.sqrt(p0c * p0c + m0 * m0) / m0
    t0 = time.perf_counter()
    tw = TW.twiss_along(el, ref, dim=4)
    dmp = TW.damping(el, ref)
    I2 = I3 = I5 = 0.0
    for i, r in enumerate(el):
        if int(r["type"]) != I.MULTIPOLE or r["p"][23] <= 0.0 or r["p"][0] == 0.0:
            continue
        L = float(r["p"][23])
        h = float(r["p"][0]) / L
        b, a, d = tw["betx"][i + 1], tw["alfx"][i + 1], tw["dx"][i + 1]
        dp = 0.5 * (tw["dpx"][i] + tw["dpx"][i + 1])  # the slope jumps across the thin slice
        H = ((1 + a * a) / b) * d * d + 2 * a * d * dp + b * dp * dp
        I2 += h * h * L
        I3 += abs(h) ** 3 * L
        I5 += H * abs(h) ** 3 * L
    alpha = np.asarray(dmp["alpha"])
    J = 4 * alpha / alpha.sum()
    CQ = 55.0 / (32.0 * math.sqrt(3.0)) * 3.8615926796e-13  # hbar / (m_e c) in m
    eps_th = CQ * gamma0 ** 2 * I5 / (J[0] * I2)
    sd_th = math.sqrt(CQ * gamma0 ** 2 * I3 / (J[2] * I2))
    optics_s = time.perf_counter() - t0
    bx, ax, dx, dpx = tw["betx"][0], tw["alfx"][0], tw["dx"][0], tw["dpx"][0]
    p = I.matched_gaussian(el, ref, n, 0.0, math.sqrt(2.0) * sd_th, seed=2025, emit_x=2 * eps_th,
                           emit_y=2 * eps_th)
    tr = xtgb.Tracker(el, ref, radiation=xtgb.RAD_QUANTUM, seed=77)
    P = xtgb.Particles.from_numpy(p)

    def emit(u, pu, d, alive):
        u, pu = u[alive], pu[alive]
        ub = u - u.mean()
        pb = pu - pu.mean()
        return float(torch.sqrt((ub * ub).mean() * (pb * pb).mean() - (ub * pb).mean() ** 2))

    hist = []
    ms_all = 0.0
    for start in range(0, turns, every):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tr.track(P, every, start)
        e1.record()
        torch.cuda.synchronize()
        ms_all += e0.elapsed_time(e1)
        alive = P.t["state"] == 1
        d = P.t["delta"]
        ex = emit(P.t["x"] - dx * d, P.t["px"] - dpx * d, d, alive)
        ey = emit(P.t["y"], P.t["py"], d, alive)
        hist.append((start + every, ex, ey, float(d[alive].std()), int(alive.sum())))
    if tr.sync_status() != xtgb.XT_OK:
        raise RuntimeError("tracking reported an error status")
    tr.close()
    h = np.array(hist)
    last = h[:, 0] > turns - tail
    ex_m, ey_m, sd_m = h[last, 1].mean(), h[last, 2].mean(), h[last, 3].mean()
    # damping times: eps - eps_end decays as exp(-2 t / tau) (amplitude decrement alpha = 1/tau)
    early = h[:, 0] <= 600

    def tau_fit(col, floor):
        y = h[early, col] - floor
        ok = y > 0
        return -2.0 / np.polyfit(h[early, 0][ok], np.log(y[ok]), 1)[0]

    tau_x = tau_fit(1, ex_m)
    tau_y = tau_fit(2, 0.0)
    # the longitudinal emittance goes as sigma_delta^2: its excess over the
    # equilibrium decays as exp(-2 t / tau_z); fitted while it is well above
    # the noise of the second moment (the first 300 turns)
    zz = (h[:, 0] <= 300) & (h[:, 3] ** 2 > sd_m ** 2)
    tau_z = -2.0 / np.polyfit(h[zz, 0], np.log(h[zz, 3] ** 2 - sd_m ** 2), 1)[0]
    units = n * turns * el.shape[0]
    return {"workload": "lepton ring 10,000 elements, 45.6 GeV electrons, mean radiation + quantum excitation, "
                        "%d particles from 2x the equilibrium emittances, %d turns" % (n, turns),
            "eps_x": {"tracked": ex_m, "integrals": eps_th, "rel": ex_m / eps_th - 1,
                      "stat_error": math.sqrt(2.0 / n)},
            "sigma_delta": {"tracked": sd_m, "integrals": sd_th, "rel": sd_m / sd_th - 1,
                            "stat_error": math.sqrt(1.0 / (2 * n))},
            "eps_y_tracked": ey_m,
            "damping_turns": {"x": {"fit": tau_x, "eigen": 1 / alpha[0]}, "y": {"fit": tau_y, "eigen": 1 / alpha[1]},
                              "z": {"fit": tau_z, "eigen": 1 / alpha[2]}},
            "I2": I2, "I3": I3, "I5": I5, "J": J.tolist(), "optics_seconds": optics_s,
            "tracking_seconds": ms_all * 1e-3, "value": units / (ms_all * 1e-3), "unit": UNIT,
            "history_every_100_turns": [[int(r[0]), r[1], r[2], r[3]] for r in h[9::10]]}


def measure_da_scan(n_turns=300):
    """Surrogate-guided DA scan against the plain FP64 scan at equal turns."""
    from paper_2310_00317_gb300 import surrogate as S
    r = S.da_study(n_turns=n_turns)
    out = {k: v for k, v in r.items() if k not in ("loss_history",)}
    out["workload"] = ("family of 48 error seeds of a reduced LHC-scale ring (20 cells, 2,000 elements, errors x1.5 "
                       "x per-seed scales): random-amplitude labels of every seed by the batched tracker, band "
                       "limits from plain scans of 3 validation seeds of the family on 2,222 radii, 4 test seeds "
                       "of the family each scanned on 22,222 radii x 45 angles (999,990 points), %d turns"
                       % n_turns)
    return out


def measure_da_scan_full(n_turns=100, base_mult=1.0, total_labels=5_000_000, n_test=4):
    """The surrogate-guided DA scan on the LHC-scale ring itself: a family of
    64 error seeds of the 20,000-element ring, total_labels labels from one
    batched launch per segment, the full 999,990-point grid of the first
    n_test of the test seeds 60, 13, 30, 45."""
    from paper_2310_00317_gb300 import surrogate as S
    test_seeds = (60, 13, 30, 45)[:n_test]
    r = S.da_study_full(n_turns=n_turns, base_mult=base_mult, total_labels=int(total_labels), test_seeds=test_seeds)
    out = {k: v for k, v in r.items() if k not in ("loss_history",)}
    out["workload"] = ("family of 64 error seeds of the LHC-scale ring (200 cells, 20,000 elements, orders 2..6 "
                       "scaled log-uniformly in [0.5, 2] x %g): %d random-amplitude labels (momentum deviations "
                       "N(0, 3e-4)) tracked by the batched tracker, band limits from plain scans of 3 validation "
                       "seeds on 2,222 radii, %d test seeds each scanned on the full grid of 22,222 radii x 9 "
                       "angles x 5 momentum offsets (999,990 points), %d turns"
                       % (base_mult, r["n_train"], len(test_seeds), n_turns))
    return out


# ----------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    procs = os.cpu_count() or 1
    steps, warm = args.steps, args.warmup
    per_proc = args.ref_particles
    times, units_all = [], 0
    for s in range(warm + steps):
        units, busy, wall = oracle_sample(20231001, per_proc, args.turns_per_step, procs, 1000 + s)
        if s >= warm:
            times.append(busy)
            units_all += units
    total = sum(times)
    value = units_all / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * total / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + "; each step a random sample of %d particles x %d turns"
                   % (per_proc * procs, args.turns_per_step),
                   "turns_per_step": args.turns_per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": "%d random DA-grid particles x %d turns per step, %d processes"
                                   % (per_proc * procs, args.turns_per_step, procs)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2310_00317_gb300 import inputs as I
    from paper_2310_00317_gb300 import xtgb

    from paper_2310_00317_gb300 import sharding
    # weak scaling: each rank tracks its own error seed of the ring
    seed = sharding.rank_seed(I.BASE_SEED, rank)
    el, ref = I.lhc_ring(seed=seed)
    n_el = len(el)
    grid = I.da_grid(el, ref)
    N = grid["x"].shape[0]
    sel = np.arange(N) if args.particles <= 0 or args.particles >= N else \
        np.unique(np.linspace(0, N - 1, args.particles).astype(np.int64))
    p0 = I.subset(grid, sel)
    n = p0["x"].shape[0]
    T = args.turns_per_step

    tr = xtgb.Tracker(el, ref)
    flops_row = tr.element_flops().astype(np.float64)
    fprefix = np.cumsum(flops_row)
    f_turn = float(fprefix[-1])
    P = xtgb.Particles.from_numpy(p0, device=dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    peak_meas = xtgb.fp64_peak()

    def counts(before, after, start):
        st0 = before
        st, at, ae = after["state"], after["at_turn"].astype(np.int64), after["at_element"].astype(np.int64)
        alive0 = st0 == 1
        surv = alive0 & (st == 1)
        lost = alive0 & (st != 1)
        units = int(surv.sum()) * T * n_el + int(((at[lost] - start) * n_el + ae[lost] + 1).sum())
        flops = float(surv.sum()) * T * f_turn + float(((at[lost] - start) * f_turn + fprefix[ae[lost]]).sum())
        return units, flops

    def snap():
        return {k: P.t[k].cpu().numpy() for k in ("state", "at_turn", "at_element")}

    turn = 0
    for _ in range(args.warmup):
        flush.zero_()
        tr.track(P, T, turn)
        turn += T
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(gpu_id_for_smi(local))
    tr.set_profiling(True)
    tr.kernel_time()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    units_all = 0
    flops_all = 0.0
    step_ms = []
    wall0 = time.perf_counter()
    for s in range(args.steps):
        before = snap()["state"]
        flush.zero_()
        ev[s][0].record(stream)
        tr.track(P, T, turn)
        ev[s][1].record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev[s][0].elapsed_time(ev[s][1]))
        u, f = counts(before, snap(), turn)
        units_all += u
        flops_all += f
        turn += T
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    kern_ms, kern_launches = tr.kernel_time()
    tr.set_profiling(False)
    clocks = sampler.stop()
    if tr.sync_status() != xtgb.XT_OK:
        raise RuntimeError("tracking reported an error status")
    total_ms = float(sum(step_ms))
    units_job, total_ms_job = sharding.reduce_throughput(units_all, total_ms, device=dev)
    value = units_job / (total_ms_job * 1e-3)
    achieved = flops_all / (kern_ms * 1e-3)

    # end to end through the public API with host buffers (pinned), copies
    # inside the timed region
    host = {}
    for k in xtgb.ALL_FIELDS:
        v = P.t[k].cpu()
        host[k] = v.pin_memory().numpy()
    H = xtgb.HostParticles(host, copy=False)
    h2d = n * (9 * 8 + 3 * 4 + 8)
    d2h = n * (9 * 8 + 3 * 4)
    e2e_steps = args.steps
    e_units = 0
    e_time = 0.0
    for s in range(e2e_steps):
        before = H.a["state"].copy()
        t0 = time.perf_counter()
        tr.track_host(H, T, turn)
        e_time += time.perf_counter() - t0
        u, _ = counts(before, H.a, turn)
        e_units += u
        turn += T
    e2e_value = e_units / e_time

    if ws > 1:
        torch.distributed.barrier()
    if rank != 0:
        return 0

    extras = {}
    if ws == 1 and not args.no_extras:
        extras["steady_state"] = measure_steady()
        extras["loss_refinement"] = measure_refinement(tr, H.a)
        extras["beambeam_lens"] = measure_beambeam()
        extras["thick_elements"] = measure_thick()
        extras["twiss"] = measure_twiss()
        extras["batched_seeds"] = measure_batched()
        extras["lepton_quantum"] = measure_lepton()
        # the LHC-scale ring itself with 1e6 labels (5e6 in --only da_scan_full:
        # 5 more minutes of labels for a narrower band)
        extras["da_scan"] = measure_da_scan_full(n_turns=100, total_labels=1_000_000, n_test=4)
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(seed, args.cpu_particles, args.cpu_turns)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_job / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if n == N else WORKLOAD + " (evenly spaced subset of %d)" % n,
                   "n_particles": n, "n_elements": n_el, "turns_per_step": T,
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": "independent error seed per GPU, no collective" if ws > 1 else "1 GPU",
                   "wall_s_timed": wall},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": NOMINAL_FP64 / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / NOMINAL_FP64,
                     "traffic": TRACK_DRAM_BYTES_PER_PARTICLE_TURN * n * T * args.steps / max(kern_launches, 1),
                     "traffic_unit": "bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum of an ncu "
                                     "capture of 400,000 particles, scaled by particles)",
                     "kernel": "xt::track_kernel<0>", "kernel_ms_total": kern_ms,
                     "kernel_launches": kern_launches,
                     "peak_source": "nominal FP64 from unit counts and clocks: 4 flop/clk/SM x 152 SMs x 2070 MHz",
                     "peak_measured_fma": peak_meas / 1e12,
                     "frac_of_measured_fma": achieved / peak_meas,
                     "frac_at_sampled_clock": (achieved / (FP64_FLOP_PER_CLK_SM * N_SM * clocks["sm_mhz"] * 1e6)
                                               if clocks.get("sm_mhz") else None),
                     "algorithmic_flops_per_pass": flops_all / max(units_all, 1)},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "api": "xt_track_host (pinned host buffers)"},
        # each tracking launch is preceded by the two compaction kernels
        "gpu_launches": int(kern_launches * 3),
        "losses": {"alive_after": int((H.a["state"] == 1).sum()), "turns_tracked": turn},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    line.update(extras)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_mlp(args):
    """Surrogate network alone (not part of the default run): CUDA-event time
    of a forward pass over args.mlp_forward samples, or of args.mlp_train
    training steps of batch 4096, on random inputs."""
    import torch
    from paper_2310_00317_gb300 import xtgb
    net = xtgb.Surrogate(seed=7)
    g = torch.Generator(device="cpu")
    g.manual_seed(0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.mlp_forward:
        X = torch.randn(args.mlp_forward, 16, generator=g).cuda()
        net.forward(X)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            net.forward(X)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        flops = 2.0 * args.mlp_forward * (16 * 256 + 3 * 256 * 256 + 256 * 2)
        out = {"mlp_forward_samples": args.mlp_forward, "ms": ms, "tflops": flops / (ms * 1e-3) / 1e12}
    else:
        B = 4096
        X = torch.randn(B, 16, generator=g).cuda()
        y = (torch.rand(B, generator=g) > 0.5).float().cuda()
        t = torch.rand(B, generator=g).cuda()
        m = (torch.rand(B, generator=g) > 0.5).float().cuda()
        L = torch.zeros(1, device="cuda")
        for _ in range(3):
            net.train_step(X, y, t, m, 1e-3, 0.5, L)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.mlp_train):
            net.train_step(X, y, t, m, 1e-3, 0.5, L)
        e1.record()
        torch.cuda.synchronize()
        out = {"mlp_train_steps": args.mlp_train, "batch": B, "ms_per_step": e0.elapsed_time(e1) / args.mlp_train}
    net.close()
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--turns-per-step", type=int, default=2)
    ap.add_argument("--particles", type=int, default=0, help="0 = the full 999,990-particle grid")
    ap.add_argument("--cpu-particles", type=int, default=600)
    ap.add_argument("--cpu-turns", type=int, default=10)
    ap.add_argument("--ref-particles", type=int, default=150)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-seed, lepton-ring and DA-scan measurements")
    ap.add_argument("--mlp-forward", type=int, default=0,
                    help="time only the surrogate's forward pass over this many samples (--steps repeats)")
    ap.add_argument("--mlp-train", type=int, default=0,
                    help="time only this many surrogate training steps (batch 4096)")
    ap.add_argument("--only", default="",
                    help="run one extra measurement alone and print its JSON: thick_elements[:n[:turns]], "
                         "beambeam_lens[:n[:turns]], lepton_quantum[:n[:turns]], twiss, steady[:turns[:window]], "
                         "batched_seeds[:turns_per_step:steps], lepton_equilibrium[:n[:turns]], fodo10[:n[:turns]], "
                         "da_scan (the reduced ring), da_scan_full[:turns[:error_mult[:labels[:test_seeds]]]]")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mlp_forward or args.mlp_train:
        return run_mlp(args)
    if args.only:
        return run_only(args.only)
    return run_ours(args)


def only_kwargs(spec: str):
    """Name and keyword arguments of an --only measurement spec."""
    name, *nums = spec.split(":")
    kw = {}
    if name == "steady":
        kw = {"turns": int(nums[0])} if nums else {}
        if len(nums) > 1:
            kw["window"] = int(nums[1])
    elif name == "batched_seeds":
        kw = {"T": int(nums[0]), "steps": int(nums[1])} if len(nums) > 1 else {}
    elif name == "da_scan":
        kw = {"n_turns": int(nums[0])} if nums else {}
    elif name == "da_scan_full":
        kw = {"n_turns": int(nums[0])} if nums else {}
        if len(nums) > 1:
            kw["base_mult"] = float(nums[1])
        if len(nums) > 2:
            kw["total_labels"] = int(float(nums[2]))
        if len(nums) > 3:
            kw["n_test"] = int(nums[3])
    else:
        if nums:
            kw["n"] = int(nums[0])
        if len(nums) > 1:
            kw["turns"] = int(nums[1])
    return name, kw


def run_only(spec: str) -> int:
    """One extra measurement on its own (for profiling its kernel)."""
    name, kw = only_kwargs(spec)
    fn = {"thick_elements": measure_thick, "beambeam_lens": measure_beambeam, "twiss": measure_twiss,
          "lepton_quantum": measure_lepton, "steady": measure_steady, "batched_seeds": measure_batched,
          "lepton_equilibrium": measure_lepton_equilibrium, "da_scan_full": measure_da_scan_full, "da_scan": measure_da_scan,
          "fodo10": measure_fodo}.get(name)
    if fn is None:
        raise SystemExit("--only: unknown measurement %r" % name)
    print(json.dumps({name: fn(**kw)}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
