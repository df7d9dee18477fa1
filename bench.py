#!/usr/bin/env python
"""Benchmark of the local Verlet buffer broad phase on one GB300.

Workload: the 200,000-particle polydisperse settling box (radii U[0.5, 2] mm,
rho 2500, linear spring-dashpot k_n = 1e4, e = 0.7, velocity Verlet
dt = 1e-6 s, local skin 0.1 d_i, cell edge 1.25 d_max), run through the
library's DEM driver.  A "step" is one DEM step: integrate, broad phase
(displacement check + partial rebuild), narrow phase and forces.  The L2
cache (129 MB) is flushed with a 1 GiB write before every timed step, and
each phase is bracketed by CUDA events on the stream it runs on.

value    = broad-phase particle-steps/s = N * K / (sum of broad-phase times)
e2e      = the same metric through the C-ABI with host buffers: per step the
           positions are copied from pinned host memory, lvb_step runs, and
           the step's flags are read back (all inside the timed region)
roofline = the dominant kernel's algorithmic bytes / its event-timed
           duration, against the measured HBM copy bandwidth
cpu_baseline = the CPU oracle on a bounded sample of the same scene

`--impl reference` times the CPU oracle alone (the reference arm).
Multi-GPU (torchrun): every rank runs its own replica of the scene (weak
scaling, no collective on the data path); rank 0 prints the line.
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

METRIC = "broad-phase particle-steps/s and % HBM roofline; rebuild fraction; vs global buffer"
WORKLOAD = ("settling box: 200,000 polydisperse spheres r~U[0.5,2] mm, rho 2500, LSD k_n 1e4 "
            "e 0.7, velocity Verlet dt 1e-6 s, local skin 0.1 d_i, cell 1.25 d_max")
# 1 GiB: well above the 129 MB L2, and long enough on the GPU (~0.15 ms) that
# the device, not Python's per-step issue rate, is the bottleneck, so the
# event intervals around each phase hold device time only.
L2_FLUSH_BYTES = 1 << 30
T0_SAMPLE = 10_000        # oracle samples start mid-run (step 10,000 of 20,000)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    from paper_2208_13770_gb300 import replicas
    return replicas.rank_info()


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _scene(rank):
    from paper_2208_13770_gb300 import replicas, scenes
    return scenes.settling(seed=replicas.replica_seed(scenes.SEED_BASE + 1, rank))


def _run_dem(lvb, torch, scene, trigger, skin_kind, skin_value, steps, warmup, flush,
             record=None, choice=None, profile_from=0):
    """Runs warmup + steps DEM steps with per-phase CUDA events.  Returns
    per-phase total ms, stats and the (optional) recorded window.  flush:
    a buffer larger than L2 written before every step, or None when the
    inputs themselves are larger than L2.  choice: an autotuned launch
    choice (cell factor, step-kernel block size, flag compaction).
    profile_from: advance this many steps first (100-step graphs), and
    bracket the timed steps with cudaProfilerStart/Stop, so that a profiler
    started with profiling off sees only them."""
    dem = lvb.DEM(scene, trigger=trigger, skin_kind=skin_kind, skin_value=skin_value,
                  cell_factor=None if choice is None else choice.cell_factor)
    if choice is not None:
        choice.apply(dem, lvb)
    stream = torch.cuda.current_stream()
    if profile_from:
        dem.advance(profile_from)
    for _ in range(warmup):
        if flush is not None:
            flush.zero_()
        dem.step()
    torch.cuda.synchronize()
    st0 = dem.lvb.stats()
    tot = np.zeros(3)
    batch = 256
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(batch)]
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    rec = None
    if record is not None:
        start, m = record
        rec = {"pos": torch.empty((m, scene.n, 4), dtype=torch.float32, pin_memory=True),
               "start": start, "m": m}
        dpos = dem.device_pos_tensor(torch)
    if profile_from:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
    t_all0.record(stream)
    done = 0
    while done < steps:
        nb = min(batch, steps - done)
        for b in range(nb):
            k = done + b
            if rec is not None and k == rec["start"]:
                torch.cuda.synchronize()
                rec["ref"] = dem.lvb.ref()
                rec["pos0"] = dem.state()[0]
            if flush is not None:
                flush.zero_()
            e = evs[b]
            e[0].record(stream)
            dem.phase(lvb.DEM_PHASE_INTEGRATE)
            e[1].record(stream)
            dem.phase(lvb.DEM_PHASE_BROAD)
            e[2].record(stream)
            dem.phase(lvb.DEM_PHASE_FORCES)
            e[3].record(stream)
            if rec is not None and rec["start"] <= k < rec["start"] + rec["m"]:
                rec["pos"][k - rec["start"]].copy_(dpos, non_blocking=True)
        torch.cuda.synchronize()
        for b in range(nb):
            e = evs[b]
            tot += [e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])]
        done += nb
    t_all1.record(stream)
    torch.cuda.synchronize()
    if profile_from:
        torch.cuda.profiler.stop()
    wall_ms = t_all0.elapsed_time(t_all1)
    rc = dem.sync()
    if rc != 0:
        raise RuntimeError("device error %d: %s" % (rc, lvb.lvb_strerror(rc)))
    st1 = dem.lvb.stats()
    out = {"phase_ms": tot, "wall_ms": wall_ms, "stats0": st0, "stats1": st1, "rec": rec,
           "near_cutoff": int(len(dem.lvb.near_cutoff(1e-6)[0]))}
    dem.close()
    return out


BATCH_STEPS = 2000

# DRAM bytes (read + write) per launch of the broad-phase step kernel, from
# one ncu capture of the current kernel on each workload (mean of two
# launches; the command and the counters are in profiles/).  They go stale
# when the kernel changes: set them to None until the capture is repeated.
NCU_TRAFFIC_SETTLING = 7.18e6      # profiles/k_step_settling200k_ncu.txt
NCU_TRAFFIC_BATCHED = 210.4e6      # profiles/k_step_batched512_ncu.txt


def _narrow_phase(n, entries, ms, hbm_peak):
    """Roofline of the separate narrow-phase + forces kernel (k_forces): per
    particle pos, v*, a, v (4 x 16 B) and the row bounds (12 B) read, v and a
    (32 B) written, and 4 B per list entry; neighbour records are gathered
    (mostly L2 hits) and not counted."""
    b = n * (16.0 * 4 + 12.0 + 32.0) + 4.0 * entries
    ach = b / (ms * 1e-3) / 1e9
    return {"kernel": "k_forces", "ms_per_step": ms, "bytes_per_step": b,
            "achieved_gbs": ach, "frac_hbm": ach / hbm_peak}


def _batched(lvb, torch, hbm_peak, warmup):
    """512 independent settling scenes (6.2M particles) advanced together:
    autotuned launch choice, then the 2,000-step workload through graphs of
    DEM_GRAPH_STEPS steps (full steps), and once more phase by phase with
    CUDA events for the broad phase's share.  The inputs exceed L2, so no
    flush is needed."""
    from paper_2208_13770_gb300 import autotune, scenes
    sc = scenes.batch()
    n = int(sum(q.n for q in sc))
    # the candidates are tried on the batch as it is half-way through the
    # workload (positions and velocities after BATCH_STEPS / 2 steps), where
    # the particles move as they do in most of the timed steps
    dem = lvb.DEM(sc)
    dem.advance(BATCH_STEPS // 2)
    x, v, _, _ = dem.state()
    off = dem.offsets
    dem.close()
    mid = []
    for q, s0 in enumerate(sc):
        m = s0.copy()
        m.pos[:] = x[off[q]:off[q + 1]]
        m.vel[:, :3] = v[off[q]:off[q + 1], :3]
        mid.append(m)
    best, trials = autotune.tune(mid)
    dem = lvb.DEM(sc, cell_factor=best.cell_factor)
    best.apply(dem, lvb)
    dem.advance(warmup)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    k0 = dem.lvb.stats()["kernels_executed"]
    e0.record(stream)
    dem.advance(BATCH_STEPS)
    e1.record(stream)
    torch.cuda.synchronize()
    rc = dem.sync()
    if rc != 0:
        raise RuntimeError("device error %d: %s" % (rc, lvb.lvb_strerror(rc)))
    graph_ms = e0.elapsed_time(e1)
    k1 = dem.lvb.stats()["kernels_executed"]
    dem.close()
    ph = _run_dem(lvb, torch, sc, lvb.LVB_TRIGGER_PARTIAL, sc[0].skin_kind, sc[0].skin_value,
                  BATCH_STEPS, warmup, None, choice=best)
    bp_ms = float(ph["phase_ms"][1])
    s0, s1 = ph["stats0"], ph["stats1"]
    F = (s1["flagged_total"] - s0["flagged_total"]) / BATCH_STEPS
    row_len = s1["entries"] / n
    bytes_bp = 32.0 * n + n / 8.0 + F * (64.0 + 8.0 * row_len)
    t_ms = bp_ms / BATCH_STEPS
    ach = bytes_bp / (t_ms * 1e-3) / 1e9
    return {
        "workload": "512 settling boxes, N log-uniform in [1000, 50000] (seeded), %d particles, "
                    "r~U[0.5,2] mm, skin 0.1 d_i, %d steps" % (n, BATCH_STEPS),
        "n_scenes": len(sc), "n": n, "steps": BATCH_STEPS,
        "value": n * BATCH_STEPS / (bp_ms * 1e-3), "unit": "particle-steps/s",
        "full_step_graph_value": n * BATCH_STEPS / (graph_ms * 1e-3),
        "graph_steps": 100, "graph_ms_per_step": graph_ms / BATCH_STEPS,
        "gpu_launches_graph_run": int(k1 - k0),
        "narrow_phase": _narrow_phase(n, s1["entries"], float(ph["phase_ms"][2]) / BATCH_STEPS,
                                      hbm_peak),
        "phases_ms_per_step": {"integrate": float(ph["phase_ms"][0]) / BATCH_STEPS,
                               "broad": t_ms, "forces": float(ph["phase_ms"][2]) / BATCH_STEPS},
        "roofline": {"bound": "hbm", "kernel": "broad phase (check + partial rebuild)",
                     "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                     "traffic": NCU_TRAFFIC_BATCHED, "traffic_source": "ncu capture",
                     "bytes_per_launch": bytes_bp, "ms_per_launch": t_ms},
        "flagged_per_step": F,
        "rebuild_fraction": (s1["updated_total"] - s0["updated_total"]) / (n * BATCH_STEPS),
        "autotune": {"choice": {"cell_factor": best.cell_factor,
                                "block_threads": best.block_threads,
                                "compaction": best.compaction},
                     "trials": trials},
        "l2": "inputs (%.0f MB of particle state) exceed L2; no flush" % (n * 96 / 1e6),
    }


LEARN_N = 1_000_000
LEARN_H = 400           # horizon of the rebuild-log labels, and K of the paper's rule
LEARN_MARGIN = 2.0      # labels scaled by this margin before training
LEARN_CLIP = 0.99       # labels clipped at this quantile
LEARN_STEPS = 1500      # steps of the logged training run and of each timed run
LEARN_LOSS = "squared"   # training loss: squared error of the label (or "relative")


def _timed_advance(lvb, torch, scene, kind, value, mlp=None, log=None, steps=LEARN_STEPS):
    """Advance a fresh DEM context `steps` steps in 100-step graphs; returns
    full-step particle-steps/s, updates/step, mean entries, rebuild steps
    (and the rebuild-log samples when log is a horizon)."""
    dem = lvb.DEM(scene, skin_kind=kind, skin_value=value, mlp=mlp)
    if log:
        dem.lvb.log_enable(log, 2_000_000)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    st0 = dem.lvb.stats()
    ms, done, ent = 0.0, 0, []
    while done < steps:
        k = min(500, steps - done)
        torch.cuda.synchronize()
        e0.record(stream)
        dem.advance(k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        ent.append(dem.lvb.stats()["entries"])
        done += k
    rc = dem.sync()
    if rc != 0:
        raise RuntimeError("device error %d: %s" % (rc, lvb.lvb_strerror(rc)))
    st = dem.lvb.stats()
    out = {"value": scene.n * steps / (ms * 1e-3), "unit": "particle-steps/s (full DEM step)",
           "updates_per_step": (st["updated_total"] - st0["updated_total"]) / steps,
           "rebuild_steps": st["rebuild_steps"] - st0["rebuild_steps"],
           "mean_entries": float(np.mean(ent)), "relayouts": st["relayouts"]}
    smp = dem.lvb.log_samples() if log else None
    dem.close()
    return out, smp


def _train_skin(lvb, torch, samples, seed):
    """Network weights trained on the GPU on rebuild-log samples, for the
    travel form of the output over LEARN_H steps (skin = y LEARN_H |v| dt,
    a per-particle factor of the paper's rule): each label (largest
    displacement over the horizon, in diameters) becomes label /
    (f0 LEARN_H) -- the displacement in units of the particle's travel over
    the horizon at its speed when updated -- scaled by LEARN_MARGIN and
    clipped at the LEARN_CLIP quantile; samples of particles at rest are
    left out.  Returns (device weights, info)."""
    import time
    smp = np.ascontiguousarray(samples[samples[:, 0] > 0]).copy()
    y = smp[:, 8].astype(np.float64) * LEARN_MARGIN / (smp[:, 0].astype(np.float64) * LEARN_H)
    smp[:, 8] = np.minimum(y, np.quantile(y, LEARN_CLIP)).astype(np.float32)
    rng = np.random.default_rng(seed)
    p0 = (rng.standard_normal(lvb.LVB_MLP_PARAMS) * 0.1).astype(np.float32)
    yr = np.zeros(2, np.float32)
    t0 = time.time()
    kind = lvb.LVB_MLP_LOSS_RELATIVE if LEARN_LOSS == "relative" else lvb.LVB_MLP_LOSS_SQUARED
    p, mu, isd, losses = lvb.mlp_train(torch.from_numpy(smp).cuda(), epochs=20, batch=512,
                                       lr=3e-3, seed=seed, params0=p0, y_range_out=yr,
                                       loss_kind=kind)
    info = {"samples": int(len(smp)), "epochs": 20, "loss": LEARN_LOSS,
            "loss_first": float(losses[0]),
            "loss_last": float(losses[-1]), "seconds": time.time() - t0,
            "y_range": [float(yr[0]), float(yr[1])], "y_steps": LEARN_H}
    return lvb.mlp_weights_device(p, mu, isd, yr, float(LEARN_H)), info


def _learned(lvb, torch):
    """The learned skin against the paper's rule on a 1,000,000-sphere drum:
    rebuild-log samples from the plain local-buffer run (skin 0.1 d_i,
    horizon LEARN_H), training on the GPU (own kernels), a run of the network
    with its own log, training again on both logs, and a run of that network,
    from three initial weight draws; the fastest of these networks is
    compared with the paper's rule (K = LEARN_H, and K / 2, 2 K) and the
    plain rule, each run from the same initial state."""
    from paper_2208_13770_gb300 import scenes
    sc = scenes.drum(n=LEARN_N, length=0.1)
    # the logged runs give the training samples; every timed run has the log off
    _, smp = _timed_advance(lvb, torch, sc, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, log=LEARN_H)
    plain, _ = _timed_advance(lvb, torch, sc, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1)
    # three initial weight draws, each trained on the plain run's log (stage
    # 1) and again with its own run's log added (stage 2); the fastest of
    # the six networks on this scene is kept
    cands = []
    for seed in (1, 2, 3):
        w1, info1 = _train_skin(lvb, torch, smp, seed)
        _, smp1 = _timed_advance(lvb, torch, sc, lvb.LVB_SKIN_LEARNED, 0.0, mlp=w1, log=LEARN_H)
        r1, _ = _timed_advance(lvb, torch, sc, lvb.LVB_SKIN_LEARNED, 0.0, mlp=w1)
        w2, info2 = _train_skin(lvb, torch, np.concatenate([smp, smp1]), seed + 10)
        r2, _ = _timed_advance(lvb, torch, sc, lvb.LVB_SKIN_LEARNED, 0.0, mlp=w2)
        r1["seed"], r1["stage"], r2["seed"], r2["stage"] = seed, 1, seed, 2
        cands += [r1, r2]
    rule, _ = _timed_advance(lvb, torch, sc, lvb.LVB_SKIN_PAPER_KVDT, float(LEARN_H))
    sweep = {}
    for K in (LEARN_H // 2, 2 * LEARN_H):
        sweep["K%d" % K], _ = _timed_advance(lvb, torch, sc, lvb.LVB_SKIN_PAPER_KVDT, float(K))
    learned = max(cands, key=lambda r: r["value"])
    best_rule = max([rule] + list(sweep.values()), key=lambda r: r["value"])
    return {
        "workload": "drum R 0.3 m x 0.1 m, %d lognormal spheres (median 1 mm, sigma_ln 0.35), "
                    "10 rpm, dt 1e-6 s, %d steps per run" % (sc.n, LEARN_STEPS),
        "training": {"source": "plain local buffer (0.1 d_i), then the network's own run",
                     "output": "travel form: skin = y * %d |v| dt (y clamped to its "
                               "range), a per-particle K = %d y of the paper's rule" % (LEARN_H, LEARN_H),
                     "label": "largest displacement over the next %d steps / (%d |v| dt), "
                              "x %.1f, clipped at the %.2f quantile"
                              % (LEARN_H, LEARN_H, LEARN_MARGIN, LEARN_CLIP),
                     "selection": "fastest of 3 weight draws x 2 training stages on this "
                                  "scene",
                     "last_stage1": info1, "last_stage2": info2},
        "paper_rule_K%d" % LEARN_H: rule,
        "plain_0.1d": plain,
        "learned_candidates": cands,
        "learned": learned,
        "paper_rule_other_K": sweep,
        "gain_vs_paper_rule": learned["value"] / rule["value"],
        "gain_vs_best_paper_rule": learned["value"] / best_rule["value"],
        "gain_vs_plain": learned["value"] / plain["value"],
        "note": "samples come from separate runs with the rebuild log on; timed runs have it off",
    }


def _fused_graph(lvb, torch, scene, steps, warmup):
    """The same scene advanced as the driver runs it: graphs of
    DEM_GRAPH_STEPS fused steps (integrate, broad phase and forces in one
    cooperative launch per step), timed with CUDA events around the whole
    run; no flush between steps."""
    dem = lvb.DEM(scene)
    dem.advance(warmup)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    dem.advance(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    rc = dem.sync()
    if rc != 0:
        raise RuntimeError("device error %d: %s" % (rc, lvb.lvb_strerror(rc)))
    ms = e0.elapsed_time(e1)
    dem.close()
    return {"value": scene.n * steps / (ms * 1e-3), "unit": "particle-steps/s (full DEM step)",
            "ms_per_step": ms / steps, "steps": steps,
            "l2": "not flushed (graphs of 100 fused steps; the state stays in L2)"}


E2E_PASSES = 5   # pipelined passes over the window; the median is reported


def _e2e(lvb, torch, scene, rec):
    """Broad phase through the C-ABI with host buffers, steps m of a recorded
    window of the run (the context resumes from the run's saved reference
    state).  Pipelined: per step lvb_step_host copies the pinned host
    positions in (overlapping the previous step's kernel) and the step's flag
    words and count out to pinned host memory (overlapping the next step's
    kernel); one synchronisation at the end; E2E_PASSES passes, the median
    reported (the host is shared with other jobs).  Also the per-step synchronous form: copy in, lvb_step, then
    lvb_get_flags (which waits) every step."""
    m = rec["m"]
    nw = (scene.n + 31) // 32
    ref = torch.from_numpy(rec["ref"]).cuda()
    out = {}
    reps = []
    pos0_pinned = torch.from_numpy(rec["pos0"]).pin_memory()
    for form in ("pipelined",) * E2E_PASSES + ("sync",):
        dev = torch.empty((scene.n, 4), dtype=torch.float32, device="cuda")
        dev.copy_(torch.from_numpy(rec["pos0"]))
        ctx = lvb.LVB(dev, scene.lo, scene.hi, scene.skin_kind, scene.skin_value, scene.dt,
                      lvb.LVB_TRIGGER_PARTIAL, scene.cell_factor, ref=ref)
        bits = torch.zeros((m, nw), dtype=torch.int32, pin_memory=True)
        nf = torch.zeros((m,), dtype=torch.int32, pin_memory=True)
        words = np.zeros(nw, dtype=np.uint32)
        nf64 = lvb.ctypes.c_int64(0)
        if form == "pipelined":
            # untimed: the first call allocates the context's staging slots;
            # a step at the window's starting positions flags nothing
            ctx.step_host(pos0_pinned, bits=bits[0], n_flagged=nf[0:1])
            rc = ctx.sync()
            if rc:
                raise RuntimeError(lvb.lvb_strerror(rc))
        torch.cuda.synchronize()
        flagged = 0
        t0 = time.perf_counter()
        if form == "pipelined":
            for k in range(m):
                ctx.step_host(rec["pos"][k], bits=bits[k], n_flagged=nf[k:k + 1])
            out["enqueue_s"] = time.perf_counter() - t0
            rc = ctx.sync()
            if rc:
                raise RuntimeError(lvb.lvb_strerror(rc))
            dt = time.perf_counter() - t0
            flagged = int(nf.sum())
        else:
            for k in range(m):
                dev.copy_(rec["pos"][k], non_blocking=True)
                ctx.step(dev)
                rc = lvb.lvb_get_flags(ctx.ctx, words.ctypes.data, lvb.ctypes.byref(nf64))
                if rc:
                    raise RuntimeError(lvb.lvb_strerror(rc))
                flagged += nf64.value
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        st = ctx.stats()
        ctx.close()
        res = {"value": scene.n * m / dt, "unit": "particle-steps/s",
               "h2d_bytes_per_step": scene.n * 16, "d2h_bytes_per_step": nw * 4 + 4,
               "steps": m, "flagged": flagged, "store_grows": st["grows"],
               "relayouts": st["relayouts"]}
        if form == "pipelined":
            res["host_enqueue_us_per_step"] = out.pop("enqueue_s") * 1e6 / m
            reps.append(res)
        else:
            out[form] = res
    # the host is shared: the median of the passes over the window
    reps.sort(key=lambda r: r["value"])
    e2e = dict(reps[len(reps) // 2])
    e2e["api"] = "lvb_step_host (pinned host positions in, flag words and count out)"
    e2e["passes"] = [r["value"] for r in reps]
    e2e["sync_per_step"] = out["sync"]
    return e2e


def _oracle_sample(scene, t0_steps, m_steps, n_sub=None, time_budget=None, stride=10):
    """Times the CPU oracle's broad phase (flags, reference update, pair set
    by Algorithm 1) on a bounded sample of the scene: the n_sub lowest
    particles, moving in free fall (the settling cloud is dilute, so free
    fall is its motion between rare contacts), from step t0 for m steps.
    The reference state at t0 is prepared (untimed) by the oracle's own
    flag/skin updates every `stride` steps from step 0, without list builds."""
    import oracle
    from oracle.statemachine import OracleLVB
    pos0 = scene.pos
    if n_sub is not None and n_sub < scene.n:
        idx = np.argsort(pos0[:, 2], kind="stable")[:n_sub]
        idx.sort()
    else:
        idx = np.arange(scene.n)
    p0 = pos0[idx].astype(np.float64)
    v0 = scene.vel[idx].astype(np.float64)
    g = np.asarray(scene.gravity, dtype=np.float64)
    dt = scene.dt

    def at(step):
        t = step * dt
        out = np.empty((len(idx), 4), dtype=np.float32)
        out[:, :3] = p0[:, :3] + v0[:, :3] * t + 0.5 * g * t * t
        out[:, 3] = p0[:, 3]
        return out

    rmax = float(np.float32(scene.pos[:, 3].max()))
    L = scene.cell_factor * 2.0 * rmax * (1 + 2 ** -7)
    H = np.float32(0.5 * L * (1 - 2 ** -8))
    first = at(0)
    ref = first.copy()
    ref[:, 3] = oracle.skin(scene.skin_kind, scene.skin_value, dt, H, first)
    for k in list(range(stride, t0_steps, stride)) + [t0_steps]:   # fast-forward
        p = at(k)
        f = oracle.flags(p, ref)
        if f.any():
            ref[f, :3] = p[f, :3]
            ref[f, 3] = oracle.skin(scene.skin_kind, scene.skin_value, dt, H, p[f])
    sm = OracleLVB(at(t0_steps), scene.skin_kind, scene.skin_value, dt, H, ref4=ref)
    snaps = [at(t0_steps + 1 + k) for k in range(m_steps)]
    t = time.perf_counter()
    done = 0
    for p in snaps:
        sm.step(p)
        done += 1
        if time_budget is not None and time.perf_counter() - t > time_budget:
            break
    el = time.perf_counter() - t
    return {"value": len(idx) * done / el, "particles": int(len(idx)), "steps": done,
            "seconds": el, "updates": int(sm.updates), "rebuild_steps": int(sm.rebuild_steps)}


def _cpu_info():
    model = "unknown"
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model, "arch": os.uname().machine}


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return 0
    scene = _scene(0)
    # size the per-step sample so that warmup + steps fit in ~150 s
    probe = _oracle_sample(scene, T0_SAMPLE, 3, n_sub=20_000)
    per_particle = 1.0 / probe["value"]
    budget = 150.0 / max(1, args.steps + args.warmup)
    n_sub = int(max(1000, min(scene.n, budget / per_particle)))
    res = _oracle_sample(scene, T0_SAMPLE, args.steps + args.warmup, n_sub=n_sub)
    v = res["value"]
    sample = ("oracle broad phase (flags, skins, pair set by linked cells) on the %d lowest "
              "particles of the settling box in free fall, steps %d..%d" %
              (res["particles"], T0_SAMPLE + 1, T0_SAMPLE + res["steps"]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * res["seconds"] / max(1, res["steps"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n": scene.n},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": 1,
                             "kind": "oracle", "sample": sample, "host": _cpu_info()},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _only_batched(lvb, torch, args, rank):
    """The batched workload alone, phase by phase with CUDA events (for
    profiling: --profile-from brackets the timed steps), default launch
    choice.  Prints one short JSON line."""
    from paper_2208_13770_gb300 import scenes
    sc = scenes.batch()
    n = int(sum(q.n for q in sc))
    res = _run_dem(lvb, torch, sc, lvb.LVB_TRIGGER_PARTIAL, sc[0].skin_kind, sc[0].skin_value,
                   args.steps, args.warmup, None, profile_from=args.profile_from)
    if rank == 0:
        ph = res["phase_ms"] / args.steps
        print(json.dumps({"only_batched": True, "n": n, "phases_ms_per_step": list(ph),
                          "value": n * args.steps / (res["phase_ms"][1] * 1e-3),
                          "stats": res["stats1"]}))
    return 0


def run_native(args):
    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2208_13770_gb300 import lvb
    hbm_peak, peak_kind = _peaks()
    if args.only_batched:
        return _only_batched(lvb, torch, args, rank)
    scene = _scene(rank)
    n = scene.n
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    m_e2e = 0 if args.only_local else min(args.e2e_steps, args.steps)
    rec_start = max(0, args.steps // 2 - m_e2e // 2)

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        loc = _run_dem(lvb, torch, scene, lvb.LVB_TRIGGER_PARTIAL, scene.skin_kind,
                       scene.skin_value, args.steps, args.warmup, flush,
                       record=(rec_start, m_e2e) if m_e2e else None,
                       profile_from=args.profile_from)
    torch.cuda.synchronize()
    from paper_2208_13770_gb300 import replicas
    bp_ms, step_ms_tot = replicas.max_over_ranks(
        [float(loc["phase_ms"][1]), float(loc["phase_ms"].sum())], device="cuda")
    value = replicas.job_throughput(world, n, args.steps, bp_ms)

    if args.only_local:
        if rank == 0:
            ph = loc["phase_ms"] / args.steps
            print(json.dumps({"only_local": True, "phases_ms_per_step": list(ph),
                              "value": value, "stats": loc["stats1"]}))
        return 0
    # global-buffer variant: uniform skin 0.1 * mean diameter, any flag
    # rebuilds the whole list (Def. autoverlet)
    dmean = float(2.0 * scene.pos[:, 3].astype(np.float64).mean())
    glob = _run_dem(lvb, torch, scene, lvb.LVB_TRIGGER_GLOBAL, lvb.LVB_SKIN_GLOBAL,
                    0.1 * dmean, args.steps, args.warmup, flush)
    g_bp_ms, = replicas.max_over_ranks([float(glob["phase_ms"][1])], device="cuda")

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
        return 0

    e2e = _e2e(lvb, torch, scene, loc["rec"])
    e2e["value"] *= world
    fused = _fused_graph(lvb, torch, scene, args.steps, args.warmup)
    batched = None if args.no_batched else _batched(lvb, torch, hbm_peak, args.warmup)
    learned = None if args.no_learned else _learned(lvb, torch)

    s0, s1 = loc["stats0"], loc["stats1"]
    flagged = s1["flagged_total"] - s0["flagged_total"]
    upd = s1["updated_total"] - s0["updated_total"]
    gs0, gs1 = glob["stats0"], glob["stats1"]
    g_rebuild_steps = gs1["rebuild_steps"] - gs0["rebuild_steps"]
    entries = s1["entries"]
    row_len = entries / n
    K = args.steps
    ph = loc["phase_ms"] / K
    # algorithmic bytes per step (one launch each of the phase kernels)
    F = flagged / K
    bytes_bp = 32.0 * n + n / 8.0 + F * (64.0 + 8.0 * row_len)
    bytes_forces = n * (16.0 * 4 + 12.0 + 32.0) + 4.0 * entries
    bytes_integrate = n * (16.0 * 4 + 32.0)
    kern = {"k_forces (narrow phase + forces)": (ph[2], bytes_forces),
            "k_integrate": (ph[0], bytes_integrate),
            "broad phase (check + partial rebuild)": (ph[1], bytes_bp)}
    dom = max(kern, key=lambda k: kern[k][0])
    t_ms, b = kern[dom]
    achieved = b / (t_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak,
            "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm_peak,
            "traffic": NCU_TRAFFIC_SETTLING if dom.startswith("broad") else None,
            "traffic_source": "ncu capture", "bytes_per_launch": b, "ms_per_launch": t_ms}
    bp_ach = bytes_bp / (ph[1] * 1e-3) / 1e9

    cpu = None
    if not args.no_cpu_baseline:
        res = _oracle_sample(scene, T0_SAMPLE, 60, time_budget=25.0)
        cpu = {"value": res["value"], "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
               "sample": "oracle broad phase on all %d particles in free fall, steps "
                         "%d..%d (%.1f s); reference state fast-forwarded by the oracle"
                         % (res["particles"], T0_SAMPLE + 1, T0_SAMPLE + res["steps"],
                            res["seconds"]),
               "host": _cpu_info()}

    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": step_ms_tot / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "dt": scene.dt, "skin": "0.1 d_i",
                   "trigger": "partial (local buffer)", "l2": "flushed before every timed step "
                   "(1 GiB write)", "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roof,
        "broad_phase": {"ms_per_step": ph[1], "achieved_gbs": bp_ach,
                        "frac_hbm": bp_ach / hbm_peak, "bytes_per_step": bytes_bp},
        "narrow_phase": _narrow_phase(n, entries, ph[2], hbm_peak),
        "phases_ms_per_step": {"integrate": ph[0], "broad": ph[1], "forces": ph[2]},
        "full_step_particle_steps_per_s": world * n * K / (step_ms_tot * 1e-3),
        "full_step_graph": fused,
        "rebuild_fraction": upd / (n * K),
        "flagged_per_step": F,
        "global_buffer": {"value": world * n * K / (g_bp_ms * 1e-3),
                          "rebuild_step_fraction": g_rebuild_steps / K,
                          "skin": "uniform 0.1 * mean diameter = %.3g m" % (0.1 * dmean),
                          "ms_per_step": float(glob["phase_ms"].sum()) / K},
        "speedup_vs_global": g_bp_ms / bp_ms,
        "list": {"entries": entries, "mean_row": row_len, "relayouts": s1["relayouts"],
                 "near_cutoff_pairs_rel_1e-6": loc["near_cutoff"]},
        "e2e": e2e,
        "gpu_launches": int(s1["kernels_executed"] - s0["kernels_executed"]),
        "grid_barriers": int(s1["barriers"] - s0["barriers"]),
        "step_kernel": {"blocks": s1["step_blocks"], "threads": s1["block_threads"],
                        "launch": "cooperative, one per broad-phase step"},
        "clocks": clk.summary(),
        "timed_region_ms_incl_flush": loc["wall_ms"],
    }
    if batched is not None:
        batched["vs_single_scene"] = batched["value"] / value
        line["batched"] = batched
    if learned is not None:
        line["learned"] = learned
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line))
    if world > 1:
        torch.distributed.barrier()
    return 0


def run_k_sweep(args):
    """Time and rebuild fractions against K of the paper's rule (Eq.
    skin_formulus1) on the settling box, every run from the same initial
    state, phase by phase with the L2 flushed before every step."""
    import torch
    from paper_2208_13770_gb300 import lvb
    scene = _scene(0)
    n = scene.n
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    rows = []
    for K in (float(k) for k in args.k_sweep.split(",")):
        r = _run_dem(lvb, torch, scene, lvb.LVB_TRIGGER_PARTIAL, lvb.LVB_SKIN_PAPER_KVDT, K,
                     args.steps, args.warmup, flush)
        ph = r["phase_ms"] / args.steps
        s0, s1 = r["stats0"], r["stats1"]
        rows.append({"K": K, "broad_ms": ph[1], "narrow_forces_ms": ph[2],
                     "integrate_ms": ph[0], "step_ms": float(ph.sum()),
                     "rebuild_fraction": (s1["updated_total"] - s0["updated_total"])
                     / (n * args.steps),
                     "rebuild_step_fraction": (s1["rebuild_steps"] - s0["rebuild_steps"])
                     / args.steps,
                     "entries": s1["entries"]})
    print(json.dumps({"k_sweep": rows, "workload": WORKLOAD.replace("local skin 0.1 d_i",
                                                                   "skin K |v| dt"),
                      "steps": args.steps, "warmup": args.warmup,
                      "l2": "flushed before every timed step (1 GiB write)"}))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-local", action="store_true",
                    help="time the local-buffer run only (for profiling)")
    ap.add_argument("--profile-from", type=int, default=0,
                    help="with --only-local: advance this many steps first and bracket the "
                         "timed steps with cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched (512-scene) run")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-skin comparison (1M-sphere drum)")
    ap.add_argument("--only-batched", action="store_true",
                    help="time the batched (512-scene) workload alone, phase by phase "
                         "(for profiling)")
    ap.add_argument("--k-sweep", default="",
                    help="comma-separated K values: the paper's skin rule K |v| dt on the "
                         "settling box, phase by phase (broad phase, narrow phase + forces, "
                         "rebuild fractions) for each K, then exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.k_sweep:
        return run_k_sweep(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
