#!/usr/bin/env python
"""Benchmark of the local Verlet buffer broad phase on one GB300.

Headline workload: 512 independent settling boxes (N per box log-uniform in
[1,000, 50,000], seeded; 6,229,742 polydisperse spheres, radii U[0.5, 2] mm,
rho 2500, linear spring-dashpot k_n = 1e4, e = 0.7, velocity Verlet
dt = 1e-6 s, local skin 0.1 d_i) advanced together in one context by the
library's DEM driver, with the autotuned launch choice.  The run is advanced
(untimed, 100-step graphs) to step 1,000 - W of its 2,000 steps, W warm-up
steps follow, and the K timed steps are steps 1,001 .. 1,000 + K, so any K
times a representative stretch of the run with list updates in it.  A
"step" is one DEM step, run phase by phase (integrate, broad phase, narrow
phase + forces), each phase bracketed by CUDA events on its stream.  The
particle state (~600 MB) exceeds the 129 MB L2, so no flush is needed.

value    = broad-phase particle-steps/s = N * K / (sum of broad-phase times);
           the broad phase is one cooperative launch of the step kernel
           (displacement check + partial rebuild) per step
roofline = the step kernel's algorithmic bytes per launch (check, flagged
           particles, stencil candidates, partner-row edits, all counted on
           the device) / its event-timed duration, against the measured HBM
           copy bandwidth
e2e      = the same metric through the C-ABI with host buffers (lvb_step_host
           on a batched context resumed at the window's start: per step the
           positions come from pinned host memory and the flags go back)
cpu_baseline = the CPU oracle (OpenMP, all host cores, and one core) on the
           GPU run's own states of a contiguous block of the scenes over the
           first steps of the same window

Extras: the 200,000-sphere settling box from step 10,001 (local vs global
buffer, L2 flushed), the 2,000,000-sphere drum with a dilute cascading layer
(5,000 timed steps after a spin-up, a K sweep of the paper's rule, the
stencil's reach bounds against a plain 27-cell stencil), the learned skin on
the 1,000,000-sphere drum, and the 2,000-sphere ballistic case.

`--impl reference` times the CPU oracle alone (the reference arm) on the same
window: a sample of the batch's scenes advanced to step 1,000 by the oracle's
own binary64 DEM, then its broad phase timed over steps 1,001 .. 1,000 + K.
Multi-GPU (torchrun): the 512 scenes are split over the ranks, greedily by
particle count; every rank runs its share with no collective on the data
path; rank 0 prints the line.
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
WORKLOAD = ("batched settling boxes: 512 independent scenes, N log-uniform in [1000, 50000] "
            "(seeded), polydisperse spheres r~U[0.5,2] mm, rho 2500, LSD k_n 1e4 e 0.7, "
            "velocity Verlet dt 1e-6 s, local skin 0.1 d_i, autotuned cell factor and launch "
            "shape; window from step 1001 of the 2000-step run")
BATCH_STEPS = 2000
T0 = 1000                 # the timed window starts after step T0 of the batch's run
T0_SETTLING = 10_000      # and after step T0_SETTLING of the 200k settling box's run
SETTLING_STEPS = 2000     # timed steps of the 200k box (its global buffer rebuilds on
                          # about one step in 500, so a long window)
EARLY_PERMILLE = 700      # the early trigger's beta (x 1000) in the settling extra
# 1 GiB: well above the 129 MB L2 (for the workloads that fit in it)
L2_FLUSH_BYTES = 1 << 30
M_E2E = 16                # steps of the window the e2e and CPU legs replay
CPU_BUDGET_S = 15.0       # seconds of oracle time per thread setting (whole scenes)
REF_SAMPLE_N = 40_000     # particles of the reference arm's sample (scenes > 4096 each)


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


def _check_rc(lvb, rc):
    if rc != 0:
        raise RuntimeError("device error %d: %s" % (rc, lvb.lvb_strerror(rc)))


# ----------------------------------------------------------------- timing
def _phases(lvb, torch, dem, steps, flush=None, on_step=None):
    """Runs `steps` DEM steps phase by phase with CUDA events around each
    phase (on the context's stream, torch's current one).  flush: a buffer
    larger than L2 zeroed before every step (None when the inputs exceed
    L2).  on_step(k): called after step k's phases are enqueued (outside the
    events).  Returns per-phase total ms (integrate, broad, forces)."""
    stream = torch.cuda.current_stream()
    tot = np.zeros(3)
    batch = 256
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(batch)]
    done = 0
    while done < steps:
        nb = min(batch, steps - done)
        for b in range(nb):
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
            if on_step is not None:
                on_step(done + b)
        torch.cuda.synchronize()
        for b in range(nb):
            e = evs[b]
            tot += [e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])]
        done += nb
    return tot


def _advance_to(dem, step, done=0):
    """Advance the DEM context from step `done` to step `step` (graphs)."""
    if step > done:
        dem.advance(step - done)


def _diff(s0, s1, key):
    return s1[key] - s0[key]


def _bp_bytes(n, steps, s0, s1, reads_vel=False):
    """Algorithmic bytes per broad-phase launch, averaged over `steps`:
      check      32 n (pos + ref read) + n / 8 (flag bits written)
      flagged    F (56 + 8 l) [+ 16 F when the policy reads v]: pos read, new
                 reference state written, old / new cell keys, the cell
                 slot's record written, the particle's own row read (old)
                 and written (new), l = mean row length
      candidates 20 per stencil candidate (slot id + reference record) and
                 16 per flagged-list record of the direct flagged test
      edits      8 l per edit of an unflagged partner's row (row read, entry
                 written)
    The counts F, candidates, direct records and edits are the device's own
    (lvb_stats), so the figure follows the work the step actually did."""
    F = _diff(s0, s1, "flagged_total") / steps
    ell = s1["entries"] / n
    cand = _diff(s0, s1, "rebuild_candidates") / steps
    direct = _diff(s0, s1, "rebuild_direct") / steps
    edits = _diff(s0, s1, "rebuild_edits") / steps
    check = 32.0 * n + n / 8.0
    flagged = F * (56.0 + 8.0 * ell + (16.0 if reads_vel else 0.0))
    b = check + flagged + 20.0 * cand + 16.0 * direct + 8.0 * ell * edits
    return b, {"check": check, "flagged": flagged, "candidates": 20.0 * cand + 16.0 * direct,
               "edits": 8.0 * ell * edits, "F": F, "mean_row": ell,
               "stencil_candidates_per_flagged": cand / F if F else 0.0,
               "direct_records_per_flagged": direct / F if F else 0.0,
               "edits_per_flagged": edits / F if F else 0.0}


def _roofline(kernel, bytes_per_launch, ms_per_launch, peak, peak_kind, traffic, parts=None):
    ach = bytes_per_launch / (ms_per_launch * 1e-3) / 1e9
    r = {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": peak,
         "peak_kind": peak_kind, "unit": "GB/s", "frac": ach / peak, "traffic": traffic,
         "traffic_source": "ncu capture (dram__bytes_read.sum + dram__bytes_write.sum per "
                           "launch)" if traffic else "none: kernel changed since the capture",
         "bytes_per_launch": bytes_per_launch, "ms_per_launch": ms_per_launch}
    if parts is not None:
        r["bytes_parts"] = parts
    return r


def _narrow_phase(n, entries, ms, hbm_peak):
    """Roofline of the separate narrow-phase + forces kernel (k_forces): per
    particle pos, v*, a, v (4 x 16 B) and the row bounds (12 B) read, v and a
    (32 B) written, and 4 B per list entry; neighbour records are gathered
    (mostly L2 hits) and not counted."""
    b = n * (16.0 * 4 + 12.0 + 32.0) + 4.0 * entries
    ach = b / (ms * 1e-3) / 1e9
    return {"kernel": "k_forces", "ms_per_step": ms, "bytes_per_step": b,
            "achieved_gbs": ach, "frac_hbm": ach / hbm_peak}


# DRAM bytes (read + write) per launch of the broad-phase step kernel on the
# headline window, from one ncu capture of the current kernel (mean of the
# captured launches; the command and the counters are in profiles/).  None
# when the kernel has changed since the capture.
NCU_TRAFFIC_BATCHED = 203.61e6   # profiles/k_step_batched512_ncu.txt


# ----------------------------------------------------------------- headline
def _batch_scenes(rank=0, world=1):
    from paper_2208_13770_gb300 import replicas, scenes
    sc = scenes.batch()
    if world > 1:
        mine = replicas.shard_greedy([q.n for q in sc], world)[rank]
        sc = [sc[q] for q in mine]
    return sc


def _tune(lvb, torch, sc):
    """Autotuned launch choice on the batch as it stands half-way through
    its run (positions and velocities after BATCH_STEPS / 2 steps)."""
    from paper_2208_13770_gb300 import autotune
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
    return autotune.tune(mid, key="settling-batch")


def _headline(lvb, torch, sc, choice, steps, warmup, record=True, profile=False):
    """The batch from step T0 - warmup: warm-up steps, then `steps` timed
    steps phase by phase.  Records (for the e2e and CPU legs) the reference
    state and positions at the window's start and all positions over the
    first M_E2E steps."""
    n = int(sum(q.n for q in sc))
    dem = lvb.DEM(sc, cell_factor=choice.cell_factor)
    choice.apply(dem, lvb)
    _advance_to(dem, T0 - warmup)
    _phases(lvb, torch, dem, warmup)
    torch.cuda.synchronize()
    rec = None
    on_step = None
    if record:
        off = dem.offsets
        m_e2e = min(M_E2E, steps)
        rec = {"ref0": dem.lvb.ref(), "pos0": dem.state()[0], "m_e2e": m_e2e,
               "pos_e2e": torch.empty((m_e2e, n, 4), dtype=torch.float32, pin_memory=True),
               "rnl_max": [dem.lvb.scene_info(q)["rnl_max"] for q in range(len(sc))],
               "offsets": off}
        dpos = dem.device_pos_tensor(torch)

        def on_step(k):
            if k < m_e2e:
                rec["pos_e2e"][k].copy_(dpos, non_blocking=True)
    s0 = dem.lvb.stats()
    if profile:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
    ph = _phases(lvb, torch, dem, steps, on_step=on_step)
    if profile:
        torch.cuda.profiler.stop()
    _check_rc(lvb, dem.sync())
    s1 = dem.lvb.stats()
    out = {"n": n, "phase_ms": ph, "stats0": s0, "stats1": s1, "rec": rec}
    dem.close()
    return out


def _e2e_batch(lvb, torch, sc, choice, rec):
    """Broad phase through the C-ABI with host buffers on the window's first
    m steps: a batched context resumed at the window's start
    (lvb_batch_init_resume from the run's reference state) steps through
    the run's recorded positions with lvb_step_host -- per step the pinned
    host positions go in (overlapping the previous step's kernel) and the
    step's flag words and count come back to pinned host memory; one
    synchronisation at the end.  Five passes, each on a fresh context; the
    median is reported."""
    m = rec["m_e2e"]
    n = rec["pos0"].shape[0]
    nw = (n + 31) // 32
    off = rec["offsets"]
    lo = [q.lo for q in sc]
    hi = [q.hi for q in sc]
    ref = torch.from_numpy(rec["ref0"]).cuda()
    pos0 = torch.from_numpy(rec["pos0"]).cuda()
    reps = []
    for _ in range(5):
        ctx = lvb.LVB(pos0, lo, hi, sc[0].skin_kind, sc[0].skin_value, sc[0].dt,
                      lvb.LVB_TRIGGER_PARTIAL, choice.cell_factor, ref=ref, offsets=off)
        ctx.set_option(lvb.LVB_OPT_BLOCK_THREADS, choice.block_threads)
        ctx.set_option(lvb.LVB_OPT_COMPACT, choice.compaction)
        ctx.set_option(lvb.LVB_OPT_CHECK_LOADS, choice.check_loads)
        bits = torch.zeros((m + 1, nw), dtype=torch.int32, pin_memory=True)
        nf = torch.zeros((m + 1,), dtype=torch.int32, pin_memory=True)
        # untimed: the first call allocates the staging slots; a step at the
        # window's starting positions flags nothing (every particle is within
        # its skin of its reference position there)
        ctx.step_host(rec["pos0"], bits=bits[m], n_flagged=nf[m:m + 1])
        _check_rc(lvb, ctx.sync())
        k0 = ctx.stats()["kernels_executed"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(m):
            ctx.step_host(rec["pos_e2e"][k], bits=bits[k], n_flagged=nf[k:k + 1])
        _check_rc(lvb, ctx.sync())
        dt = time.perf_counter() - t0
        st = ctx.stats()
        ctx.close()
        reps.append({"value": n * m / dt, "flagged": int(nf[:m].sum()),
                     "launches": int(st["kernels_executed"] - k0)})
    reps.sort(key=lambda r: r["value"])
    med = reps[len(reps) // 2]
    return {"value": med["value"], "unit": "particle-steps/s", "h2d_bytes_per_step": n * 16,
            "d2h_bytes_per_step": nw * 4 + 4, "steps": m, "window": "steps %d..%d" %
            (T0 + 1, T0 + m), "flagged": med["flagged"], "launches": med["launches"],
            "api": "lvb_step_host on lvb_batch_init_resume (pinned host positions in, flag "
                   "words and count out)", "passes": [r["value"] for r in reps]}


def _oracle_replay(sc, rec, threads, budget_s):
    """The oracle's broad phase (flags, skins, pair set by linked cells) on
    the GPU run's own states: each scene starts from the run's reference
    state at the window's start and steps through the recorded positions of
    the window's first steps.  Scenes are replayed one after another, from
    scene 0, until the time budget is spent; returns particle-steps/s and
    what was covered."""
    import oracle
    from oracle.statemachine import OracleLVB
    oracle.set_threads(threads)
    used = oracle.threads()
    off = rec["offsets"]
    pos = rec["pos_e2e"].numpy()
    m = rec["m_e2e"]
    done_ps, el, scenes_done = 0, 0.0, 0
    for q in range(len(sc)):
        a, b = int(off[q]), int(off[q + 1])
        s0 = sc[q]
        sm = OracleLVB(rec["pos0"][a:b], s0.skin_kind, s0.skin_value, s0.dt, rec["rnl_max"][q],
                       ref4=rec["ref0"][a:b])
        snaps = [np.ascontiguousarray(pos[k, a:b]) for k in range(m)]
        t = time.perf_counter()
        for p in snaps:
            sm.step(p)
        el += time.perf_counter() - t
        done_ps += (b - a) * m
        scenes_done += 1
        if el > budget_s:
            break
    oracle.set_threads(0)
    return {"value": done_ps / el, "cores": used, "seconds": el, "scenes": scenes_done,
            "particles": int(off[scenes_done]), "steps": m}


def _cpu_baseline(sc, rec):
    allc = _oracle_replay(sc, rec, 0, CPU_BUDGET_S)
    one = _oracle_replay(sc, rec, 1, CPU_BUDGET_S)
    return {"value": allc["value"], "unit": "particle-steps/s", "cores": allc["cores"],
            "kind": "oracle",
            "sample": "oracle broad phase (flags, skins, pair set by linked cells; OpenMP) on "
                      "the GPU run's own states of scenes 0..%d (%d particles), steps %d..%d of "
                      "the window, from the run's reference state at step %d (%.1f s)"
                      % (allc["scenes"] - 1, allc["particles"], T0 + 1, T0 + allc["steps"], T0,
                         allc["seconds"]),
            "single_core": {"value": one["value"], "cores": one["cores"],
                            "scenes": one["scenes"], "seconds": one["seconds"]},
            "host": _cpu_info()}


# ----------------------------------------------------------------- extras
def _settling(lvb, torch, steps, warmup, hbm_peak, peak_kind):
    """The 200,000-sphere settling box from step T0_SETTLING: local buffer
    (skin 0.1 d_i) against the paper's global buffer (uniform skin 0.1 x
    mean diameter, any flag rebuilds the whole list), phase by phase, L2
    flushed before every step; and the driver's fused 100-step graphs."""
    from paper_2208_13770_gb300 import scenes
    scene = scenes.settling()
    n = scene.n
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    dmean = float(2.0 * scene.pos[:, 3].astype(np.float64).mean())
    out = {"workload": "settling box: 200,000 polydisperse spheres r~U[0.5,2] mm, steps "
                       "%d..%d of the 20,000-step run" % (T0_SETTLING + 1, T0_SETTLING + steps),
           "n": n, "l2": "flushed before every timed step (1 GiB write)"}
    for name, trig, kind, val, early in (("local", lvb.LVB_TRIGGER_PARTIAL, scene.skin_kind,
                                          scene.skin_value, 1000),
                                         ("local_early", lvb.LVB_TRIGGER_PARTIAL,
                                          scene.skin_kind, scene.skin_value, EARLY_PERMILLE),
                                         ("global_buffer", lvb.LVB_TRIGGER_GLOBAL,
                                          lvb.LVB_SKIN_GLOBAL, 0.1 * dmean, 1000)):
        dem = lvb.DEM(scene, trigger=trig, skin_kind=kind, skin_value=val)
        if early < 1000:
            dem.lvb.set_option(lvb.LVB_OPT_EARLY, early)
        _advance_to(dem, T0_SETTLING - warmup)
        _phases(lvb, torch, dem, warmup, flush)
        s0 = dem.lvb.stats()
        ph = _phases(lvb, torch, dem, steps, flush)
        _check_rc(lvb, dem.sync())
        s1 = dem.lvb.stats()
        dem.close()
        r = {"value": n * steps / (ph[1] * 1e-3), "unit": "particle-steps/s",
             "phases_ms_per_step": {"integrate": ph[0] / steps, "broad": ph[1] / steps,
                                    "forces": ph[2] / steps},
             "flagged_per_step": _diff(s0, s1, "flagged_total") / steps,
             "rebuild_fraction": _diff(s0, s1, "updated_total") / (n * steps),
             "rebuild_step_fraction": _diff(s0, s1, "rebuild_steps") / steps,
             "entries": s1["entries"], "relayouts": s1["relayouts"]}
        if name.startswith("local"):
            b, parts = _bp_bytes(n, steps, s0, s1)
            r["roofline"] = _roofline("k_step (broad phase)", b, ph[1] / steps, hbm_peak,
                                      peak_kind, None, parts)
            r["narrow_phase"] = _narrow_phase(n, s1["entries"], ph[2] / steps, hbm_peak)
            if early < 1000:
                r["early_beta"] = early / 1000.0
        else:
            r["skin"] = "uniform 0.1 * mean diameter = %.3g m" % (0.1 * dmean)
        out[name] = r
    out["speedup_vs_global"] = {
        "local": out["local"]["value"] / out["global_buffer"]["value"],
        "local_early": out["local_early"]["value"] / out["global_buffer"]["value"]}
    # the driver's own form: one cooperative launch per full DEM step, graphs
    dem = lvb.DEM(scene)
    _advance_to(dem, T0_SETTLING)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    gsteps = 1000
    torch.cuda.synchronize()
    e0.record(stream)
    dem.advance(gsteps)
    e1.record(stream)
    torch.cuda.synchronize()
    _check_rc(lvb, dem.sync())
    ms = e0.elapsed_time(e1)
    dem.close()
    out["full_step_graph"] = {"value": n * gsteps / (ms * 1e-3),
                              "unit": "particle-steps/s (full DEM step)",
                              "ms_per_step": ms / gsteps, "steps": "%d..%d" % (
                                  T0_SETTLING + 1, T0_SETTLING + gsteps),
                              "l2": "not flushed (100-step graphs)"}
    return out


DRUM_N = 2_000_000
DRUM_SPINUP = 20_000
DRUM_STEPS = 5000


def _drum_scene(n=DRUM_N, length=0.20):
    from paper_2208_13770_gb300 import scenes
    return scenes.drum(n=n, length=length, tilt_deg=30.0, cascade=0.05)


def _spun_up(lvb, sc, steps):
    """The drum after `steps` steps of the driver (graphs), as a new scene
    object (positions and velocities), for runs that start from it."""
    dem = lvb.DEM(sc)
    dem.advance(steps)
    x, v, _, _ = dem.state()
    _check_rc(lvb, dem.sync())
    dem.close()
    m = sc.copy()
    m.pos[:] = x
    m.vel[:, :3] = v[:, :3]
    return m


def _drum(lvb, torch, hbm_peak, peak_kind, k_sweep=(0, 50, 100, 200, 400, 1000, 5000)):
    """The 2,000,000-sphere drum (lognormal radii, 0.20 m long, bed turned
    30 degrees, 5% of the particles in a dilute cascading layer): spin-up of
    DRUM_SPINUP steps, then DRUM_STEPS full steps in graphs; the broad phase
    phase by phase over 500 steps; a K sweep of the paper's rule; and the
    stencil's reach bounds against a plain 27-cell stencil."""
    sc = _drum_scene()
    n = sc.n
    mid = _spun_up(lvb, sc, DRUM_SPINUP)
    stream = torch.cuda.current_stream()
    out = {"workload": "drum R 0.3 m x 0.20 m, %d lognormal spheres (median 1 mm, sigma_ln "
                       "0.35, clipped [0.4, 3] mm), bed turned 30 deg with 5%% in a dilute "
                       "cascading layer, 10 rpm, dt 1e-6 s; %d steps of spin-up, then the "
                       "timed steps" % (n, DRUM_SPINUP), "n": n}
    # full steps, graphs
    dem = lvb.DEM(mid)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    s0 = dem.lvb.stats()
    torch.cuda.synchronize()
    e0.record(stream)
    dem.advance(DRUM_STEPS)
    e1.record(stream)
    torch.cuda.synchronize()
    _check_rc(lvb, dem.sync())
    s1 = dem.lvb.stats()
    ms = e0.elapsed_time(e1)
    dem.close()
    out["full_step_graph"] = {"value": n * DRUM_STEPS / (ms * 1e-3),
                              "unit": "particle-steps/s (full DEM step)",
                              "ms_per_step": ms / DRUM_STEPS, "steps": DRUM_STEPS,
                              "flagged_per_step": _diff(s0, s1, "flagged_total") / DRUM_STEPS,
                              "entries": s1["entries"]}
    # broad phase alone, phase by phase, each stencil form
    pb_steps = 500
    forms = {}
    for name, reach in (("reach_bounds", 2), ("H_bound_only", 1), ("plain_27_cells", 0)):
        dem = lvb.DEM(mid)
        dem.lvb.set_option(lvb.LVB_OPT_STENCIL_REACH, reach)
        _phases(lvb, torch, dem, 3)
        s0 = dem.lvb.stats()
        ph = _phases(lvb, torch, dem, pb_steps)
        _check_rc(lvb, dem.sync())
        s1 = dem.lvb.stats()
        dem.close()
        b, parts = _bp_bytes(n, pb_steps, s0, s1)
        forms[name] = {"value": n * pb_steps / (ph[1] * 1e-3), "unit": "particle-steps/s",
                       "broad_us_per_step": 1e3 * ph[1] / pb_steps,
                       "flagged_per_step": parts["F"],
                       "stencil_candidates_per_flagged": parts["stencil_candidates_per_flagged"],
                       "roofline": _roofline("k_step (broad phase)", b, ph[1] / pb_steps,
                                             hbm_peak, peak_kind, None, parts)}
        if name == "reach_bounds":
            forms[name]["phases_ms_per_step"] = {"integrate": ph[0] / pb_steps,
                                                 "broad": ph[1] / pb_steps,
                                                 "forces": ph[2] / pb_steps}
    out["broad_phase"] = forms
    out["reach_bounds_speedup_vs_plain"] = (forms["reach_bounds"]["value"] /
                                            forms["plain_27_cells"]["value"])
    # K sweep of the paper's rule (Eq. skin_formulus1), each from the spun-up state
    rows = []
    ks = 1000
    for K in k_sweep:
        dem = lvb.DEM(mid, skin_kind=lvb.LVB_SKIN_PAPER_KVDT, skin_value=float(K))
        _phases(lvb, torch, dem, 3)
        s0 = dem.lvb.stats()
        ph = _phases(lvb, torch, dem, ks)
        _check_rc(lvb, dem.sync())
        s1 = dem.lvb.stats()
        dem.close()
        rows.append({"K": K, "broad_ms": ph[1] / ks, "narrow_forces_ms": ph[2] / ks,
                     "integrate_ms": ph[0] / ks, "step_ms": float(ph.sum()) / ks,
                     "rebuild_fraction": _diff(s0, s1, "updated_total") / (n * ks),
                     "rebuild_step_fraction": _diff(s0, s1, "rebuild_steps") / ks,
                     "entries": s1["entries"]})
    best = min(rows, key=lambda r: r["step_ms"])
    t_none = next((r["step_ms"] for r in rows if r["K"] == 0), None)
    for r in rows:
        if t_none:
            r["improvement_pct_vs_K0"] = (t_none - r["step_ms"]) / t_none * 100.0   # Eq. impr
        r["overhead_vs_best_pct"] = (r["step_ms"] - best["step_ms"]) / best["step_ms"] * 100.0
    out["k_sweep"] = {"steps_each": ks, "rows": rows, "best_K": best["K"],
                      "phases": "phase by phase, no flush (the state exceeds L2)"}
    return out


LEARN_N = 1_000_000
LEARN_H = 400           # horizon of the rebuild-log labels, and K of the paper's rule
LEARN_MARGIN = 2.0      # labels scaled by this margin before training
LEARN_CLIP = 0.99       # labels clipped at this quantile
LEARN_STEPS = 1500      # steps of the logged training run and of each timed run


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
    _check_rc(lvb, dem.sync())
    st = dem.lvb.stats()
    out = {"value": scene.n * steps / (ms * 1e-3), "unit": "particle-steps/s (full DEM step)",
           "updates_per_step": (st["updated_total"] - st0["updated_total"]) / steps,
           "rebuild_steps": st["rebuild_steps"] - st0["rebuild_steps"],
           "mean_entries": float(np.mean(ent)), "relayouts": st["relayouts"]}
    smp = dem.lvb.log_samples() if log else None
    dem.close()
    return out, smp


def _train_skin(lvb, torch, samples, seed):
    """Network weights trained on the GPU on rebuild-log samples for the
    travel form of the output over LEARN_H steps (skin = y LEARN_H |v| dt, a
    per-particle factor of the paper's rule); the library turns the log's
    labels into that form (lvb_mlp_travel_labels).  Returns (device
    weights, info)."""
    smp = lvb.mlp_travel_labels(samples, LEARN_H, LEARN_MARGIN, LEARN_CLIP)
    rng = np.random.default_rng(seed)
    p0 = (rng.standard_normal(lvb.LVB_MLP_PARAMS) * 0.1).astype(np.float32)
    yr = np.zeros(2, np.float32)
    t0 = time.time()
    p, mu, isd, losses = lvb.mlp_train(torch.from_numpy(smp).cuda(), epochs=20, batch=512,
                                       lr=3e-3, seed=seed, params0=p0, y_range_out=yr,
                                       loss_kind=lvb.LVB_MLP_LOSS_SQUARED)
    info = {"samples": int(len(smp)), "epochs": 20, "loss": "squared",
            "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
            "seconds": time.time() - t0, "y_range": [float(yr[0]), float(yr[1])],
            "y_steps": LEARN_H}
    return lvb.mlp_weights_device(p, mu, isd, yr, float(LEARN_H)), info


def _learned(lvb, torch):
    """The learned skin against the paper's rule on a 1,000,000-sphere drum.
    Training: rebuild-log samples of the plain local-buffer run (skin
    0.1 d_i), then of the network's own run, on the GPU by the library's
    kernels, from three initial weight draws.  Selection: the six networks
    are timed on a validation drum (another seed); the fastest there is then
    timed on the benchmark drum against the paper's rule (K = LEARN_H / 2,
    LEARN_H, 2 LEARN_H) and the plain rule, each from the same state."""
    from paper_2208_13770_gb300 import scenes
    bench_sc = scenes.drum(n=LEARN_N, length=0.1)
    val_sc = scenes.drum(n=LEARN_N, length=0.1, seed=scenes.SEED_BASE + 12)
    _, smp = _timed_advance(lvb, torch, val_sc, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, log=LEARN_H)
    cands = []
    for seed in (1, 2, 3):
        w1, info1 = _train_skin(lvb, torch, smp, seed)
        _, smp1 = _timed_advance(lvb, torch, val_sc, lvb.LVB_SKIN_LEARNED, 0.0, mlp=w1,
                                 log=LEARN_H)
        v1, _ = _timed_advance(lvb, torch, val_sc, lvb.LVB_SKIN_LEARNED, 0.0, mlp=w1)
        w2, info2 = _train_skin(lvb, torch, np.concatenate([smp, smp1]), seed + 10)
        v2, _ = _timed_advance(lvb, torch, val_sc, lvb.LVB_SKIN_LEARNED, 0.0, mlp=w2)
        cands += [(v1["value"], seed, 1, w1), (v2["value"], seed, 2, w2)]
    vbest, bseed, bstage, w = max(cands, key=lambda c: c[0])
    learned, _ = _timed_advance(lvb, torch, bench_sc, lvb.LVB_SKIN_LEARNED, 0.0, mlp=w)
    plain, _ = _timed_advance(lvb, torch, bench_sc, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1)
    rules = {}
    for K in (LEARN_H // 2, LEARN_H, 2 * LEARN_H):
        rules["K%d" % K], _ = _timed_advance(lvb, torch, bench_sc, lvb.LVB_SKIN_PAPER_KVDT,
                                             float(K))
    best_rule = max(rules.values(), key=lambda r: r["value"])
    return {
        "workload": "drum R 0.3 m x 0.1 m, %d lognormal spheres (median 1 mm, sigma_ln 0.35), "
                    "10 rpm, dt 1e-6 s, %d steps per run" % (bench_sc.n, LEARN_STEPS),
        "training": {"source": "validation drum (seed +12): plain local buffer (0.1 d_i), then "
                               "the network's own run",
                     "output": "travel form: skin = y * %d |v| dt (y clamped to its range), a "
                               "per-particle K = %d y of the paper's rule" % (LEARN_H, LEARN_H),
                     "label": "largest displacement over the next %d steps / (%d |v| dt), x "
                              "%.1f, clipped at the %.2f quantile (lvb_mlp_travel_labels)"
                              % (LEARN_H, LEARN_H, LEARN_MARGIN, LEARN_CLIP),
                     "selection": "fastest of 3 weight draws x 2 training stages on the "
                                  "validation drum (%.3g particle-steps/s; seed %d, stage %d); "
                                  "timed once on the benchmark drum" % (vbest, bseed, bstage),
                     "last_stage1": info1, "last_stage2": info2},
        "learned": learned, "plain_0.1d": plain, "paper_rule": rules,
        "gain_vs_paper_default_K200": (learned["value"] / rules["K200"]["value"]
                                       if "K200" in rules else None),
        "gain_vs_paper_rule_K%d" % LEARN_H: learned["value"] / rules["K%d" % LEARN_H]["value"],
        "gain_vs_best_paper_rule": learned["value"] / best_rule["value"],
        "gain_vs_plain": learned["value"] / plain["value"],
        "note": "samples come from runs with the rebuild log on; timed runs have it off",
    }


def _friction(lvb, torch):
    """Friction with contact history on the 1,000,000-sphere drum (mu 0.5,
    k_t = 2/7 k_n, gamma_t = 0.5 gamma_n): full DEM steps in graphs with and
    without friction from the same state, and the broad phase alone phase by
    phase with the history on (flagged rows edited in place) and off."""
    from paper_2208_13770_gb300 import scenes
    sc = scenes.drum(n=LEARN_N, length=0.1)
    out = {"workload": "drum R 0.3 m x 0.1 m, %d lognormal spheres, 10 rpm, dt 1e-6 s; "
                       "friction mu 0.5 between particles (walls frictionless)" % sc.n}
    stream = torch.cuda.current_stream()
    for name, mu in (("frictionless", 0.0), ("friction", 0.5)):
        s = sc.copy()
        s.mu = mu
        dem = lvb.DEM(s)
        dem.advance(500)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        dem.advance(1000)
        e1.record(stream)
        torch.cuda.synchronize()
        _check_rc(lvb, dem.sync())
        ms = e0.elapsed_time(e1)
        s0 = dem.lvb.stats()
        ph = _phases(lvb, torch, dem, 300)
        _check_rc(lvb, dem.sync())
        s1 = dem.lvb.stats()
        dem.close()
        out[name] = {"full_step_value": sc.n * 1000 / (ms * 1e-3),
                     "full_step_us": 1e3 * ms / 1000,
                     "unit": "particle-steps/s (full DEM step, graphs)",
                     "broad_us_per_step": 1e3 * ph[1] / 300,
                     "forces_us_per_step": 1e3 * ph[2] / 300,
                     "flagged_per_step": _diff(s0, s1, "flagged_total") / 300}
    out["friction_cost"] = out["frictionless"]["full_step_value"] / out["friction"]["full_step_value"]
    return out


def _clumps(lvb, torch, n=400_000, seed=2208_13770 + 21):
    """The clumps' narrow phase (lvb_clump_contacts) on the bounding-sphere
    list: n rigid clumps of one to four spheres, random orientations, their
    bounding spheres on a jittered lattice at 1.6 median bounding radii (so
    neighbours' bounds overlap); the narrow phase's time per call between
    CUDA events, outputs in device memory (the call includes its input
    checks and two synchronisations)."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 5, size=n)
    off = np.concatenate([[0], np.cumsum(k)]).astype(np.int32)
    m = int(off[-1])
    sub = np.zeros((m, 4), np.float32)
    sub[:, :3] = rng.normal(0, 0.5e-3, size=(m, 3))
    sub[:, 3] = rng.uniform(0.3e-3, 0.8e-3, size=m)
    ext = np.linalg.norm(sub[:, :3].astype(np.float64), axis=1) + sub[:, 3]
    R = np.maximum.reduceat(ext, off[:-1])
    R = (R / (1.0 - 2.0 ** -12) * (1.0 + 1e-6)).astype(np.float32)
    spacing = 1.6 * float(np.median(R))   # neighbours' bounding spheres overlap
    side = int(np.ceil(n ** (1 / 3)))
    idx = rng.permutation(side ** 3)[:n]
    c = np.stack([idx % side, (idx // side) % side, idx // side ** 2], 1) * spacing
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = c + rng.uniform(-0.05, 0.05, size=(n, 3)) * spacing
    pos[:, 3] = R
    q = rng.normal(size=(n, 4))
    q = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    dev = lambda a, t=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", t)
    pad = 2.0 * float(R.max())
    ctx = lvb.LVB(dev(pos), (-pad,) * 3, (side * spacing + pad,) * 3,
                  lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, 1e-5, lvb.LVB_TRIGGER_PARTIAL, 1.25)
    d_pos, d_q, d_off, d_sub = dev(pos), dev(q), dev(off, torch.int32), dev(sub)
    stream = torch.cuda.current_stream()
    contacts = len(ctx.clump_contacts(d_pos, d_q, d_off, d_sub)[0])
    cap = contacts + 1024
    outs = [torch.empty(cap, dtype=torch.int32, device="cuda") for _ in range(4)] + \
        [torch.empty(cap, dtype=torch.float32, device="cuda")]
    calls, ms = 20, 0.0
    for _ in range(3):
        ctx.clump_contacts_into(d_pos, d_q, d_off, d_sub, *outs)
    for _ in range(calls):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        got = ctx.clump_contacts_into(d_pos, d_q, d_off, d_sub, *outs)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        assert got == contacts
    st = ctx.stats()
    ctx.close()
    return {"workload": "%d clumps of 1-4 spheres (%d sub-spheres), bounding spheres on a "
                        "jittered lattice, random orientations" % (n, m),
            "n_clumps": n, "n_spheres": m, "list_pairs": st["pairs"],
            "contacts": contacts, "ms_per_call": ms / calls,
            "clumps_per_s": n / (ms / calls * 1e-3), "unit": "clumps/s (narrow phase)"}


def _ballistic(lvb, torch):
    """The 2,000-sphere ballistic case (r = 1 mm, phi 0.30, specular walls,
    dt 1e-5 s, 1,000 steps): local skin 0.1 d (plain, and with the early
    trigger) against the global skin 0.1 d; the state fits in L2, so this
    is a latency figure."""
    from paper_2208_13770_gb300 import scenes
    sc = scenes.ballistic()
    out = {"workload": "2,000 spheres r 1 mm, phi 0.30, N(0, 0.01 m/s), specular walls, "
                       "dt 1e-5 s, 1,000 steps", "n": sc.n}
    for name, trig, kind, val, early in (
            ("local", lvb.LVB_TRIGGER_PARTIAL, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, 1000),
            ("local_early", lvb.LVB_TRIGGER_PARTIAL, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1,
             EARLY_PERMILLE),
            ("global_buffer", lvb.LVB_TRIGGER_GLOBAL, lvb.LVB_SKIN_GLOBAL, 0.2e-3, 1000)):
        dem = lvb.DEM(sc, trigger=trig, skin_kind=kind, skin_value=val)
        if early < 1000:
            dem.lvb.set_option(lvb.LVB_OPT_EARLY, early)
        s0 = dem.lvb.stats()
        ph = _phases(lvb, torch, dem, sc.steps)
        _check_rc(lvb, dem.sync())
        s1 = dem.lvb.stats()
        dem.close()
        out[name] = {"broad_us_per_step": 1e3 * ph[1] / sc.steps,
                     "value": sc.n * sc.steps / (ph[1] * 1e-3), "unit": "particle-steps/s",
                     "updated_total": _diff(s0, s1, "updated_total"),
                     "rebuild_steps": _diff(s0, s1, "rebuild_steps")}
    return out


# ----------------------------------------------------------------- arms
def run_native(args):
    import torch
    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2208_13770_gb300 import lvb, replicas
    hbm_peak, peak_kind = _peaks()
    sc = _batch_scenes(rank, world)
    if args.only_batched and args.scenes:
        sc = sc[:args.scenes]
    n = int(sum(q.n for q in sc))
    K, W = args.steps, args.warmup
    if args.only_batched:
        from paper_2208_13770_gb300 import autotune
        ch = autotune.Choice()
        if args.choice:
            f = args.choice.split(",")
            ch = autotune.Choice(float(f[0]), int(f[1]), int(f[2]),
                                 int(f[3]) if len(f) > 3 else 1)
        res = _headline(lvb, torch, sc, ch, K, W, record=False, profile=args.profile)
        if rank == 0:
            ph = res["phase_ms"] / K
            print(json.dumps({"only_batched": True, "n": n, "phases_ms_per_step": list(ph),
                              "value": n * K / (res["phase_ms"][1] * 1e-3),
                              "window": "steps %d..%d" % (T0 + 1, T0 + K),
                              "flagged_per_step": _diff(res["stats0"], res["stats1"],
                                                        "flagged_total") / K}))
        return 0
    choice, trials = _tune(lvb, torch, sc)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        res = _headline(lvb, torch, sc, choice, K, W, record=(rank == 0))
    torch.cuda.synchronize()
    bp_ms, step_ms = replicas.max_over_ranks([float(res["phase_ms"][1]),
                                              float(res["phase_ms"].sum())], device="cuda")
    n_all = n
    if world > 1:
        t = torch.tensor([float(n)], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t)
        n_all = int(t.item())
    value = n_all * K / (bp_ms * 1e-3)
    if rank != 0:
        torch.distributed.barrier()
        return 0
    s0, s1 = res["stats0"], res["stats1"]
    ph = res["phase_ms"] / K
    b, parts = _bp_bytes(n, K, s0, s1)
    roof = _roofline("k_step (broad phase: displacement check + partial rebuild)", b, ph[1],
                     hbm_peak, peak_kind, NCU_TRAFFIC_BATCHED, parts)
    e2e = _e2e_batch(lvb, torch, sc, choice, res["rec"])
    e2e["value"] *= world
    cpu = None if args.no_cpu_baseline else _cpu_baseline(sc, res["rec"])
    extras = {}
    if not args.no_extras:
        extras["settling_200k"] = _settling(lvb, torch, SETTLING_STEPS, W, hbm_peak, peak_kind)
        extras["drum_2M"] = _drum(lvb, torch, hbm_peak, peak_kind)
        extras["ballistic_2k"] = _ballistic(lvb, torch)
        extras["friction_1M"] = _friction(lvb, torch)
        extras["clumps_400k"] = _clumps(lvb, torch)
        if not args.no_learned:
            extras["learned"] = _learned(lvb, torch)
    line = {
        "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": step_ms / K,
        "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n_all, "n_scenes": 512,
                   "window": "steps %d..%d (after %d untimed steps and %d warm-up steps)"
                             % (T0 + 1, T0 + K, T0 - W, W),
                   "dt": sc[0].dt, "skin": "0.1 d_i", "trigger": "partial (local buffer)",
                   "l2": "inputs (%.0f MB of particle state) exceed L2; no flush"
                         % (n * 96 / 1e6),
                   "parallelism": ("scenes sharded over %d ranks (greedy by N)" % world)
                   if world > 1 else "single",
                   "autotuned": {"cell_factor": choice.cell_factor,
                                 "block_threads": choice.block_threads,
                                 "compaction": choice.compaction,
                                 "check_loads": "registers" if choice.check_loads else
                                                "bulk-copy ring"}},
        "roofline": roof,
        "flagged_per_step": parts["F"],
        "rebuild_fraction": _diff(s0, s1, "updated_total") / (n * K),
        "rebuild_step_fraction": _diff(s0, s1, "rebuild_steps") / K,
        "phases_ms_per_step": {"integrate": ph[0], "broad": ph[1], "forces": ph[2]},
        "narrow_phase": _narrow_phase(n, s1["entries"], ph[2], hbm_peak),
        "full_step_particle_steps_per_s": n_all * K / (step_ms * 1e-3),
        "list": {"entries": s1["entries"], "mean_row": s1["entries"] / n,
                 "relayouts": _diff(s0, s1, "relayouts")},
        "e2e": e2e,
        "gpu_launches": int(_diff(s0, s1, "kernels_executed")),
        "grid_barriers": int(_diff(s0, s1, "barriers")),
        "step_kernel": {"blocks": s1["step_blocks"], "threads": s1["block_threads"],
                        "launch": "cooperative, one per broad-phase step"},
        "autotune_trials": trials,
        "clocks": clk.summary(),
    }
    if "settling_200k" in extras:
        line["speedup_vs_global"] = extras["settling_200k"]["speedup_vs_global"]["local"]
        line["speedup_vs_global_early"] = \
            extras["settling_200k"]["speedup_vs_global"]["local_early"]
    if cpu is not None:
        line["cpu_baseline"] = cpu
    line.update(extras)
    print(json.dumps(line))
    if world > 1:
        torch.distributed.barrier()
    return 0


def _ref_trajectory(scene, steps, threads):
    """The oracle's own binary64 DEM (orc_dem_step64, velocity Verlet with
    the linear spring-dashpot law) from the scene's seeded initial state,
    and the broad phase's reference state carried along by the oracle's
    flag and skin rules at every step (Eq. update, partial trigger) without
    list builds.  Returns (positions at `steps` as float32 records,
    reference state there, the state (x, v, a) for continuing)."""
    import oracle
    oracle.set_threads(threads)
    P = oracle.dem_params(kn=scene.kn, restitution=scene.restitution, rho=scene.rho,
                          g=scene.gravity, lo=scene.lo, hi=scene.hi, wall_kind=oracle.WALL_BOX)
    r = scene.pos[:, 3].astype(np.float64)
    x = scene.pos[:, :3].astype(np.float64)
    v = scene.vel[:, :3].astype(np.float64)
    a = np.zeros_like(x)
    H = _ref_H(scene)
    p32 = scene.pos.copy()
    ref = p32.copy()
    ref[:, 3] = oracle.skin(scene.skin_kind, scene.skin_value, scene.dt, H, p32)
    for _ in range(steps):
        x, v, a = _ref_dem_step(oracle, x, v, a, r, scene.dt, P)
        p32[:, :3] = x.astype(np.float32)
        f = oracle.flags(p32, ref)
        if f.any():
            ref[f, :3] = p32[f, :3]
            ref[f, 3] = oracle.skin(scene.skin_kind, scene.skin_value, scene.dt, H, p32[f])
    return p32, ref, (x, v, a, r, P, H)


def _ref_dem_step(oracle, x, v, a, r, dt, P):
    xn, _, an, vn = oracle.dem_step64(x, v, a, r, dt, P)
    return xn, vn, an


def _ref_H(scene):
    rmax = float(np.float32(scene.pos[:, 3].max()))
    L = scene.cell_factor * 2.0 * rmax * (1 + 2 ** -7)
    return np.float32(0.5 * L * (1 - 2 ** -8))


def run_reference(args):
    """The reference arm: the CPU oracle (all host cores) on the headline's
    window.  A sample of the batch's scenes (in scene order, those of more
    than 4,096 particles, about REF_SAMPLE_N particles) is advanced to step
    T0 by the oracle's own binary64 DEM (untimed), then through the warm-up
    and the K window steps, the oracle's broad phase (flags, skins, pair set
    by linked cells) timed at each."""
    rank, world, local = _dist()
    if rank != 0:
        return 0
    import oracle
    from oracle.statemachine import OracleLVB
    from paper_2208_13770_gb300 import scenes
    sc = scenes.batch()
    sample = []
    for q, s in enumerate(sc):
        if s.n > 4096:
            sample.append(q)
            if sum(sc[k].n for k in sample) >= REF_SAMPLE_N:
                break
    K, W = args.steps, args.warmup
    oracle.set_threads(0)
    cores = oracle.threads()
    el, ps = 0.0, 0
    for q in sample:
        s = sc[q]
        p32, ref, (x, v, a, r, P, H) = _ref_trajectory(s, T0 - W, 0)
        sm = OracleLVB(p32, s.skin_kind, s.skin_value, s.dt, H, ref4=ref)
        for k in range(W + K):
            x, v, a = _ref_dem_step(oracle, x, v, a, r, s.dt, P)
            p32[:, :3] = x.astype(np.float32)
            t = time.perf_counter()
            sm.step(p32)
            d = time.perf_counter() - t
            if k >= W:
                el += d
                ps += s.n
    value = ps / el
    nsamp = sum(sc[q].n for q in sample)
    sample_txt = ("oracle broad phase (flags, skins, pair set by linked cells; OpenMP, %d "
                  "threads) on scenes %s of the batch (%d particles), steps %d..%d; states from "
                  "the oracle's own binary64 DEM from the seeded start (untimed)"
                  % (cores, sample, nsamp, T0 + 1, T0 + K))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s",
            "n_gpus": args.gpus, "steps": K, "warmup": W,
            "ms_per_step": 1e3 * el / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": int(sum(q.n for q in sc)), "n_scenes": 512,
                       "window": "steps %d..%d" % (T0 + 1, T0 + K)},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": cores,
                             "kind": "oracle", "sample": sample_txt, "host": _cpu_info()},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_k_sweep(args):
    """K sweep of the paper's rule on the 2M drum alone (and the stencil
    comparison), printed as one JSON line."""
    import torch
    from paper_2208_13770_gb300 import lvb
    hbm_peak, peak_kind = _peaks()
    ks = tuple(int(k) for k in args.k_sweep.split(","))
    print(json.dumps({"drum_2M": _drum(lvb, torch, hbm_peak, peak_kind, k_sweep=ks)}))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only (no 200k box, 2M drum, learned skin, ballistic case)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-skin comparison (1M-sphere drum)")
    ap.add_argument("--only-batched", action="store_true",
                    help="time the headline window alone, default launch choice, no e2e or "
                         "CPU leg (for profiling)")
    ap.add_argument("--scenes", type=int, default=0,
                    help="with --only-batched: the first S scenes of the batch only (a smaller "
                         "case of the same kernel, for profiling)")
    ap.add_argument("--choice", default="",
                    help="with --only-batched: launch choice 'cell_factor,block_threads,"
                         "compaction' (default 1.25,1024,0)")
    ap.add_argument("--profile", action="store_true",
                    help="with --only-batched: bracket the timed steps with "
                         "cudaProfilerStart/Stop (for ncu --profile-from-start off)")
    ap.add_argument("--k-sweep", default="",
                    help="comma-separated K values: the paper's skin rule K |v| dt on the "
                         "2M drum (and the stencil comparison), then exit")
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
