"""Autotuner for the batched DEM step: cell-size factor, block shape of the
step kernel, the compaction scheme of the flagged ids (one atomic per warp
chunk, or one per block tile), and how the broad phase's check reads its
inputs (register loads or a ring of bulk copies).

Each candidate is a fresh context on the same batch from the same initial
state; it runs ``warm`` steps (graph replays of DEM_GRAPH_STEPS steps), then
``steps`` steps phase by phase, the broad phase of each between CUDA events
on the context's stream: the tuner minimises the broad phase's time.  The
search is coordinate-wise: the cell factor first (it changes the grid, so a
new context), then the block shape, then the compaction scheme, each on
the best of the previous ones.  The block shape, the compaction scheme and
the check's loads are launch choices only: the lists do not change.  The cell factor also sets
the cap on every skin (R_NL <= half a cell edge, Eq.
skin_formulus_mincell), so at 1.0 the largest particles get smaller skins
and update more often; the lists change with the skins, but no contact is
ever missed (Theorem 1 holds for any skin).
"""
from __future__ import annotations

import dataclasses
import json
import os

CELL_FACTORS = (1.0, 1.25, 1.5)
BLOCK_THREADS = (1024, 512, 256)
COMPACTION = (0, 1)   # LVB_COMPACT_WARP, LVB_COMPACT_BLOCK
CHECK_LOADS = (1, 0)  # LVB_CHECK_REGS, LVB_CHECK_RING


@dataclasses.dataclass
class Choice:
    cell_factor: float = 1.25
    block_threads: int = 1024
    compaction: int = 0
    check_loads: int = 1

    def apply(self, dem, lvb):
        dem.lvb.set_option(lvb.LVB_OPT_BLOCK_THREADS, self.block_threads)
        dem.lvb.set_option(lvb.LVB_OPT_COMPACT, self.compaction)
        dem.lvb.set_option(lvb.LVB_OPT_CHECK_LOADS, self.check_loads)


def _trial(torch, lvb, scene_list, choice, warm, steps):
    """Broad-phase time per step of one candidate: `warm` steps of the DEM
    driver (graphs), then `steps` steps phase by phase with CUDA events
    around each broad-phase launch (the quantity the candidates differ in:
    the cell factor changes the grid and the skins' cap, the other choices
    the broad phase's launch)."""
    dem = lvb.DEM(scene_list, cell_factor=choice.cell_factor)
    try:
        choice.apply(dem, lvb)
        dem.advance(warm)
        stream = torch.cuda.current_stream()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize()
        for e0, e1 in evs:
            dem.phase(lvb.DEM_PHASE_INTEGRATE)
            e0.record(stream)
            dem.phase(lvb.DEM_PHASE_BROAD)
            e1.record(stream)
            dem.phase(lvb.DEM_PHASE_FORCES)
        torch.cuda.synchronize()
        rc = dem.sync()
        if rc != 0:
            raise RuntimeError("device error %d: %s" % (rc, lvb.lvb_strerror(rc)))
        return sum(e0.elapsed_time(e1) for e0, e1 in evs) / steps
    finally:
        dem.close()


def _cache_path():
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "lvb_autotune.json")


def cache_key(kind, n, gpu_name):
    """(scene kind, particle-count bucket (powers of two), GPU name)."""
    return "%s|n2^%d|%s" % (kind, max(0, int(n) - 1).bit_length(), gpu_name)


def _cache_load():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _cache_store(key, choice, trials):
    d = _cache_load()
    d[key] = {"choice": dataclasses.asdict(choice), "trials": trials}
    try:
        os.makedirs(os.path.dirname(_cache_path()), exist_ok=True)
        tmp = _cache_path() + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(d, f)
        os.replace(tmp, _cache_path())
    except OSError:
        pass


def tune(scene_list, warm=200, steps=400, key=None):
    """Returns (best Choice, list of trials {choice fields, ms_per_step of
    the broad phase}).
    With key (a scene kind), the choice is looked up in a per-user cache
    under (kind, particle-count bucket, GPU name) and stored there after a
    search, so that a second run on the same kind of workload and GPU skips
    the search (its trials list is then the cached one)."""
    import torch
    from . import lvb
    trials = []
    ck = None
    if key is not None:
        ck = cache_key(key, sum(q.n for q in scene_list), torch.cuda.get_device_name())
        hit = _cache_load().get(ck)
        if hit is not None:
            return Choice(**hit["choice"]), hit["trials"]

    def run(choice):
        ms = _trial(torch, lvb, scene_list, choice, warm, steps)
        trials.append(dict(dataclasses.asdict(choice), ms_per_step=ms))
        return ms

    best = Choice()
    best_ms = None
    for cf in CELL_FACTORS:
        c = dataclasses.replace(best, cell_factor=cf)
        ms = run(c)
        if best_ms is None or ms < best_ms:
            best, best_ms = c, ms
    base = best
    for ct in BLOCK_THREADS:
        if ct == base.block_threads:
            continue
        c = dataclasses.replace(base, block_threads=ct)
        ms = run(c)
        if ms < best_ms:
            best, best_ms = c, ms
    base = best
    for cp in COMPACTION:
        if cp == base.compaction:
            continue
        c = dataclasses.replace(base, compaction=cp)
        ms = run(c)
        if ms < best_ms:
            best, best_ms = c, ms
    base = best
    for ck in CHECK_LOADS:
        if ck == base.check_loads:
            continue
        c = dataclasses.replace(base, check_loads=ck)
        ms = run(c)
        if ms < best_ms:
            best, best_ms = c, ms
    if ck is not None:
        _cache_store(ck, best, trials)
    return best, trials
