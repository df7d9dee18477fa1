"""ctypes binding of liblvb (include/lvb.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes
device pointers (``tensor.data_ptr()``), sizes and the CUDA stream handle
straight through; every step of the broad phase runs in the library's CUDA
kernels.  Importing this module loads ``liblvb.so`` and raises ImportError
if it has not been built -- there is no fallback.

``LVB`` is a small convenience wrapper over one context that allocates the
host output arrays of the lvb_get_* calls.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblvb.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError("liblvb.so is not built; run `python -m paper_2208_13770_gb300.build` "
                      "(needs nvcc) -- the broad phase has no CPU fallback")
_lib = ctypes.CDLL(_LIB_PATH)

LVB_OK, LVB_EINVAL, LVB_ENOMEM, LVB_ECAPACITY, LVB_EDEVICE, LVB_ENAN, LVB_EOVERFLOW, \
    LVB_ESTATE, LVB_ELIMIT, LVB_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
LVB_NOALLOC_MAX_N = 65536
LVB_SKIN_GLOBAL, LVB_SKIN_DIAMETER_FACTOR, LVB_SKIN_PAPER_KVDT, LVB_SKIN_LEARNED = 0, 1, 2, 3
LVB_TRIGGER_PARTIAL, LVB_TRIGGER_GLOBAL, LVB_TRIGGER_ALWAYS = 0, 1, 2


class lvb_skin_policy(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("value", ctypes.c_float), ("dt", ctypes.c_float),
                ("mlp", ctypes.c_void_p)]


class lvb_box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3)]


class lvb_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in
                ("n", "steps", "rebuild_steps", "flagged_total", "updated_total", "last_flagged",
                 "entries", "pairs", "relayouts", "grows", "cell_capacity", "row_store_capacity",
                 "kernels_executed", "barriers", "step_blocks", "block_threads", "compaction",
                 "n_scenes", "rebuild_candidates", "rebuild_direct", "rebuild_edits")] + \
               [("reserved", ctypes.c_int64 * 1)] + \
               [("cell_edge", ctypes.c_float), ("rnl_max", ctypes.c_float),
                ("grid", ctypes.c_int32 * 3), ("pad", ctypes.c_int32)]


class lvb_scene_info_t(ctypes.Structure):
    _fields_ = [("first", ctypes.c_int64), ("count", ctypes.c_int64),
                ("cell_edge", ctypes.c_float), ("rnl_max", ctypes.c_float),
                ("grid", ctypes.c_int32 * 3), ("pad", ctypes.c_int32)]


class dem_params(ctypes.Structure):
    _fields_ = [("kn", ctypes.c_float), ("restitution", ctypes.c_float), ("rho", ctypes.c_float),
                ("g", ctypes.c_float * 3), ("wall_kind", ctypes.c_int32),
                ("clamp_tensile", ctypes.c_int32), ("drum_cx", ctypes.c_float),
                ("drum_cz", ctypes.c_float), ("drum_R", ctypes.c_float),
                ("drum_omega", ctypes.c_float), ("contacts_on", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("mu", ctypes.c_float), ("kt_ratio", ctypes.c_float),
                ("gt_ratio", ctypes.c_float), ("pad2", ctypes.c_int32)]


DEM_WALL_NONE, DEM_WALL_BOX, DEM_WALL_DRUM, DEM_WALL_SPECULAR = 0, 1, 2, 3
DEM_PHASE_INTEGRATE, DEM_PHASE_BROAD, DEM_PHASE_FORCES = 0, 1, 2

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_pi64 = ctypes.POINTER(ctypes.c_int64)
_SIGS = {
    "lvb_init": ([ctypes.POINTER(_p), _i64, _p, ctypes.POINTER(lvb_box),
                  ctypes.POINTER(lvb_skin_policy), ctypes.c_int32, ctypes.c_float, _p, _p, _p],
                 ctypes.c_int),
    "lvb_batch_init": ([ctypes.POINTER(_p), ctypes.c_int32, _p, _p, ctypes.POINTER(lvb_box),
                        ctypes.POINTER(lvb_skin_policy), ctypes.c_int32, ctypes.c_float, _p, _p,
                        _p], ctypes.c_int),
    "lvb_scene_info": ([_p, ctypes.c_int32, ctypes.POINTER(lvb_scene_info_t)], ctypes.c_int),
    "lvb_init_resume": ([ctypes.POINTER(_p), _i64, _p, _p, ctypes.POINTER(lvb_box),
                         ctypes.POINTER(lvb_skin_policy), ctypes.c_int32, ctypes.c_float, _p, _p,
                         _p], ctypes.c_int),
    "lvb_batch_init_resume": ([ctypes.POINTER(_p), ctypes.c_int32, _p, _p, _p,
                               ctypes.POINTER(lvb_box), ctypes.POINTER(lvb_skin_policy),
                               ctypes.c_int32, ctypes.c_float, _p, _p, _p], ctypes.c_int),
    "lvb_step": ([_p, _p, _p, _p], ctypes.c_int),
    "lvb_step_host": ([_p, _p, _p, _p, _p, _p], ctypes.c_int),
    "lvb_sync": ([_p], ctypes.c_int),
    "lvb_set_option": ([_p, ctypes.c_int32, _i64], ctypes.c_int),
    "lvb_trace": ([_p, _p, _p], ctypes.c_int),
    "lvb_get_pairs": ([_p, _p, _p, _i64, _pi64], ctypes.c_int),
    "lvb_get_pairs_ij": ([_p, _p, _p, _i64, _pi64], ctypes.c_int),
    "lvb_get_near_cutoff": ([_p, ctypes.c_double, _p, _p, _i64, _pi64], ctypes.c_int),
    "lvb_get_contacts": ([_p, _p, _p, _p, _p, _i64, _pi64], ctypes.c_int),
    "lvb_get_flags": ([_p, _p, _pi64], ctypes.c_int),
    "lvb_get_ref": ([_p, _p], ctypes.c_int),
    "lvb_stats": ([_p, ctypes.POINTER(lvb_stats_t)], ctypes.c_int),
    "lvb_set_stream": ([_p, _p], ctypes.c_int),
    "lvb_destroy": ([_p], ctypes.c_int),
    "lvb_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "lvb_mlp_pack": ([_p, _p, _p, _p, ctypes.c_float, _p], ctypes.c_int),
    "lvb_mlp_infer": ([_p, _p, _i64, _p, _p, _p, _p], ctypes.c_int),
    "lvb_mlp_grad": ([_p, _i64, _p, _p, _p, ctypes.c_float, _p, ctypes.POINTER(ctypes.c_double),
                      _p], ctypes.c_int),
    "lvb_mlp_train": ([_p, _i64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_uint64,
                       ctypes.c_int32, _p, _p, _p, _p, _p, _p], ctypes.c_int),
    "lvb_mlp_travel_labels": ([_p, _i64, ctypes.c_int32, ctypes.c_float, ctypes.c_float, _p,
                               _pi64, _p], ctypes.c_int),
    "lvb_log_enable": ([_p, ctypes.c_int32, _i64], ctypes.c_int),
    "lvb_log_read": ([_p, _p, _i64, _pi64], ctypes.c_int),
    "lvb_pairs_noalloc": ([_i64, _p, _p, ctypes.POINTER(lvb_box), _p, _p, _i64, _pi64, _p],
                          ctypes.c_int),
    "lvb_clump_contacts": ([_p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _i64, _pi64], ctypes.c_int),
    "dem_init": ([ctypes.POINTER(_p), _i64, _p, _p, ctypes.POINTER(dem_params), ctypes.c_float,
                  ctypes.POINTER(lvb_box), ctypes.POINTER(lvb_skin_policy), ctypes.c_int32,
                  ctypes.c_float, _p], ctypes.c_int),
    "dem_batch_init": ([ctypes.POINTER(_p), ctypes.c_int32, _p, _p, _p, ctypes.POINTER(dem_params),
                        ctypes.c_float, ctypes.POINTER(lvb_box), ctypes.POINTER(lvb_skin_policy),
                        ctypes.c_int32, ctypes.c_float, _p], ctypes.c_int),
    "dem_advance": ([_p, _i64], ctypes.c_int),
    "dem_phase": ([_p, ctypes.c_int32], ctypes.c_int),
    "dem_get_state": ([_p, _p, _p, _p, _p], ctypes.c_int),
    "dem_set_state": ([_p, _p, _p, _p], ctypes.c_int),
    "dem_get_contact_forces": ([_p, _p, _p, _p, _p, _i64, _pi64], ctypes.c_int),
    "dem_get_contact_history": ([_p, ctypes.c_int32, _p, _p, _p, _p, _p, _i64, _pi64],
                                ctypes.c_int),
    "dem_get_rot_state": ([_p, _p, _p, _p], ctypes.c_int),
    "dem_lvb": ([_p, ctypes.POINTER(_p)], ctypes.c_int),
    "dem_device_state": ([_p, ctypes.POINTER(_p), ctypes.POINTER(_p), ctypes.POINTER(_p),
                          ctypes.POINTER(_p)], ctypes.c_int),
    "dem_sync": ([_p], ctypes.c_int),
    "dem_destroy": ([_p], ctypes.c_int),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = sorted(k for k in _SIGS if k.startswith("lvb_"))
EXPORTED_DEM = sorted(k for k in _SIGS if k.startswith("dem_"))


class LVBError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, lvb_strerror(code), code))


def _check(rc, what):
    if rc != LVB_OK:
        raise LVBError(rc, what)
    return rc


def lvb_strerror(code: int) -> str:
    return _lib.lvb_strerror(int(code)).decode()


def lvb_init(n, pos_r, box, skin, trigger, cell_factor, vel=None, acc=None, stream=None):
    ctx = _p()
    rc = _lib.lvb_init(ctypes.byref(ctx), int(n), pos_r, ctypes.byref(box), ctypes.byref(skin),
                       int(trigger), float(cell_factor), vel, acc, stream)
    _check(rc, "lvb_init")
    return ctx


def lvb_batch_init(n_scenes, offsets, pos_r, boxes, skin, trigger, cell_factor, vel=None,
                   acc=None, stream=None):
    """offsets: host int64 array (n_scenes + 1); boxes: ctypes array of lvb_box."""
    ctx = _p()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    rc = _lib.lvb_batch_init(ctypes.byref(ctx), int(n_scenes), off.ctypes.data, pos_r, boxes,
                             ctypes.byref(skin), int(trigger), float(cell_factor), vel, acc,
                             stream)
    _check(rc, "lvb_batch_init")
    return ctx


def lvb_scene_info(ctx, scene, out):
    return _lib.lvb_scene_info(ctx, int(scene), out)


def lvb_init_resume(n, pos_r, ref4, box, skin, trigger, cell_factor, vel=None, acc=None,
                    stream=None):
    ctx = _p()
    rc = _lib.lvb_init_resume(ctypes.byref(ctx), int(n), pos_r, ref4, ctypes.byref(box),
                              ctypes.byref(skin), int(trigger), float(cell_factor), vel, acc,
                              stream)
    _check(rc, "lvb_init_resume")
    return ctx


def lvb_batch_init_resume(n_scenes, offsets, pos_r, ref4, boxes, skin, trigger, cell_factor,
                          vel=None, acc=None, stream=None):
    ctx = _p()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    rc = _lib.lvb_batch_init_resume(ctypes.byref(ctx), int(n_scenes), off.ctypes.data, pos_r,
                                    ref4, boxes, ctypes.byref(skin), int(trigger),
                                    float(cell_factor), vel, acc, stream)
    _check(rc, "lvb_batch_init_resume")
    return ctx


def lvb_step(ctx, pos_r, vel=None, acc=None):
    return _lib.lvb_step(ctx, pos_r, vel, acc)


def lvb_step_host(ctx, pos_r, vel=None, acc=None, bits=None, n_flagged=None):
    """Host pointers (ints); see include/lvb.h."""
    return _lib.lvb_step_host(ctx, pos_r, vel, acc, bits, n_flagged)


LVB_OPT_TRACE, LVB_OPT_BLOCK_THREADS, LVB_OPT_COMPACT = 3, 4, 5
LVB_OPT_BARRIER_EXTRA, LVB_OPT_BARRIER_SPINS = 6, 7
LVB_OPT_DIRECT_MAX = 8
LVB_OPT_STENCIL_REACH = 9
LVB_OPT_GROW = 10
LVB_OPT_STORE_LIMIT = 11
LVB_OPT_CELL_CAPACITY = 12
LVB_OPT_HISTORY = 13
LVB_OPT_FORCE_RELAYOUT = 14
LVB_OPT_CHECK_LOADS = 15
LVB_OPT_EARLY = 16
LVB_CHECK_RING, LVB_CHECK_REGS = 0, 1
LVB_COMPACT_WARP, LVB_COMPACT_BLOCK = 0, 1
TRACE_SLOTS = ["check", "rebuild", "relayout", "tail_forces", "integrate", "forces", "rows",
               "rebuild_items", "rebuild_item_max"]


def lvb_trace(ctx, sum_ns, count):
    return _lib.lvb_trace(ctx, sum_ns, count)


def lvb_set_option(ctx, option, value):
    return _lib.lvb_set_option(ctx, int(option), int(value))


def lvb_sync(ctx):
    return _lib.lvb_sync(ctx)


def lvb_get_pairs(ctx, row_ptr, col, cap, n_entries):
    return _lib.lvb_get_pairs(ctx, row_ptr, col, cap, n_entries)


def lvb_get_pairs_ij(ctx, pi, pj, cap, n_pairs):
    return _lib.lvb_get_pairs_ij(ctx, pi, pj, cap, n_pairs)


def lvb_get_contacts(ctx, pos_r, ci, cj, delta, cap, n_contacts):
    return _lib.lvb_get_contacts(ctx, pos_r, ci, cj, delta, cap, n_contacts)


def lvb_get_flags(ctx, bits, n_flagged):
    return _lib.lvb_get_flags(ctx, bits, n_flagged)


def lvb_get_ref(ctx, ref4):
    return _lib.lvb_get_ref(ctx, ref4)


def lvb_stats(ctx, out):
    return _lib.lvb_stats(ctx, out)


def lvb_set_stream(ctx, stream):
    return _lib.lvb_set_stream(ctx, stream)


def lvb_destroy(ctx):
    return _lib.lvb_destroy(ctx)


def dem_init(n, pos_r, vel, prm, dt, box, skin, trigger, cell_factor, stream=None):
    ctx = _p()
    rc = _lib.dem_init(ctypes.byref(ctx), int(n), pos_r, vel, ctypes.byref(prm), float(dt),
                       ctypes.byref(box), ctypes.byref(skin), int(trigger), float(cell_factor),
                       stream)
    _check(rc, "dem_init")
    return ctx


def dem_batch_init(n_scenes, offsets, pos_r, vel, prm, dt, boxes, skin, trigger, cell_factor,
                   stream=None):
    ctx = _p()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    rc = _lib.dem_batch_init(ctypes.byref(ctx), int(n_scenes), off.ctypes.data, pos_r, vel,
                             ctypes.byref(prm), float(dt), boxes, ctypes.byref(skin),
                             int(trigger), float(cell_factor), stream)
    _check(rc, "dem_batch_init")
    return ctx


def dem_advance(ctx, steps):
    return _lib.dem_advance(ctx, int(steps))


def dem_phase(ctx, phase):
    return _lib.dem_phase(ctx, int(phase))


def dem_get_state(ctx, pos_r, vel, acc, vstar):
    return _lib.dem_get_state(ctx, pos_r, vel, acc, vstar)


def dem_set_state(ctx, pos_r, vel, acc):
    return _lib.dem_set_state(ctx, pos_r, vel, acc)


def dem_lvb(ctx):
    out = _p()
    _check(_lib.dem_lvb(ctx, ctypes.byref(out)), "dem_lvb")
    return out


def dem_device_state(ctx):
    ptrs = [_p() for _ in range(4)]
    _check(_lib.dem_device_state(ctx, *[ctypes.byref(q) for q in ptrs]), "dem_device_state")
    return [q.value for q in ptrs]


def dem_sync(ctx):
    return _lib.dem_sync(ctx)


def dem_destroy(ctx):
    return _lib.dem_destroy(ctx)


LVB_MLP_IN, LVB_MLP_HIDDEN, LVB_MLP_PARAMS = 8, 32, 1377
LVB_MLP_LOSS_SQUARED, LVB_MLP_LOSS_RELATIVE = 0, 1
MLP_WEIGHTS_BYTES = 4 * (32 * 8 + 32 + 32 * 32 + 32 + 32 + 1 + 8 + 8 + 3)


def lvb_mlp_pack(params, mu, isd, y_range, y_steps, out):
    return _lib.lvb_mlp_pack(params, mu, isd, y_range, y_steps, out)


def lvb_mlp_infer(feats, diam, n, w, skin, y, stream=None):
    return _lib.lvb_mlp_infer(feats, diam, int(n), w, skin, y, stream)


def lvb_mlp_grad(samples, n, params, mu, isd, rel_floor, grad, loss, stream=None):
    return _lib.lvb_mlp_grad(samples, int(n), params, mu, isd, float(rel_floor), grad, loss,
                             stream)


def lvb_mlp_train(samples, n, epochs, batch, lr, seed, loss_kind, params, mu, isd, y_range,
                  losses, stream=None):
    return _lib.lvb_mlp_train(samples, int(n), int(epochs), int(batch), float(lr), int(seed),
                              int(loss_kind), params, mu, isd, y_range, losses, stream)


def lvb_mlp_travel_labels(samples, n, horizon, margin, clip_q, out, n_out, stream=None):
    return _lib.lvb_mlp_travel_labels(samples, int(n), int(horizon), float(margin),
                                      float(clip_q), out, n_out, stream)


def lvb_log_enable(ctx, horizon, capacity):
    return _lib.lvb_log_enable(ctx, int(horizon), int(capacity))


def lvb_log_read(ctx, samples, cap, n_samples):
    return _lib.lvb_log_read(ctx, samples, int(cap), n_samples)


def lvb_pairs_noalloc(n, pos4, ref4, box, pi, pj, cap, n_pairs, stream=None):
    return _lib.lvb_pairs_noalloc(int(n), pos4, ref4, box, pi, pj, int(cap), n_pairs, stream)


def _np_ptr(a):
    return a.ctypes.data_as(_p)


def _dptr(t):
    """Device pointer of a torch tensor (or an int/None passed through)."""
    if t is None or isinstance(t, int):
        return t
    return t.data_ptr()


class LVB:
    """One broad-phase context over device tensors of float4 records."""

    def __init__(self, pos, box_lo, box_hi, skin_kind=LVB_SKIN_DIAMETER_FACTOR, skin_value=0.1,
                 dt=0.0, trigger=LVB_TRIGGER_PARTIAL, cell_factor=1.25, vel=None, acc=None,
                 stream=None, ref=None, offsets=None, mlp=None):
        """One scene (box_lo/box_hi: 3 floats), or several independent scenes
        when offsets (n_scenes + 1 particle offsets) is given and box_lo /
        box_hi hold one corner per scene."""
        import torch
        self.n = int(pos.shape[0])
        self._mlp = mlp            # keeps the weights alive with the context
        skin = lvb_skin_policy(int(skin_kind), float(skin_value), float(dt), _dptr(mlp))
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        if offsets is not None:
            ns = len(offsets) - 1
            boxes = (lvb_box * ns)()
            for q in range(ns):
                for k in range(3):
                    boxes[q].lo[k], boxes[q].hi[k] = float(box_lo[q][k]), float(box_hi[q][k])
            if ref is None:
                self.ctx = lvb_batch_init(ns, offsets, _dptr(pos), boxes, skin, trigger,
                                          cell_factor, _dptr(vel), _dptr(acc), stream)
            else:
                self.ctx = lvb_batch_init_resume(ns, offsets, _dptr(pos), _dptr(ref), boxes, skin,
                                                 trigger, cell_factor, _dptr(vel), _dptr(acc),
                                                 stream)
            return
        box = lvb_box()
        for k in range(3):
            box.lo[k], box.hi[k] = float(box_lo[k]), float(box_hi[k])
        if ref is None:
            self.ctx = lvb_init(self.n, _dptr(pos), box, skin, trigger, cell_factor, _dptr(vel),
                                _dptr(acc), stream)
        else:
            self.ctx = lvb_init_resume(self.n, _dptr(pos), _dptr(ref), box, skin, trigger,
                                       cell_factor, _dptr(vel), _dptr(acc), stream)

    def step(self, pos, vel=None, acc=None):
        _check(lvb_step(self.ctx, _dptr(pos), _dptr(vel), _dptr(acc)), "lvb_step")

    def step_host(self, pos, vel=None, acc=None, bits=None, n_flagged=None):
        """lvb_step_host on host tensors / arrays (pinned for overlap): pos,
        vel, acc (n, 4) float32; bits (ceil(n/32),) uint32 and n_flagged
        (1,) int32 receive the step's flags once the context is synchronised.
        Every buffer must stay alive until then."""
        def hp(a):
            if a is None:
                return None
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        _check(lvb_step_host(self.ctx, hp(pos), hp(vel), hp(acc), hp(bits), hp(n_flagged)),
               "lvb_step_host")

    def sync(self):
        return lvb_sync(self.ctx)

    def set_option(self, option, value):
        _check(lvb_set_option(self.ctx, option, value), "lvb_set_option")

    def pairs_ij(self):
        n = ctypes.c_int64(0)
        rc = lvb_get_pairs_ij(self.ctx, None, None, 0, ctypes.byref(n))
        if rc not in (LVB_OK, LVB_ECAPACITY):
            _check(rc, "lvb_get_pairs_ij")
        cap = n.value
        pi = np.empty(max(cap, 1), dtype=np.int32)
        pj = np.empty(max(cap, 1), dtype=np.int32)
        _check(lvb_get_pairs_ij(self.ctx, _np_ptr(pi), _np_ptr(pj), cap, ctypes.byref(n)),
               "lvb_get_pairs_ij")
        return pi[:n.value], pj[:n.value]

    def near_cutoff(self, rel=1e-6):
        """Pairs i < j whose squared reference distance is within rel of the
        squared cutoff (lvb_get_near_cutoff), sorted by (i, j)."""
        n = ctypes.c_int64(0)
        rc = _lib.lvb_get_near_cutoff(self.ctx, float(rel), None, None, 0, ctypes.byref(n))
        if rc not in (LVB_OK, LVB_ECAPACITY):
            _check(rc, "lvb_get_near_cutoff")
        cap = n.value
        pi = np.empty(max(cap, 1), dtype=np.int32)
        pj = np.empty(max(cap, 1), dtype=np.int32)
        _check(_lib.lvb_get_near_cutoff(self.ctx, float(rel), _np_ptr(pi), _np_ptr(pj), cap,
                                        ctypes.byref(n)), "lvb_get_near_cutoff")
        pi, pj = pi[:n.value], pj[:n.value]
        order = np.lexsort((pj, pi))
        return pi[order], pj[order]

    def pairs_csr(self):
        n = ctypes.c_int64(0)
        row_ptr = np.empty(self.n + 1, dtype=np.int32)
        rc = lvb_get_pairs(self.ctx, _np_ptr(row_ptr), None, 0, ctypes.byref(n))
        if rc not in (LVB_OK, LVB_ECAPACITY):
            _check(rc, "lvb_get_pairs")
        col = np.empty(max(n.value, 1), dtype=np.int32)
        _check(lvb_get_pairs(self.ctx, _np_ptr(row_ptr), _np_ptr(col), n.value, ctypes.byref(n)),
               "lvb_get_pairs")
        return row_ptr, col[:n.value]

    def contacts(self, pos):
        n = ctypes.c_int64(0)
        rc = lvb_get_contacts(self.ctx, _dptr(pos), None, None, None, 0, ctypes.byref(n))
        if rc not in (LVB_OK, LVB_ECAPACITY):
            _check(rc, "lvb_get_contacts")
        cap = n.value
        ci = np.empty(max(cap, 1), dtype=np.int32)
        cj = np.empty(max(cap, 1), dtype=np.int32)
        dl = np.empty(max(cap, 1), dtype=np.float32)
        _check(lvb_get_contacts(self.ctx, _dptr(pos), _np_ptr(ci), _np_ptr(cj), _np_ptr(dl), cap,
                                ctypes.byref(n)), "lvb_get_contacts")
        return ci[:n.value], cj[:n.value], dl[:n.value]

    def clump_contacts(self, pos, quat, sub_off, sub):
        """lvb_clump_contacts on device tensors (pos, quat: (n, 4); sub_off:
        (n + 1,) int32; sub: (m, 4)): (ci, ca, cj, cb, delta) sorted by
        (i, j, a, b)."""
        n = ctypes.c_int64(0)
        rc = _lib.lvb_clump_contacts(self.ctx, _dptr(pos), _dptr(quat), _dptr(sub_off),
                                     _dptr(sub), None, None, None, None, None, 0,
                                     ctypes.byref(n))
        if rc not in (LVB_OK, LVB_ECAPACITY):
            _check(rc, "lvb_clump_contacts")
        cap = max(n.value, 1)
        outs = [np.empty(cap, np.int32) for _ in range(4)] + [np.empty(cap, np.float32)]
        _check(_lib.lvb_clump_contacts(self.ctx, _dptr(pos), _dptr(quat), _dptr(sub_off),
                                       _dptr(sub), *[_np_ptr(o) for o in outs], cap,
                                       ctypes.byref(n)), "lvb_clump_contacts")
        m = n.value
        ci, ca, cj, cb, dl = (o[:m] for o in outs)
        o = np.lexsort((cb, ca, cj, ci))
        return ci[o], ca[o], cj[o], cb[o], dl[o]

    def clump_contacts_into(self, pos, quat, sub_off, sub, ci, ca, cj, cb, delta):
        """lvb_clump_contacts into device tensors of equal length (the
        capacity); returns the contact count (over the capacity: only the
        first capacity written)."""
        n = ctypes.c_int64(0)
        rc = _lib.lvb_clump_contacts(self.ctx, _dptr(pos), _dptr(quat), _dptr(sub_off),
                                     _dptr(sub), _dptr(ci), _dptr(ca), _dptr(cj), _dptr(cb),
                                     _dptr(delta), int(ci.numel()), ctypes.byref(n))
        if rc not in (LVB_OK, LVB_ECAPACITY):
            _check(rc, "lvb_clump_contacts")
        return n.value

    def flags(self):
        words = np.zeros((self.n + 31) // 32, dtype=np.uint32)
        nf = ctypes.c_int64(0)
        _check(lvb_get_flags(self.ctx, _np_ptr(words), ctypes.byref(nf)), "lvb_get_flags")
        bits = np.unpackbits(words.view(np.uint8), bitorder="little")[:self.n].astype(bool)
        return bits

    def ref(self):
        out = np.empty((self.n, 4), dtype=np.float32)
        _check(lvb_get_ref(self.ctx, _np_ptr(out)), "lvb_get_ref")
        return out

    def trace(self):
        """Mean device time per step (us) of each traced kernel."""
        a = np.zeros(16, np.uint64)
        b = np.zeros(16, np.uint64)
        _check(lvb_trace(self.ctx, _np_ptr(a), _np_ptr(b)), "lvb_trace")
        return {name: (float(a[k]) / 1e3 / max(int(b[k]), 1), int(b[k]))
                for k, name in enumerate(TRACE_SLOTS)}

    def log_enable(self, horizon, capacity):
        _check(lvb_log_enable(self.ctx, horizon, capacity), "lvb_log_enable")

    def log_samples(self):
        n = ctypes.c_int64(0)
        rc = lvb_log_read(self.ctx, None, 0, ctypes.byref(n))
        if rc not in (LVB_OK, LVB_ECAPACITY):
            _check(rc, "lvb_log_read")
        out = np.empty((max(n.value, 1), LVB_MLP_IN + 1), dtype=np.float32)
        _check(lvb_log_read(self.ctx, _np_ptr(out), n.value, ctypes.byref(n)), "lvb_log_read")
        return out[:n.value]

    def scene_info(self, scene):
        si = lvb_scene_info_t()
        _check(lvb_scene_info(self.ctx, scene, ctypes.byref(si)), "lvb_scene_info")
        return {"first": si.first, "count": si.count, "cell_edge": si.cell_edge,
                "rnl_max": si.rnl_max, "grid": list(si.grid)}

    def stats(self):
        st = lvb_stats_t()
        _check(lvb_stats(self.ctx, ctypes.byref(st)), "lvb_stats")
        return {k: (list(getattr(st, k)) if k in ("grid", "reserved") else getattr(st, k))
                for k, _ in lvb_stats_t._fields_ if k != "pad"}

    def close(self):
        if self.ctx:
            lvb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


WALLS = {"none": DEM_WALL_NONE, "box": DEM_WALL_BOX, "drum": DEM_WALL_DRUM,
         "specular": DEM_WALL_SPECULAR}


class _BorrowedLVB(LVB):
    """The broad-phase context owned by a DEM context (not destroyed here)."""

    def __init__(self, ctx, n):
        self.ctx = ctx
        self.n = n

    def close(self):
        self.ctx = None


class DEM:
    """A DEM driver context over a scene (``scenes.Scene``-like object)."""

    def __init__(self, scene, trigger=LVB_TRIGGER_PARTIAL, skin_kind=None, skin_value=None,
                 cell_factor=None, stream=None, mlp=None):
        """scene: one scene, or a list of scenes (same physics, own boxes)
        advanced together as one batch.  mlp: device weights of the skin
        network (mlp_weights_device) for LVB_SKIN_LEARNED."""
        import torch
        batch = isinstance(scene, (list, tuple))
        scenes_ = list(scene) if batch else [scene]
        scene = scenes_[0]
        self.n = int(sum(q.n for q in scenes_))
        prm = dem_params()
        prm.kn, prm.restitution, prm.rho = scene.kn, scene.restitution, scene.rho
        for k in range(3):
            prm.g[k] = scene.gravity[k]
        prm.wall_kind = WALLS[scene.wall]
        prm.clamp_tensile = 0
        if scene.drum is not None:
            prm.drum_cx, prm.drum_cz, prm.drum_R, prm.drum_omega = scene.drum
        prm.contacts_on = int(bool(scene.contacts))
        prm.mu = float(getattr(scene, "mu", 0.0))
        prm.kt_ratio = float(getattr(scene, "kt_ratio", 2.0 / 7.0))
        prm.gt_ratio = float(getattr(scene, "gt_ratio", 0.5))
        self.prm = prm
        boxes = (lvb_box * len(scenes_))()
        for q, sc in enumerate(scenes_):
            for k in range(3):
                boxes[q].lo[k], boxes[q].hi[k] = sc.lo[k], sc.hi[k]
        kind = scene.skin_kind if skin_kind is None else skin_kind
        value = scene.skin_value if skin_value is None else skin_value
        self._mlp = mlp            # keeps the weights alive with the context
        skin = lvb_skin_policy(int(kind), float(value), float(scene.dt), _dptr(mlp))
        cf = scene.cell_factor if cell_factor is None else cell_factor
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        pos = torch.from_numpy(np.ascontiguousarray(np.concatenate([q.pos for q in scenes_]),
                                                    dtype=np.float32)).cuda()
        vel = torch.from_numpy(np.ascontiguousarray(np.concatenate([q.vel for q in scenes_]),
                                                    dtype=np.float32)).cuda()
        if batch:
            self.offsets = np.concatenate([[0], np.cumsum([q.n for q in scenes_])]).astype(np.int64)
            self.ctx = dem_batch_init(len(scenes_), self.offsets, pos.data_ptr(), vel.data_ptr(),
                                      prm, scene.dt, boxes, skin, trigger, cf, stream)
        else:
            self.offsets = np.array([0, self.n], dtype=np.int64)
            self.ctx = dem_init(self.n, pos.data_ptr(), vel.data_ptr(), prm, scene.dt, boxes[0],
                                skin, trigger, cf, stream)
        torch.cuda.synchronize()
        self.lvb = _BorrowedLVB(dem_lvb(self.ctx), self.n)

    def advance(self, steps):
        _check(dem_advance(self.ctx, steps), "dem_advance")

    def phase(self, ph):
        _check(dem_phase(self.ctx, ph), "dem_phase")

    def step(self):
        for ph in (DEM_PHASE_INTEGRATE, DEM_PHASE_BROAD, DEM_PHASE_FORCES):
            self.phase(ph)

    def state(self):
        outs = [np.empty((self.n, 4), dtype=np.float32) for _ in range(4)]
        _check(dem_get_state(self.ctx, *[_np_ptr(o) for o in outs]), "dem_get_state")
        return tuple(outs)   # pos, vel, acc, vstar

    def device_pos_tensor(self, torch):
        """A torch view (no copy) of the context's device positions."""
        ptr = dem_device_state(self.ctx)[0]

        class _View:
            __cuda_array_interface__ = {"shape": (self.n, 4), "typestr": "<f4",
                                        "data": (ptr, False), "version": 2}
        return torch.as_tensor(_View(), device="cuda")

    def contact_forces(self):
        """dem_get_contact_forces: (ci, cj, force on i (m, 3), delta), sorted
        by (i, j)."""
        n = ctypes.c_int64(0)
        rc = _lib.dem_get_contact_forces(self.ctx, None, None, None, None, 0, ctypes.byref(n))
        if rc not in (LVB_OK, LVB_ECAPACITY):
            _check(rc, "dem_get_contact_forces")
        cap = max(n.value, 1)
        ci = np.empty(cap, np.int32)
        cj = np.empty(cap, np.int32)
        f3 = np.empty((cap, 3), np.float32)
        dl = np.empty(cap, np.float32)
        _check(_lib.dem_get_contact_forces(self.ctx, _np_ptr(ci), _np_ptr(cj), _np_ptr(f3),
                                           _np_ptr(dl), cap, ctypes.byref(n)),
               "dem_get_contact_forces")
        m = n.value
        o = np.lexsort((cj[:m], ci[:m]))
        return ci[:m][o], cj[:m][o], f3[:m][o], dl[:m][o]

    def contact_history(self, sides=1):
        """dem_get_contact_history: (ci, cj, force on i (m, 3), delta, spring
        xi of row i (m, 3)), sorted by (i, j); sides=2: both rows of each
        pair."""
        n = ctypes.c_int64(0)
        rc = _lib.dem_get_contact_history(self.ctx, sides, None, None, None, None, None, 0,
                                          ctypes.byref(n))
        if rc not in (LVB_OK, LVB_ECAPACITY):
            _check(rc, "dem_get_contact_history")
        cap = max(n.value, 1)
        ci = np.empty(cap, np.int32)
        cj = np.empty(cap, np.int32)
        f3 = np.empty((cap, 3), np.float32)
        dl = np.empty(cap, np.float32)
        xi = np.empty((cap, 3), np.float32)
        _check(_lib.dem_get_contact_history(self.ctx, sides, _np_ptr(ci), _np_ptr(cj),
                                            _np_ptr(f3), _np_ptr(dl), _np_ptr(xi), cap,
                                            ctypes.byref(n)),
               "dem_get_contact_history")
        m = n.value
        o = np.lexsort((cj[:m], ci[:m]))
        return ci[:m][o], cj[:m][o], f3[:m][o], dl[:m][o], xi[:m][o]

    def rot_state(self):
        """(omega (w, 1/I), alpha, omega*) float4 records."""
        outs = [np.empty((self.n, 4), dtype=np.float32) for _ in range(3)]
        _check(_lib.dem_get_rot_state(self.ctx, *[_np_ptr(o) for o in outs]),
               "dem_get_rot_state")
        return tuple(outs)

    def set_state(self, pos, vel, acc):
        arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (pos, vel, acc)]
        _check(dem_set_state(self.ctx, *[_np_ptr(a) for a in arrs]), "dem_set_state")

    def sync(self):
        return dem_sync(self.ctx)

    def close(self):
        if self.ctx:
            dem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ skin network
def mlp_weights_device(params, mu, isd, y_range=None, y_steps=0.0):
    """Pack master parameters (+ normalisation, + output range {y_lo, y_hi}
    or None for {0, inf}, + y_steps: 0 for the diameter form of the output,
    else the travel form's step count) into a device lvb_mlp_weights record;
    returns the torch byte tensor holding it."""
    import torch
    buf = torch.empty(MLP_WEIGHTS_BYTES, dtype=torch.uint8, device="cuda")
    p = np.ascontiguousarray(params, np.float32)
    m = np.ascontiguousarray(mu, np.float32)
    d = np.ascontiguousarray(isd, np.float32)
    yr = None if y_range is None else np.ascontiguousarray(y_range, np.float32)
    _check(lvb_mlp_pack(_np_ptr(p), _np_ptr(m), _np_ptr(d), None if yr is None else _np_ptr(yr),
                        float(y_steps), buf.data_ptr()), "lvb_mlp_pack")
    return buf


def mlp_train(samples_dev, epochs, batch, lr, seed, params0, y_range_out=None,
              loss_kind=None):
    """Train on device samples (torch (n, 9) float32); returns (params, mu,
    isd, losses).  y_range_out (a float32 array of 2) receives the output
    range computed from the labels; loss_kind: LVB_MLP_LOSS_SQUARED
    (default) or LVB_MLP_LOSS_RELATIVE."""
    kind = LVB_MLP_LOSS_SQUARED if loss_kind is None else loss_kind
    p = np.ascontiguousarray(params0, np.float32).copy()
    mu = np.zeros(LVB_MLP_IN, np.float32)
    isd = np.zeros(LVB_MLP_IN, np.float32)
    yr = np.zeros(2, np.float32) if y_range_out is None else y_range_out
    losses = np.zeros(int(epochs), np.float32)
    _check(lvb_mlp_train(samples_dev.data_ptr(), samples_dev.shape[0], epochs, batch, lr, seed,
                         kind, _np_ptr(p), _np_ptr(mu), _np_ptr(isd), _np_ptr(yr),
                         _np_ptr(losses)),
           "lvb_mlp_train")
    return p, mu, isd, losses


def mlp_travel_labels(samples, horizon, margin, clip_q):
    """lvb_mlp_travel_labels on an (n, 9) float32 array (host) or device
    tensor; returns the kept samples as a host array (m, 9)."""
    import torch
    if isinstance(samples, np.ndarray):
        src = torch.from_numpy(np.ascontiguousarray(samples, dtype=np.float32)).cuda()
    else:
        src = samples.contiguous()
    out = torch.empty_like(src)
    m = ctypes.c_int64(0)
    _check(lvb_mlp_travel_labels(src.data_ptr() if src.numel() else None, src.shape[0],
                                 horizon, margin, clip_q,
                                 out.data_ptr() if out.numel() else None, ctypes.byref(m),
                                 torch.cuda.current_stream().cuda_stream),
           "lvb_mlp_travel_labels")
    return out[:m.value].cpu().numpy()
