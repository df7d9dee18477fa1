"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/*.h declares (no compute call: runs without a GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b((?:lvb|dem)_\w+)\s*\(",
                             txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_declared_symbols():
    from paper_2208_13770_gb300 import build
    lib = build.build()
    declared = _declared()
    assert "lvb_init" in declared and "lvb_step" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = declared - exported
    assert not missing, missing
    L = ctypes.CDLL(lib)
    for name in declared:
        getattr(L, name)


def test_binding_names_match_header():
    from paper_2208_13770_gb300 import lvb
    declared = _declared()
    assert {n for n in declared if n.startswith("lvb_")} == set(lvb.EXPORTED)
    assert {n for n in declared if n.startswith("dem_")} == set(lvb.EXPORTED_DEM)


def test_strerror_without_gpu():
    from paper_2208_13770_gb300 import lvb
    assert lvb.lvb_strerror(0) == "ok"
    assert "overflow" in lvb.lvb_strerror(lvb.LVB_EOVERFLOW)


def test_argument_checks_without_gpu():
    # every call below fails its argument checks before any device work, so
    # it runs (and must return EINVAL) on a machine without a GPU: empty and
    # oversized inputs, misaligned records, bad skin / trigger / cell factor,
    # inverted boxes, null contexts
    import numpy as np
    from paper_2208_13770_gb300 import lvb
    pos = np.zeros((8, 4), np.float32)
    p = pos.ctypes.data
    box = lvb.lvb_box((0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    skin = lvb.lvb_skin_policy(lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, 1e-5, None)

    def init(n=8, ptr=p, b=box, s=skin, trigger=0, cf=1.25, vel=None, acc=None):
        ctx = lvb.ctypes.c_void_p()
        return lvb._lib.lvb_init(lvb.ctypes.byref(ctx), n, ptr, lvb.ctypes.byref(b),
                                 lvb.ctypes.byref(s), trigger, cf, vel, acc, None)

    E = lvb.LVB_EINVAL
    assert init(n=0) == E                      # empty
    assert init(n=-1) == E
    assert init(n=2 ** 31) == E                # above the index range
    assert init(ptr=None) == E
    assert init(ptr=p + 4) == E                # not 16-byte aligned
    assert init(trigger=3) == E
    assert init(cf=0.99) == E                  # cells smaller than a diameter
    assert init(cf=float("nan")) == E
    assert init(b=lvb.lvb_box((0.0, 0.0, 0.0), (1.0, 0.0, 1.0))) == E
    assert init(s=lvb.lvb_skin_policy(lvb.LVB_SKIN_DIAMETER_FACTOR, -0.1, 1e-5, None)) == E
    assert init(s=lvb.lvb_skin_policy(7, 0.1, 1e-5, None)) == E
    # the paper's rule needs velocities and a positive time step
    assert init(s=lvb.lvb_skin_policy(lvb.LVB_SKIN_PAPER_KVDT, 200.0, 1e-5, None)) == E
    assert init(s=lvb.lvb_skin_policy(lvb.LVB_SKIN_PAPER_KVDT, 200.0, 0.0, None), vel=p) == E
    # the network needs weights, velocities and accelerations
    assert init(s=lvb.lvb_skin_policy(lvb.LVB_SKIN_LEARNED, 0.0, 1e-5, None), vel=p) == E
    # ... and 16-byte aligned weights (the step kernel copies them in pieces)
    assert init(s=lvb.lvb_skin_policy(lvb.LVB_SKIN_LEARNED, 0.0, 1e-5, p + 8), vel=p,
                acc=p) == E
    # the network's weights: a bad output range or travel step count
    prm = np.zeros(lvb.LVB_MLP_PARAMS, np.float32)
    one = np.ones(lvb.LVB_MLP_IN, np.float32)
    rec = np.zeros(lvb.MLP_WEIGHTS_BYTES, np.uint8)

    def pack(yr=None, steps=0.0):
        yp = None if yr is None else np.asarray(yr, np.float32)
        return lvb._lib.lvb_mlp_pack(prm.ctypes.data, one.ctypes.data, one.ctypes.data,
                                     None if yp is None else yp.ctypes.data, steps,
                                     rec.ctypes.data)
    assert pack(yr=(0.5, 0.1)) == E
    assert pack(steps=-1.0) == E
    assert pack(steps=float("nan")) == E
    assert pack(steps=float("inf")) == E
    # inference, gradient and training entry points: null buffers, negative
    # or empty sample counts, a negative relative floor, a bad loss kind
    buf = np.zeros(64, np.float32).ctypes.data
    dbl = lvb.ctypes.byref(lvb.ctypes.c_double(0.0))
    L = lvb._lib
    assert L.lvb_mlp_infer(None, buf, 4, buf, buf, None, None) == E
    assert L.lvb_mlp_infer(buf, buf, -1, buf, buf, None, None) == E
    assert L.lvb_mlp_grad(buf, 0, buf, buf, buf, 0.0, buf, dbl, None) == E
    assert L.lvb_mlp_grad(buf, 4, buf, buf, buf, -1.0, buf, dbl, None) == E
    assert L.lvb_mlp_grad(buf, 4, None, buf, buf, 0.0, buf, dbl, None) == E
    assert L.lvb_mlp_train(buf, 0, 1, 8, 1e-3, 1, 0, buf, buf, buf, buf, buf, None) == E
    assert L.lvb_mlp_train(buf, 4, 1, 8, 1e-3, 1, 7, buf, buf, buf, buf, buf, None) == E
    assert lvb._lib.lvb_step(None, p, None, None) == E
    assert lvb._lib.lvb_step_host(None, p, None, None, None, None) == E
    assert lvb._lib.lvb_sync(None) == E
    assert lvb._lib.lvb_destroy(None) == E
