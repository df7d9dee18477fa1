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
