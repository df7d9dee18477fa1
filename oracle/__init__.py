"""CPU oracle for the local Verlet buffer broad phase and its DEM driver.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product library never imports,
links or runs anything here, and nothing here imports the product package.

* ``lvb_oracle.c``  -- the definitions in plain C (binary32 fixed formula for
  the broad-phase decisions, binary64 for the dynamics), built by
  :func:`build` with ``-ffp-contract=off``.
* ``statemachine``  -- the automatic Verlet update (Def. autoverlet) driven
  step by step over position snapshots.
* ``mlp``           -- the skin network in binary64 (training oracle) and the
  exact binary32/bfloat16 inference formula.
* :func:`near_cutoff` -- the pairs near their cutoff, in numpy binary32.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lvb_oracle.c")
_LIB = os.path.join(_HERE, "liblvb_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary32 arithmetic without contraction),
    with OpenMP where the compiler has it (the flag test and the pair search
    then use several host threads; the results do not depend on how many)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        if subprocess.call(base + ["-fopenmp"], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


class DemParams(ctypes.Structure):
    """Mirror of ``orc_dem_params`` in lvb_oracle.c."""
    _fields_ = [
        ("kn", ctypes.c_double),
        ("restitution", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("wall_kind", ctypes.c_int32),
        ("clamp_tensile", ctypes.c_int32),
        ("drum_center", ctypes.c_double * 2),
        ("drum_radius", ctypes.c_double),
        ("drum_omega", ctypes.c_double),
        ("contacts_on", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


WALL_NONE, WALL_BOX, WALL_DRUM, WALL_SPECULAR = 0, 1, 2, 3


def _configure(L):
    if True:
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        L.orc_flags.argtypes = [i64, p, p, p]
        L.orc_flags.restype = i64
        L.orc_flags_beta.argtypes = [i64, p, p, ctypes.c_float, p]
        L.orc_flags_beta.restype = i64
        L.orc_skin.argtypes = [i64, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, p, p, p, p]
        L.orc_skin.restype = None
        for name in ("orc_pairs_brute", "orc_pairs_cells"):
            f = getattr(L, name)
            f.argtypes = [i64, p, p, p, p, i64]
            f.restype = i64
        L.orc_contacts.argtypes = [i64, p, p, p, p, p, p, i64]
        L.orc_contacts.restype = i64
        for name in ("orc_contacts_brute", "orc_contacts_cells"):
            f = getattr(L, name)
            f.argtypes = [i64, p, p, p, p, i64]
            f.restype = i64
        L.orc_dem_forces.argtypes = [i64, p, p, ctypes.POINTER(DemParams), p]
        L.orc_dem_forces.restype = ctypes.c_int
        L.orc_dem_forces64.argtypes = [i64, p, p, p, ctypes.POINTER(DemParams), p, p]
        L.orc_dem_forces64.restype = ctypes.c_int
        L.orc_dem_step64.argtypes = [i64, p, p, p, p, ctypes.c_double,
                                     ctypes.POINTER(DemParams), p, p, p, p, p, p, p]
        L.orc_dem_step64.restype = ctypes.c_int
        L.orc_dem_contacts64.argtypes = [i64, p, p, p, ctypes.POINTER(DemParams), p, p, p, p,
                                         p, i64]
        L.orc_dem_contacts64.restype = i64
        L.orc_dem_step64f.argtypes = ([i64] + [p] * 6 + [ctypes.c_double,
                                      ctypes.POINTER(DemParams)] + [ctypes.c_double] * 3 +
                                     [p] * 3 + [i64] + [p] * 3 + [p] * 7 + [p] * 7 + [i64])
        L.orc_dem_step64f.restype = i64
        L.orc_clump_contacts.argtypes = [i64, p, p, p, p, p, p, p, p, p, i64]
        L.orc_clump_contacts.restype = i64
        L.orc_improvement_pct.argtypes = [ctypes.c_double, ctypes.c_double]
        L.orc_improvement_pct.restype = ctypes.c_double
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = None
        L.orc_threads.argtypes = []
        L.orc_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB))
    return _lib


class use_library:
    """Context manager that routes every oracle call through another build
    of lvb_oracle.c (used by the mutation tests, which compile deliberately
    broken copies to show that the pins catch them)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = lib()
        _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def set_threads(t):
    """Host threads of the flag test and the pair search (t <= 0: all
    processors)."""
    lib().orc_set_threads(int(t))


def threads():
    """Host threads the oracle's parallel loops use (1 without OpenMP)."""
    return int(lib().orc_threads())


def _f32x4(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    assert a.ndim == 2 and a.shape[1] == 4, a.shape
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


def flags(pos4, ref4):
    """Eq. update: boolean array, True where |x - xref|^2 > skin^2."""
    pos4, ref4 = _f32x4(pos4), _f32x4(ref4)
    out = np.zeros(len(pos4), dtype=np.uint8)
    lib().orc_flags(len(pos4), _ptr(pos4), _ptr(ref4), _ptr(out))
    return out.astype(bool)


def flags_beta(pos4, ref4, beta):
    """The early trigger's set: True where |x - xref|^2 > (beta skin)^2
    (binary32, beta rounded to binary32)."""
    pos4, ref4 = _f32x4(pos4), _f32x4(ref4)
    out = np.zeros(len(pos4), dtype=np.uint8)
    lib().orc_flags_beta(len(pos4), _ptr(pos4), _ptr(ref4), np.float32(beta), _ptr(out))
    return out.astype(bool)


SKIN_GLOBAL, SKIN_DIAMETER_FACTOR, SKIN_PAPER_KVDT, SKIN_LEARNED = 0, 1, 2, 3


def skin(kind, value, dt, H, pos4, vel4=None, proposal=None):
    """Per-particle skin from a policy, capped so that r + skin <= H."""
    pos4 = _f32x4(pos4)
    vel4 = None if vel4 is None else _f32x4(vel4)
    if kind == SKIN_PAPER_KVDT and vel4 is None:
        raise ValueError("the K*|v|*dt policy needs velocities")
    prop = None if proposal is None else np.ascontiguousarray(proposal, dtype=np.float32)
    if kind == SKIN_LEARNED and prop is None:
        raise ValueError("the learned policy needs a proposal")
    out = np.zeros(len(pos4), dtype=np.float32)
    lib().orc_skin(len(pos4), int(kind), np.float32(value), np.float32(dt), np.float32(H),
                   _ptr(pos4), _ptr(vel4), _ptr(prop), _ptr(out))
    return out


def _pairs(fn, ref4, rad):
    ref4 = _f32x4(ref4)
    rad = np.ascontiguousarray(rad, dtype=np.float32)
    n = len(ref4)
    cap = max(16, 8 * n)
    while True:
        pi = np.empty(cap, dtype=np.int32)
        pj = np.empty(cap, dtype=np.int32)
        m = fn(n, _ptr(ref4), _ptr(rad), _ptr(pi), _ptr(pj), cap)
        if m < 0:
            raise MemoryError("oracle pair search failed")
        if m <= cap:
            return pi[:m].copy(), pj[:m].copy()
        cap = int(m)


def pairs_brute(ref4, rad):
    """Pair set by definition (brute force), sorted (i, j) with i < j."""
    return _pairs(lib().orc_pairs_brute, ref4, rad)


def pairs_cells(ref4, rad):
    """Pair set through Algorithm 1 (linked cells), sorted (i, j) with i < j."""
    return _pairs(lib().orc_pairs_cells, ref4, rad)


def near_cutoff(ref4, rad, rel):
    """Pairs i < j whose squared reference distance d2 lies within rel of the
    squared cutoff c2 (Def. verletlist's inequality d2 <= c2, near its
    boundary): d2 = ((dx dx) + (dy dy)) + dz dz of the binary32 differences,
    c = R_i + R_j with R = r + skin, c2 = c c, every operation in binary32
    (numpy, no fused multiply-add); |d2 - c2| <= rel c2 compared in binary64.
    Brute force over all pairs (small inputs); sorted (i, j)."""
    ref = np.ascontiguousarray(ref4, dtype=np.float32)
    R = (np.asarray(rad, dtype=np.float32) + ref[:, 3]).astype(np.float32)
    n = len(ref)
    out_i, out_j = [], []
    for i in range(n - 1):
        j = np.arange(i + 1, n)
        dx = ref[i, 0] - ref[j, 0]
        dy = ref[i, 1] - ref[j, 1]
        dz = ref[i, 2] - ref[j, 2]
        d2 = (dx * dx + dy * dy) + dz * dz
        c = R[i] + R[j]
        c2 = c * c
        m = np.abs(d2.astype(np.float64) - c2.astype(np.float64)) <= rel * c2.astype(np.float64)
        out_i.append(np.full(int(m.sum()), i, dtype=np.int32))
        out_j.append(j[m].astype(np.int32))
    if not out_i:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    return np.concatenate(out_i), np.concatenate(out_j)


def pairs(ref4, rad):
    """The pair set: brute force for small inputs, linked cells otherwise."""
    return pairs_brute(ref4, rad) if len(ref4) <= 3000 else pairs_cells(ref4, rad)


def contacts(pi, pj, pos4):
    """Eq. delta on a pair list: (ci, cj, delta) for the pairs with delta > 0."""
    pos4 = _f32x4(pos4)
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    pj = np.ascontiguousarray(pj, dtype=np.int32)
    n = len(pi)
    ci = np.empty(max(n, 1), dtype=np.int32)
    cj = np.empty(max(n, 1), dtype=np.int32)
    dl = np.empty(max(n, 1), dtype=np.float32)
    m = lib().orc_contacts(n, _ptr(pi), _ptr(pj), _ptr(pos4), _ptr(ci), _ptr(cj), _ptr(dl), n)
    return ci[:m].copy(), cj[:m].copy(), dl[:m].copy()


def _contacts_all(fn, pos4):
    pos4 = _f32x4(pos4)
    n = len(pos4)
    cap = max(16, 8 * n)
    while True:
        ci = np.empty(cap, dtype=np.int32)
        cj = np.empty(cap, dtype=np.int32)
        dl = np.empty(cap, dtype=np.float32)
        m = fn(n, _ptr(pos4), _ptr(ci), _ptr(cj), _ptr(dl), cap)
        if m < 0:
            raise MemoryError("oracle contact search failed")
        if m <= cap:
            return ci[:m].copy(), cj[:m].copy(), dl[:m].copy()
        cap = int(m)


def contacts_brute(pos4):
    """Every overlapping pair of a configuration (brute force over all pairs)."""
    return _contacts_all(lib().orc_contacts_brute, pos4)


def contacts_cells(pos4):
    """Every overlapping pair of a configuration (cell search)."""
    return _contacts_all(lib().orc_contacts_cells, pos4)


def contacts_all(pos4):
    return contacts_brute(pos4) if len(pos4) <= 3000 else contacts_cells(pos4)


def dem_params(kn=1e4, restitution=0.7, rho=2500.0, g=(0.0, 0.0, -9.81), lo=(0, 0, 0),
               hi=(1, 1, 1), wall_kind=WALL_BOX, clamp_tensile=False, drum_center=(0.0, 0.0),
               drum_radius=0.0, drum_omega=0.0, contacts_on=True):
    P = DemParams()
    P.kn, P.restitution, P.rho = kn, restitution, rho
    for k in range(3):
        P.g[k], P.lo[k], P.hi[k] = g[k], lo[k], hi[k]
    P.wall_kind = int(wall_kind)
    P.clamp_tensile = int(bool(clamp_tensile))
    P.drum_center[0], P.drum_center[1] = drum_center
    P.drum_radius, P.drum_omega = drum_radius, drum_omega
    P.contacts_on = int(bool(contacts_on))
    return P


def dem_forces(x4, v4, P):
    """Net contact + wall force per particle (binary64, shape (n, 3))."""
    x4, v4 = _f32x4(x4), _f32x4(v4)
    F = np.zeros((len(x4), 3), dtype=np.float64)
    rc = lib().orc_dem_forces(len(x4), _ptr(x4), _ptr(v4), ctypes.byref(P), _ptr(F))
    if rc != 0:
        raise MemoryError("oracle force evaluation failed")
    return F


def _d3(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a)[:, :3], dtype=np.float64)


def dem_step64(x, v, a, r, dt, P, xf=None, vf=None, with_fmag=False):
    """One velocity-Verlet step on a binary64 state (x, v, a: (n, 3); r: (n,)).
    xf / vf replace x' / v* as the state at which forces are evaluated.
    Returns (x', v*, a', v'), each (n, 3) binary64, plus the per-particle
    scale of the summed force terms when with_fmag."""
    x, v, a, xf, vf = _d3(x), _d3(v), _d3(a), _d3(xf), _d3(vf)
    r = np.ascontiguousarray(r, dtype=np.float64)
    n = len(x)
    outs = [np.zeros((n, 3), dtype=np.float64) for _ in range(4)]
    fmag = np.zeros(n, dtype=np.float64) if with_fmag else None
    rc = lib().orc_dem_step64(n, _ptr(x), _ptr(v), _ptr(a), _ptr(r), float(dt), ctypes.byref(P),
                              _ptr(xf), _ptr(vf), *[_ptr(o) for o in outs], _ptr(fmag))
    if rc != 0:
        raise MemoryError("oracle step failed")
    return tuple(outs) + ((fmag,) if with_fmag else ())


def dem_step(x4, v4, a4, dt, P, x_in=None, vstar_in=None, with_fmag=False):
    """One step from the binary32 state (float4 records) of the code under
    test, widened exactly.  Returns (x', v*, a', v'[, fmag]) in binary64."""
    x4, v4, a4 = _f32x4(x4), _f32x4(v4), _f32x4(a4)
    return dem_step64(x4, v4, a4, x4[:, 3], dt, P,
                      None if x_in is None else _f32x4(x_in),
                      None if vstar_in is None else _f32x4(vstar_in), with_fmag=with_fmag)


def dem_contacts(x4, v4, P):
    """Every contact i < j of the configuration (binary64 overlap > 0) with
    the force on i, the overlap and the scale of the force's terms, from the
    binary32 state of the code under test widened exactly: (ci, cj, f (m,
    3), delta, scale), sorted by (i, j)."""
    x4, v4 = _f32x4(x4), _f32x4(v4)
    x, v = _d3(x4), _d3(v4)
    r = np.ascontiguousarray(x4[:, 3], dtype=np.float64)
    n = len(x)
    cap = max(16, 8 * n)
    while True:
        ci = np.empty(cap, np.int32)
        cj = np.empty(cap, np.int32)
        f3 = np.empty((cap, 3), np.float64)
        dl = np.empty(cap, np.float64)
        sc = np.empty(cap, np.float64)
        m = lib().orc_dem_contacts64(n, _ptr(x), _ptr(r), _ptr(v), ctypes.byref(P), _ptr(ci),
                                     _ptr(cj), _ptr(f3), _ptr(dl), _ptr(sc), cap)
        if m < 0:
            raise MemoryError("oracle contact search failed")
        if m <= cap:
            return ci[:m].copy(), cj[:m].copy(), f3[:m].copy(), dl[:m].copy(), sc[:m].copy()
        cap = int(m)


def dem_step_friction(x4, v4, a4, w4, al4, dt, P, mu, kt_ratio, gt_ratio, hist=None,
                      x_in=None, vstar_in=None, wstar_in=None):
    """One step with rotation and the tangential law with contact history
    (orc_dem_step64f), binary64, from the binary32 state of the code under
    test widened exactly.  hist: (hi, hj, xi (m, 3)) of the pairs in contact
    at the previous step (i < j, sorted), or None.  x_in / vstar_in /
    wstar_in replace x', v*, w* as the state at which forces are evaluated.
    Returns a dict: x, vstar, a, v, wstar, al, w (n, 3); contacts ci, cj, xi
    (m, 3), f (m, 3: force on i), scale (m,); fmag, tmag (n,)."""
    x4, v4, a4, w4, al4 = (_f32x4(q) for q in (x4, v4, a4, w4, al4))
    x, v, a, w, al = (_d3(q) for q in (x4, v4, a4, w4, al4))
    r = np.ascontiguousarray(x4[:, 3], dtype=np.float64)
    n = len(x)
    xf, vf, wf = (None if q is None else _d3(_f32x4(q)) for q in (x_in, vstar_in, wstar_in))
    if hist is None:
        hi = np.zeros(0, np.int32)
        hj = np.zeros(0, np.int32)
        hx = np.zeros((0, 3), np.float64)
    else:
        hi = np.ascontiguousarray(hist[0], np.int32)
        hj = np.ascontiguousarray(hist[1], np.int32)
        hx = np.ascontiguousarray(np.asarray(hist[2])[:, :3], np.float64)
    outs = [np.zeros((n, 3), np.float64) for _ in range(7)]
    fmag = np.zeros(n, np.float64)
    tmag = np.zeros(n, np.float64)
    cap = max(16, 8 * n)
    while True:
        ci = np.empty(cap, np.int32)
        cj = np.empty(cap, np.int32)
        oxi = np.empty((cap, 3), np.float64)
        of3 = np.empty((cap, 3), np.float64)
        osc = np.empty(cap, np.float64)
        m = lib().orc_dem_step64f(n, _ptr(x), _ptr(v), _ptr(a), _ptr(w), _ptr(al), _ptr(r),
                                  float(dt), ctypes.byref(P), float(mu), float(kt_ratio),
                                  float(gt_ratio), _ptr(xf), _ptr(vf), _ptr(wf), len(hi),
                                  _ptr(hi), _ptr(hj), _ptr(hx), *[_ptr(o) for o in outs],
                                  _ptr(ci), _ptr(cj), _ptr(oxi), _ptr(of3), _ptr(osc),
                                  _ptr(fmag), _ptr(tmag), cap)
        if m < 0:
            raise MemoryError("oracle step failed")
        if m <= cap:
            break
        cap = int(m)
    keys = ("x", "vstar", "a", "v", "wstar", "al", "w")
    out = dict(zip(keys, outs))
    out.update(ci=ci[:m].copy(), cj=cj[:m].copy(), xi=oxi[:m].copy(), f=of3[:m].copy(),
               scale=osc[:m].copy(), fmag=fmag, tmag=tmag)
    return out


def clump_contacts(pos4, quat4, sub_off, sub4):
    """Every sub-sphere contact between clumps i < j (brute force over all
    pairs of clumps): (ci, ca, cj, cb, delta), in (i, j, a, b) order; ca, cb
    index the sub-spheres within their clumps."""
    pos4, quat4, sub4 = _f32x4(pos4), _f32x4(quat4), _f32x4(sub4)
    off = np.ascontiguousarray(sub_off, np.int32)
    n = len(pos4)
    cap = max(16, 64 * n)
    while True:
        outs = [np.empty(cap, np.int32) for _ in range(4)] + [np.empty(cap, np.float32)]
        m = lib().orc_clump_contacts(n, _ptr(pos4), _ptr(quat4), _ptr(off), _ptr(sub4),
                                     *[_ptr(o) for o in outs], cap)
        if m <= cap:
            return tuple(o[:m].copy() for o in outs)
        cap = int(m)


def improvement_pct(t_without, t_case):
    """Eq. impr."""
    return lib().orc_improvement_pct(float(t_without), float(t_case))
