"""Tangential friction with contact history on the GPU against the binary64
oracle (the LSD model with static friction, Sec. Methodology).

The driver keeps each contact's tangential spring in the broad phase's
contact history (LVB_OPT_HISTORY): a record beside every list entry, kept
in place while a flagged particle's row is edited, carried to the new slot
by a re-layout of the row store (forced here with LVB_OPT_FORCE_RELAYOUT)
and by the host's re-layout when the cell slots grow (LVB_OPT_CELL_CAPACITY
here).  A packed bed with random velocities flags particles on most steps,
so the rows holding live springs are rebuilt throughout.

Per checked step the oracle is fed the GPU's state before the step (x, v,
a, w, al and the springs of the contacts then), and the GPU's own x', v*,
w* for the force evaluation, and must give the same contacts, springs and
forces (1e-5 of the summed terms of each contact), accelerations and
velocities (1e-5 of the particle's summed terms).  A spring lost in a
rebuild would show as an error of the size of the spring force.  Both rows
of a pair hold exactly opposite springs.
"""
import numpy as np
import pytest

from paper_2208_13770_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-5
MU, KT_RATIO, GT_RATIO = 0.5, 2.0 / 7.0, 0.5


def _lvb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_13770_gb300 import lvb
    return lvb


def _f32(v):
    return float(np.float32(v))


def _params(orc, s):
    return orc.dem_params(kn=_f32(s.kn), restitution=_f32(s.restitution), rho=_f32(s.rho),
                          g=tuple(map(_f32, s.gravity)), lo=tuple(map(_f32, s.lo)),
                          hi=tuple(map(_f32, s.hi)), wall_kind=orc.WALL_BOX)


def _state(dem):
    x, v, a, vs = dem.state()
    w, al, ws = dem.rot_state()
    ci, cj, f, dl, xi = dem.contact_history()
    return {"x": x, "v": v, "a": a, "vs": vs, "w": w, "al": al, "ws": ws,
            "hist": (ci, cj, xi), "f": f, "dl": dl}


def _check(orc, s, P, before, after, flags):
    """One step (before -> after) against the oracle; returns the number of
    springs that lived through the step on a pair with a flagged side."""
    o = orc.dem_step_friction(before["x"], before["v"], before["a"], before["w"], before["al"],
                              s.dt, P, _f32(MU), _f32(KT_RATIO), _f32(GT_RATIO),
                              hist=before["hist"], x_in=after["x"], vstar_in=after["vs"],
                              wstar_in=after["ws"])
    gi, gj, gxi = after["hist"]
    n = len(after["x"])
    gk = gi.astype(np.int64) * n + gj
    ok = o["ci"].astype(np.int64) * n + o["cj"]
    # the contact sets (overlaps within 1e-14 m of zero may differ)
    both, ig, io = np.intersect1d(gk, ok, return_indices=True)
    only_o = np.setdiff1d(np.arange(len(ok)), io)
    if len(only_o):
        ci, cj, _, od, _ = orc.dem_contacts(after["x"], after["vs"], P)
        odl = dict(zip((ci.astype(np.int64) * n + cj).tolist(), od.tolist()))
        assert all(abs(odl[int(q)]) <= 1e-14 for q in ok[only_o])
    only_g = np.setdiff1d(np.arange(len(gk)), ig)
    assert np.all(np.abs(after["dl"][only_g]) <= 1e-14)
    assert len(both) > 1000
    sc = o["scale"][io][:, None]
    kt = _f32(KT_RATIO) * _f32(s.kn)
    assert np.all(np.abs(gxi[ig] - o["xi"][io]) <= RTOL * sc / kt), \
        np.max(np.abs(gxi[ig] - o["xi"][io]) / (sc / kt))
    assert np.all(np.abs(after["f"][ig] - o["f"][io]) <= RTOL * sc), \
        np.max(np.abs(after["f"][ig] - o["f"][io]) / sc)
    # per particle: a', v', al', w' against the summed terms
    r = after["x"][:, 3].astype(np.float64)
    m = s.rho * 4.0 / 3.0 * np.pi * r ** 3
    I = 0.4 * m * r * r
    g = np.linalg.norm(s.gravity)
    fa = (o["fmag"] / m + g)[:, None]
    ta = (o["tmag"] / I)[:, None]
    checks = [("a'", after["a"][:, :3], o["a"], fa),
              ("v'", after["v"][:, :3], o["v"],
               np.abs(before["v"][:, :3]) + s.dt * (np.abs(before["a"][:, :3]) + fa)),
              ("al'", after["al"][:, :3], o["al"], ta + 1e-30),
              ("w'", after["w"][:, :3], o["w"],
               np.abs(before["w"][:, :3]) + s.dt * (np.abs(before["al"][:, :3]) + ta) + 1e-30)]
    for name, gv, ov, terms in checks:
        ex = np.abs(gv - ov) - RTOL * terms
        assert ex.max() <= 0, (name, float(ex.max()))
    # springs that lived through the step on a pair with a flagged side
    bi, bj, bxi = before["hist"]
    bk = bi.astype(np.int64) * n + bj
    kept = np.intersect1d(bk, gk[ig])
    flagged = flags[(kept // n)] | flags[(kept % n)]
    return int(flagged.sum())


def test_friction_history_survives_rebuilds(orc):
    lvb = _lvb()
    s = scenes.packed(n=4000, seed=19, vsigma=5.0)
    s.mu, s.kt_ratio, s.gt_ratio = MU, KT_RATIO, GT_RATIO
    P = _params(orc, s)
    dem = lvb.DEM(s)
    st0 = dem.lvb.stats()
    survived = 0
    checked = 0
    for k in range(90):
        if k == 30:
            dem.lvb.set_option(lvb.LVB_OPT_FORCE_RELAYOUT, 1)
        if k == 60:
            dem.lvb.set_option(lvb.LVB_OPT_CELL_CAPACITY, 2 * st0["cell_capacity"])
        check = k % 5 == 0 or k in (30, 31, 60, 61)
        if check:
            before = _state(dem)
        dem.step()
        if check:
            after = _state(dem)
            survived += _check(orc, s, P, before, after, dem.lvb.flags())
            checked += 1
    assert dem.sync() == lvb.LVB_OK
    st = dem.lvb.stats()
    assert st["relayouts"] > st0["relayouts"]        # the forced re-layout ran
    assert st["grows"] > st0["grows"]                # and the host's re-layout
    assert st["cell_capacity"] >= 2 * st0["cell_capacity"]
    assert st["flagged_total"] > 5000
    assert survived > 500, survived                  # live springs through rebuilt rows
    # both rows of every pair hold exactly opposite springs
    ci, cj, _, _, xi = dem.contact_history(sides=2)
    n = s.n
    fwd = dict(zip((ci.astype(np.int64) * n + cj).tolist(), range(len(ci))))
    pairs = [(fwd[int(i) * n + int(j)], fwd[int(j) * n + int(i)])
             for i, j in zip(ci, cj) if i < j]
    a, b = np.array(pairs).T
    assert len(a) > 1000 and np.any(xi[a] != 0)
    assert np.array_equal(xi[a], -xi[b])
    dem.close()


def test_friction_needs_the_partial_trigger():
    lvb = _lvb()
    s = scenes.packed(n=500, seed=3)
    s.mu = MU
    with pytest.raises(lvb.LVBError):
        lvb.DEM(s, trigger=lvb.LVB_TRIGGER_GLOBAL)
