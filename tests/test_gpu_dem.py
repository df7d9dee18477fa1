"""GPU DEM driver against the binary64 oracle, one step at a time.

The oracle is fed the GPU's binary32 state (x, v, a) before each checked step
and, for the force evaluation, the GPU's own x' and v*, so the trajectories
cannot drift apart; it also gets the physical constants as the GPU holds
them (rounded to binary32).  Tolerances are relative 1e-5 of the terms that
are summed, because a sum that cancels cannot be held to a relative bound
of its own (possibly tiny) size:
  x'       : |gpu - oracle| <= 1e-5 (|x| + |v| dt + |a| dt^2)
  v*       : |gpu - oracle| <= 1e-5 (|v| + |a| dt)
  a'       : |gpu - oracle| <= 1e-5 (S/m + |g|), S = sum over the particle's
             contacts of |k_n delta| + |damping term|
  v'       : |gpu - oracle| <= 1e-5 (|v| + dt (|a| + S/m + |g|))
A contact missing from the list would show as a force error of the size of
that contact's force.
"""
import numpy as np
import pytest

from paper_2208_13770_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = 1e-5


def _lvb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_13770_gb300 import lvb
    return lvb


def _f32(v):
    return float(np.float32(v))


def _params(orc, s):
    kind = {"box": orc.WALL_BOX, "drum": orc.WALL_DRUM, "specular": orc.WALL_SPECULAR,
            "none": orc.WALL_NONE}[s.wall]
    dc, dr = ((_f32(s.drum[0]), _f32(s.drum[1])), _f32(s.drum[2])) if s.drum else ((0.0, 0.0), 0.0)
    return orc.dem_params(kn=_f32(s.kn), restitution=_f32(s.restitution), rho=_f32(s.rho),
                          g=tuple(map(_f32, s.gravity)), lo=tuple(map(_f32, s.lo)),
                          hi=tuple(map(_f32, s.hi)), wall_kind=kind, drum_center=dc,
                          drum_radius=dr, contacts_on=s.contacts)


def _check_step(orc, dem, s, P, idx=None):
    """One GPU step checked against the oracle; returns (#particles in contact)."""
    x, v, a, _ = dem.state()
    dem.step()
    x1, v1, a1, vs1 = dem.state()
    xo, vso, ao, vo, fmag = orc.dem_step(x, v, a, s.dt, P, x_in=x1, vstar_in=vs1,
                                         with_fmag=True)
    sel = slice(None) if idx is None else idx
    dt = s.dt
    x64, v64, a64 = (q[sel, :3].astype(np.float64) for q in (x, v, a))
    m = s.rho * 4.0 / 3.0 * np.pi * x[sel, 3].astype(np.float64) ** 3
    fs = (fmag[sel] / m)[:, None] + np.linalg.norm(s.gravity)
    checks = [
        ("x'", x1[sel, :3], xo[sel], np.abs(x64) + np.abs(v64) * dt + np.abs(a64) * dt * dt),
        ("v*", vs1[sel, :3], vso[sel], np.abs(v64) + np.abs(a64) * dt),
        ("a'", a1[sel, :3], ao[sel], np.broadcast_to(fs, ao[sel].shape)),
        ("v'", v1[sel, :3], vo[sel], np.abs(v64) + dt * (np.abs(a64) + fs)),
    ]
    for name, g, o, terms in checks:
        ex = np.abs(g - o) - RTOL * terms
        k = np.unravel_index(np.argmax(ex), ex.shape)
        assert ex.max() <= 1e-30, "%s off at %s: gpu %r oracle %r terms %r (%d bad)" % (
            name, k, g[k], o[k], terms[k], int((ex > 1e-30).sum()))
    return int((fmag > 0).sum())


@pytest.mark.parametrize("threads,compact", [(1024, 0), (512, 1), (256, 0)])
def test_packed_box_per_step_parity(orc, threads, compact):
    # every launch shape of the fused step (block size; flagged-list indices
    # per warp or per block): graph replays and direct launches alike
    lvb = _lvb()
    s = scenes.packed(n=8000, vsigma=1.0)     # fast enough to flag within the run
    P = _params(orc, s)
    dem = lvb.DEM(s)
    dem.lvb.set_option(lvb.LVB_OPT_BLOCK_THREADS, threads)
    dem.lvb.set_option(lvb.LVB_OPT_COMPACT, compact)
    dem.advance(120)                          # one graph of 100 steps, 20 direct
    touching = 0
    for k in range(300):
        if k % 25 == 0:
            touching = max(touching, _check_step(orc, dem, s, P))
        else:
            dem.step()
    assert dem.sync() == 0
    assert touching > 1000
    st = dem.lvb.stats()
    assert st["rebuild_steps"] > 0
    dem.close()


def test_packed_box_no_contact_missed(orc):
    # every overlapping pair at the checked steps is in the list (Theorem 1)
    lvb = _lvb()
    s = scenes.packed(n=4000, seed=99, vsigma=0.3)
    dem = lvb.DEM(s)
    for k in range(200):
        dem.step()
        if k % 20 == 19:
            x = dem.state()[0]
            ci, cj, _ = orc.contacts_all(x)
            pi, pj = dem.lvb.pairs_ij()
            lst = set(zip(pi.tolist(), pj.tolist()))
            assert set(zip(ci.tolist(), cj.tolist())) <= lst
            assert len(ci) > 100
    dem.close()


def test_drum_wall_parity(orc):
    lvb = _lvb()
    s = scenes.drum(n=20_000, length=0.02, seed=7)
    # push the outermost particles into the drum wall by 1 micrometre
    rho = np.hypot(s.pos[:, 0], s.pos[:, 2])
    out = rho > np.quantile(rho, 0.97)
    target = np.float32(0.3) - s.pos[out, 3] + np.float32(1e-6)
    s.pos[out, 0] *= target / rho[out]
    s.pos[out, 2] *= target / rho[out]
    P = _params(orc, s)
    dem = lvb.DEM(s)
    for k in range(120):
        if k % 30 == 0:
            _check_step(orc, dem, s, P)
        else:
            dem.step()
    assert dem.sync() == 0
    dem.close()


def test_ballistic_driver_matches_oracle_and_broad_phase(orc):
    lvb = _lvb()
    from oracle.statemachine import OracleLVB
    s = scenes.ballistic()
    s.vel[:, :3] *= 10.0
    P = _params(orc, s)
    dem = lvb.DEM(s)
    H = dem.lvb.stats()["rnl_max"]
    sm = OracleLVB(s.pos, 1, 0.1, s.dt, H, 0)
    for k in range(200):
        if k % 50 == 0:
            _check_step(orc, dem, s, P)
        else:
            dem.step()
        x = dem.state()[0]
        f, _ = sm.step(x)
        assert np.array_equal(dem.lvb.flags(), f)
    pi, pj = dem.lvb.pairs_ij()
    assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj)
    dem.close()


def test_contact_forces_match_oracle(orc):
    # every contact's normal force (dem_get_contact_forces: the pair i < j,
    # the force on i, the overlap) against the binary64 oracle at the
    # driver's own x' and v*: the contact sets agree except for overlaps
    # within 1e-14 m of zero (below the compensated binary32 overlap's
    # error), each force component within 1e-5 of the contact's summed
    # terms |k_n delta| + |damping|, and the overlap within the rounding of
    # the binary32 it is returned in
    lvb = _lvb()
    s = scenes.packed(n=6000, seed=12, vsigma=0.5)
    P = _params(orc, s)
    dem = lvb.DEM(s)
    for k in range(3):
        dem.advance(40)
        x, _, _, vstar = dem.state()
        gi, gj, gf, gd = dem.contact_forces()
        oi, oj, of, od, sc = orc.dem_contacts(x, vstar, P)
        g = set(zip(gi.tolist(), gj.tolist()))
        o = dict(zip(zip(oi.tolist(), oj.tolist()), range(len(oi))))
        assert len(oi) > 5000
        only_o = [p for p in o if p not in g]
        assert all(abs(od[o[p]]) <= 1e-14 for p in only_o), only_o[:5]
        idx = [(t, o[p]) for t, p in enumerate(zip(gi.tolist(), gj.tolist())) if p in o]
        assert len(idx) == len(gi) - sum(1 for p in g if p not in o)
        for p in g:
            if p not in o:     # a contact only the GPU sees: overlap ~0 there too
                t = list(zip(gi.tolist(), gj.tolist())).index(p)
                assert abs(gd[t]) <= 1e-14
        a, b = np.array(idx).T
        err = np.abs(gf[a].astype(np.float64) - of[b])
        assert (err <= 1e-5 * sc[b][:, None]).all(), err.max()
        # the overlap, returned in binary32: within its rounding
        assert np.all(np.abs(gd[a] - od[b]) <= 2.0 ** -23 * np.abs(od[b]) + 1e-15)
    dem.close()


def test_advance_graph_matches_phase_launches(orc):
    # the fused step (dem_advance: graphs of one cooperative launch per
    # step) and the phase-by-phase step (dem_phase) use the same arithmetic,
    # but the order of a row's entries -- set by concurrent slot claims --
    # orders each force sum, so the two runs agree to rounding, and a
    # packed bed carries the difference forward: positions to 1e-9 m and
    # velocities to 1e-4 relative after 250 steps
    lvb = _lvb()
    s = scenes.packed(n=3000, seed=4)
    a = lvb.DEM(s)
    b = lvb.DEM(s)
    a.advance(250)          # two graph replays of 100 steps + 50 direct steps
    for _ in range(250):
        b.step()
    xa, va, _, _ = a.state()
    xb, vb, _, _ = b.state()
    assert np.allclose(xa, xb, rtol=0, atol=1e-9)
    assert np.allclose(va, vb, rtol=1e-4, atol=1e-6)
    assert a.lvb.stats()["steps"] == b.lvb.stats()["steps"] == 250
    a.close()
    b.close()


def test_set_state_keeps_inverse_mass():
    # the driver keeps 1/m in the w of v (and of v*), which the integrator
    # reads: dem_set_state ignores the caller's v.w and restores it, so the
    # next position half-step is the one of a context that was not reset
    lvb = _lvb()
    s = scenes.packed(n=800, seed=13, vsigma=0.2)
    dems = [lvb.DEM(s), lvb.DEM(s)]
    for dem in dems:
        dem.step()
    x, v, a, vs = dems[0].state()
    im = vs[:, 3].copy()
    assert np.all(im > 0) and np.array_equal(v[:, 3], im)
    v0 = v.copy()
    v0[:, 3] = -1.0
    dems[1].set_state(x, v0, a)
    assert np.array_equal(dems[1].state()[1], v)
    for dem in dems:
        dem.phase(lvb.DEM_PHASE_INTEGRATE)
    s0, s1 = dems[0].state(), dems[1].state()
    assert np.array_equal(s0[0], s1[0]) and np.array_equal(s0[3], s1[3])
    for dem in dems:
        dem.close()


def test_settling_full_size_step_parity(orc):
    # 200,000 polydisperse particles, graph-replayed steps, then one checked
    # step over every particle
    lvb = _lvb()
    s = scenes.settling()
    P = _params(orc, s)
    dem = lvb.DEM(s)
    dem.advance(200)
    _check_step(orc, dem, s, P)
    assert dem.sync() == 0
    st = dem.lvb.stats()
    assert st["steps"] == 201
    dem.close()


def test_drum_full_size_step_parity(orc):
    # 2,000,000 spheres in the rotating drum as the benchmark runs it (bed
    # turned 30 degrees, 5% in a dilute cascading layer): 1,000
    # graph-replayed steps, then one step checked over every particle
    lvb = _lvb()
    s = scenes.drum(tilt_deg=30.0, cascade=0.05)
    P = _params(orc, s)
    dem = lvb.DEM(s)
    dem.advance(1000)
    in_contact = _check_step(orc, dem, s, P)
    assert dem.sync() == 0
    assert dem.lvb.stats()["steps"] == 1001
    assert in_contact > 0
    dem.close()
