"""Pins of the binary64 DEM oracle (velocity Verlet + linear spring-dashpot).

* free fall: velocity Verlet is exact for a constant acceleration, so the
  closed form x0 + v0 t + g t^2 / 2 must be met to rounding;
* head-on collision of two spheres: the coefficient of restitution
  e = exp(-zeta pi / sqrt(1 - zeta^2)) of the linear dashpot and the contact
  duration pi / omega_d, omega_d = sqrt(k/m_eff) sqrt(1 - zeta^2);
* e = 1: kinetic energy is conserved to O(dt^2);
* a sphere dropped on the floor of a box rebounds with e;
* the drum wall pushes inward along the radius;
* specular walls mirror position and velocity.
"""
import math

import numpy as np
import pytest


def _run(orc, x, v, r, dt, P, steps, record=None):
    x = np.array(x, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    # initial acceleration from the forces at t = 0
    a = _accel(orc, x, v, r, P)
    for k in range(steps):
        x, vstar, a, v = orc.dem_step64(x, v, a, r, dt, P)
        if record is not None:
            record(k + 1, x, v)
    return x, v, a


def _accel(orc, x, v, r, P):
    import ctypes
    n = len(x)
    F = np.zeros((n, 3))
    xx = np.ascontiguousarray(x, dtype=np.float64)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    rr = np.ascontiguousarray(r, dtype=np.float64)
    rc = orc.lib().orc_dem_forces64(n, xx.ctypes.data, rr.ctypes.data, vv.ctypes.data,
                                    ctypes.byref(P), F.ctypes.data, None)
    assert rc == 0
    m = P.rho * 4.0 / 3.0 * math.pi * rr ** 3
    return F / m[:, None] + np.array(P.g[:])


def test_free_fall_exact(orc):
    P = orc.dem_params(g=(0.0, 0.0, -9.81), wall_kind=orc.WALL_NONE)
    x0 = np.array([[0.1, 0.2, 0.5]])
    v0 = np.array([[0.3, -0.1, 2.0]])
    dt, steps = 1e-4, 250
    x, v, a = _run(orc, x0, v0, [1e-3], dt, P, steps)
    t = dt * steps
    g = np.array([0.0, 0.0, -9.81])
    assert np.allclose(x, x0 + v0 * t + 0.5 * g * t * t, rtol=0, atol=1e-13)
    assert np.allclose(v, v0 + g * t, rtol=0, atol=1e-13)
    assert np.allclose(a, g, rtol=0, atol=0)


def _head_on(orc, e, dt, vrel=0.2):
    r = 1e-3
    P = orc.dem_params(restitution=e, g=(0, 0, 0), wall_kind=orc.WALL_NONE)
    x = [[-r - 1e-6, 0, 0], [r + 1e-6, 0, 0]]
    v = [[vrel / 2, 0, 0], [-vrel / 2, 0, 0]]
    state = {"t_in": None, "t_out": None}

    def rec(k, x, v):
        d = x[1, 0] - x[0, 0]
        if d < 2 * r and state["t_in"] is None:
            state["t_in"] = k
        if state["t_in"] is not None and state["t_out"] is None and d >= 2 * r:
            state["t_out"] = k

    m = 2500 * 4 / 3 * math.pi * r ** 3
    w0 = math.sqrt(1e4 / (m / 2))
    zeta = -math.log(e) / math.sqrt(math.pi ** 2 + math.log(e) ** 2) if e < 1 else 0.0
    wd = w0 * math.sqrt(1 - zeta ** 2)
    steps = int((1e-5 + 1.3 * math.pi / wd) / dt)
    x, v, _ = _run(orc, x, v, [r, r], dt, P, steps, rec)
    return x, v, state, wd, vrel


def test_head_on_restitution_and_duration(orc):
    dt = 2e-8
    x, v, st, wd, vrel = _head_on(orc, 0.7, dt)
    e_meas = (v[1, 0] - v[0, 0]) / vrel
    assert abs(e_meas - 0.7) < 2e-3
    dur = (st["t_out"] - st["t_in"]) * dt
    assert abs(dur - math.pi / wd) < 3 * dt
    # momentum is conserved exactly by the pairwise law
    assert abs(v[0, 0] + v[1, 0]) < 1e-12


def test_elastic_energy_conserved(orc):
    dt = 2e-8
    x, v, st, wd, vrel = _head_on(orc, 1.0, dt)
    assert abs((v[1, 0] - v[0, 0]) / vrel - 1.0) < 1e-4


def test_floor_bounce(orc):
    r = 1e-3
    P = orc.dem_params(restitution=0.7, g=(0, 0, 0), lo=(0, 0, 0), hi=(1, 1, 1),
                       wall_kind=orc.WALL_BOX)
    x = [[0.5, 0.5, r + 1e-6]]
    v = [[0.0, 0.0, -0.1]]
    dt = 2e-8
    x, v, _ = _run(orc, x, v, [r], dt, P, 6000)
    assert abs(v[0, 2] / 0.1 - 0.7) < 2e-3 and v[0, 0] == 0.0


def test_drum_wall_pushes_inward(orc):
    r, R = 1e-3, 0.3
    P = orc.dem_params(g=(0, 0, 0), lo=(-R, 0, -R), hi=(R, 0.2, R), wall_kind=orc.WALL_DRUM,
                       drum_center=(0.0, 0.0), drum_radius=R)
    ang = 0.3
    depth = 1e-5
    rho_i = R - r + depth
    x = np.array([[rho_i * math.cos(ang), 0.1, rho_i * math.sin(ang)]])
    v = np.zeros((1, 3))
    F = _accel(orc, x, v, np.array([r]), P) * (2500 * 4 / 3 * math.pi * r ** 3)
    expect = -1e4 * depth * np.array([math.cos(ang), 0, math.sin(ang)])
    assert np.allclose(F, expect, rtol=1e-9, atol=0)


def test_specular_walls(orc):
    r = 1e-3
    P = orc.dem_params(g=(0, 0, 0), lo=(0, 0, 0), hi=(0.01, 0.01, 0.01),
                       wall_kind=orc.WALL_SPECULAR, contacts_on=False)
    x = np.array([[r + 1e-5, 0.005, 0.01 - r - 2e-5]])
    v = np.array([[-1.0, 0.0, 1.0]])
    x1, _, _, v1 = orc.dem_step64(x, v, np.zeros((1, 3)), [r], 3e-5, P)
    assert np.allclose(x1, [[r + 2e-5, 0.005, 0.01 - r - 1e-5]], rtol=0, atol=1e-15)
    assert np.array_equal(v1, [[1.0, 0.0, -1.0]])


def test_fed_state_is_used(orc):
    # forces are evaluated at the fed state, not at the oracle's own x'
    r = 1e-3
    P = orc.dem_params(g=(0, 0, 0), wall_kind=orc.WALL_NONE)
    x = np.array([[0.0, 0, 0], [0.01, 0, 0]])
    v = np.zeros((2, 3))
    xf = np.array([[0.0, 0, 0], [2 * r - 1e-5, 0, 0]])
    _, _, a, _ = orc.dem_step64(x, v, np.zeros((2, 3)), [r, r], 1e-6, P, xf=xf, vf=v)
    m = 2500 * 4 / 3 * math.pi * r ** 3
    assert np.allclose(a[1], [1e4 * 1e-5 / m, 0, 0], rtol=1e-12)
    assert np.allclose(a[0], -a[1], rtol=1e-12)


def test_contact_list_sums_to_the_net_forces(orc):
    # the per-contact forces of orc_dem_contacts64, summed per particle (the
    # force on i, its negation on j), are the net contact forces of
    # orc_dem_forces64 (pinned by the restitution and energy cases above);
    # and the head-on pair in closed form: f = k_n delta + gamma |v_n|
    from paper_2208_13770_gb300 import scenes
    s = scenes.packed(n=1500, seed=3, vsigma=0.3)
    P = orc.dem_params(lo=s.lo, hi=s.hi, wall_kind=orc.WALL_NONE)
    ci, cj, f3, dl, sc = orc.dem_contacts(s.pos, s.vel, P)
    assert len(ci) > 500 and (dl > 0).all()
    assert np.all(ci < cj) and np.all(np.diff(ci.astype(np.int64) * len(s.pos) + cj) > 0)
    F = np.zeros((len(s.pos), 3))
    np.add.at(F, ci, f3)
    np.add.at(F, cj, -f3)
    Fo = orc.dem_forces(s.pos, s.vel, P)
    assert np.allclose(F, Fo, rtol=0, atol=1e-12 * np.abs(Fo).max())
    r, m_rho = 1e-3, 2500.0
    x = np.array([[0, 0, 0, r], [2 * r - 1e-5, 0, 0, r]], np.float32)
    v = np.zeros((2, 4), np.float32)
    v[0, 0], v[1, 0] = 0.05, -0.05
    ci, cj, f3, dl, sc = orc.dem_contacts(x, v, orc.dem_params(wall_kind=orc.WALL_NONE))
    # the inputs are binary32 values, widened exactly
    r32, d32, v32 = (float(np.float32(q)) for q in (r, 2 * r - 1e-5, 0.05))
    m = m_rho * 4.0 / 3.0 * np.pi * r32 ** 3
    e = 0.7
    zeta = -np.log(e) / np.sqrt(np.pi ** 2 + np.log(e) ** 2)
    delta = 2 * r32 - d32
    f = 1e4 * delta + 2 * zeta * np.sqrt(m / 2 * 1e4) * (2 * v32)
    assert len(ci) == 1 and np.isclose(dl[0], delta, rtol=1e-12)
    assert np.isclose(f3[0, 0], -f, rtol=1e-12) and f3[0, 1] == 0 and f3[0, 2] == 0
