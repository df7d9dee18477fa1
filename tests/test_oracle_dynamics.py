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


def _pair(u, w0=(0.0, 0.0, 0.0)):
    # sphere 0 at the origin, sphere 1 along +x overlapping it by 1e-5 m;
    # sphere 0 moves along +y at u, with angular velocity w0
    r = 1e-3
    x = np.array([[0, 0, 0, r], [2 * r - 1e-5, 0, 0, r]], np.float32)
    v = np.zeros((2, 4), np.float32)
    v[0, 1] = u
    w = np.zeros((2, 4), np.float32)
    w[0, :3] = w0
    z = np.zeros((2, 4), np.float32)
    return x, v, w, z


def _fric_consts(orc, r=1e-3, rho=2500.0, kn=1e4, e=0.7, kt_ratio=2.0 / 7.0, gt_ratio=0.5):
    r32 = float(np.float32(r))
    m = rho * 4.0 / 3.0 * np.pi * r32 ** 3
    zeta = -np.log(e) / np.sqrt(np.pi ** 2 + np.log(e) ** 2)
    gam_n = 2 * zeta * np.sqrt(m / 2 * kn)
    return m, kt_ratio * kn, gt_ratio * gam_n


def test_friction_oracle_sticking_pair_closed_form(orc):
    # a slow tangential motion sticks: the spring is v_t dt after one step,
    # F_t = -(k_t dt + gamma_t) v_t, and the torque on each sphere is
    # -r n x F_t (n from sphere 1 to sphere 0, about -x)
    P = orc.dem_params(wall_kind=orc.WALL_NONE, g=(0, 0, 0))
    u, dt = 1e-3, 1e-6
    x, v, w, z = _pair(u)
    u = float(np.float32(u))          # the inputs are binary32 values
    m, kt, gt = _fric_consts(orc)
    out = orc.dem_step_friction(x, v, z, w, z, dt, P, 0.5, 2.0 / 7.0, 0.5,
                                x_in=x, vstar_in=v, wstar_in=w)
    assert len(out["ci"]) == 1
    xi, f = out["xi"][0], out["f"][0]
    assert np.isclose(xi[1], u * dt, rtol=1e-12, atol=0) and xi[0] == 0 and xi[2] == 0
    ft = -(kt * dt + gt) * u
    assert np.isclose(f[1], ft, rtol=1e-12, atol=0)
    # torques: -r n x F_t with n = -x: (-x) x (F y) = -F z, so T = r F z;
    # the same for sphere 1 (both spheres turn the same way)
    I = 0.4 * m * float(np.float32(1e-3)) ** 2
    assert np.isclose(out["al"][0, 2], float(np.float32(1e-3)) * ft / I, rtol=1e-12, atol=0)
    assert np.isclose(out["al"][1, 2], out["al"][0, 2], rtol=1e-12, atol=0)
    # three steps at the same state, history carried: the spring grows by
    # v_t dt each step
    hist = (out["ci"], out["cj"], out["xi"])
    for k in range(2):
        out = orc.dem_step_friction(x, v, z, w, z, dt, P, 0.5, 2.0 / 7.0, 0.5, hist=hist,
                                    x_in=x, vstar_in=v, wstar_in=w)
        hist = (out["ci"], out["cj"], out["xi"])
    assert np.isclose(out["xi"][0, 1], 3 * u * dt, rtol=1e-12, atol=0)
    # a rotation of sphere 0 about z at w makes its contact point (at +r x)
    # move at w r along +y: v_rel = v - (r w x n) with n = -x gives u + r w
    x, v, w, z = _pair(u, w0=(0.0, 0.0, 0.5))
    out = orc.dem_step_friction(x, v, z, w, z, dt, P, 0.5, 2.0 / 7.0, 0.5,
                                x_in=x, vstar_in=v, wstar_in=w)
    rw = float(np.float32(1e-3)) * float(np.float32(0.5))
    assert np.isclose(out["xi"][0, 1], (u + rw) * dt, rtol=1e-9, atol=0)


def test_friction_oracle_sliding_pair_at_the_coulomb_limit(orc):
    # a fast tangential motion slides: |F_t| = mu F_n, F_t against v_t, and
    # the spring is the one that gives the capped force,
    # xi = -(F_t + gamma_t v_t) / k_t
    P = orc.dem_params(wall_kind=orc.WALL_NONE, g=(0, 0, 0))
    u, dt, mu = 10.0, 1e-6, 0.4
    x, v, w, z = _pair(u)
    mu = float(np.float32(mu))
    m, kt, gt = _fric_consts(orc)
    out = orc.dem_step_friction(x, v, z, w, z, dt, P, mu, 2.0 / 7.0, 0.5,
                                x_in=x, vstar_in=v, wstar_in=w)
    f, xi = out["f"][0], out["xi"][0]
    fn = -f[0]                    # normal force on sphere 0 along n = -x
    delta = 2 * float(np.float32(1e-3)) - float(np.float32(2e-3 - 1e-5))
    assert np.isclose(fn, 1e4 * delta, rtol=1e-12, atol=0)       # no normal motion
    assert np.isclose(f[1], -mu * fn, rtol=1e-12, atol=0) and f[2] == 0
    assert np.isclose(xi[1], -(f[1] + gt * u) / kt, rtol=1e-12, atol=0)


def test_friction_oracle_conserves_momentum(orc):
    # contact forces come in equal and opposite pairs: with no walls and no
    # gravity the total force on a dense random pack with random velocities
    # and spins sums to zero, and so does the change of momentum
    from paper_2208_13770_gb300 import scenes
    s = scenes.packed(n=1200, seed=8, vsigma=0.5)
    rng = np.random.default_rng(2)
    w = np.zeros_like(s.pos)
    w[:, :3] = rng.normal(0, 50.0, size=(len(s.pos), 3))
    z = np.zeros_like(s.pos)
    P = orc.dem_params(lo=s.lo, hi=s.hi, wall_kind=orc.WALL_NONE, g=(0, 0, 0))
    out = orc.dem_step_friction(s.pos, s.vel, z, w, z, 1e-6, P, 0.5, 2.0 / 7.0, 0.5)
    assert len(out["ci"]) > 300
    m = 2500.0 * 4.0 / 3.0 * np.pi * s.pos[:, 3].astype(np.float64) ** 3
    ptot = (m[:, None] * out["a"]).sum(axis=0)
    assert np.all(np.abs(ptot) <= 1e-12 * out["fmag"].sum())


def test_friction_oracle_without_friction_is_the_normal_step(orc):
    # mu = 0 caps every tangential force at zero: the step is the
    # frictionless velocity-Verlet step of orc_dem_step64 (pinned above by
    # free fall, restitution and energy), and no particle turns
    from paper_2208_13770_gb300 import scenes
    s = scenes.packed(n=800, seed=4, vsigma=0.3)
    P = orc.dem_params(lo=s.lo, hi=s.hi, wall_kind=orc.WALL_BOX)
    rng = np.random.default_rng(1)
    a = np.zeros_like(s.pos)
    a[:, :3] = rng.normal(0, 1.0, size=(len(s.pos), 3))
    w = np.zeros_like(s.pos)
    w[:, :3] = rng.normal(0, 10.0, size=(len(s.pos), 3))
    z = np.zeros_like(s.pos)
    out = orc.dem_step_friction(s.pos, s.vel, a, w, z, 1e-6, P, 0.0, 2.0 / 7.0, 0.5)
    xo, vso, ao, vo = orc.dem_step(s.pos, s.vel, a, 1e-6, P)
    assert len(out["ci"]) > 100
    for got, want in ((out["x"], xo), (out["vstar"], vso), (out["a"], ao), (out["v"], vo)):
        assert np.allclose(got, want, rtol=1e-13, atol=1e-300)
    assert np.all(out["al"] == 0)
    assert np.array_equal(out["w"], w[:, :3].astype(np.float64))
