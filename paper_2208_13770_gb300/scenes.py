"""Seeded synthetic scenes shaped like the paper's workloads.

This module only produces inputs: particle positions, radii, velocities and
the physical set-up.  It holds none of the method's arithmetic (no
displacement check, skin rule, pair or contact test), so both the CUDA path
and the CPU oracle can be fed from it.

The paper's own test cases (hopper discharge, vibrating incline, avalanche,
biomass furnace, powder levelling; Sec. Test-cases) need its in-house solver
and geometries, which are not available.  These scenes stand in for them:

* ``ballistic``   2,000 monodisperse spheres (r = 1 mm), packing fraction
                  0.30 in a cube, N(0, 0.01 m/s) velocities, specular walls.
* ``settling``    200,000 spheres with r ~ U[0.5, 2] mm (rho = 2500) in a
                  closed 0.15 x 0.15 x 0.80 m box, a dilute jittered-lattice
                  cloud (phi ~ 0.17) with small random velocities, under
                  gravity.
* ``drum``        lognormal radii (median 1 mm, sigma_ln = 0.35, clipped to
                  [0.4, 3] mm) in a horizontal drum (R = 0.3 m), a dense
                  size-stratified bed in solid-body rotation at 10 rpm.
* ``batch``       many independent ``settling``-style boxes with uneven
                  particle counts (log-uniform).

Placement is a jittered lattice, so particles never overlap at t = 0 by
construction.  Every generator is deterministic for a given seed (numpy
PCG64); the default seed of scene k is 2208_13770 + k.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2208_13770


@dataclasses.dataclass
class Scene:
    name: str
    pos: np.ndarray            # (n, 4) float32: x, y, z, r
    vel: np.ndarray            # (n, 4) float32: vx, vy, vz, 0
    lo: tuple                  # box lower corner [m]
    hi: tuple                  # box upper corner [m]
    dt: float                  # time step [s]
    steps: int                 # steps of the workload
    wall: str                  # "specular" | "box" | "drum"
    gravity: tuple = (0.0, 0.0, 0.0)
    kn: float = 1e4
    restitution: float = 0.7
    rho: float = 2500.0
    contacts: bool = True
    drum: tuple | None = None  # (cx, cz, R, omega) for wall == "drum"
    skin_kind: int = 1         # diameter factor
    skin_value: float = 0.1    # alpha
    cell_factor: float = 1.25  # cell edge / largest diameter
    mu: float = 0.0            # Coulomb friction between particles (0: none)
    kt_ratio: float = 2.0 / 7.0  # tangential / normal stiffness
    gt_ratio: float = 0.5      # tangential / normal damping

    @property
    def n(self) -> int:
        return len(self.pos)

    def copy(self) -> "Scene":
        return dataclasses.replace(self, pos=self.pos.copy(), vel=self.vel.copy())


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _jittered_lattice(rng, n, lo, hi, spacing, radii):
    """n sites of a simple-cubic lattice of the given spacing inside [lo, hi],
    chosen at random, each jittered within its free play (spacing - 2 r)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    dims = np.floor((hi - lo) / spacing).astype(np.int64)
    total = int(np.prod(dims))
    if total < n:
        raise ValueError("lattice too small: %d sites for %d particles" % (total, n))
    sites = rng.choice(total, size=n, replace=False)
    ix = sites % dims[0]
    iy = (sites // dims[0]) % dims[1]
    iz = sites // (dims[0] * dims[1])
    centre = lo + (np.stack([ix, iy, iz], axis=1) + 0.5) * spacing
    play = np.maximum(0.5 * spacing - radii, 0.0)[:, None]
    jitter = rng.uniform(-1.0, 1.0, size=(n, 3)) * play * 0.98
    return centre + jitter


def ballistic(n=2000, seed=SEED_BASE + 0, phi=0.30, r=1e-3, vsigma=0.01, dt=1e-5,
              steps=1000, skin_kind=1, skin_value=0.1, cell_factor=1.25) -> Scene:
    """Monodisperse spheres in free flight with specular walls."""
    rng = _rng(seed)
    side = (n * (4.0 / 3.0) * math.pi * r ** 3 / phi) ** (1.0 / 3.0)
    m = int(math.ceil(n ** (1.0 / 3.0)))
    while m ** 3 < n:
        m += 1
    spacing = side / m
    if spacing < 2 * r:
        raise ValueError("packing fraction too high for a lattice start")
    radii = np.full(n, r)
    xyz = _jittered_lattice(rng, n, (0, 0, 0), (side, side, side), spacing, radii)
    pos = np.zeros((n, 4), dtype=np.float32)
    pos[:, :3] = xyz
    pos[:, 3] = r
    vel = np.zeros((n, 4), dtype=np.float32)
    vel[:, :3] = rng.normal(0.0, vsigma, size=(n, 3))
    return Scene("ballistic", pos, vel, (0.0, 0.0, 0.0), (side, side, side), dt, steps,
                 "specular", contacts=False, skin_kind=skin_kind, skin_value=skin_value,
                 cell_factor=cell_factor)


def settling(n=200_000, seed=SEED_BASE + 1, rmin=0.5e-3, rmax=2e-3, footprint=0.15,
             height=0.80, vsigma=0.05, dt=1e-6, steps=20_000, skin_kind=1, skin_value=0.1,
             cell_factor=1.25) -> Scene:
    """Polydisperse spheres settling under gravity in a closed box.  The
    cloud occupies as many lattice layers as it needs from the floor up; the
    lattice spacing is the largest diameter (plus 1%)."""
    rng = _rng(seed)
    radii = rng.uniform(rmin, rmax, size=n)
    spacing = 2.0 * rmax * 1.01
    per_layer = int(math.floor(footprint / spacing)) ** 2
    layers = int(math.ceil(n / per_layer))
    fill_h = layers * spacing * (1.0 + 1e-9)   # exact multiple: keep the last layer
    if fill_h > height:
        raise ValueError("box too short for %d particles" % n)
    xyz = _jittered_lattice(rng, n, (0, 0, 0), (footprint, footprint, fill_h), spacing, radii)
    pos = np.zeros((n, 4), dtype=np.float32)
    pos[:, :3] = xyz
    pos[:, 3] = radii
    vel = np.zeros((n, 4), dtype=np.float32)
    vel[:, :3] = rng.normal(0.0, vsigma, size=(n, 3))
    return Scene("settling", pos, vel, (0.0, 0.0, 0.0), (footprint, footprint, height), dt,
                 steps, "box", gravity=(0.0, 0.0, -9.81), skin_kind=skin_kind,
                 skin_value=skin_value, cell_factor=cell_factor)


def _drum_layers(rng, radii, z0, R, length, margin):
    """Horizontal lattice layers inside the circle of radius R (x-z plane)
    from height z0 up: each layer's spacing is `margin` times the largest
    diameter among the next particles (radii sorted large-first), sites
    chosen at random and jittered within their free play.  Returns (xyz,
    height of the top of the last layer)."""
    n = len(radii)
    xyz = np.zeros((n, 3))
    placed = 0
    z = z0
    while placed < n:
        a = 2.0 * radii[placed] * margin
        zc = z + 0.5 * a
        if zc + 0.5 * a > R:
            raise ValueError("drum too small for %d particles" % n)
        half = math.sqrt(max(R * R - max(zc * zc, (zc - 0.5 * a) ** 2, (zc + 0.5 * a) ** 2), 0.0))
        half -= 0.5 * a
        nx = int(math.floor(2.0 * half / a)) if half > 0 else 0
        ny = int(math.floor(length / a))
        cnt = nx * ny
        if cnt > 0:
            take = min(cnt, n - placed)
            sites = rng.choice(cnt, size=take, replace=False)
            ix = sites % nx
            iy = sites // nx
            xs = -half + (ix + 0.5) * a
            ys = (iy + 0.5) * a
            r_l = radii[placed:placed + take]
            play = np.maximum(0.5 * a - r_l, 0.0) * 0.98
            xyz[placed:placed + take, 0] = xs + rng.uniform(-1, 1, take) * play
            xyz[placed:placed + take, 1] = ys + rng.uniform(-1, 1, take) * play
            xyz[placed:placed + take, 2] = zc + rng.uniform(-1, 1, take) * play
            placed += take
        z += a
    return xyz, z


def drum(n=2_000_000, seed=SEED_BASE + 2, R=0.3, length=0.20, rpm=10.0, median=1e-3,
         sigma_ln=0.35, rclip=(0.4e-3, 3e-3), dt=1e-6, steps=5000, skin_kind=1,
         skin_value=0.1, cell_factor=1.25, tilt_deg=0.0, cascade=0.0,
         cascade_speed=0.3, cascade_spacing=1.6) -> Scene:
    """A horizontal drum (axis along y, centre (0, 0) in x-z) holding a dense
    bed, stratified by size: radii are sorted large-first and laid in
    horizontal lattice layers from the bottom, each layer's spacing the
    largest diameter in it.  The bed starts in solid-body rotation.

    tilt_deg turns the whole load about the drum axis, so that the bed's free
    surface slopes as in a drum rotating in the rolling regime.  cascade > 0
    takes that fraction of the particles (a random subset of the radii) out
    of the bed and lays them, the same way but with cascade_spacing times the
    spacing (a packing fraction about cascade_spacing^-3 of the bed's), in
    layers on top of the bed, moving down the slope at cascade_speed [m/s]
    plus N(0, 0.05 m/s) per component: the dense bed and dilute cascading
    layer of a rotating drum, made by construction because a real drum needs
    about a revolution (6e6 steps of 1 us) to develop them."""
    rng = _rng(seed)
    radii = np.exp(rng.normal(math.log(median), sigma_ln, size=n))
    radii = np.clip(radii, rclip[0], rclip[1])
    n_c = int(round(cascade * n))
    r_c = np.zeros(0)
    if n_c > 0:
        pick = np.zeros(n, dtype=bool)
        pick[rng.choice(n, size=n_c, replace=False)] = True
        r_c = np.sort(radii[pick])[::-1].copy()
        radii = radii[~pick]
    radii = np.sort(radii)[::-1].copy()
    xyz, top = _drum_layers(rng, radii, -R, R, length, 1.0001)
    omega = rpm * 2.0 * math.pi / 60.0
    vel3 = np.zeros((len(radii), 3))
    # solid-body rotation about +y: v = omega x (x - c) with c on the axis
    vel3[:, 0] = omega * xyz[:, 2]
    vel3[:, 2] = -omega * xyz[:, 0]
    if n_c:
        xc, _ = _drum_layers(rng, r_c, top, R, length, cascade_spacing)
        vc = rng.normal(0.0, 0.05, size=(n_c, 3))
        xyz = np.concatenate([xyz, xc])
        vel3 = np.concatenate([vel3, vc])
        radii = np.concatenate([radii, r_c])
    th = math.radians(tilt_deg)
    if th:
        # turn positions and velocities about +y by th (distances from the
        # axis are kept, so every particle stays inside the drum)
        c, s_ = math.cos(th), math.sin(th)
        x, z = xyz[:, 0].copy(), xyz[:, 2].copy()
        xyz[:, 0], xyz[:, 2] = c * x - s_ * z, s_ * x + c * z
        vx, vz = vel3[:, 0].copy(), vel3[:, 2].copy()
        vel3[:, 0], vel3[:, 2] = c * vx - s_ * vz, s_ * vx + c * vz
    if n_c:
        # downhill along the turned surface: the surface direction (cos th,
        # sin th) in x-z, signed so that it points down
        down = np.array([math.cos(th), math.sin(th)])
        if down[1] > 0:
            down = -down
        vel3[-n_c:, 0] += cascade_speed * down[0]
        vel3[-n_c:, 2] += cascade_speed * down[1]
    pos = np.zeros((n, 4), dtype=np.float32)
    pos[:, :3] = xyz
    pos[:, 3] = radii
    vel = np.zeros((n, 4), dtype=np.float32)
    vel[:, :3] = vel3
    lo = (-R, 0.0, -R)
    hi = (R, length, R)
    return Scene("drum", pos, vel, lo, hi, dt, steps, "drum", gravity=(0.0, 0.0, -9.81),
                 drum=(0.0, 0.0, R, omega), skin_kind=skin_kind, skin_value=skin_value,
                 cell_factor=cell_factor)


def batch_sizes(n_scenes=512, seed=SEED_BASE + 3, nmin=1000, nmax=50_000):
    """Particle counts of the batched workload, log-uniform in [nmin, nmax]."""
    rng = _rng(seed)
    return np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=n_scenes)).astype(np.int64)


def batch(n_scenes=512, seed=SEED_BASE + 3, nmin=1000, nmax=50_000, steps=2000):
    """Independent settling boxes; box footprint scaled so that every scene
    has the same dilute packing fraction."""
    sizes = batch_sizes(n_scenes, seed, nmin, nmax)
    scenes = []
    for k, ns in enumerate(sizes):
        # same cloud density as ``settling``: 200k particles per 0.15^2 m^2 column
        fp = 0.15 * math.sqrt(ns / 200_000.0) * 1.6
        fp = max(fp, 0.03)
        h = 0.80
        scenes.append(settling(int(ns), seed=seed * 1000 + k, footprint=fp, height=h,
                               steps=steps))
    return scenes


def packed(n=8000, seed=SEED_BASE + 5, r=1e-3, spread=0.004, vsigma=0.05, dt=1e-6,
           steps=1000, skin_kind=1, skin_value=0.1, cell_factor=1.25) -> Scene:
    """A dense simple-cubic pack of near-monodisperse spheres resting on the
    floor of a box under gravity: lattice spacing 2r, radii r * U[1 - spread,
    1 + spread], so that about half of the neighbour pairs start in contact
    with overlaps of a few micrometres."""
    rng = _rng(seed)
    a = 2.0 * r
    m = int(math.ceil(n ** (1.0 / 3.0)))
    side = m * a
    radii = r * rng.uniform(1.0 - spread, 1.0 + spread, size=n)
    sites = rng.choice(m ** 3, size=n, replace=False)
    ix, iy, iz = sites % m, (sites // m) % m, sites // (m * m)
    pos = np.zeros((n, 4), dtype=np.float32)
    pos[:, 0] = (ix + 0.5) * a
    pos[:, 1] = (iy + 0.5) * a
    pos[:, 2] = (iz + 0.5) * a
    pos[:, 3] = radii
    vel = np.zeros((n, 4), dtype=np.float32)
    vel[:, :3] = rng.normal(0.0, vsigma, size=(n, 3))
    return Scene("packed", pos, vel, (0.0, 0.0, 0.0), (side, side, 2.0 * side), dt, steps, "box",
                 gravity=(0.0, 0.0, -9.81), skin_kind=skin_kind, skin_value=skin_value,
                 cell_factor=cell_factor)


def ballistic_trajectory(scene: Scene, steps: int):
    """Positions of a ballistic scene at steps 1..steps (free flight with
    specular walls, binary32 x <- x + v dt), for feeding a broad phase with
    snapshots.  Yields (pos, vel) copies."""
    pos = scene.pos.copy()
    vel = scene.vel.copy()
    lo = np.asarray(scene.lo, dtype=np.float32)
    hi = np.asarray(scene.hi, dtype=np.float32)
    dt = np.float32(scene.dt)
    r = pos[:, 3:4]
    for _ in range(steps):
        pos[:, :3] = pos[:, :3] + vel[:, :3] * dt
        low = pos[:, :3] < lo + r
        high = pos[:, :3] > hi - r
        pos[:, :3] = np.where(low, 2 * (lo + r) - pos[:, :3], pos[:, :3])
        pos[:, :3] = np.where(high, 2 * (hi - r) - pos[:, :3], pos[:, :3])
        vel[:, :3] = np.where(low | high, -vel[:, :3], vel[:, :3])
        yield pos.copy(), vel.copy()


SCENES = {"ballistic": ballistic, "settling": settling, "drum": drum, "packed": packed}
