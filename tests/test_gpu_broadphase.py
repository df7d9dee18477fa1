"""GPU parity of the broad phase (through the C-ABI) against the oracle.

On identical position snapshots the flags, the reference state, the pair set
and the contact set must match the oracle exactly (binary32 fixed formula),
at every checked step.
"""
import numpy as np
import pytest

from paper_2208_13770_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_13770_gb300 import lvb
    return lvb


def _H(scene_pos, cell_factor):
    rmax = np.float32(scene_pos[:, 3].max())
    L = cell_factor * 2.0 * float(rmax) * (1 + 2 ** -7)
    return np.float32(0.5 * L * (1 - 2 ** -8))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _csr_from_pairs(n, pi, pj):
    """Symmetric CSR (rows ascending) of an unordered pair list."""
    a = np.concatenate([pi, pj]).astype(np.int64)
    b = np.concatenate([pj, pi]).astype(np.int64)
    order = np.lexsort((b, a))
    a, b = a[order], b[order]
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(ptr, a + 1, 1)
    return np.cumsum(ptr), b


def _compare(ctx, sm, pos_h, step, check_contacts=True):
    pi, pj = ctx.pairs_ij()
    assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj), \
        "pair set differs at step %d: gpu %d oracle %d" % (step, len(pi), len(sm.pi))
    # every row, seen from both ends: symmetric, no duplicates, same set
    ptr, col = ctx.pairs_csr()
    optr, ocol = _csr_from_pairs(len(pos_h), sm.pi, sm.pj)
    assert np.array_equal(ptr, optr) and np.array_equal(col, ocol), \
        "symmetric rows differ at step %d" % step
    ref = ctx.ref()
    assert np.array_equal(ref, sm.ref), "reference state differs at step %d" % step
    if check_contacts:
        ci, cj, dl = ctx.contacts(_dev(pos_h))
        oi, oj, od = sm.contacts(pos_h)
        assert np.array_equal(ci, oi) and np.array_equal(cj, oj)
        assert np.array_equal(dl, od)


def _run_trajectory(orc, scene, snaps, trigger, skin_kind, skin_value, every=1, cell_factor=1.25,
                    options=()):
    lvb = _cuda()
    from oracle.statemachine import OracleLVB
    H = _H(scene.pos, cell_factor)
    pos0 = scene.pos
    vel0 = scene.vel
    ctx = lvb.LVB(_dev(pos0), scene.lo, scene.hi, skin_kind, skin_value, scene.dt, trigger,
                  cell_factor, vel=_dev(vel0))
    for opt, val in options:
        ctx.set_option(opt, val)
    assert ctx.stats()["rnl_max"] == H
    sm = OracleLVB(pos0, skin_kind, skin_value, scene.dt, H, trigger, vel4=vel0)
    _compare(ctx, sm, pos0, 0)
    nflag = 0
    for k, (pos, vel) in enumerate(snaps, start=1):
        ctx.step(_dev(pos), _dev(vel))
        f, _ = sm.step(pos, vel4=vel)
        nflag += int(f.sum())
        if k % every == 0:
            assert ctx.sync() == 0
            assert np.array_equal(ctx.flags(), f), "flags differ at step %d" % k
            _compare(ctx, sm, pos, k)
    st = ctx.stats()
    assert st["flagged_total"] == nflag
    assert st["pairs"] == len(sm.pi)
    ctx.close()
    return st, sm


@pytest.mark.parametrize("trigger", [0, 1, 2], ids=["partial", "global", "always"])
def test_ballistic_parity(orc, trigger):
    s = scenes.ballistic()
    steps = 1000 if trigger == 0 else 300
    every = 1 if trigger == 0 else 3
    st, sm = _run_trajectory(orc, s, scenes.ballistic_trajectory(s, steps), trigger, 1, 0.1,
                             every=every)
    assert st["steps"] == steps
    if trigger == 0:
        assert 0 < st["updated_total"] < s.n * steps


def test_ballistic_paper_rule_parity(orc):
    # skin = K |v| dt (Eq. skin_formulus1) with K = 200, the paper's default
    s = scenes.ballistic(n=2000, seed=21)
    _run_trajectory(orc, s, scenes.ballistic_trajectory(s, 600), 0, 2, 200.0, every=2)


SHAPES = [(1024, 0), (1024, 1), (512, 0), (256, 1)]


@pytest.mark.parametrize("threads,compact", SHAPES)
def test_hot_gas_many_rebuilds_parity(orc, threads, compact):
    # fast particles: many flags, cell moves and row changes per step, with
    # every launch shape of the step kernel (block size; flag compaction
    # per warp chunk or per block tile)
    lvb = _cuda()
    opts = ((lvb.LVB_OPT_BLOCK_THREADS, threads), (lvb.LVB_OPT_COMPACT, compact))
    s = scenes.ballistic(n=3000, seed=5, phi=0.3, vsigma=3.0)
    st, _ = _run_trajectory(orc, s, scenes.ballistic_trajectory(s, 150), 0, 1, 0.1,
                            options=opts)
    assert st["updated_total"] > s.n
    assert st["block_threads"] == threads and st["compaction"] == compact
    assert st["barriers"] >= st["steps"]


@pytest.mark.parametrize("direct_max", [0, 64])
def test_hot_gas_two_phase_rebuild_parity(orc, direct_max):
    # the rebuild with the cell moves first and a barrier before the rows
    # (every step, or only on steps with more than 64 flagged) gives the
    # same lists as the one-phase rebuild with the direct flagged test
    lvb = _cuda()
    s = scenes.ballistic(n=3000, seed=6, phi=0.3, vsigma=3.0)
    st, _ = _run_trajectory(orc, s, scenes.ballistic_trajectory(s, 150), 0, 1, 0.1,
                            options=((lvb.LVB_OPT_DIRECT_MAX, direct_max),))
    assert st["updated_total"] > s.n
    # one barrier after the check, one between moves and rows, one at the end
    assert st["barriers"] >= st["steps"] + (st["rebuild_steps"] if direct_max == 0 else 0)


def _random_walk(scene, steps, sigma, seed=0):
    rng = np.random.default_rng(seed)
    pos = scene.pos.copy()
    vel = scene.vel.copy()
    for _ in range(steps):
        pos[:, :3] += rng.normal(0.0, sigma, size=(len(pos), 3)).astype(np.float32)
        yield pos.copy(), vel


@pytest.mark.parametrize("n", [1, 2, 33, 1027])
def test_small_and_ragged_sizes(orc, n):
    s = scenes.ballistic(n=n, seed=40 + n, phi=0.2 if n > 8 else 0.05)
    s.vel[:, :3] *= 50.0
    _run_trajectory(orc, s, scenes.ballistic_trajectory(s, 40), 0, 1, 0.1)


def test_all_in_one_cell_and_outside_box(orc):
    # a dense clump (many same-cell pairs) and particles outside the box
    lvb = _cuda()
    rng = np.random.default_rng(3)
    n = 300
    pos = np.zeros((n, 4), dtype=np.float32)
    pos[:, :3] = rng.uniform(0.0, 2e-3, size=(n, 3))
    pos[:, 3] = 1e-3
    pos[:50, 0] -= 0.02            # left of the box
    pos[50:100, 2] += 0.05         # above the box
    s = scenes.Scene("clump", pos, np.zeros_like(pos), (0, 0, 0), (0.01, 0.01, 0.01), 1e-5, 10,
                     "box")
    st, sm = _run_trajectory(orc, s, _random_walk(s, 20, 5e-5), 0, 1, 0.1)
    assert st["pairs"] > 10000


def test_exact_cutoff_pair_on_gpu(orc):
    lvb = _cuda()
    # r = 0.5, skin = 0.125 (global), pair exactly at the cutoff 1.25 and one
    # ulp beyond; box large enough
    pos = np.array([[10, 10, 10, 0.5], [10.75, 11, 10, 0.5],
                    [20, 20, 20, 0.5], [20, 20, np.nextafter(np.float32(21.25), 99), 0.5]],
                   dtype=np.float32)
    ctx = lvb.LVB(_dev(pos), (0, 0, 0), (40, 40, 40), lvb.LVB_SKIN_GLOBAL, 0.125, 0.0,
                  lvb.LVB_TRIGGER_PARTIAL, 1.25)
    pi, pj = ctx.pairs_ij()
    assert list(zip(pi, pj)) == [(0, 1)]
    ctx.close()


def test_static_particles_never_flag(orc):
    lvb = _cuda()
    s = scenes.ballistic(n=500, seed=2)
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, 1, 0.1, s.dt, 0, 1.25)
    d = _dev(s.pos)
    for _ in range(20):
        ctx.step(d)
    st = ctx.stats()
    assert st["flagged_total"] == 0 and st["rebuild_steps"] == 0
    ctx.close()


@pytest.mark.parametrize("threads,compact", [(1024, 0), (256, 1)])
def test_relayout_when_rows_grow(orc, threads, compact):
    # contract the cloud towards its centre: rows grow past their slack and
    # the row store is re-laid out on the device; parity must hold throughout
    lvb = _cuda()
    s = scenes.ballistic(n=2000, seed=8, phi=0.25)

    def shrink(steps):
        # 1% per step: after 60 steps the cloud is 0.55 of its size and the
        # rows hold about six times their entries, past any row's slack
        pos = s.pos.copy()
        c = pos[:, :3].mean(axis=0)
        for _ in range(steps):
            pos[:, :3] = c + (pos[:, :3] - c) * np.float32(0.99)
            yield pos.copy(), s.vel

    st, _ = _run_trajectory(orc, s, shrink(60), 0, 1, 0.1,
                            options=((lvb.LVB_OPT_BLOCK_THREADS, threads),
                                     (lvb.LVB_OPT_COMPACT, compact)))
    assert st["relayouts"] > 0


def test_polydisperse_settling_subset_parity(orc):
    # polydisperse radii U[0.5, 2] mm, random displacements of mixed size
    s = scenes.settling(n=20_000, seed=77, footprint=0.06, height=0.6)
    st, _ = _run_trajectory(orc, s, _random_walk(s, 25, 1e-4, seed=1), 0, 1, 0.1, every=5)
    assert st["updated_total"] > 0


def test_store_growth_keeps_parity(orc):
    # skins that grow step by step (K|v|dt with the velocity handed to the
    # step ramping up 1000-fold): rows grow well past the initial row store,
    # which must grow on the fly (at 75% use), every step exact
    lvb = _cuda()
    from oracle.statemachine import OracleLVB
    s = scenes.ballistic(n=3000, seed=51, vsigma=2.0, phi=0.3)
    slow = s.vel.copy()
    slow[:, :3] *= 1e-3
    K = 400.0
    # ALWAYS: every particle takes the growing skin at every step; large
    # cells (factor 3) let the skins reach ~2 mm, rows ~60 partners
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, lvb.LVB_SKIN_PAPER_KVDT, K, s.dt, 2, 3.0,
                  vel=_dev(slow))
    sm = OracleLVB(s.pos, 2, K, s.dt, _H(s.pos, 3.0), 2, vel4=slow)
    cap0 = ctx.stats()["row_store_capacity"]
    steps = 60
    for k, (pos, vel) in enumerate(scenes.ballistic_trajectory(s, steps), start=1):
        v = vel.copy()
        v[:, :3] *= np.float32(10.0 ** (-3.0 + 3.0 * k / steps))
        ctx.step(_dev(pos), _dev(v))
        sm.step(pos, vel4=v)
        _compare(ctx, sm, pos, k, check_contacts=(k % 10 == 0))
    st = ctx.stats()
    assert st["grows"] > 0 and st["row_store_capacity"] > cap0
    ctx.close()


@pytest.mark.parametrize("threads", [1024, 256])
def test_global_and_always_small_blocks(orc, threads):
    lvb = _cuda()
    s = scenes.ballistic(n=1500, seed=12, vsigma=1.0)
    for trig in (1, 2):
        _run_trajectory(orc, s, scenes.ballistic_trajectory(s, 40), trig, 1, 0.1,
                        options=((lvb.LVB_OPT_BLOCK_THREADS, threads),))


def test_resume_from_saved_reference(orc):
    # lvb_init_resume on a saved reference state continues exactly
    lvb = _cuda()
    from oracle.statemachine import OracleLVB
    s = scenes.ballistic(n=2000, seed=31, vsigma=0.5)
    traj = list(scenes.ballistic_trajectory(s, 80))
    a = lvb.LVB(_dev(s.pos), s.lo, s.hi, 1, 0.1, s.dt, 0, 1.25)
    for pos, _ in traj[:40]:
        a.step(_dev(pos))
    ref = a.ref()
    b = lvb.LVB(_dev(traj[39][0]), s.lo, s.hi, 1, 0.1, s.dt, 0, 1.25, ref=_dev(ref))
    sm = OracleLVB(traj[39][0], 1, 0.1, s.dt, _H(s.pos, 1.25), 0, ref4=ref)
    for pos, _ in traj[40:]:
        a.step(_dev(pos))
        b.step(_dev(pos))
        sm.step(pos)
    for ctx in (a, b):
        pi, pj = ctx.pairs_ij()
        assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj)
        assert np.array_equal(ctx.ref(), sm.ref)
    bad = ref.copy()
    bad[0, 3] = 1.0                    # skin above the cap
    with pytest.raises(lvb.LVBError):
        lvb.LVB(_dev(traj[39][0]), s.lo, s.hi, 1, 0.1, s.dt, 0, 1.25, ref=_dev(bad))
    a.close()
    b.close()


def test_settling_full_size_parity(orc):
    # the 200,000-particle settling box at full size: complete pair-set parity
    # after init and after steps with many flags
    s = scenes.settling()
    st, _ = _run_trajectory(orc, s, _random_walk(s, 6, 6e-5, seed=2), 0, 1, 0.1, every=3)
    assert st["n"] == 200_000


def test_drum_full_size_parity(orc):
    # the 2,000,000-sphere drum (lognormal radii, 0.2 m axis) at full size:
    # complete pair-set, row, reference-state and contact parity after init
    # and after three random-walk steps that flag a fifth of the particles
    s = scenes.drum()
    st, sm = _run_trajectory(orc, s, _random_walk(s, 3, 6e-5, seed=2), 0, 1, 0.1, every=3)
    assert st["n"] == 2_000_000
    assert st["flagged_total"] > 500_000


def _crowd_moves(s, n_cells=20, per_cell=20, seed=31):
    """One step in which `per_cell` particles jump into each of `n_cells`
    cells at once while the particles that were in those cells jump out:
    many concurrent movers reuse the cells' emptied slots and append new
    ones.  Returns the snapshots (this step, then a step with no motion)."""
    rng = np.random.default_rng(seed)
    pos = s.pos.copy()
    rmax = np.float32(pos[:, 3].max())
    L = 1.25 * 2.0 * float(rmax) * (1 + 2 ** -7)
    lo = np.array(s.lo, np.float64)
    dims = np.ceil((np.array(s.hi, np.float64) - lo) / L).astype(int)
    cell = np.clip(np.floor((pos[:, :3] - lo) / L).astype(int), 0, dims - 1)
    key = (cell[:, 2] * dims[1] + cell[:, 1]) * dims[0] + cell[:, 0]
    inner = np.array([c for c in range(dims.prod())
                      if all(0 < v < d - 1 for v, d in zip(
                          ((c % dims[0]), (c // dims[0]) % dims[1], c // (dims[0] * dims[1])),
                          dims))])
    targets = rng.choice(inner, n_cells, replace=False)
    residents = np.nonzero(np.isin(key, targets))[0]
    others = rng.permutation(np.nonzero(~np.isin(key, targets))[0])
    movers = others[:n_cells * per_cell]
    for t, c in enumerate(targets):
        cx, cy, cz = c % dims[0], (c // dims[0]) % dims[1], c // (dims[0] * dims[1])
        idx = movers[t * per_cell:(t + 1) * per_cell]
        u = rng.uniform(0.2, 0.8, size=(per_cell, 3))
        pos[idx, :3] = (lo + (np.array([cx, cy, cz]) + u) * L).astype(np.float32)
    # the residents leave for random places elsewhere in the box
    hi = np.array(s.hi, np.float64)
    pos[residents, :3] = rng.uniform(lo + 2 * L, hi - 2 * L,
                                     size=(len(residents), 3)).astype(np.float32)
    return [(pos.copy(), s.vel), (pos.copy(), s.vel)], len(residents)


def _tiny_and_big(n=6000, n_big=100, seed=32):
    """Many tiny spheres among a few big ones, scattered in a 25 mm box: the
    cell edge follows the big ones, so a cell has room for thousands of slots."""
    rng = np.random.default_rng(seed)
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = rng.uniform(1e-3, 24e-3, size=(n, 3))
    pos[:, 3] = 5e-5
    pos[:n_big, 3] = 1e-3
    return scenes.Scene("tiny_and_big", pos, np.zeros_like(pos), (0, 0, 0),
                        (0.025, 0.025, 0.025), 1e-5, 2, "box")


@pytest.mark.parametrize("direct_max", [4096, 0], ids=["one_phase", "two_phase"])
@pytest.mark.parametrize("crowd", ["20x20", "1x2000"])
def test_crowded_cell_moves_parity(orc, direct_max, crowd):
    # particles move into a few cells in one step while the cells' former
    # occupants move out: concurrent moves claim the freed slots and append
    # new ones (up to 2,000 movers into one cell); every particle must end in
    # exactly one slot, so the lists must still equal the oracle's
    lvb = _cuda()
    if crowd == "20x20":
        s = scenes.ballistic(n=3000, seed=31, phi=0.3)
        snaps, n_res = _crowd_moves(s)
        moved = 400
    else:
        s = _tiny_and_big()
        snaps, n_res = _crowd_moves(s, n_cells=1, per_cell=2000, seed=33)
        moved = 2000
    assert n_res > 0
    # slots for the whole crowd (the cells are sized for the scene as it
    # starts, and grow only between steps)
    st, _ = _run_trajectory(orc, s, snaps, 0, 1, 0.1,
                            options=((lvb.LVB_OPT_DIRECT_MAX, direct_max),
                                     (lvb.LVB_OPT_CELL_CAPACITY, 4096)))
    assert st["flagged_total"] >= moved + n_res
    assert st["cell_capacity"] >= 4096


def test_near_cutoff_pairs_match_oracle(orc):
    # the pairs whose squared distance is within rel of the squared cutoff:
    # planted pairs at the cutoff and one or a few ulps away from it among
    # background particles (skin 0), then a ballistic scene at rel 1e-3
    # after steps with many flags
    lvb = _cuda()
    from tests.test_oracle_broadphase import _near_pairs_scene
    ref, rad, expected = _near_pairs_scene()
    rng = np.random.default_rng(14)
    bg = np.zeros((300, 4), np.float32)
    bg[:, :3] = rng.uniform((-1.5, -1.5, -1.5), (2.5, 41.5, 1.5), size=(300, 3))
    bg[:, 3] = 0.3
    pos = np.concatenate([ref, bg])
    pos[:len(ref), 3] = rad
    ctx = lvb.LVB(_dev(pos), (-2, -2, -2), (3, 43, 2), lvb.LVB_SKIN_GLOBAL, 0.0, 0.0,
                  lvb.LVB_TRIGGER_PARTIAL, 1.25)
    ref0 = pos.copy()
    ref0[:, 3] = 0.0                     # (xref, skin) at init, skin 0
    assert np.array_equal(ctx.ref(), ref0)
    for rel in (0.0, 1e-6, 1e-5, 1e-3):
        gi, gj = ctx.near_cutoff(rel)
        oi, oj = orc.near_cutoff(ref0, pos[:, 3], rel)
        assert np.array_equal(gi, oi) and np.array_equal(gj, oj), rel
    gi, gj = ctx.near_cutoff(1e-6)
    assert expected <= set(zip(gi.tolist(), gj.tolist()))
    with pytest.raises(lvb.LVBError):
        ctx.near_cutoff(0.01)            # beyond what the 27 cells cover
    ctx.close()

    s = scenes.ballistic(n=2000, seed=15, vsigma=1.0)
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, 1, 0.1, s.dt, 0, s.cell_factor)
    for k, (p, _) in enumerate(scenes.ballistic_trajectory(s, 20)):
        ctx.step(_dev(p))
    gi, gj = ctx.near_cutoff(1e-3)
    oi, oj = orc.near_cutoff(ctx.ref(), s.pos[:, 3], 1e-3)
    assert len(oi) > 0
    assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
    ctx.close()


@pytest.mark.parametrize("kind,value", [(1, 0.1), (2, 300.0)], ids=["diameter", "paper_rule"])
def test_early_trigger_matches_oracle(orc, kind, value):
    # the early trigger (beta 0.9): on a step with a violation, the
    # particles past 0.9 of their skin are updated too; flags (the
    # violations), reference states and pair sets equal the oracle's state
    # machine with the same trigger at every step, and updates come on
    # fewer steps than without it
    lvb = _cuda()
    from oracle.statemachine import OracleLVB
    s = scenes.ballistic(n=3000, seed=61, vsigma=1.0)
    H = _H(s.pos, s.cell_factor)
    runs = {}
    for beta in (900, 1000):
        ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, kind, value, s.dt, lvb.LVB_TRIGGER_PARTIAL,
                      s.cell_factor, vel=_dev(s.vel))
        ctx.set_option(lvb.LVB_OPT_EARLY, beta)
        sm = OracleLVB(s.pos, kind, value, s.dt, H, 0, vel4=s.vel,
                       early_beta=np.float32(beta / 1000.0))
        for k, (pos, vel) in enumerate(scenes.ballistic_trajectory(s, 80), start=1):
            ctx.step(_dev(pos), _dev(vel))
            f, upd = sm.step(pos, vel4=vel)
            assert np.array_equal(ctx.flags(), f), k
            if k % 8 == 0 or k > 70:
                assert np.array_equal(ctx.ref(), sm.ref), k
                pi, pj = ctx.pairs_ij()
                assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj), k
        st = ctx.stats()
        assert st["updated_total"] == sm.updates and st["rebuild_steps"] == sm.rebuild_steps
        runs[beta] = st
        ctx.close()
    assert runs[900]["rebuild_steps"] < runs[1000]["rebuild_steps"]
    assert runs[900]["flagged_total"] < runs[900]["updated_total"]
    with pytest.raises(lvb.LVBError):
        ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, kind, value, s.dt, lvb.LVB_TRIGGER_GLOBAL,
                      s.cell_factor, vel=_dev(s.vel))
        try:
            ctx.set_option(lvb.LVB_OPT_EARLY, 900)
        finally:
            ctx.close()


def test_early_trigger_fused_dem_step(orc):
    # the same inside the DEM driver's fused step (position half-step in the
    # check, forces as the tail), one direct launch per step
    lvb = _cuda()
    from oracle.statemachine import OracleLVB
    s = scenes.packed(n=6000, seed=63, vsigma=3.0)
    dem = lvb.DEM(s)
    dem.lvb.set_option(lvb.LVB_OPT_EARLY, 850)
    H = dem.lvb.stats()["rnl_max"]
    sm = OracleLVB(s.pos, 1, 0.1, s.dt, H, 0, ref4=dem.lvb.ref(), early_beta=np.float32(0.85))
    for k in range(60):
        dem.advance(1)
        x = dem.state()[0]
        f, _ = sm.step(x)
        assert np.array_equal(dem.lvb.flags(), f), k
    assert np.array_equal(dem.lvb.ref(), sm.ref)
    pi, pj = dem.lvb.pairs_ij()
    assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj)
    st = dem.lvb.stats()
    assert st["updated_total"] == sm.updates and sm.updates > st["flagged_total"] > 0
    dem.close()
