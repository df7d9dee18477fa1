"""Error paths made from the host, without a device fault.

* A non-finite position given to lvb_step: the step flags nothing for it,
  the context reports LVB_ENAN from then on, and a fresh context on valid
  positions again matches the oracle.
* A full cell: with the host's growth of the stores switched off (test hook
  LVB_OPT_GROW = 0), a step that moves more particles into one cell than it
  has slots reports LVB_EOVERFLOW.
* A full row store: with growth off and the usable store capped near the
  list's size (LVB_OPT_STORE_LIMIT), a step whose rows outgrow it -- so
  that even a re-layout without slack does not fit -- reports
  LVB_EOVERFLOW; the DEM driver's forces then read no rows.
Every access stays inside its buffer on these paths (the stores are only
capped logically, below their allocations), and after each error a fresh
context agrees with the oracle.
"""
import numpy as np
import pytest

from paper_2208_13770_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lvb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_13770_gb300 import lvb
    return lvb


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _fresh_matches_oracle(lvb, orc, s, steps=20):
    from oracle.statemachine import OracleLVB
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor)
    sm = OracleLVB(s.pos, orc.SKIN_DIAMETER_FACTOR, 0.1, s.dt, ctx.stats()["rnl_max"], 0)
    for pos, _ in scenes.ballistic_trajectory(s, steps):
        ctx.step(_dev(pos))
        f, _ = sm.step(pos)
        assert np.array_equal(ctx.flags(), f)
    pi, pj = ctx.pairs_ij()
    assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj)
    assert ctx.sync() == lvb.LVB_OK
    ctx.close()


def test_nan_position_reports_enan(orc):
    lvb = _lvb()
    s = scenes.ballistic(n=2000, seed=41, vsigma=2.0)
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor)
    traj = list(scenes.ballistic_trajectory(s, 6))
    for pos, _ in traj[:3]:
        ctx.step(_dev(pos))
    assert ctx.sync() == lvb.LVB_OK
    bad = traj[3][0].copy()
    bad[17, 1] = np.nan
    bad[1900, 2] = np.inf
    ctx.step(_dev(bad))
    assert ctx.sync() == lvb.LVB_ENAN
    # sticky: later steps and every synchronising call report it
    ctx.step(_dev(traj[4][0]))
    assert ctx.sync() == lvb.LVB_ENAN
    with pytest.raises(lvb.LVBError):
        ctx.pairs_ij()
    ctx.close()
    # a non-finite radius or position at init is refused
    p0 = s.pos.copy()
    p0[5, 3] = np.nan
    with pytest.raises(lvb.LVBError) as ei:
        lvb.LVB(_dev(p0), s.lo, s.hi, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, s.dt,
                lvb.LVB_TRIGGER_PARTIAL, s.cell_factor)
    assert ei.value.code == lvb.LVB_ENAN
    _fresh_matches_oracle(lvb, orc, s)


def test_full_cell_reports_eoverflow(orc):
    lvb = _lvb()
    s = scenes.ballistic(n=2000, seed=43, vsigma=0.5)
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor)
    st = ctx.stats()
    ccap = st["cell_capacity"]
    L = st["cell_edge"]
    ctx.set_option(lvb.LVB_OPT_GROW, 0)
    # ccap + 40 particles moved onto points inside one cell (overlapping:
    # the broad phase does not mind), all flagged in the same step
    pos = s.pos.copy()
    c = np.array(s.lo, np.float32) + np.float32(2.5 * L)
    k = ccap + 40
    assert k < s.n
    rng = np.random.default_rng(3)
    pos[:k, :3] = c + rng.uniform(-0.2 * L, 0.2 * L, size=(k, 3)).astype(np.float32)
    ctx.step(_dev(pos))
    assert ctx.sync() == lvb.LVB_EOVERFLOW
    with pytest.raises(lvb.LVBError):
        ctx.stats()
    ctx.close()
    # with the slots raised beforehand (LVB_OPT_CELL_CAPACITY) the same move
    # fits, and the list is the oracle's
    from oracle.statemachine import OracleLVB
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor)
    ctx.set_option(lvb.LVB_OPT_CELL_CAPACITY, 2 * k)
    sm = OracleLVB(s.pos, orc.SKIN_DIAMETER_FACTOR, 0.1, s.dt, st["rnl_max"], 0)
    ctx.step(_dev(pos))
    sm.step(pos)
    assert ctx.sync() == lvb.LVB_OK
    pi, pj = ctx.pairs_ij()
    assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj)
    assert ctx.stats()["cell_capacity"] >= 2 * k
    ctx.close()
    _fresh_matches_oracle(lvb, orc, s)


def test_full_row_store_reports_eoverflow(orc):
    lvb = _lvb()
    s = scenes.ballistic(n=2000, seed=47, vsigma=0.5)
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor)
    # cells with room for the crowd below (so that only the row store
    # fills up), grown at the next step
    ctx.set_option(lvb.LVB_OPT_CELL_CAPACITY, 512)
    ctx.step(_dev(s.pos))
    assert ctx.sync() == lvb.LVB_OK
    st = ctx.stats()
    assert st["cell_capacity"] >= 512
    ctx.set_option(lvb.LVB_OPT_GROW, 0)
    ctx.set_option(lvb.LVB_OPT_STORE_LIMIT, st["entries"] + 64)
    # 150 particles packed into a small cube: their rows grow far past their
    # slack, the step re-lays the store out, and the rows do not fit even
    # without slack under the limit
    pos = s.pos.copy()
    L = st["cell_edge"]
    c = np.array(s.lo, np.float32) + np.float32(4.5 * L)
    rng = np.random.default_rng(5)
    pos[:150, :3] = c + rng.uniform(-0.8 * L, 0.8 * L, size=(150, 3)).astype(np.float32)
    ctx.step(_dev(pos))
    assert ctx.sync() == lvb.LVB_EOVERFLOW
    ctx.close()
    _fresh_matches_oracle(lvb, orc, s)


def test_dem_store_failure_reads_no_rows():
    # the DEM driver on a context whose row store failed: the step reports
    # LVB_EOVERFLOW, and the forces phase (which reads the rows) reads none
    lvb = _lvb()
    s = scenes.packed(n=3000, seed=7, vsigma=0.5)
    dem = lvb.DEM(s)
    dem.lvb.set_option(lvb.LVB_OPT_CELL_CAPACITY, 512)
    dem.step()
    assert dem.sync() == lvb.LVB_OK
    st = dem.lvb.stats()
    assert st["cell_capacity"] >= 512
    dem.lvb.set_option(lvb.LVB_OPT_GROW, 0)
    dem.lvb.set_option(lvb.LVB_OPT_STORE_LIMIT, st["entries"] + 64)
    x, v, a, _ = dem.state()
    L = st["cell_edge"]
    c = np.array(s.lo, np.float32) + np.float32(3.5 * L)
    rng = np.random.default_rng(9)
    x[:150, :3] = c + rng.uniform(-0.8 * L, 0.8 * L, size=(150, 3)).astype(np.float32)
    v[:150, :3] = 0.0
    dem.set_state(x, v, a)
    dem.step()
    assert dem.sync() == lvb.LVB_EOVERFLOW
    dem.step()          # forces skip the rows; no access outside them
    assert dem.sync() == lvb.LVB_EOVERFLOW
    dem.close()
