"""Failure detection without a GPU fault: a grid-wide barrier of the step
kernel whose wait runs out.

The barrier is made to wait for one arrival more than the grid has (a flag
that nothing sets) with a short poll limit.  Every block gives up after its
polls, records the error and returns; the host reads LVB_ETIMEOUT, later
steps on that context do nothing and report the same, and the device stays
usable: a fresh context afterwards matches the oracle.  The same holds for
the DEM driver's fused step.
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


def test_barrier_timeout_is_reported_and_the_device_stays_usable(orc):
    lvb = _lvb()
    from oracle.statemachine import OracleLVB
    s = scenes.ballistic(n=2000, seed=61, vsigma=1.0)
    traj = list(scenes.ballistic_trajectory(s, 5))
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, 1, 0.1, s.dt, 0, s.cell_factor)
    ctx.set_option(lvb.LVB_OPT_BARRIER_SPINS, 1 << 12)
    ctx.set_option(lvb.LVB_OPT_BARRIER_EXTRA, 1)
    ctx.step(_dev(traj[0][0]))
    assert ctx.sync() == lvb.LVB_ETIMEOUT
    assert "barrier" in lvb.lvb_strerror(lvb.LVB_ETIMEOUT)
    ctx.step(_dev(traj[1][0]))          # the context is unusable: nothing runs
    assert ctx.sync() == lvb.LVB_ETIMEOUT
    ctx.close()
    # the device still works: a new context follows the oracle exactly
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, 1, 0.1, s.dt, 0, s.cell_factor)
    H = np.float32(0.5 * s.cell_factor * 2.0 * float(np.float32(s.pos[:, 3].max()))
                   * (1 + 2 ** -7) * (1 - 2 ** -8))
    sm = OracleLVB(s.pos, 1, 0.1, s.dt, H, 0)
    for pos, _ in traj:
        ctx.step(_dev(pos))
        sm.step(pos)
    assert ctx.sync() == 0
    pi, pj = ctx.pairs_ij()
    assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj)
    ctx.close()


def test_fused_dem_step_timeout(orc):
    lvb = _lvb()
    s = scenes.packed(n=3000, seed=9)
    dem = lvb.DEM(s)
    dem.lvb.set_option(lvb.LVB_OPT_BARRIER_SPINS, 1 << 12)
    dem.lvb.set_option(lvb.LVB_OPT_BARRIER_EXTRA, 1)
    dem.advance(3)                      # direct fused launches
    assert dem.sync() == lvb.LVB_ETIMEOUT
    dem.close()
    dem = lvb.DEM(s)
    dem.advance(120)                    # one graph of 100 steps + 20 direct
    assert dem.sync() == 0
    assert dem.lvb.stats()["steps"] == 120
    dem.close()
