"""Pins of the rebuild-log oracle and of the travel-form labels.

The rebuild log is the skin network's training data: each update of a
particle opens a record with its features, and `horizon` steps later the
record closes with the largest displacement since it opened, in diameters.
The cases below are worked out by hand on scripted motion (coordinates
exactly representable in binary32), so that a horizon off by one, a record
opened at the wrong step or from the post-update state, the last instead of
the largest displacement, or a label in the wrong unit each fails one of
them.
"""
import numpy as np
import pytest

from oracle import mlp


def _scene(xs):
    """Three particles of radius 0.5 (d = 1) far apart along y; particle 0
    moves along x through the scripted positions xs (one per step)."""
    pos = np.zeros((3, 4), np.float32)
    pos[:, 1] = [0.0, 100.0, 200.0]
    pos[:, 3] = 0.5
    traj = []
    for x in xs:
        p = pos.copy()
        p[0, 0] = x
        traj.append(p)
    return pos, traj


def _grid():
    # cells of 8 d_max: the cap H - r (3.5) is above every skin used here
    return mlp.grid_params(0.5, 8.0, (-50.0, -50.0, -50.0), (250.0, 250.0, 250.0))


def test_rebuild_log_closed_form(orc):
    from oracle.statemachine import OracleLVB, RebuildLog
    grid = _grid()
    # skin 1 (global); horizon 3
    pos0, traj = _scene([1.5, 4.0, 3.5, 2.75, 2.75, 4.25, 4.25, 4.25, 4.25])
    vel = np.zeros((3, 4), np.float32)
    vel[0, 0] = 2.0
    sm = OracleLVB(pos0, orc.SKIN_GLOBAL, 1.0, 0.25, grid["H"])
    log = RebuildLog(sm, grid, 3)
    for p in traj:
        log.step(p, vel4=vel)
    s = log.log()
    # step 1: |1.5 - 0| > 1 -> update, record opens at x = 1.5 (features of
    # the state before the update: age 1, f5 = 1.5 / 1).  Step 2: 4.0 flags
    # again (2.5 from 1.5), but the record is open: no second record.  Step
    # 3: 3.5, 0.5 from the new reference, no flag.  Step 4 (= 1 + 3): 2.75
    # flags (1.25 from 4.0) while the record is still open, so nothing opens;
    # the record closes with the largest displacement from 1.5 over steps
    # 2..4, max(2.5, 2.0, 1.25) = 2.5, in diameters (d = 1).  Step 6: 4.25
    # flags (1.5 from 2.75) and opens a record (age 6 - 4 = 2) that closes
    # at step 9 with 0.
    assert s.shape == (2, 9)
    a, b = s[0], s[1]
    assert a[8] == np.float32(2.5)
    assert a[4] == 1 and a[5] == np.float32(1.5)
    assert a[0] == np.float32(2.0 * 0.25)              # |v| dt / d
    assert a[2] == np.float32(np.float32(0.5) / grid["H"])
    assert b[8] == 0.0
    assert b[4] == 2 and b[5] == np.float32(1.5)       # updated at step 4, flagged at 6
    assert sm.updates == 4                             # steps 1, 2, 4 and 6


def test_rebuild_log_label_is_largest_not_last(orc):
    from oracle.statemachine import OracleLVB, RebuildLog
    grid = _grid()
    # large skin after the first update keeps it from flagging again
    pos0, traj = _scene([3.0, 6.0, 3.5, 3.0])
    sm = OracleLVB(pos0, orc.SKIN_DIAMETER_FACTOR, 2.0, 1.0, grid["H"])
    # skin = 2 d = 2: step 1 (|3 - 0| > 2) updates and opens at 3.0
    log = RebuildLog(sm, grid, 3)
    for p in traj:
        log.step(p)
    s = log.log()
    assert s.shape == (1, 9)
    assert s[0, 8] == np.float32(3.0)      # max(3.0, 0.5, 0.0), not the last (0)


def test_rebuild_log_horizon_one(orc):
    from oracle.statemachine import OracleLVB, RebuildLog
    grid = _grid()
    pos0, traj = _scene([1.5, 2.25, 2.0])
    sm = OracleLVB(pos0, orc.SKIN_GLOBAL, 1.0, 1.0, grid["H"])
    log = RebuildLog(sm, grid, 1)
    for p in traj:
        log.step(p)
    s = log.log()
    # opens at step 1 (x 1.5), closes at step 2 with |2.25 - 1.5| = 0.75
    assert s.shape == (1, 9) and s[0, 8] == np.float32(0.75)


def test_travel_labels_closed_form():
    s = np.zeros((7, 9), np.float32)
    s[:, 0] = [0.5, 0.0, 0.25, 1.0, 0.5, 2.0, 0.125]
    s[:, 3] = np.arange(7)                      # marks the rows
    s[:, 8] = [1, 5, 2, 8, 0.25, 4, 3]
    # kept: f0 > 0, in order; y = (t * 2) / (f0 * 4) = [1, 4, 4, 0.25, 1, 12]
    out = mlp.travel_labels(s, 4, 2.0, 0.5)
    assert list(out[:, 3]) == [0, 2, 3, 4, 5, 6]
    # sorted [0.25, 1, 1, 4, 4, 12]; rank floor(0.5 * 5) = 2 -> clip at 1
    assert list(out[:, 8]) == [1, 1, 1, 0.25, 1, 1]
    assert np.array_equal(out[:, :8], s[[0, 2, 3, 4, 5, 6], :8])
    # clip_q = 1: the largest value, nothing clipped
    out1 = mlp.travel_labels(s, 4, 2.0, 1.0)
    assert list(out1[:, 8]) == [1, 4, 4, 0.25, 1, 12]
    # every operation rounds to binary32: t = 1 + 2^-23, margin 5, f0 3,
    # horizon 3: 5 t = 5 + 1.25 ulp rounds to 5 + 2^-21, f0 horizon = 9 is
    # exact, and (5 + 2^-21) / 9 rounds to 0x1.1c71c8p-1, where one rounding
    # of the exact 5 t / 9 would give 0x1.1c71cap-1
    t = np.float32(1 + 2.0 ** -23)
    r = np.zeros((1, 9), np.float32)
    r[0, 0], r[0, 8] = 3.0, t
    got = mlp.travel_labels(r, 3, 5.0, 1.0)[0, 8]
    assert got == np.float32(float.fromhex("0x1.1c71c8p-1"))
    assert got != np.float32(float.fromhex("0x1.1c71cap-1"))
    # nothing kept
    assert mlp.travel_labels(s[[1]], 4, 2.0, 0.5).shape == (0, 9)
