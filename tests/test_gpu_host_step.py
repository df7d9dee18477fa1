"""lvb_step_host: the broad-phase step on host buffers (positions, and
velocities for the paper's rule), with the copies of one step's inputs
overlapping the previous step and the flags copied back per step.  Without
any synchronisation between steps it must give, step by step, the oracle's
flags and flagged counts, and at the end its pair set."""
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


@pytest.mark.parametrize("kind,value,pinned_out", [(1, 0.1, True), (2, 200.0, True),
                                                   (1, 0.1, False)],
                         ids=["diameter", "paper_rule", "pageable_outputs"])
def test_step_host_matches_oracle_step_by_step(orc, kind, value, pinned_out):
    # the step writes its flag words into a device staging slot, which a
    # copy stream of the context copies out to the caller's buffers while
    # the next step runs; page-locked outputs overlap that copy, pageable
    # ones make it synchronous
    lvb = _lvb()
    from oracle.statemachine import OracleLVB
    s = scenes.ballistic(n=3000, seed=21, vsigma=1.0)
    traj = list(scenes.ballistic_trajectory(s, 40))
    m, n, nw = len(traj), s.n, (s.n + 31) // 32
    pos = torch.empty((m, n, 4), dtype=torch.float32, pin_memory=True)
    vel = torch.empty((m, n, 4), dtype=torch.float32, pin_memory=True)
    for k, (p, v) in enumerate(traj):
        pos[k].copy_(torch.from_numpy(p))
        vel[k].copy_(torch.from_numpy(v))
    if pinned_out:
        bits = torch.zeros((m, nw), dtype=torch.int32, pin_memory=True)
        nf = torch.full((m,), -1, dtype=torch.int32, pin_memory=True)
    else:
        bits = torch.from_numpy(np.zeros((m, nw), np.int32))
        nf = torch.from_numpy(np.full(m, -1, np.int32))
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, kind, value, s.dt, 0, s.cell_factor,
                  vel=_dev(s.vel))
    for k in range(m):
        ctx.step_host(pos[k], vel=vel[k] if kind == 2 else None, bits=bits[k],
                      n_flagged=nf[k:k + 1])
    assert ctx.sync() == 0
    H = np.float32(0.5 * s.cell_factor * 2.0 * float(np.float32(s.pos[:, 3].max()))
                   * (1 + 2 ** -7) * (1 - 2 ** -8))
    sm = OracleLVB(s.pos, kind, value, s.dt, H, 0, vel4=s.vel)
    total = 0
    for k, (p, v) in enumerate(traj):
        f, _ = sm.step(p, vel4=v)
        got = np.unpackbits(bits[k].numpy().view(np.uint8), bitorder="little")[:n].astype(bool)
        assert np.array_equal(got, f), "flags differ at step %d" % (k + 1)
        assert int(nf[k]) == int(f.sum())
        total += int(f.sum())
    assert total > 100
    pi, pj = ctx.pairs_ij()
    assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj)
    ctx.close()


def test_step_host_rejects_missing_velocity():
    lvb = _lvb()
    s = scenes.ballistic(n=500, seed=22)
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, 2, 100.0, s.dt, 0, s.cell_factor, vel=_dev(s.vel))
    with pytest.raises(lvb.LVBError):
        ctx.step_host(np.ascontiguousarray(s.pos, np.float32))
    ctx.close()
