"""The device-time trace of the step kernel (LVB_OPT_TRACE): the phases it
records are consistent with one another and with the step counters, and
tracing changes no result.

Per rebuild step the trace records the rebuild phase (after the check's
barrier to after the last barrier), the span of the rebuild's work items
(first start to last end) and the longest item; so the longest item lies
within the span and the span within the phase, and each of the three is
recorded once per step that rebuilt.  Two contexts, one traced, step
through the same scripted positions (a random walk) and must agree on
every flag count and on the list.
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


def test_trace_phases_are_consistent_and_change_nothing():
    lvb = _lvb()
    s = scenes.packed(n=6000, seed=23)
    pos0 = s.pos.astype(np.float32)
    ctxs = []
    for trace in (0, 1):
        ctx = lvb.LVB(torch.from_numpy(pos0).cuda(), s.lo, s.hi, lvb.LVB_SKIN_DIAMETER_FACTOR,
                      0.1, s.dt, lvb.LVB_TRIGGER_PARTIAL, 1.25)
        ctx.set_option(lvb.LVB_OPT_TRACE, trace)
        ctxs.append(ctx)
    rng = np.random.default_rng(5)
    x = pos0.copy()
    steps = 40
    for _ in range(steps):
        x[:, :3] += rng.normal(0.0, 3e-5, size=(len(x), 3)).astype(np.float32)
        p = torch.from_numpy(x).cuda()
        for ctx in ctxs:
            ctx.step(p)
    for ctx in ctxs:
        assert ctx.sync() == lvb.LVB_OK
    st = [c.stats() for c in ctxs]
    assert st[0]["flagged_total"] == st[1]["flagged_total"] > 0
    assert st[0]["rebuild_steps"] == st[1]["rebuild_steps"] > 0
    a, b = (c.pairs_ij() for c in ctxs)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    t = ctxs[1].trace()
    assert t["check"][1] == steps and t["check"][0] > 0
    rebuilt = t["rebuild"][1]
    assert rebuilt == st[1]["rebuild_steps"]
    assert t["rebuild_items"][1] == rebuilt == t["rebuild_item_max"][1]
    assert 0 < t["rebuild_item_max"][0] <= t["rebuild_items"][0] <= t["rebuild"][0]
    assert ctxs[0].trace()["check"][1] == 0
    for c in ctxs:
        c.close()
