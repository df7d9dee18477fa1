"""lvb_pairs_noalloc, the allocation-free list build, against a context.

Collected last on purpose: the entry point's working memory is one fixed
device array shared by every call, so these tests also show that it works
after the rest of the suite has used the device, and that one call leaves
nothing behind that changes the next (two calls in a row, on different and
on repeated inputs).  Every call's pair set is compared with two others:
the CPU oracle's pair set for the same reference state (its own brute-force
or linked-cell search), and lvb_get_pairs_ij of a context that holds that
state.  Pairs come back in no particular order, so the sets are compared.
"""
import ctypes

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


def _box(lvb, lo, hi):
    b = lvb.lvb_box()
    for k in range(3):
        b.lo[k], b.hi[k] = float(lo[k]), float(hi[k])
    return b


def _noalloc(lvb, pos_d, ref_d, box, cap):
    n = int(pos_d.shape[0])
    pi = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    pj = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    cnt = ctypes.c_int64(-1)
    rc = lvb.lvb_pairs_noalloc(n, pos_d.data_ptr(), ref_d.data_ptr(), ctypes.byref(box),
                               pi.data_ptr(), pj.data_ptr(), cap, ctypes.byref(cnt),
                               torch.cuda.current_stream().cuda_stream)
    return rc, cnt.value, pi.cpu().numpy(), pj.cpu().numpy()


def _keys(n, pi, pj):
    return np.sort(pi.astype(np.int64) * n + pj.astype(np.int64))


def _check_against_context(lvb, ctx, pos_d, box):
    """One call through the C-ABI; its pair set must be the oracle's and the
    context's."""
    import oracle
    ei, ej = ctx.pairs_ij()
    n = ctx.n
    ref = ctx.ref()
    oi, oj = oracle.pairs(ref, pos_d.cpu().numpy()[:, 3])
    assert np.array_equal(_keys(n, ei, ej), _keys(n, oi, oj))
    ref_d = _dev(ref)
    rc, cnt, pi, pj = _noalloc(lvb, pos_d, ref_d, box, len(ei) + 64)
    assert rc == lvb.LVB_OK, lvb.lvb_strerror(rc)
    assert cnt == len(ei)
    pi, pj = pi[:cnt], pj[:cnt]
    assert (pi < pj).all() and (pi >= 0).all() and (pj < n).all()
    got = _keys(n, pi, pj)
    assert np.array_equal(got, _keys(n, ei, ej))
    assert len(np.unique(got)) == cnt      # each pair once
    return got


def test_two_calls_in_a_row_match_context():
    lvb = _lvb()
    s = scenes.ballistic(n=2000, seed=71, vsigma=1.0)
    pos0 = _dev(s.pos)
    ctx = lvb.LVB(pos0, s.lo, s.hi, lvb.LVB_SKIN_PAPER_KVDT, 150.0, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor, vel=_dev(s.vel))
    box = _box(lvb, s.lo, s.hi)
    traj = list(scenes.ballistic_trajectory(s, 40))
    for pos, vel in traj[:20]:
        ctx.step(_dev(pos), _dev(vel))
    a = _check_against_context(lvb, ctx, _dev(traj[19][0]), box)
    for pos, vel in traj[20:]:
        ctx.step(_dev(pos), _dev(vel))
    st = ctx.stats()
    assert st["flagged_total"] > 0            # the reference state has moved on
    pos_last = _dev(traj[-1][0])
    b = _check_against_context(lvb, ctx, pos_last, box)
    c = _check_against_context(lvb, ctx, pos_last, box)
    assert not np.array_equal(a, b)
    assert np.array_equal(b, c)
    ctx.close()


def test_polydisperse_coarsened_grid():
    # 60,000 spheres of radius 0.5..2 mm in a 0.15 x 0.15 x 0.80 m box: cells
    # of 2 max R_NL would need ~2e5 cells, so the grid is coarsened to fit
    lvb = _lvb()
    s = scenes.settling(n=60_000, seed=73)
    pos_d = _dev(s.pos)
    ctx = lvb.LVB(pos_d, s.lo, s.hi, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.35, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor)
    box = _box(lvb, s.lo, s.hi)
    a = _check_against_context(lvb, ctx, pos_d, box)
    assert len(a) > 1000
    b = _check_against_context(lvb, ctx, pos_d, box)
    assert np.array_equal(a, b)
    ctx.close()


def test_capacity_and_limits():
    lvb = _lvb()
    s = scenes.ballistic(n=3000, seed=79, vsigma=0.5)
    pos_d = _dev(s.pos)
    ctx = lvb.LVB(pos_d, s.lo, s.hi, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.5, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor)
    box = _box(lvb, s.lo, s.hi)
    ei, ej = ctx.pairs_ij()
    full = set(_keys(ctx.n, ei, ej).tolist())
    assert len(full) > 20
    ref_d = _dev(ctx.ref())
    # too small an output: the full count comes back, the first cap pairs are
    # real pairs, nothing is written past cap
    rc, cnt, pi, pj = _noalloc(lvb, pos_d, ref_d, box, 10)
    assert rc == lvb.LVB_ECAPACITY and cnt == len(full)
    assert set(_keys(ctx.n, pi[:10], pj[:10]).tolist()) <= full
    # more particles than the fixed working memory holds: refused before any
    # launch (the buffers are never read)
    cnt = ctypes.c_int64(-1)
    rc = lvb.lvb_pairs_noalloc(lvb.LVB_NOALLOC_MAX_N + 1, pos_d.data_ptr(), ref_d.data_ptr(),
                               ctypes.byref(box), None, None, 0, ctypes.byref(cnt), None)
    assert rc == lvb.LVB_ELIMIT and cnt.value == 0
    assert "maximum" in lvb.lvb_strerror(rc)
    # misaligned records, an empty box, no particles
    rc = lvb.lvb_pairs_noalloc(10, pos_d.data_ptr() + 4, ref_d.data_ptr(), ctypes.byref(box),
                               None, None, 0, ctypes.byref(cnt), None)
    assert rc == lvb.LVB_EINVAL
    flat = _box(lvb, s.lo, s.lo)
    rc = lvb.lvb_pairs_noalloc(10, pos_d.data_ptr(), ref_d.data_ptr(), ctypes.byref(flat),
                               None, None, 0, ctypes.byref(cnt), None)
    assert rc == lvb.LVB_EINVAL
    rc = lvb.lvb_pairs_noalloc(0, pos_d.data_ptr(), ref_d.data_ptr(), ctypes.byref(box),
                               None, None, 0, ctypes.byref(cnt), None)
    assert rc == lvb.LVB_EINVAL
    # a stream being captured into a graph: refused before any launch (the
    # call synchronises its stream, which a capture does not allow)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    x = torch.zeros(4, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        graph.capture_begin()
        x.add_(1.0)
        cnt = ctypes.c_int64(-1)
        rc = lvb.lvb_pairs_noalloc(10, pos_d.data_ptr(), ref_d.data_ptr(), ctypes.byref(box),
                                   None, None, 0, ctypes.byref(cnt), side.cuda_stream)
        graph.capture_end()
    assert rc == lvb.LVB_EINVAL and cnt.value == 0
    graph.replay()
    torch.cuda.synchronize()
    assert x.sum().item() == 4.0
    # non-finite reference coordinate
    bad = ctx.ref()
    bad[7, 1] = np.nan
    rc, cnt, _, _ = _noalloc(lvb, pos_d, _dev(bad), box, 16)
    assert rc == lvb.LVB_ENAN
    # and a valid call right after the refused ones still agrees
    _check_against_context(lvb, ctx, pos_d, box)
    ctx.close()
