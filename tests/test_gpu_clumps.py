"""Multi-sphere clumps: the broad phase on bounding spheres, the narrow phase
on sub-spheres (lvb_clump_contacts), against the oracle's brute force over
every pair of clumps.

1,500 rigid clumps of one to four spheres (random body offsets and radii,
each bounding radius covering its clump with the stated margin) move and
turn: positions ballistic, orientations q(t) = q0 * exp(w t / 2) rounded to
binary32 (the same inputs on both sides).  The context's list is kept on the
bounding spheres with skin 0.1 of the bounding diameter; at every checked
step the sub-sphere contacts found from the list equal the oracle's over
all pairs -- (i, a, j, b) and the overlap bit for bit -- so no contact is
missed and none is invented.
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


def _dev(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _clumps(n, seed):
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 5, size=n)
    off = np.concatenate([[0], np.cumsum(k)]).astype(np.int32)
    m = int(off[-1])
    r = rng.uniform(0.3e-3, 0.8e-3, size=m)
    b = rng.normal(0, 0.5e-3, size=(m, 3))
    sub = np.zeros((m, 4), np.float32)
    sub[:, :3] = b
    sub[:, 3] = r
    ext = np.linalg.norm(sub[:, :3].astype(np.float64), axis=1) + sub[:, 3]
    R = np.array([ext[off[i]:off[i + 1]].max() for i in range(n)])
    R = (R / (1.0 - 2.0 ** -12) * (1.0 + 1e-6)).astype(np.float32)
    # bounding spheres on a jittered lattice, close enough for contacts
    spacing = 1.7 * float(R.max())
    side = int(np.ceil(n ** (1 / 3)))
    idx = rng.permutation(side ** 3)[:n]
    c = np.stack([idx % side, (idx // side) % side, idx // side ** 2], 1) * spacing
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = c + rng.uniform(-0.05, 0.05, size=(n, 3)) * spacing
    pos[:, 3] = R
    vel = rng.normal(0, 0.8, size=(n, 3))
    q0 = rng.normal(size=(n, 4))
    q0 /= np.linalg.norm(q0, axis=1, keepdims=True)
    w = rng.normal(0, 200.0, size=(n, 3))
    lo = (-spacing, -spacing, -spacing)
    hi = (side * spacing + spacing,) * 3
    return pos, vel, q0, w, off, sub, lo, hi


def _qmul(a, b):
    w1, x1, y1, z1 = a.T
    w2, x2, y2, z2 = b.T
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)


def _state(pos0, vel, q0, w, t):
    pos = pos0.copy()
    pos[:, :3] = (pos0[:, :3].astype(np.float64) + vel * t).astype(np.float32)
    ang = np.linalg.norm(w, axis=1) * t
    axis = w / np.maximum(np.linalg.norm(w, axis=1, keepdims=True), 1e-30)
    dq = np.concatenate([np.cos(ang / 2)[:, None], axis * np.sin(ang / 2)[:, None]], 1)
    q = _qmul(q0, dq)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return pos, q.astype(np.float32)


def test_clump_contacts_match_oracle(orc):
    lvb = _lvb()
    pos0, vel, q0, w, off, sub, lo, hi = _clumps(1500, seed=7)
    dt = 2e-5
    ctx = lvb.LVB(_dev(pos0), lo, hi, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, dt,
                  lvb.LVB_TRIGGER_PARTIAL, 1.25)
    d_off, d_sub = _dev(off, np.int32), _dev(sub)
    total = 0
    for k in range(1, 161):
        pos, q = _state(pos0, vel, q0, w, k * dt)
        ctx.step(_dev(pos))
        if k % 20 == 0:
            got = ctx.clump_contacts(_dev(pos), _dev(q), d_off, d_sub)
            want = orc.clump_contacts(pos, q, off, sub)
            for g, o in zip(got, want):
                assert np.array_equal(g, o), k
            total += len(want[0])
    assert total > 200
    assert ctx.stats()["flagged_total"] > 0
    # the same contacts written in place to device outputs, and a short
    # capacity (the count, the first cap written)
    d_pos, d_q = _dev(pos), _dev(q)
    want = orc.clump_contacts(pos, q, off, sub)
    m = len(want[0])
    for cap in (m + 7, m // 2):
        outs = [torch.empty(cap, dtype=torch.int32, device="cuda") for _ in range(4)] + \
            [torch.empty(cap, dtype=torch.float32, device="cuda")]
        assert ctx.clump_contacts_into(d_pos, d_q, d_off, d_sub, *outs) == m
        got = [o[:min(cap, m)].cpu().numpy() for o in outs]
        o = np.lexsort((got[3], got[1], got[2], got[0]))
        key = lambda c: (c[0].astype(np.int64) * 64 + c[1]) * (1 << 30) + c[2].astype(np.int64) * 64 + c[3]
        kw = key(want)
        kg = key([g[o] for g in got])
        if cap >= m:
            assert np.array_equal(kg, kw)
            assert np.array_equal(got[4][o], want[4])
        else:
            assert np.all(np.isin(kg, kw))
    # input checks: a bound without the margin, a quaternion off unit length
    import ctypes
    n = ctypes.c_int64(0)
    bad = pos0.copy()
    bad[3, 3] *= np.float32(0.999)
    rc = lvb._lib.lvb_clump_contacts(ctx.ctx, _dev(bad).data_ptr(), _dev(q).data_ptr(),
                                     d_off.data_ptr(), d_sub.data_ptr(), None, None, None, None,
                                     None, 0, ctypes.byref(n))
    assert rc == lvb.LVB_EINVAL
    bad_off = off.copy()
    bad_off[0] = -1
    rc = lvb._lib.lvb_clump_contacts(ctx.ctx, _dev(pos).data_ptr(), _dev(q).data_ptr(),
                                     _dev(bad_off, np.int32).data_ptr(), d_sub.data_ptr(), None,
                                     None, None, None, None, 0, ctypes.byref(n))
    assert rc == lvb.LVB_EINVAL
    qb = q.copy()
    qb[5] *= np.float32(1.01)
    rc = lvb._lib.lvb_clump_contacts(ctx.ctx, _dev(pos).data_ptr(), _dev(qb).data_ptr(),
                                     d_off.data_ptr(), d_sub.data_ptr(), None, None, None, None,
                                     None, 0, ctypes.byref(n))
    assert rc == lvb.LVB_EINVAL
    ctx.close()
