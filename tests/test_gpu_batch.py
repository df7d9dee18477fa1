"""Batched contexts: many independent scenes of uneven size in one context
must give, scene by scene, exactly the oracle's result for that scene alone
(no pair joins two scenes), and the batched DEM driver must match the
binary64 oracle per scene with each scene's own walls."""
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


def _scenes(k, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(k):
        n = int(rng.integers(50, 3000))
        s = scenes.settling(n=n, seed=1000 + seed * 100 + q, footprint=0.03 + 0.01 * (q % 3),
                            height=0.5, rmin=0.5e-3, rmax=float(rng.uniform(1.0e-3, 2e-3)))
        out.append(s)
    return out


def _walks(sc, steps, sigma, seed):
    rng = np.random.default_rng(seed)
    pos = [s.pos.copy() for s in sc]
    for _ in range(steps):
        for p in pos:
            p[:, :3] += rng.normal(0, sigma, size=(len(p), 3)).astype(np.float32)
        yield [p.copy() for p in pos]


def test_batch_broad_phase_parity_per_scene(orc):
    lvb = _lvb()
    from oracle.statemachine import OracleLVB
    sc = _scenes(9, seed=3)
    off = np.concatenate([[0], np.cumsum([s.n for s in sc])]).astype(np.int64)
    pos0 = np.concatenate([s.pos for s in sc])
    ctx = lvb.LVB(_dev(pos0), [s.lo for s in sc], [s.hi for s in sc], 1, 0.1, 1e-6, 0, 1.25,
                  offsets=off)
    assert ctx.stats()["n_scenes"] == len(sc)
    sms = []
    for q, s in enumerate(sc):
        info = ctx.scene_info(q)
        assert info["first"] == off[q] and info["count"] == s.n
        rmax = np.float32(s.pos[:, 3].max())
        L = 1.25 * 2.0 * float(rmax) * (1 + 2 ** -7)
        H = np.float32(0.5 * L * (1 - 2 ** -8))
        assert info["rnl_max"] == H
        sms.append(OracleLVB(s.pos, 1, 0.1, 1e-6, H, 0))
    for k, snaps in enumerate(_walks(sc, 12, 1.2e-4, 5)):
        ctx.step(_dev(np.concatenate(snaps)))
        for sm, p in zip(sms, snaps):
            sm.step(p)
        if k % 4 == 3:
            pi, pj = ctx.pairs_ij()
            ei = np.concatenate([sm.pi + off[q] for q, sm in enumerate(sms)])
            ej = np.concatenate([sm.pj + off[q] for q, sm in enumerate(sms)])
            assert np.array_equal(pi, ei) and np.array_equal(pj, ej)
            ref = ctx.ref()
            assert np.array_equal(ref, np.concatenate([sm.ref for sm in sms]))
            fl = ctx.flags()
    st = ctx.stats()
    assert st["updated_total"] == sum(sm.updates for sm in sms) > 0
    ctx.close()


def test_identical_scenes_never_pair_across_scenes(orc):
    # four copies of the same scene in one context, moved by the same walk:
    # every flagged particle has a flagged twin at the same position in each
    # other scene, and the flagged counts stay small enough for the rebuild
    # to test flagged particles against each other directly.  Each scene must
    # still give exactly its own oracle result.
    lvb = _lvb()
    from oracle.statemachine import OracleLVB
    one = scenes.settling(n=2500, seed=77, footprint=0.04, height=0.3)
    sc = [one] * 4
    off = np.concatenate([[0], np.cumsum([s.n for s in sc])]).astype(np.int64)
    ctx = lvb.LVB(_dev(np.concatenate([s.pos for s in sc])), [s.lo for s in sc],
                  [s.hi for s in sc], 1, 0.1, 1e-6, 0, 1.25, offsets=off)
    rmax = np.float32(one.pos[:, 3].max())
    H = np.float32(0.5 * 1.25 * 2.0 * float(rmax) * (1 + 2 ** -7) * (1 - 2 ** -8))
    sm = OracleLVB(one.pos, 1, 0.1, 1e-6, H, 0)
    rng = np.random.default_rng(8)
    p = one.pos.copy()
    flagged = 0
    for k in range(8):
        # a few percent of the particles jump past their skin each step
        idx = rng.choice(one.n, 60, replace=False)
        p[idx, :3] += rng.normal(0, 4e-4, size=(60, 3)).astype(np.float32)
        ctx.step(_dev(np.concatenate([p] * 4)))
        f, _ = sm.step(p)
        flagged += int(f.sum())
        pi, pj = ctx.pairs_ij()
        ei = np.concatenate([sm.pi + off[q] for q in range(4)])
        ej = np.concatenate([sm.pj + off[q] for q in range(4)])
        assert np.array_equal(pi, ei) and np.array_equal(pj, ej), "step %d" % k
    assert ctx.sync() == 0
    st = ctx.stats()
    assert st["flagged_total"] == 4 * flagged > 0
    assert st["flagged_total"] // 8 < 4096
    ctx.close()


def test_batch_rejects_global_trigger():
    lvb = _lvb()
    sc = _scenes(2, seed=1)
    off = np.concatenate([[0], np.cumsum([s.n for s in sc])]).astype(np.int64)
    with pytest.raises(lvb.LVBError):
        lvb.LVB(_dev(np.concatenate([s.pos for s in sc])), [s.lo for s in sc],
                [s.hi for s in sc], 1, 0.1, 1e-6, 1, 1.25, offsets=off)


def test_batch_dem_matches_oracle_per_scene(orc):
    lvb = _lvb()
    from tests.test_gpu_dem import _params, RTOL
    sc = [scenes.packed(n=n, seed=70 + n, vsigma=0.3) for n in (500, 1500, 3000)]
    # shift boxes so that scenes overlap in space: they must still not interact
    dem = lvb.DEM(sc)
    off = dem.offsets
    for k in range(60):
        if k % 20 == 0:
            x, v, a, _ = dem.state()
            dem.step()
            x1, v1, a1, vs1 = dem.state()
            for q, s in enumerate(sc):
                sl = slice(off[q], off[q + 1])
                P = _params(orc, s)
                xo, vso, ao, vo, fmag = orc.dem_step(x[sl], v[sl], a[sl], s.dt, P, x_in=x1[sl],
                                                     vstar_in=vs1[sl], with_fmag=True)
                m = s.rho * 4 / 3 * np.pi * x[sl, 3].astype(np.float64) ** 3
                fs = (fmag / m)[:, None] + 9.81
                assert (np.abs(a1[sl, :3] - ao) - RTOL * fs).max() <= 0
        else:
            dem.step()
    assert dem.sync() == 0
    dem.close()


def test_autotuner_picks_a_measured_candidate_and_keeps_results():
    # the coordinate search times every candidate once and returns the
    # fastest; the launch choices (block size, compaction, the check's
    # loads) change no result
    lvb = _lvb()
    from paper_2208_13770_gb300 import autotune
    sc = _scenes(6, seed=11)
    best, trials = autotune.tune(sc, warm=20, steps=30)
    n_cf, n_bt, n_cp = len(autotune.CELL_FACTORS), len(autotune.BLOCK_THREADS), len(autotune.COMPACTION)
    n_ck = len(autotune.CHECK_LOADS)
    assert len(trials) == n_cf + (n_bt - 1) + (n_cp - 1) + (n_ck - 1)
    assert all(t["ms_per_step"] > 0 for t in trials)
    picked = [t for t in trials if (t["cell_factor"], t["block_threads"], t["compaction"],
                                    t["check_loads"]) ==
              (best.cell_factor, best.block_threads, best.compaction, best.check_loads)]
    assert picked and picked[0]["ms_per_step"] == min(t["ms_per_step"] for t in trials)
    # the chosen cell factor with two launch shapes: identical lists on the
    # same position snapshots (the broad phase is exact for any shape)
    off = np.concatenate([[0], np.cumsum([q.n for q in sc])]).astype(np.int64)
    pos0 = np.concatenate([q.pos for q in sc])
    ctxs = []
    for threads, comp, check in ((1024, 0, lvb.LVB_CHECK_REGS), (256, 1, lvb.LVB_CHECK_RING)):
        ctx = lvb.LVB(_dev(pos0), [q.lo for q in sc], [q.hi for q in sc], 1, 0.1, 1e-6, 0,
                      best.cell_factor, offsets=off)
        ctx.set_option(lvb.LVB_OPT_BLOCK_THREADS, threads)
        ctx.set_option(lvb.LVB_OPT_COMPACT, comp)
        ctx.set_option(lvb.LVB_OPT_CHECK_LOADS, check)
        ctxs.append(ctx)
    for snap in _walks(sc, 20, 2e-4, seed=5):
        p = _dev(np.concatenate(snap))
        for ctx in ctxs:
            ctx.step(p)
    a, b = (ctx.pairs_ij() for ctx in ctxs)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and len(a[0]) > 0
    assert ctxs[0].stats()["flagged_total"] == ctxs[1].stats()["flagged_total"] > 0
    for ctx in ctxs:
        ctx.close()


def test_full_size_batch_sampled_parity(orc):
    # the 512-scene, 6.2M-particle batch in the launch shape the autotuner
    # picked (cell factor 1.0, 512-thread blocks): three random-walk steps,
    # then, for a sample of scenes (the smallest, the largest and four
    # others), flags, reference states and pair sets against the oracle run
    # on that scene alone
    lvb = _lvb()
    from oracle.statemachine import OracleLVB
    sc = scenes.batch()
    off = np.concatenate([[0], np.cumsum([s.n for s in sc])]).astype(np.int64)
    assert off[-1] > 6_000_000
    pos0 = np.concatenate([s.pos for s in sc])
    ctx = lvb.LVB(_dev(pos0), [s.lo for s in sc], [s.hi for s in sc], 1, 0.1, 1e-6, 0, 1.0,
                  offsets=off)
    ctx.set_option(lvb.LVB_OPT_BLOCK_THREADS, 512)
    sizes = np.array([s.n for s in sc])
    rng = np.random.default_rng(12)
    pick = sorted({int(sizes.argmin()), int(sizes.argmax())}
                  | set(rng.choice(len(sc), 4, replace=False).tolist()))
    sms = {}
    for q in pick:
        rmax = np.float32(sc[q].pos[:, 3].max())
        H = np.float32(0.5 * 1.0 * 2.0 * float(rmax) * (1 + 2 ** -7) * (1 - 2 ** -8))
        assert ctx.scene_info(q)["rnl_max"] == H
        sms[q] = OracleLVB(sc[q].pos, 1, 0.1, 1e-6, H, 0)
    p = pos0.copy()
    last = {}
    for k in range(3):
        p[:, :3] += rng.normal(0, 6e-5, size=(len(p), 3)).astype(np.float32)
        ctx.step(_dev(p))
        for q in pick:
            last[q], _ = sms[q].step(p[off[q]:off[q + 1]])
    assert ctx.sync() == 0
    fl, ref = ctx.flags(), ctx.ref()
    pi, pj = ctx.pairs_ij()
    for q in pick:
        a, b = off[q], off[q + 1]
        sm = sms[q]
        assert np.array_equal(fl[a:b], last[q]), "scene %d" % q
        assert np.array_equal(ref[a:b], sm.ref), "scene %d" % q
        sel = (pi >= a) & (pi < b)
        assert ((pj[sel] >= a) & (pj[sel] < b)).all()
        assert np.array_equal(pi[sel] - a, sm.pi) and np.array_equal(pj[sel] - a, sm.pj), \
            "scene %d" % q
    assert ctx.stats()["flagged_total"] > 100_000
    ctx.close()
