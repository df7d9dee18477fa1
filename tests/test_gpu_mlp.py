"""The learned skin on the GPU against the oracle.

* inference: the exact binary32/bfloat16 formula, bit for bit;
* gradients of the mean squared error: against the binary64 oracle with the
  same bfloat16 roundings (straight-through), 1e-4 of the largest component
  (binary32 accumulation order differs);
* training on the GPU lowers the loss;
* the LEARNED skin policy inside the broad phase: the oracle recomputes every
  feature and proposal and must get the same skins, flags and pair sets;
* the rebuild log: the samples of a context's log equal the oracle's
  rebuild log (oracle.statemachine.RebuildLog) bit for bit, on a ballistic
  run and on a packed bed run by the DEM driver;
* the travel-form labels of the library equal the oracle's.
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


def _weights(seed):
    from oracle import mlp
    W = mlp.Weights.random(seed=seed, scale=0.6)
    W.mu = np.linspace(-0.5, 0.5, 8).astype(np.float32)
    W.isd = np.linspace(0.5, 2.0, 8).astype(np.float32)
    return W


@pytest.mark.parametrize("y_steps", [0.0, 400.0])
def test_inference_bit_exact(y_steps):
    # diameter form and travel form of the output
    lvb = _lvb()
    from oracle import mlp
    W = _weights(1)
    W.y_lo, W.y_hi = np.float32(0.05), np.float32(0.8)
    W.y_steps = np.float32(y_steps)
    rng = np.random.default_rng(2)
    n = 5000
    f = rng.normal(0, 2, (n, 8)).astype(np.float32)
    f[:, 0] = np.abs(f[:, 0]) * np.float32(1e-3)
    d = rng.uniform(1e-3, 4e-3, n).astype(np.float32)
    wbuf = lvb.mlp_weights_device(W.flat(), W.mu, W.isd, (W.y_lo, W.y_hi), y_steps)
    skin = torch.empty(n, device="cuda")
    y = torch.empty(n, device="cuda")
    fd, dd = _dev(f), _dev(d)
    rc = lvb.lvb_mlp_infer(fd.data_ptr(), dd.data_ptr(), n, wbuf.data_ptr(), skin.data_ptr(),
                           y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 0
    torch.cuda.synchronize()
    es, ey = mlp.infer(W, f, d)
    assert np.array_equal(y.cpu().numpy(), ey)
    assert np.array_equal(skin.cpu().numpy(), es)
    # the range is exercised on both sides
    assert (ey < W.y_lo).any() and (ey > W.y_hi).any() and ((ey > W.y_lo) & (ey < W.y_hi)).any()


@pytest.mark.parametrize("rel_floor", [0.0, 0.2])
def test_gradient_matches_oracle(rel_floor):
    # squared error, and relative error with a floor some labels fall below
    lvb = _lvb()
    from oracle import mlp
    W = _weights(5)
    rng = np.random.default_rng(6)
    n = 3000
    samp = np.zeros((n, 9), np.float32)
    samp[:, :8] = rng.normal(0, 2, (n, 8))
    samp[:, 8] = rng.normal(0.3, 0.2, n)
    grad = np.zeros(mlp.N_PARAMS, np.float32)
    loss = lvb.ctypes.c_double(0)
    p = W.flat()
    rc = lvb.lvb_mlp_grad(_dev(samp).data_ptr(), n, p.ctypes.data, W.mu.ctypes.data,
                          W.isd.ctypes.data, rel_floor, grad.ctypes.data, lvb.ctypes.byref(loss))
    assert rc == 0
    eloss, eg = mlp.loss_and_grad64(W, samp[:, :8], samp[:, 8], quantize=True,
                                    rel_floor=rel_floor)
    assert abs(loss.value - eloss) <= 1e-5 * eloss
    err = np.abs(grad - eg).max()
    assert err <= 1e-4 * np.abs(eg).max(), err


def test_training_lowers_loss():
    lvb = _lvb()
    from oracle import mlp
    rng = np.random.default_rng(8)
    n = 20000
    samp = np.zeros((n, 9), np.float32)
    samp[:, :8] = rng.normal(0, 1, (n, 8))
    samp[:, 8] = 0.3 + 0.2 * np.tanh(samp[:, 0]) + 0.1 * np.abs(samp[:, 1])
    p0 = mlp.Weights.random(seed=9, scale=0.3).flat()
    yr = np.zeros(2, np.float32)
    p, mu, isd, losses = lvb.mlp_train(_dev(samp), epochs=15, batch=256, lr=3e-3, seed=1,
                                       params0=p0, y_range_out=yr)
    assert losses[-1] < 0.2 * losses[0], losses
    # output range from the labels: mean / 16 and mean + 4 sd
    lab = samp[:, 8].astype(np.float64)
    assert np.isclose(yr[0], lab.mean() / 16, rtol=1e-5)
    assert np.isclose(yr[1], lab.mean() + 4 * lab.std(), rtol=1e-5)
    # the trained network, evaluated by the oracle's exact formula, fits the data
    W = mlp.Weights.from_flat(p, mu, isd)
    _, y = mlp.infer(W, samp[:2000, :8], np.ones(2000, np.float32))
    assert np.mean((y - samp[:2000, 8]) ** 2) < 0.3 * np.var(samp[:, 8]) + losses[-1]


def _learned_setup(lvb, s, seed=3):
    from oracle import mlp
    W = _weights(seed)
    # keep the proposals of the order of a tenth of a diameter, bounded
    W.b3 = np.float32(0.05)
    W.w3 *= np.float32(0.05)
    W.y_lo, W.y_hi = np.float32(0.01), np.float32(0.08)
    grid = mlp.grid_params(s.pos[:, 3].max(), s.cell_factor, s.lo, s.hi)
    return W, grid


@pytest.mark.parametrize("log,y_steps", [(False, 0.0), (True, 0.0), (False, 300.0)])
def test_learned_policy_broad_phase_parity(orc, log, y_steps):
    # with the rebuild log on or off (the log adds a pass and samples, and
    # must change nothing else), and in the travel form of the output: the
    # oracle's skins bit for bit
    lvb = _lvb()
    from oracle.statemachine import OracleLVB
    s = scenes.ballistic(n=2000, seed=17, vsigma=1.0)
    W, grid = _learned_setup(lvb, s)
    W.y_steps = np.float32(y_steps)
    wbuf = lvb.mlp_weights_device(W.flat(), W.mu, W.isd, (W.y_lo, W.y_hi), y_steps)
    acc = np.zeros_like(s.pos)
    acc[:, 2] = -9.81
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, lvb.LVB_SKIN_LEARNED, 0.0, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor, vel=_dev(s.vel), acc=_dev(acc),
                  mlp=wbuf)
    if log:
        ctx.log_enable(10, 100000)
    sm = OracleLVB(s.pos, orc.SKIN_LEARNED, 0.0, s.dt, grid["H"], 0, vel4=s.vel,
                   learned={"weights": W, "grid": grid}, acc4=acc)
    assert np.array_equal(ctx.ref(), sm.ref)
    nflag = 0
    for k, (pos, vel) in enumerate(scenes.ballistic_trajectory(s, 120), start=1):
        ctx.step(_dev(pos), _dev(vel), _dev(acc))
        f, _ = sm.step(pos, vel4=vel, acc4=acc)
        nflag += int(f.sum())
        if k % 4 == 0:
            assert np.array_equal(ctx.flags(), f), k
            assert np.array_equal(ctx.ref(), sm.ref), k
            pi, pj = ctx.pairs_ij()
            assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj), k
    assert nflag > 50
    ctx.close()


def test_learned_policy_full_size_drum_parity(orc):
    # the learned policy on the 1,000,000-sphere drum (lognormal radii):
    # skins proposed by the network at init and for every flagged particle of
    # two random-walk steps; flags, reference states and pair sets equal the
    # oracle's state machine with the same network
    lvb = _lvb()
    from oracle.statemachine import OracleLVB
    s = scenes.drum(n=1_000_000, length=0.1)
    W, grid = _learned_setup(lvb, s)
    wbuf = lvb.mlp_weights_device(W.flat(), W.mu, W.isd, (W.y_lo, W.y_hi))
    acc = np.zeros_like(s.pos)
    acc[:, 2] = -9.81
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, lvb.LVB_SKIN_LEARNED, 0.0, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor, vel=_dev(s.vel), acc=_dev(acc),
                  mlp=wbuf)
    sm = OracleLVB(s.pos, orc.SKIN_LEARNED, 0.0, s.dt, grid["H"], 0, vel4=s.vel,
                   learned={"weights": W, "grid": grid}, acc4=acc)
    assert np.array_equal(ctx.ref(), sm.ref)
    rng = np.random.default_rng(4)
    p = s.pos.copy()
    nflag = 0
    for k in range(2):
        p[:, :3] += rng.normal(0, 3e-5, size=(len(p), 3)).astype(np.float32)
        ctx.step(_dev(p), _dev(s.vel), _dev(acc))
        f, _ = sm.step(p, vel4=s.vel, acc4=acc)
        nflag += int(f.sum())
        assert np.array_equal(ctx.flags(), f), k
        assert np.array_equal(ctx.ref(), sm.ref), k
    pi, pj = ctx.pairs_ij()
    assert np.array_equal(pi, sm.pi) and np.array_equal(pj, sm.pj)
    assert nflag > 10_000
    ctx.close()


def _sorted_rows(a):
    a = np.asarray(a, np.float32)
    return a[np.lexsort(a.T[::-1])]


def test_rebuild_log_matches_oracle_ballistic(orc):
    # the log of a context (features of each update, largest displacement
    # over the horizon) against the oracle's rebuild log on the same
    # positions, velocities and accelerations: the same samples bit for bit
    # (the device appends them in no particular order, so sorted rows are
    # compared)
    lvb = _lvb()
    from oracle import mlp
    from oracle.statemachine import OracleLVB, RebuildLog
    s = scenes.ballistic(n=2000, seed=23, vsigma=1.0)
    acc = np.zeros_like(s.pos)
    acc[:, 2] = -9.81
    horizon = 10
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, lvb.LVB_SKIN_PAPER_KVDT, 60.0, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor, vel=_dev(s.vel), acc=_dev(acc))
    ctx.log_enable(horizon, 100000)
    grid = mlp.grid_params(s.pos[:, 3].max(), s.cell_factor, s.lo, s.hi)
    assert np.float32(ctx.stats()["rnl_max"]) == grid["H"]
    sm = OracleLVB(s.pos, orc.SKIN_PAPER_KVDT, 60.0, s.dt, grid["H"], 0, vel4=s.vel)
    log = RebuildLog(sm, grid, horizon)
    for pos, vel in scenes.ballistic_trajectory(s, 80):
        ctx.step(_dev(pos), _dev(vel), _dev(acc))
        log.step(pos, vel4=vel, acc4=acc)
    got, want = ctx.log_samples(), log.log()
    assert len(want) > 100
    assert got.shape == want.shape
    assert np.array_equal(_sorted_rows(got), _sorted_rows(want))
    ctx.close()


def test_rebuild_log_matches_oracle_packed_dem(orc):
    # the same on a packed bed run by the DEM driver, phase by phase: the
    # oracle is fed the driver's own state after each position half-step
    # (x', v* and a, what the broad phase sees)
    lvb = _lvb()
    from oracle import mlp
    from oracle.statemachine import OracleLVB, RebuildLog
    s = scenes.packed(n=4000, seed=31, vsigma=3.0)
    horizon = 7
    dem = lvb.DEM(s)
    dem.lvb.log_enable(horizon, 100000)
    H = np.float32(dem.lvb.stats()["rnl_max"])
    grid = mlp.grid_params(s.pos[:, 3].max(), s.cell_factor, s.lo, s.hi)
    assert grid["H"] == H
    sm = OracleLVB(s.pos, orc.SKIN_DIAMETER_FACTOR, s.skin_value, s.dt, H, 0,
                   ref4=dem.lvb.ref())
    log = RebuildLog(sm, grid, horizon)
    for _ in range(120):
        dem.phase(lvb.DEM_PHASE_INTEGRATE)
        x, _, a, vstar = dem.state()
        dem.phase(lvb.DEM_PHASE_BROAD)
        dem.phase(lvb.DEM_PHASE_FORCES)
        log.step(x, vel4=vstar, acc4=a)
    got, want = dem.lvb.log_samples(), log.log()
    assert len(want) > 100
    assert got.shape == want.shape
    assert np.array_equal(_sorted_rows(got), _sorted_rows(want))
    assert np.array_equal(dem.lvb.ref(), sm.ref)
    dem.close()


def test_travel_labels_match_oracle(orc):
    # lvb_mlp_travel_labels against the oracle's travel_labels: random
    # samples with some particles at rest (f0 = 0), and a real log
    lvb = _lvb()
    from oracle import mlp
    rng = np.random.default_rng(5)
    smp = rng.uniform(0.0, 2.0, size=(200_003, 9)).astype(np.float32)
    smp[rng.random(len(smp)) < 0.1, 0] = 0.0
    for h, margin, q in ((400, 2.0, 0.99), (7, 1.5, 0.5), (1, 1.0, 1.0)):
        got = lvb.mlp_travel_labels(smp, h, margin, q)
        want = mlp.travel_labels(smp, h, margin, q)
        assert got.shape == want.shape
        assert np.array_equal(got, want), (h, margin, q)
    s = scenes.ballistic(n=2000, seed=29, vsigma=1.0)
    ctx = lvb.LVB(_dev(s.pos), s.lo, s.hi, lvb.LVB_SKIN_DIAMETER_FACTOR, 0.1, s.dt,
                  lvb.LVB_TRIGGER_PARTIAL, s.cell_factor, vel=_dev(s.vel))
    ctx.log_enable(10, 100000)
    for pos, vel in scenes.ballistic_trajectory(s, 60):
        ctx.step(_dev(pos), _dev(vel))
    real = ctx.log_samples()
    ctx.close()
    assert len(real) > 50
    assert np.array_equal(lvb.mlp_travel_labels(real, 10, 2.0, 0.99),
                          mlp.travel_labels(real, 10, 2.0, 0.99))
    # argument checks
    import ctypes
    m = ctypes.c_int64(0)
    d = _dev(smp[:10])
    o = torch.empty_like(d)
    for args in ((0, 2.0, 0.5), (10, 0.0, 0.5), (10, 2.0, 0.0), (10, 2.0, 1.5)):
        rc = lvb.lvb_mlp_travel_labels(d.data_ptr(), 10, *args, o.data_ptr(), ctypes.byref(m))
        assert rc == lvb.LVB_EINVAL, args
    rc = lvb.lvb_mlp_travel_labels(d.data_ptr(), 10, 10, 2.0, 0.5, d.data_ptr(), ctypes.byref(m))
    assert rc == lvb.LVB_EINVAL
