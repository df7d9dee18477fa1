"""Pins of the skin-network oracle: bfloat16 rounding against torch's own
conversion (a library routine) and hand cases, the fixed-order binary32 dot
product, a one-path network in closed form, and the binary64 backward pass
against central finite differences."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_round_hand_cases():
    one = np.float32(1.0)
    cases = {1.0: 1.0, 1 + 2 ** -8: 1.0, 1 + 3 * 2 ** -8: 1 + 2 ** -6,
             1 + 2 ** -7: 1 + 2 ** -7, -(1 + 3 * 2 ** -8): -(1 + 2 ** -6), 0.0: 0.0}
    for x, want in cases.items():
        assert mlp.bf16_round(np.array([x], np.float32))[0] == np.float32(want), x
    assert np.isinf(mlp.bf16_round(np.array([3.4e38], np.float32))[0])
    assert one == mlp.bf16_round(np.array([one]))[0]


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-30, 2000),
                        rng.normal(0, 1e30, 2000)]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mlp.bf16_round(x), want)


def test_fixed_order_dot_is_sequential_binary32():
    # a case where the order matters: 1 + 2^-24 + 2^-24 in order gives 1,
    # while pairing the small terms first would give 1 + 2^-23
    w = np.array([[1.0, 1.0, 1.0]], np.float32)
    x = np.array([[1.0, 2.0 ** -24, 2.0 ** -24]], np.float32)
    got = mlp._dot_fixed(np.zeros(1, np.float32), w, x)[0, 0]
    assert got == np.float32(1.0)
    x2 = np.array([[2.0 ** -24, 2.0 ** -24, 1.0]], np.float32)
    assert mlp._dot_fixed(np.zeros(1, np.float32), w, x2)[0, 0] == np.float32(1 + 2.0 ** -23)


def test_one_path_network_closed_form():
    z = np.zeros((mlp.N_H, mlp.N_IN), np.float32)
    W1 = z.copy(); W1[0, 0] = 1.0
    W2 = np.zeros((mlp.N_H, mlp.N_H), np.float32); W2[0, 0] = 2.0
    w3 = np.zeros(mlp.N_H, np.float32); w3[0] = 0.5
    W = mlp.Weights(W1, np.zeros(mlp.N_H), W2, np.zeros(mlp.N_H), w3, 0.25,
                    np.full(mlp.N_IN, 1.0), np.full(mlp.N_IN, 2.0))
    f = np.array([[3.0] + [0.0] * 7, [-1.0] + [0.0] * 7, [1.3] + [0.0] * 7], np.float32)
    d = np.array([2e-3, 2e-3, 1e-3], np.float32)
    skin, y = mlp.infer(W, f, d)
    z0 = mlp.bf16_round((f[:, 0] - 1.0) * 2.0)
    expect_y = 0.25 + 0.5 * mlp.bf16_round(2.0 * np.maximum(z0, 0))
    assert np.array_equal(y, expect_y.astype(np.float32))
    assert np.array_equal(skin, (d * np.maximum(expect_y, 0)).astype(np.float32))
    assert y[1] == np.float32(0.25)                 # negative input: ReLU blocks the path
    # the output range: proposals clamp to [y_lo, y_hi] diameters, by hand
    # y = (4.25, 0.25, 0.8515625) for these inputs: z0 = bf16(0.6) = 0.6015625,
    # h2 = 2 z0 = 1.203125, y = 0.25 + 0.5 h2
    assert np.array_equal(y, np.array([4.25, 0.25, 0.8515625], np.float32))
    W.y_lo, W.y_hi = np.float32(0.3), np.float32(2.0)
    skin2, y2 = mlp.infer(W, f, d)
    assert np.array_equal(y2, y)
    assert np.array_equal(skin2, np.array([2e-3 * 2.0, 2e-3 * 0.3, 1e-3 * y[2]], np.float32))
    # NaN output: the bounds decide (fmax / fmin semantics)
    W.b3 = np.float32(np.nan)
    skin3, _ = mlp.infer(W, f, d)
    assert np.array_equal(skin3, (d * np.float32(0.3)).astype(np.float32))


def test_bfloat16_roundings_closed_form():
    # three one-path units whose sums are not bfloat16 numbers, so that each
    # rounding of the inference formula (z, h1, h2) changes y; by hand,
    # with u = 1 + 3 * 2^-9 (bfloat16 neighbours 1 and 1 + 2^-7, u nearer
    # the upper one):
    #   unit 0: a1 = 1 * 1 + 3*2^-9 = u -> h1 = 1 + 2^-7; a2 = h1 - 1 = 2^-7
    #   unit 1: h1 = 1; a2 = h1 + 3*2^-9 = u -> h2 = 1 + 2^-7
    #   unit 2: z = bf16(u) = 1 + 2^-7; a1 = z - 1 = 2^-7 = h1 = h2
    #   y = ((-1 + 2^-7) + (1 + 2^-7)) + 2^-7 = 3 * 2^-7 (exact)
    u = 1 + 3 * 2.0 ** -9
    W1 = np.zeros((mlp.N_H, mlp.N_IN), np.float32)
    W1[0, 0] = W1[1, 0] = W1[2, 1] = 1.0
    b1 = np.zeros(mlp.N_H, np.float32)
    b1[0], b1[2] = 3 * 2.0 ** -9, -1.0
    W2 = np.zeros((mlp.N_H, mlp.N_H), np.float32)
    W2[0, 0] = W2[1, 1] = W2[2, 2] = 1.0
    b2 = np.zeros(mlp.N_H, np.float32)
    b2[0], b2[1] = -1.0, 3 * 2.0 ** -9
    w3 = np.zeros(mlp.N_H, np.float32)
    w3[:3] = 1.0
    W = mlp.Weights(W1, b1, W2, b2, w3, -1.0, np.zeros(mlp.N_IN), np.ones(mlp.N_IN))
    f = np.zeros((1, mlp.N_IN), np.float32)
    f[0, 0], f[0, 1] = 1.0, u
    _, y = mlp.infer(W, f, np.ones(1, np.float32))
    assert y[0] == np.float32(3 * 2.0 ** -7)
    # the training forward pass (binary64 sums, same roundings) agrees here
    y64, _ = mlp.forward64(W, f, quantize=True)
    assert y64[0] == 3 * 2.0 ** -7


def test_training_forward_matches_inference():
    # the binary64 training forward with the bfloat16 roundings evaluates
    # the same network as the binary32 inference formula: equal up to the
    # sums' roundings (which may move a hidden value by one bfloat16 step)
    rng = np.random.default_rng(21)
    W = mlp.Weights.random(seed=22, scale=0.5)
    f = rng.normal(0, 1, (3000, mlp.N_IN)).astype(np.float32)
    _, y = mlp.infer(W, f, np.ones(len(f), np.float32))
    y64, _ = mlp.forward64(W, f, quantize=True)
    d = np.abs(y64 - y.astype(np.float64)) / (np.abs(y64) + 1e-3)
    assert np.median(d) < 1e-6 and np.quantile(d, 0.99) < 1e-2


def test_travel_form_is_the_paper_rule_per_particle():
    # a network with constant output c in the travel form over S steps
    # proposes skin = d (f0 (c S)) with f0 = (|v| dt) / d: the paper's rule
    # K |v| dt (Eq. skin_formulus1) with K = c S, up to the roundings of f0
    # and of the three products (each at most half an ulp)
    rng = np.random.default_rng(5)
    n = 4000
    v = rng.normal(0, 0.5, (n, 3)).astype(np.float32)
    r = rng.uniform(0.5e-3, 2e-3, n).astype(np.float32)
    dt = np.float32(1e-6)
    d = (np.float32(2) * r).astype(np.float32)
    vm = np.sqrt(((v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]).astype(np.float32)
                  + v[:, 2] * v[:, 2]).astype(np.float32))
    f = np.zeros((n, mlp.N_IN), np.float32)
    f[:, 0] = ((vm * dt).astype(np.float32) / d).astype(np.float32)
    f[:, 1] = rng.normal(0, 1, n)          # the other features play no part
    c, S = np.float32(1.5), np.float32(400.0)
    p = np.zeros(mlp.N_PARAMS, np.float32)
    p[-1] = c
    W = mlp.Weights.from_flat(p, np.zeros(mlp.N_IN), np.ones(mlp.N_IN), 0.0, np.inf, S)
    skin, y = mlp.infer(W, f, d)
    assert (y == c).all()
    rule = 600.0 * vm.astype(np.float64) * float(dt)
    assert np.abs(skin / rule - 1).max() < 6 * 2.0 ** -24
    # the range applies to y before the scaling: y_lo above c gives K = y_lo S
    W.y_lo = np.float32(2.0)
    skin2, _ = mlp.infer(W, f, d)
    assert np.abs(skin2 / (800.0 * vm.astype(np.float64) * float(dt)) - 1).max() < 6 * 2.0 ** -24
    # a particle at rest gets no skin; the diameter form ignores f0
    f[:3, 0] = 0
    assert (mlp.infer(W, f, d)[0][:3] == 0).all()
    W.y_steps = np.float32(0)
    assert np.array_equal(mlp.infer(W, f, d)[0], (d * np.float32(2.0)).astype(np.float32))


@pytest.mark.parametrize("rel_floor", [0.0, 0.15])
def test_backward_matches_finite_differences(rel_floor):
    # squared error, and relative error with a floor that some labels fall below
    rng = np.random.default_rng(3)
    W = mlp.Weights.random(seed=4, scale=0.5)
    f = rng.normal(0, 1, (64, mlp.N_IN))
    t = rng.normal(0.2, 0.1, 64)
    if rel_floor:
        assert (t < rel_floor).any() and (t > rel_floor).any()
    loss, g = mlp.loss_and_grad64(W, f, t, quantize=False, rel_floor=rel_floor)
    p0 = W.flat().astype(np.float64)
    eps = 1e-6
    idx = rng.choice(len(p0), 60, replace=False)
    for k in idx:
        def L(delta):
            p = p0.copy(); p[k] += delta
            Wk = mlp.Weights.from_flat(p, W.mu, W.isd)
            # float32 parameters would lose the perturbation: evaluate in binary64
            Wk.W1, Wk.b1, Wk.W2, Wk.b2, Wk.w3 = (a.astype(np.float64) for a in
                                                  (Wk.W1, Wk.b1, Wk.W2, Wk.b2, Wk.w3))
            o = 0
            parts = []
            for shape in [(mlp.N_H, mlp.N_IN), (mlp.N_H,), (mlp.N_H, mlp.N_H), (mlp.N_H,),
                          (mlp.N_H,), ()]:
                size = int(np.prod(shape)) if shape else 1
                parts.append(p[o:o + size].reshape(shape) if shape else p[o]); o += size
            Wk.W1, Wk.b1, Wk.W2, Wk.b2, Wk.w3, Wk.b3 = parts
            return mlp.loss_and_grad64(Wk, f, t, quantize=False, rel_floor=rel_floor)[0]
        fd = (L(eps) - L(-eps)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])
    assert len(g) == mlp.N_PARAMS == 1377


def test_relative_loss_special_cases():
    # equal labels c above the floor: the relative error is the squared error
    # over c^2 (loss and gradient); labels below the floor count as the floor
    rng = np.random.default_rng(11)
    W = mlp.Weights.random(seed=12, scale=0.5)
    f = rng.normal(0, 1, (50, mlp.N_IN))
    c = 0.25
    t = np.full(50, c)
    l2, g2 = mlp.loss_and_grad64(W, f, t, quantize=True)
    lr, gr = mlp.loss_and_grad64(W, f, t, quantize=True, rel_floor=0.125)
    assert lr == pytest.approx(l2 / c ** 2, rel=1e-12)
    assert np.allclose(gr, g2 / c ** 2, rtol=1e-12, atol=0)
    lo = np.full(50, 0.01)
    l2, g2 = mlp.loss_and_grad64(W, f, lo, quantize=True)
    lr, gr = mlp.loss_and_grad64(W, f, lo, quantize=True, rel_floor=0.125)
    assert lr == pytest.approx(l2 / 0.125 ** 2, rel=1e-12)
    assert np.allclose(gr, g2 / 0.125 ** 2, rtol=1e-12, atol=0)


def test_features_closed_form():
    # one particle with representable values, the eight features by hand:
    # r = 2^-8 (d = 2^-7), v = (3, 4, 0) (|v| = 5), a = (0, 0, -8), dt = 2^-10,
    # moved by (3, 4, 0) 2^-12 from its old reference (skin 2^-9), in the box
    # [0, 1]^3 at (1/4, 1/2, 1/8), H = 2^-6
    pos = np.array([[0.25, 0.5, 0.125, 2.0 ** -8]], np.float32)
    vel = np.array([[3.0, 4.0, 0.0, 0.0]], np.float32)
    acc = np.array([[0.0, 0.0, -8.0, 0.0]], np.float32)
    ref_old = np.array([[0.25 - 3 * 2.0 ** -12, 0.5 - 4 * 2.0 ** -12, 0.125, 2.0 ** -9]],
                       np.float32)
    grid = {"lo": np.zeros(3, np.float32), "hi": np.ones(3, np.float32),
            "H": np.float32(2.0 ** -6)}
    f = mlp.features(pos, vel, acc, 2.0 ** -10, grid, ref_old, [7], [12], [3])[0]
    want = [5 * 2.0 ** -10 / 2.0 ** -7,          # f0 = |v| dt / d = 5/8
            8 * 2.0 ** -20 / 2.0 ** -7,          # f1 = |a| dt^2 / d = 2^-10
            2.0 ** -8 / 2.0 ** -6,               # f2 = r / H = 1/4
            7, 12,                               # f3 partners, f4 age
            5 * 2.0 ** -12 / 2.0 ** -9,          # f5 = travel / old skin = 5/8
            3,                                   # f6 occupancy
            (0.125 - 2.0 ** -8) / 2.0 ** -7]     # f7 = nearest wall gap / d = 15.5
    assert np.array_equal(f, np.array(want, np.float32))
    # no old skin: f5 = 0
    ref0 = ref_old.copy()
    ref0[0, 3] = 0
    assert mlp.features(pos, vel, acc, 2.0 ** -10, grid, ref0, [7], [12], [3])[0][5] == 0


def test_state_machine_learned_feature_counts():
    # a learned context of five particles (r = 1 mm, skin 0.1 d from a
    # constant network): A (index 2) at the middle of cell (4, 4, 4),
    # partners B, C (lower indices) and E within the cutoff 2 (r + skin) =
    # 2.4 mm of it and of no other (B-C 3.1 mm, B-E 3.3 mm, C-E 2.6 mm), D
    # far away; E's reference lies in A's cell, 0.1 mm above its lower x
    # face.  At step 1, A moves 0.3 mm (> its 0.2 mm skin) and E 0.15 mm
    # (< its skin) across that face into cell 3; A moves 0.3 mm again at
    # step 3.  A's features then count, from the state before its update: 3
    # live partners (B, C, E), 2 reference positions in the cell of its new
    # position (its own and E's, whose current position has left it), and
    # the steps since its last update (1, then 2)
    from oracle.statemachine import OracleLVB
    import oracle
    lo, hi = (0.0, 0.0, 0.0), (0.1, 0.1, 0.1)
    grid = mlp.grid_params(1e-3, 1.25, lo, hi)
    L = 1.0 / float(grid["invL"])
    a = 4.5 * L
    pos = np.array([[a + 2.1e-3, a, a], [a, a + 2.3e-3, a], [a, a, a], [0.05, 0.05, 0.05],
                    [4 * L + 0.1e-3, a, a]])
    pos4 = np.concatenate([pos, np.full((5, 1), 1e-3)], axis=1).astype(np.float32)
    p = np.zeros(mlp.N_PARAMS, np.float32)
    p[-1] = 0.1
    W = mlp.Weights.from_flat(p, np.zeros(mlp.N_IN), np.ones(mlp.N_IN))
    z4 = np.zeros_like(pos4)
    sm = OracleLVB(pos4, oracle.SKIN_LEARNED, 0.0, 1e-6, grid["H"], 0, vel4=z4,
                   learned={"weights": W, "grid": grid}, acc4=z4)
    assert np.allclose(sm.ref[:, 3], 2e-4, rtol=1e-6)
    assert set(zip(sm.pi.tolist(), sm.pj.tolist())) == {(0, 2), (1, 2), (2, 4)}
    p1 = pos4.copy()
    p1[2, 0] += np.float32(3e-4)
    p1[4, 0] -= np.float32(1.5e-4)
    f, _ = sm.step(p1, vel4=z4, acc4=z4)
    assert f.tolist() == [False, False, True, False, False]
    idx, feats = sm.last_features
    assert idx.tolist() == [2] and feats[0, 3] == 3 and feats[0, 4] == 1 and feats[0, 6] == 2
    sm.step(p1, vel4=z4, acc4=z4)                # nothing moves: no update
    p3 = p1.copy()
    p3[2, 0] += np.float32(3e-4)
    f, _ = sm.step(p3, vel4=z4, acc4=z4)
    idx, feats = sm.last_features
    assert f.tolist() == [False, False, True, False, False] and idx.tolist() == [2]
    assert feats[0, 3] == 3 and feats[0, 4] == 2 and feats[0, 6] == 2
