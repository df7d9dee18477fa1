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
