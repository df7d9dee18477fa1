"""The skin network's pins have teeth: each plausible mistake, planted in a
copy of the oracle's network module (oracle/mlp.py) loaded on the CPU, must
make one of the pins of tests/test_oracle_mlp.py fail."""
import os
import types

import pytest

import oracle
import tests.test_oracle_mlp as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "mlp.py")

MUTANTS = {
    # bfloat16 conversion truncates instead of rounding to nearest even
    "bf16_truncates": ("r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)",
                       "r = (u & 0xFFFF0000).astype(np.uint32)"),
    # sums taken in the reverse order
    "dot_reversed": ("    for k in range(w.shape[1]):\n        prod",
                     "    for k in reversed(range(w.shape[1])):\n        prod"),
    # a rounding of the inference formula left out
    "z_not_rounded": ("    z = bf16_round(((f - W.mu).astype(np.float32) * W.isd).astype(np.float32))\n"
                      "    h1 = bf16_round(",
                      "    z = ((f - W.mu).astype(np.float32) * W.isd).astype(np.float32)\n"
                      "    h1 = bf16_round("),
    "h1_not_rounded": ("h1 = bf16_round(np.maximum(_dot_fixed(W.b1, bf16_round(W.W1), z), np.float32(0)))",
                       "h1 = np.maximum(_dot_fixed(W.b1, bf16_round(W.W1), z), np.float32(0))"),
    "h2_not_rounded": ("h2 = bf16_round(np.maximum(_dot_fixed(W.b2, bf16_round(W.W2), h1), np.float32(0)))",
                       "h2 = np.maximum(_dot_fixed(W.b2, bf16_round(W.W2), h1), np.float32(0))"),
    # a dropped bias, a transposed weight matrix
    "b2_dropped": ("_dot_fixed(W.b2, bf16_round(W.W2), h1)",
                   "_dot_fixed(W.b2 * 0, bf16_round(W.W2), h1)"),
    "W2_transposed_in_inference": ("_dot_fixed(W.b2, bf16_round(W.W2), h1)",
                                   "_dot_fixed(W.b2, bf16_round(W.W2.T), h1)"),
    # the output range: bounds swapped, applied after the travel scaling
    "clamp_bounds_swapped": ("yc = np.fmin(np.fmax(y, W.y_lo), W.y_hi).astype(np.float32)",
                             "yc = np.fmax(np.fmin(y, W.y_lo), W.y_hi).astype(np.float32)"),
    "travel_unclamped": ("k = (yc * W.y_steps).astype(np.float32)",
                         "k = (y * W.y_steps).astype(np.float32)"),
    # the travel form reads the acceleration feature instead of the speed
    "travel_wrong_feature": ("yc = (f[:, 0] * k).astype(np.float32)",
                             "yc = (f[:, 1] * k).astype(np.float32)"),
    # training: forward with W2 transposed, a ReLU mask dropped, a
    # transposed operand in a weight gradient, the relative floor ignored
    "W2_transposed_in_training": ("a2 = h1 @ W2.T + W.b2.astype(np.float64)",
                                  "a2 = h1 @ W2 + W.b2.astype(np.float64)"),
    "relu_mask_dropped": ("dh1 = (dh2 @ W2) * (a1 > 0)", "dh1 = (dh2 @ W2)"),
    "gW2_transposed": ("gW2 = dh2.T @ h1", "gW2 = h1.T @ dh2"),
    "rel_floor_ignored": ("w = 1.0 / np.maximum(t, float(np.float32(rel_floor))) ** 2",
                          "w = 1.0 / t ** 2"),
}


def _load(src, name):
    mod = types.ModuleType("mlp_mutant_" + name)
    exec(compile(src, "<mlp mutant %s>" % name, "exec"), mod.__dict__)
    return mod


def _pins():
    """The pins of tests/test_oracle_mlp.py (without the torch comparison);
    True if all pass."""
    checks = [
        P.test_bf16_round_hand_cases,
        P.test_fixed_order_dot_is_sequential_binary32,
        P.test_one_path_network_closed_form,
        P.test_bfloat16_roundings_closed_form,
        P.test_training_forward_matches_inference,
        P.test_travel_form_is_the_paper_rule_per_particle,
        lambda: P.test_backward_matches_finite_differences(0.0),
        lambda: P.test_backward_matches_finite_differences(0.15),
        P.test_relative_loss_special_cases,
    ]
    for c in checks:
        try:
            c()
        except AssertionError:
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(monkeypatch, name):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, name
    monkeypatch.setattr(P, "mlp", _load(src.replace(before, after), name))
    assert not _pins(), "mutant %s survived the pins" % name


def test_unmutated_passes_pins(monkeypatch):
    monkeypatch.setattr(P, "mlp", _load(open(SRC).read(), "none"))
    assert _pins()
