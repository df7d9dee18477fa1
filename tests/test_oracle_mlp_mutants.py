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
    # features: the speed feature from the acceleration, one dt too few,
    # the wall gap without the radius, the travel over the new skin
    "f0_from_acc": ("f[:, 0] = ((_norm3(vel4) * dt)", "f[:, 0] = ((_norm3(acc4) * dt)"),
    "f1_one_dt": ("f[:, 1] = ((((_norm3(acc4) * dt).astype(np.float32)) * dt).astype(np.float32) / d)",
                  "f[:, 1] = (((_norm3(acc4) * dt).astype(np.float32)) / d)"),
    "f7_gap_without_radius": ("lo_gap = ((pos4[:, k] - grid[\"lo\"][k]).astype(np.float32) - r)",
                              "lo_gap = ((pos4[:, k] - grid[\"lo\"][k]).astype(np.float32) - 0)"),
}

# the learned state machine: partners counted on one side of the pair list
# only, occupancy from current instead of reference positions, age off by one
SM_SRC = os.path.join(os.path.dirname(oracle.__file__), "statemachine.py")
SM_MUTANTS = {
    "nrow_one_side": ("np.bincount(np.concatenate([self.pi, self.pj]), minlength=self.n)",
                      "np.bincount(self.pi, minlength=self.n)"),
    "occ_from_positions": ("mlp.cell_index(self.ref[:, :3], grid)",
                           "mlp.cell_index(pos4[:, :3], grid)"),
    "age_off_by_one": ("step - self.born[idx], occ)", "step - 1 - self.born[idx], occ)"),
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
        P.test_features_closed_form,
        P.test_state_machine_learned_feature_counts,
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


@pytest.mark.parametrize("name", sorted(SM_MUTANTS))
def test_state_machine_mutant_is_caught(monkeypatch, name):
    import oracle.statemachine as SM
    before, after = SM_MUTANTS[name]
    src = open(SM_SRC).read()
    assert src.count(before) == 1, name
    mod = types.ModuleType("oracle.statemachine_mutant_" + name)
    mod.__package__ = "oracle"
    exec(compile(src.replace(before, after), "<state machine mutant %s>" % name, "exec"),
         mod.__dict__)
    monkeypatch.setattr(SM, "OracleLVB", mod.OracleLVB)
    assert not _pins(), "mutant %s survived the pins" % name
