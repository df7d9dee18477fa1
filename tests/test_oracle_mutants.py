"""The pins have teeth: each plausible mistake, planted in a copy of the
oracle's C source and compiled on the CPU, must make a pin fail."""
import os
import subprocess

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "lvb_oracle.c")

MUTANTS = {
    "strict_cutoff": ("return d2 <= c2;", "return d2 < c2;"),
    "dropped_dz": ("    s = s + zz;\n    return s;", "    (void)zz;\n    return s;"),
    "skin_not_rnl": ("float rnl_i = rad_i + ri4[3];", "float rnl_i = ri4[3] + ri4[3];"),
    "alg1_literal_no_same_cell": ("if (cb == ca && b >= a) continue;", "if (cb == ca) continue;"),
    "flag_non_strict": ("flag[i] = (uint8_t)(d2 > s2);", "flag[i] = (uint8_t)(d2 >= s2);"),
    "no_skin_cap": ("    if (s > capv) s = capv;\n", ""),
    "wrong_sign_damping": ("double f = P->kn * dl - gam * vn;", "double f = P->kn * dl + gam * vn;"),
    "missing_half_dt2": ("x[k] + v[k] * dt + 0.5 * a[k] * dt * dt", "x[k] + v[k] * dt + a[k] * dt * dt"),
}


def _pins(orc):
    """Run the pin tests of the other oracle test modules; True if all pass."""
    import tests.test_oracle_broadphase as B
    import tests.test_oracle_dynamics as D
    checks = [
        lambda: [B.test_pair_exact_cutoff_is_inclusive(orc, o) for o in
                 [(0.75, 1.0, 0.0), (0.0, 0.75, 1.0), (1.0, 0.0, 0.75)]],
        lambda: B.test_pair_uses_extended_radius_of_both(orc),
        lambda: [B.test_brute_equals_linked_cells(orc, s) for s in (1, 2)],
        lambda: B.test_linked_cells_same_cell_pairs(orc),
        lambda: B.test_flags_ballistic_closed_form(orc),
        lambda: B.test_skin_policies_closed_form(orc),
        lambda: D.test_free_fall_exact(orc),
        lambda: D.test_head_on_restitution_and_duration(orc),
    ]
    for c in checks:
        try:
            c()
        except AssertionError:
            return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(orc, tmp_path, name):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, name
    mut = tmp_path / ("m_%s.c" % name)
    mut.write_text(src.replace(before, after))
    so = tmp_path / ("m_%s.so" % name)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                           "-fno-fast-math", "-fPIC", "-shared", "-o", str(so), str(mut), "-lm"])
    with oracle.use_library(str(so)):
        assert not _pins(orc), "mutant %s survived the pins" % name


def test_unmutated_passes_pins(orc):
    assert _pins(orc)


# the state machine's triggers: the global buffer updating only the
# violating particles, the early trigger acting on steps without a
# violation, the no-buffer mode updating only on a violation
SM_SRC = os.path.join(os.path.dirname(oracle.__file__), "statemachine.py")
SM_MUTANTS = {
    "global_updates_flagged_only": ("upd = np.full(self.n, bool(f.any()))", "upd = f.copy()"),
    "early_without_violation": ("if self.early_beta < 1 and f.any():",
                                "if self.early_beta < 1:"),
    "always_only_on_violation": ("            upd = np.ones(self.n, dtype=bool)",
                                 "            upd = np.full(self.n, bool(f.any()))"),
}


@pytest.mark.parametrize("name", sorted(SM_MUTANTS))
def test_state_machine_trigger_mutant_is_caught(orc, monkeypatch, name):
    import types
    import oracle.statemachine as SM
    import tests.test_oracle_broadphase as B
    before, after = SM_MUTANTS[name]
    src = open(SM_SRC).read()
    assert src.count(before) == 1, name
    mod = types.ModuleType("oracle.statemachine_mutant_" + name)
    mod.__package__ = "oracle"
    exec(compile(src.replace(before, after), "<state machine mutant %s>" % name, "exec"),
         mod.__dict__)
    monkeypatch.setattr(SM, "OracleLVB", mod.OracleLVB)
    caught = 0
    for pin in (B.test_trigger_modes_update_sets, B.test_early_trigger_hand_case):
        try:
            pin(orc)
        except AssertionError:
            caught += 1
    assert caught > 0, name
