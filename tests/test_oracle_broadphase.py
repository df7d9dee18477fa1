"""Pins of the broad-phase oracle against what the paper and mathematics fix.

* pair set (Def. verletlist / Eq. broad_phase): exact-cutoff closed forms
  built from representable binary32 values, brute force vs Algorithm 1, a
  k-d tree from scipy (a library routine) on monodisperse sets;
* flags (Eq. update): ballistic closed form of the first violation, the
  equality case, K = 0 and the static case;
* skin policies (Eq. skin_formulus1, Eq. skin_formulus_mincell);
* contacts (Eq. delta): closed forms, brute force vs cells;
* Theorem 1: zero missed contacts at every step, and contacts identical
  whichever update mode is used (Sec. "Local Verlet buffer").
"""
import numpy as np
import pytest

from paper_2208_13770_gb300 import scenes


def _ref(xyz, skin):
    xyz = np.asarray(xyz, dtype=np.float32).reshape(-1, 3)
    ref = np.zeros((len(xyz), 4), dtype=np.float32)
    ref[:, :3] = xyz
    ref[:, 3] = skin
    return ref


# ---------------------------------------------------------------- pair set
@pytest.mark.parametrize("offset", [(0.75, 1.0, 0.0), (0.0, 0.75, 1.0), (1.0, 0.0, 0.75),
                                    (1.25, 0.0, 0.0), (0.0, 0.0, 1.25)])
def test_pair_exact_cutoff_is_inclusive(orc, offset):
    # r = 0.5, skin = 0.125 -> R_NL = 0.625, cutoff 1.25; |offset| = 1.25 exactly
    ref = _ref([(0.0, 0.0, 0.0), offset], 0.125)
    rad = np.array([0.5, 0.5], dtype=np.float32)
    pi, pj = orc.pairs_brute(ref, rad)
    assert list(zip(pi, pj)) == [(0, 1)]
    # one ulp further along each nonzero axis: no pair
    far = np.array(offset, dtype=np.float32)
    k = int(np.argmax(far))
    far[k] = np.nextafter(far[k], np.float32(10))
    ref2 = _ref([(0.0, 0.0, 0.0), far], 0.125)
    assert len(orc.pairs_brute(ref2, rad)[0]) == 0


def test_pair_uses_extended_radius_of_both(orc):
    # r_i = 0.5, r_j = 0.25, skins 0.125 / 0.375: cutoff (0.625 + 0.625) = 1.25
    ref = np.array([[0, 0, 0, 0.125], [1.25, 0, 0, 0.375]], dtype=np.float32)
    rad = np.array([0.5, 0.25], dtype=np.float32)
    assert len(orc.pairs_brute(ref, rad)[0]) == 1
    # one ulp of the cutoff less (2^-23 at 1.25): no pair
    ref[1, 3] = np.float32(0.375) - np.float32(2.0 ** -23)
    assert len(orc.pairs_brute(ref, rad)[0]) == 0


def _random_set(rng, n, side, rmin, rmax, smax):
    xyz = rng.uniform(0, side, size=(n, 3))
    rad = rng.uniform(rmin, rmax, size=n).astype(np.float32)
    skin = rng.uniform(0, smax, size=n).astype(np.float32)
    skin[rng.random(n) < 0.2] = 0.0
    return _ref(xyz, skin), rad


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_brute_equals_linked_cells(orc, seed):
    rng = np.random.default_rng(seed)
    # polydisperse with a 1:7.5 radius ratio, dense enough for many pairs
    ref, rad = _random_set(rng, 1500, 0.05, 0.4e-3, 3e-3, 0.6e-3)
    a = orc.pairs_brute(ref, rad)
    b = orc.pairs_cells(ref, rad)
    assert len(a[0]) > 500
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_linked_cells_same_cell_pairs(orc):
    # all particles in one tiny cluster: every pair is a same-cell pair,
    # which Algorithm 1 as printed (index(C_b) < index(C_a)) would miss
    rng = np.random.default_rng(7)
    ref = _ref(rng.uniform(0, 1e-4, size=(40, 3)), 1e-4)
    rad = np.full(40, 1e-3, dtype=np.float32)
    a = orc.pairs_brute(ref, rad)
    b = orc.pairs_cells(ref, rad)
    assert len(a[0]) == 40 * 39 // 2
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_pairs_match_kdtree(orc):
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(11)
    n, r, s = 3000, 1e-3, 0.3e-3
    ref, _ = _random_set(rng, n, 0.06, r, r, 0)
    ref[:, 3] = s
    rad = np.full(n, r, dtype=np.float32)
    pi, pj = orc.pairs_brute(ref, rad)
    mine = set(zip(pi.tolist(), pj.tolist()))
    cut = 2 * (r + s)
    tree = spatial.cKDTree(ref[:, :3].astype(np.float64))
    lib = tree.query_pairs(cut * (1 + 1e-5))
    d = lambda p: np.linalg.norm(ref[p[0], :3].astype(np.float64) - ref[p[1], :3])
    # pairs farther than 1e-5 relative from the cutoff must agree exactly
    lib_clear = {p for p in lib if d(p) < cut * (1 - 1e-5)}
    mine_clear = {p for p in mine if d(p) < cut * (1 - 1e-5)}
    assert lib_clear == mine_clear
    assert all(d(p) <= cut * (1 + 1e-5) for p in mine)
    assert len(mine) > 100


def test_pairs_are_permutation_invariant(orc):
    rng = np.random.default_rng(5)
    ref, rad = _random_set(rng, 800, 0.03, 0.5e-3, 2e-3, 0.4e-3)
    perm = rng.permutation(len(ref))
    a = set(zip(*[x.tolist() for x in orc.pairs_brute(ref, rad)]))
    b = orc.pairs_brute(ref[perm], rad[perm])
    mapped = {tuple(sorted((int(perm[i]), int(perm[j])))) for i, j in zip(*b)}
    assert a == mapped


# ---------------------------------------------------------------- flags
def test_flags_ballistic_closed_form(orc):
    # x advances by exactly 2^-20 per step (representable at x = 0.5): the
    # first violation of Eq. update is the first n with n*2^-20 > skin.
    h = np.float32(2.0 ** -20)
    skins = np.array([10.5, 10.0, 3.25, 0.0, 7.0], dtype=np.float32) * h
    n = len(skins)
    pos = np.zeros((n, 4), dtype=np.float32)
    pos[:, 0] = 0.5
    pos[:, 3] = 1e-3
    ref = pos.copy()
    ref[:, 3] = skins
    first = {}
    for step in range(1, 20):
        pos[:, 0] = np.float32(0.5) + np.float32(step) * h
        f = orc.flags(pos, ref)
        for i in np.nonzero(f)[0]:
            first.setdefault(int(i), step)
    # 10.5 -> 11; equality at 10 does not flag -> 11; 3.25 -> 4; 0 -> 1; 7 -> 8
    assert first == {0: 11, 1: 11, 2: 4, 3: 1, 4: 8}


def test_flags_partial_updates_repeat_with_period(orc):
    from oracle.statemachine import OracleLVB, TRIGGER_PARTIAL
    h = np.float32(2.0 ** -20)
    pos = np.array([[0.5, 0.25, 0.25, 1e-3], [0.25, 0.5, 0.25, 1e-3]], dtype=np.float32)
    H = np.float32(1.0)
    sm = OracleLVB(pos, 0, 3.5 * h, 0.0, H, TRIGGER_PARTIAL)
    hist = []
    for step in range(1, 17):
        p = pos.copy()
        p[0, 0] = np.float32(0.5) + np.float32(step) * h        # moves
        f, upd = sm.step(p)
        hist.append(bool(f[0]))
        assert not f[1]                                      # static: never
    # skin 3.5 steps: violation at 4, 8, 12, 16 (reference reset each time)
    assert [i + 1 for i, x in enumerate(hist) if x] == [4, 8, 12, 16]


def test_trigger_modes_update_sets(orc):
    # the same two particles as above (one moving 2^-20 a step with a skin
    # of 3.5 steps, one static) under the three triggers: the local buffer
    # updates the violating particle alone; the global one (Def. autoverlet)
    # updates both whenever one violates, so the static particle's skin is
    # reset too; with no buffer every particle is updated every step
    from oracle.statemachine import OracleLVB, TRIGGER_PARTIAL, TRIGGER_GLOBAL, TRIGGER_ALWAYS
    h = np.float32(2.0 ** -20)
    pos = np.array([[0.5, 0.25, 0.25, 1e-3], [0.25, 0.5, 0.25, 1e-3]], dtype=np.float32)
    got = {}
    for trig in (TRIGGER_PARTIAL, TRIGGER_GLOBAL, TRIGGER_ALWAYS):
        sm = OracleLVB(pos, 0, 3.5 * h, 0.0, np.float32(1.0), trig)
        rows = []
        for step in range(1, 9):
            p = pos.copy()
            p[0, 0] = np.float32(0.5) + np.float32(step) * h
            f, upd = sm.step(p)
            rows.append((f.tolist(), upd.tolist()))
        got[trig] = (rows, sm.updates, sm.rebuild_steps)
    rows, upd_total, rb = got[TRIGGER_PARTIAL]
    assert [r[1] for r in rows] == [[k in (4, 8), False] for k in range(1, 9)]
    assert (upd_total, rb) == (2, 2)
    rows, upd_total, rb = got[TRIGGER_GLOBAL]
    assert [r[1] for r in rows] == [[k in (4, 8)] * 2 for k in range(1, 9)]
    assert (upd_total, rb) == (4, 2)
    rows, upd_total, rb = got[TRIGGER_ALWAYS]
    assert all(r[1] == [True, True] for r in rows) and (upd_total, rb) == (16, 8)


def test_flags_k_zero_is_every_step(orc):
    # K = 0 in skin = K |v| dt: every moving particle is flagged every step
    from oracle.statemachine import OracleLVB, TRIGGER_PARTIAL
    s = scenes.ballistic(n=300, seed=3)
    sm = OracleLVB(s.pos, orc.SKIN_PAPER_KVDT, 0.0, s.dt, 1.0, TRIGGER_PARTIAL, vel4=s.vel)
    for pos, vel in scenes.ballistic_trajectory(s, 5):
        f, upd = sm.step(pos, vel4=vel)
        assert f.all()


# ---------------------------------------------------------------- skins
def test_skin_policies_closed_form(orc):
    pos = np.array([[0, 0, 0, 0.5], [0, 0, 0, 0.25]], dtype=np.float32)
    vel = np.array([[3.0, 4.0, 0.0, 0], [0.0, 0.0, 0.0, 0]], dtype=np.float32)
    H = np.float32(10.0)
    assert np.array_equal(orc.skin(0, 0.125, 0, H, pos), [0.125, 0.125])
    assert np.array_equal(orc.skin(1, 0.25, 0, H, pos), [0.25, 0.125])
    # K = 200, |v| = 5 exactly, dt = 2^-12: 1000 * 2^-12
    assert np.array_equal(orc.skin(2, 200.0, 2.0 ** -12, H, pos, vel),
                          np.array([1000 * 2.0 ** -12, 0.0], dtype=np.float32))
    # cap: R_NL = r + skin <= H
    assert np.array_equal(orc.skin(0, 5.0, 0, np.float32(0.75), pos), [0.25, 0.5])
    assert np.array_equal(orc.skin(0, 5.0, 0, np.float32(0.375), pos), [0.0, 0.125])
    prop = np.array([-1.0, np.nan], dtype=np.float32)
    assert np.array_equal(orc.skin(3, 0, 0, H, pos, proposal=prop), [0.0, 0.0])


# ---------------------------------------------------------------- contacts
def test_contact_closed_forms(orc):
    pos = np.array([[0, 0, 0, 0.5], [0.75, 0, 0, 0.5], [3, 0, 0, 0.5], [4, 0, 0, 0.5]],
                   dtype=np.float32)
    ci, cj, dl = orc.contacts_brute(pos)
    # (0,1): delta = 1 - 0.75 = 0.25; (2,3) touching: delta = 0, no contact
    assert list(zip(ci, cj)) == [(0, 1)] and dl[0] == np.float32(0.25)


@pytest.mark.parametrize("seed", [1, 2])
def test_contacts_brute_equals_cells(orc, seed):
    rng = np.random.default_rng(seed)
    n = 2500
    pos = np.zeros((n, 4), dtype=np.float32)
    pos[:, :3] = rng.uniform(0, 0.04, size=(n, 3))
    pos[:, 3] = rng.uniform(0.5e-3, 2e-3, size=n)
    a = orc.contacts_brute(pos)
    b = orc.contacts_cells(pos)
    assert len(a[0]) > 100
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# ---------------------------------------------------------------- Theorem 1
def _run_modes(orc, s, steps, modes):
    from oracle.statemachine import OracleLVB
    H = np.float32(0.5 * 1.25 * 2 * s.pos[:, 3].max() * (1 + 2 ** -7) * (1 - 2 ** -8))
    sms = {m: OracleLVB(s.pos, *m[0], s.dt, H, m[1], vel4=s.vel) for m in modes}
    for pos, vel in scenes.ballistic_trajectory(s, steps):
        truth = orc.contacts_brute(pos)
        truth_set = set(zip(truth[0].tolist(), truth[1].tolist()))
        for m, sm in sms.items():
            sm.step(pos, vel4=vel)
            pairs = set(zip(sm.pi.tolist(), sm.pj.tolist()))
            assert truth_set <= pairs, m            # zero missed contacts
            got = sm.contacts(pos)
            for x, y in zip(got, truth):            # strictly identical results
                assert np.array_equal(x, y), m
    return sms


def test_theorem1_all_modes_identical_contacts(orc):
    from oracle.statemachine import TRIGGER_PARTIAL, TRIGGER_GLOBAL, TRIGGER_ALWAYS
    # a hot, dense ballistic gas so that contacts and rebuilds are frequent
    s = scenes.ballistic(n=600, seed=9, phi=0.35, vsigma=2.0)
    modes = [((1, 0.1), TRIGGER_PARTIAL), ((1, 0.1), TRIGGER_GLOBAL),
             ((0, 0.0), TRIGGER_ALWAYS), ((2, 50.0), TRIGGER_PARTIAL),
             ((0, 0.2e-3), TRIGGER_GLOBAL)]
    sms = _run_modes(orc, s, 60, modes)
    part = sms[modes[0]]
    assert 0 < part.updates < part.n * part.steps          # partial really is partial
    assert sms[modes[2]].rebuild_steps == sms[modes[2]].steps


def test_theorem1_violated_without_the_check(orc):
    # Control: freezing the list (never updating) must eventually miss a
    # contact in the same gas -- the invariant test above has teeth.
    s = scenes.ballistic(n=600, seed=9, phi=0.35, vsigma=2.0)
    ref = s.pos.copy()
    ref[:, 3] = 0.1 * 2 * s.pos[:, 3]
    pi, pj = orc.pairs_brute(ref, s.pos[:, 3])
    frozen = set(zip(pi.tolist(), pj.tolist()))
    missed = 0
    for pos, _ in scenes.ballistic_trajectory(s, 60):
        c = orc.contacts_brute(pos)
        missed += len(set(zip(c[0].tolist(), c[1].tolist())) - frozen)
    assert missed > 0


def _near_pairs_scene():
    """Pairs along x, one per y row, at separations s around the cutoff
    c = 0.5 + 0.5 = 1 (skin 0): s^2 in binary32 is 1, 1 +- 2^-21 (within
    1e-6 of c^2) or 1 +- 2^-18 (outside).  Returns (ref4, rad, expected)."""
    seps = [1.0, 1.0 + 2.0 ** -22, 1.0 - 2.0 ** -22, 1.0 + 2.0 ** -19, 1.0 - 2.0 ** -19]
    ref = np.zeros((2 * len(seps), 4), np.float32)
    for k, sep in enumerate(seps):
        ref[2 * k] = (0.0, 10.0 * k, 0.0, 0.0)
        ref[2 * k + 1] = (np.float32(sep), 10.0 * k, 0.0, 0.0)
    rad = np.full(len(ref), 0.5, np.float32)
    expected = {(0, 1), (2, 3), (4, 5)}
    return ref, rad, expected


def test_near_cutoff_closed_form(orc):
    # separations of 1, 1 +- 2^-22 give s^2 = 1, 1 +- 2^-21 (4.8e-7 from the
    # squared cutoff); 1 +- 2^-19 give 1 +- 2^-18 (3.8e-6): only the first
    # three pairs are within 1e-6, and all five within 1e-5
    ref, rad, expected = _near_pairs_scene()
    pi, pj = orc.near_cutoff(ref, rad, 1e-6)
    assert set(zip(pi.tolist(), pj.tolist())) == expected
    pi, pj = orc.near_cutoff(ref, rad, 1e-5)
    assert set(zip(pi.tolist(), pj.tolist())) == {(2 * k, 2 * k + 1) for k in range(5)}
    pi, pj = orc.near_cutoff(ref, rad, 0.0)
    assert set(zip(pi.tolist(), pj.tolist())) == {(0, 1)}
    # the exact-cutoff pair is in the list, the outer ones are not
    li, lj = orc.pairs_brute(ref, rad)
    assert (0, 1) in set(zip(li.tolist(), lj.tolist()))
    assert (6, 7) not in set(zip(li.tolist(), lj.tolist()))


def test_early_trigger_hand_case(orc):
    # three particles far apart, global skin 1, beta 0.75 (all values exact
    # in binary32).  Step 1: particle 0 moves 0.8 (past 0.75 of its skin,
    # within the skin), particle 1 moves 0.75 (exactly beta skin: not past
    # it) -- no violation, so nothing is updated.  Step 2: particle 2 moves
    # 1.5 (a violation): it and particle 0 are updated, particle 1 is not.
    from oracle.statemachine import OracleLVB
    pos = np.zeros((3, 4), np.float32)
    pos[:, 1] = [0.0, 100.0, 200.0]
    pos[:, 3] = 0.25
    sm = OracleLVB(pos, orc.SKIN_GLOBAL, 1.0, 1.0, np.float32(50.0), early_beta=0.75)
    p1 = pos.copy()
    p1[0, 0], p1[1, 0] = 0.8, 0.75
    f, upd = sm.step(p1)
    assert not f.any() and not upd.any() and sm.rebuild_steps == 0
    p2 = p1.copy()
    p2[2, 0] = 1.5
    f, upd = sm.step(p2)
    assert list(f) == [False, False, True]
    assert list(upd) == [True, False, True]
    assert sm.ref[0, 0] == np.float32(0.8) and sm.ref[1, 0] == 0.0 and sm.ref[2, 0] == 1.5
    # beta = 1: the plain partial trigger
    sm1 = OracleLVB(pos, orc.SKIN_GLOBAL, 1.0, 1.0, np.float32(50.0), early_beta=1.0)
    sm1.step(p1)
    f, upd = sm1.step(p2)
    assert list(upd) == [False, False, True]
    # the set itself: strict ">" at the boundary, beta rounded to binary32
    ref = np.zeros((2, 4), np.float32)
    ref[:, 3] = 1.0
    x = np.zeros((2, 4), np.float32)
    x[0, 0], x[1, 0] = 0.75, np.nextafter(np.float32(0.75), np.float32(1))
    assert list(orc.flags_beta(x, ref, 0.75)) == [False, True]


def _dumbbell_and_sphere(bx):
    # clump 0: a dumbbell, sub-spheres at (-1, 0, 0) and (1, 0, 0), r 0.5;
    # clump 1: one sphere of r 0.5 at its centre (bx, 0, 0)
    pos = np.array([[0, 0, 0, 1.6], [bx, 0, 0, 0.6]], np.float32)
    sub_off = np.array([0, 2, 3], np.int32)
    sub = np.array([[-1, 0, 0, 0.5], [1, 0, 0, 0.5], [0, 0, 0, 0.5]], np.float32)
    return pos, sub_off, sub


def test_clump_oracle_closed_forms(orc):
    # identity: the dumbbell's +x sphere (sub 1) at (1, 0, 0) touches the
    # sphere at (1.75, 0, 0): delta = 1 - 0.75 = 0.25 exactly
    pos, off, sub = _dumbbell_and_sphere(1.75)
    ident = np.array([[1, 0, 0, 0], [1, 0, 0, 0]], np.float32)
    ci, ca, cj, cb, dl = orc.clump_contacts(pos, ident, off, sub)
    assert list(zip(ci, ca, cj, cb)) == [(0, 1, 1, 0)] and dl[0] == np.float32(0.25)
    # half turns (exact quaternions): about z (w, x, y, z) = (0, 0, 0, 1) and
    # about y (0, 0, 1, 0) swap the dumbbell's ends, so sub 0 touches; about
    # x (0, 1, 0, 0) leaves the x axis where it is
    for q, a in (((0, 0, 0, 1), 0), ((0, 0, 1, 0), 0), ((0, 1, 0, 0), 1)):
        quat = np.array([q, [1, 0, 0, 0]], np.float32)
        ci, ca, cj, cb, dl = orc.clump_contacts(pos, quat, off, sub)
        assert list(zip(ci, ca, cj, cb)) == [(0, a, 1, 0)] and dl[0] == np.float32(0.25), q
    # moved away: no contact (distance 1 = r_a + r_b exactly: delta 0)
    pos, off, sub = _dumbbell_and_sphere(2.0)
    assert len(orc.clump_contacts(pos, ident, off, sub)[0]) == 0
    # the turned second clump's own offset: a sphere at b = (0, 0.5, 0) of
    # clump 1 turned half about x sits at (bx, -0.5, 0)
    pos = np.array([[0, 0, 0, 1.6], [1.5, 0.2, 0, 1.1]], np.float32)
    off = np.array([0, 2, 3], np.int32)
    sub = np.array([[-1, 0, 0, 0.5], [1, 0, 0, 0.5], [0, 0.5, 0, 0.5]], np.float32)
    q = np.array([[1, 0, 0, 0], [0, 1, 0, 0]], np.float32)
    ci, ca, cj, cb, dl = orc.clump_contacts(pos, q, off, sub)
    # (1.5, -0.3, 0) against (1, 0, 0): |d|^2 = 0.25 + 0.09 = 0.34
    d2 = np.float32(np.float32(0.5) * np.float32(0.5)) + np.float32(np.float32(-0.3) ** 2)
    assert list(zip(ci, ca, cj, cb)) == [(0, 1, 1, 0)]
    assert dl[0] == np.float32(1.0) - np.sqrt(np.float32(d2))
