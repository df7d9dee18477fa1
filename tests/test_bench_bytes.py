"""The measurement arithmetic of bench.py on made-up counters (host logic,
no GPU): the algorithmic bytes of a broad-phase launch, the roofline
fraction, and the narrow phase's bytes.

The byte formula is the one the roofline is reported on: per launch 32 N
(pos + ref read) + N / 8 (flag bits), and per flagged particle 56 + 8 l
bytes (+16 when the policy reads v), 20 per stencil candidate, 16 per
flagged-list record of the direct test, 8 l per edit of a partner's row,
with the counts taken from two lvb_stats snapshots over the window.
"""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
bench = pytest.importorskip("bench")


def _stats(flagged, cand, direct, edits, entries):
    return {"flagged_total": flagged, "rebuild_candidates": cand, "rebuild_direct": direct,
            "rebuild_edits": edits, "entries": entries}


def test_broad_phase_bytes_follow_the_counts():
    n, steps = 1000, 10
    s0 = _stats(0, 0, 0, 0, 0)
    s1 = _stats(50, 400, 120, 30, 4000)          # l = 4 entries a particle
    b, parts = bench._bp_bytes(n, steps, s0, s1)
    F, ell = 5.0, 4.0
    check = 32.0 * n + n / 8.0
    flagged = F * (56.0 + 8.0 * ell)
    cand = 20.0 * 40 + 16.0 * 12
    edits = 8.0 * ell * 3
    assert parts["check"] == check
    assert parts["flagged"] == flagged
    assert parts["candidates"] == cand
    assert parts["edits"] == edits
    assert b == check + flagged + cand + edits
    assert parts["F"] == F and parts["mean_row"] == ell
    assert parts["stencil_candidates_per_flagged"] == 8.0
    # a policy that reads v: 16 more bytes per flagged particle
    b_v, _ = bench._bp_bytes(n, steps, s0, s1, reads_vel=True)
    assert b_v == b + 16.0 * F
    # nothing flagged: the check alone
    b0, parts0 = bench._bp_bytes(n, steps, s0, _stats(0, 0, 0, 0, 4000))
    assert b0 == check and parts0["stencil_candidates_per_flagged"] == 0.0


def test_roofline_fraction():
    r = bench._roofline("k", 200e6, 0.05, 6658.0, "measured", 203.6e6)
    assert r["achieved"] == pytest.approx(4000.0)          # GB/s: 200 MB / 50 us
    assert r["frac"] == pytest.approx(4000.0 / 6658.0)
    assert r["traffic"] == 203.6e6 and r["bound"] == "hbm" and r["unit"] == "GB/s"
    r0 = bench._roofline("k", 200e6, 0.05, 6658.0, "measured", None)
    assert r0["traffic"] is None and "none" in r0["traffic_source"]


def test_narrow_phase_bytes():
    out = bench._narrow_phase(1000, 800, 0.01, 6658.0)
    want = 1000 * (16.0 * 4 + 12.0 + 32.0) + 4.0 * 800
    assert out["bytes_per_step"] == want
    assert out["achieved_gbs"] == pytest.approx(want / 1e-5 / 1e9)
    assert out["frac_hbm"] == pytest.approx(out["achieved_gbs"] / 6658.0)
