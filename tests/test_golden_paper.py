"""Pins the improvement metric of Eq. impr against Table tab:summary."""
import os

import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table_summary.txt")


def _rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, tw, k, topt, iopt, tdef, idef, ovh = line.split()
        rows.append((name, float(tw), int(k), float(topt), float(iopt), float(tdef),
                     float(idef), float(ovh)))
    return rows


@pytest.mark.parametrize("row", _rows(), ids=lambda r: r[0])
def test_improvement_matches_table(orc, row):
    name, tw, k, topt, iopt, tdef, idef, ovh = row
    # The table prints two decimals of a value computed from unrounded times,
    # so agreement is to a few hundredths of a percentage point.
    assert abs(orc.improvement_pct(tw, topt) - iopt) < 0.03
    assert abs(orc.improvement_pct(tw, tdef) - idef) < 0.03
    # Overhead column: the default's excess over the optimum, relative to the
    # default time (the reading that reproduces every printed row).
    assert abs((tdef - topt) / tdef * 100.0 - ovh) < 0.01
