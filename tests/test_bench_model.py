"""The loop-balance model that bench.py's roofline fractions divide by.

bench.loop_balance gives the algorithmic bytes per fluid-node update of each
variant (Sect. 4 "Loop Balance", Sect. 4.1).  It is held to the paper's
printed values (tests/golden/paper_numbers.json): D_pdf, the FP64 balances
of OS-NT and AA, the RIA bounds at r = 0 and r = 1, and Table 2's channel
and reactor rows (the reactor's r is not printed; one r in the interval its
two rounded RIA entries allow reproduces the row).
The reduced-precision rows scale only the PDF term (2 x 19 x p).
"""
import json
import os

import pytest

import bench

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_fp64_balances_are_the_papers():
    assert bench.loop_balance("osnt", 8, 0.0) == GOLD["B_l_OSNT"]["value"]
    assert bench.loop_balance("aa", 8, 0.0) == GOLD["B_l_AA"]["value"]
    assert 2 * 19 * 8 == GOLD["D_pdf_B"]["value"]
    lo, hi = GOLD["B_l_OSNT_R_bounds"]["value"]
    assert bench.loop_balance("osnt_r", 8, 0.0) == lo and bench.loop_balance("osnt_r", 8, 1.0) == hi
    lo, hi = GOLD["B_l_AA_R_bounds"]["value"]
    assert bench.loop_balance("aa_r", 8, 0.0) == lo and bench.loop_balance("aa_r", 8, 1.0) == hi


def test_table2_rows():
    t = GOLD["loop_balance_table"]
    assert t["order"] == ["OS-NT", "OS-NT-R", "AA", "AA-R"]
    r = 3 / 98  # the channel's run ratio (one run per row of 98 interior nodes, 3 runs)
    got = [bench.loop_balance(v, 8, r) for v in ("osnt", "osnt_r", "aa", "aa_r")]
    assert [round(x) for x in got] == t["channel"]
    # the reactor's r is not printed: one r must reproduce both of its rounded
    # RIA entries (304 + 76 r -> 333 and 304 + 38 r -> 319)
    osnt_r, aa_r = t["fixed_bed_reactor"][1], t["fixed_bed_reactor"][3]
    r_lo = max((osnt_r - 0.5 - 304) / 76, (aa_r - 0.5 - 304) / 38)
    r_hi = min((osnt_r + 0.5 - 304) / 76, (aa_r + 0.5 - 304) / 38)
    assert r_lo < r_hi
    r_bed = (r_lo + r_hi) / 2
    got = [bench.loop_balance(v, 8, r_bed) for v in ("osnt", "osnt_r", "aa", "aa_r")]
    assert [round(x) for x in got] == t["fixed_bed_reactor"]


@pytest.mark.parametrize("p", [8, 4, 2])
def test_precisions_scale_only_the_pdf_term(p):
    r = 0.207
    assert bench.loop_balance("osnt", p, r) == 38 * p + 72
    assert bench.loop_balance("osnt_r", p, r) == pytest.approx(38 * p + 76 * r)
    assert bench.loop_balance("aa", p, r) == 38 * p + 36
    assert bench.loop_balance("aa_r", p, r) == pytest.approx(38 * p + 38 * r)
