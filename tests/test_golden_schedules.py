"""The driver's iteration schedules against the values the paper prints for four scales
(tests/golden/iteration_schedules.txt, Sections 5.1 and 5.2)."""
import os

from paper_2212_13459_gb300 import driver

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "iteration_schedules.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            name, vals = line.split(":")
            out[name.strip()] = [int(v) for v in vals.split(",")]
    return out


def test_spst_schedule_matches_paper():
    assert driver.spst_schedule(4) == _golden()["spst"]


def test_spst_fast_schedule_matches_paper():
    assert driver.spst_fast_schedule(4) == _golden()["spst_fast"]


def test_spst_fast_floor():
    assert min(driver.spst_fast_schedule(8)) == 30
