"""Pins against numbers the paper prints (Table I and the percentages Sec. IV
derives from it).  They fix how this project reports a relative reduction:
(reference - ours) / reference, in percent, rounded to two decimals."""
import os

import pytest

from paper_2309_11072_gb300.metrics import reduction_pct

HERE = os.path.dirname(os.path.abspath(__file__))


def _table():
    rows = {}
    with open(os.path.join(HERE, "golden", "table1_sec4.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, *v = line.split()
                rows[k] = [float(x) for x in v]
    return rows


def test_slrme_gain_over_plain_mantissa_coding():
    t = _table()["avg42_bpp"]
    assert round(reduction_pct(t[2], t[3]), 2) == 5.02


def test_bitrate_reduction_range_against_existing_methods():
    t = _table()["avg42_bpp"]
    assert round(reduction_pct(t[1], t[3]), 2) == 1.57
    assert round(reduction_pct(t[0], t[3]), 2) == 6.68


def test_encoder_time_reduction_range():
    t42, t4 = _table()["avg42_time"], _table()["avg4_time"]
    assert round(reduction_pct(t4[1], t4[3]), 2) == 87.13
    assert round(reduction_pct(t42[0], t42[3]), 2) == 98.96


def test_reduction_rejects_nonpositive_reference():
    with pytest.raises(ValueError):
        reduction_pct(0.0, 1.0)
