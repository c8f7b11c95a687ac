"""Pins for the oracle's noise: Philox4x32-10 known-answer vectors and the
Box-Muller normal deviates (PILE-L thermostat noise, Tables S2-S3)."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], tuple(v[6:10])))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert O.philox(ctr, key) == out


def test_normal_deviates_are_standard_normal():
    from scipy import stats
    z = np.array([O.normal(12345, i, 7, 3, 2) for i in range(20000)])
    assert abs(z.mean()) < 4.0 / np.sqrt(len(z))
    assert abs(z.var() - 1.0) < 4.0 * np.sqrt(2.0 / len(z))
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_normal_streams_are_distinct():
    a = [O.normal(1, i, 0, 0, 2) for i in range(64)]
    b = [O.normal(1, i, 0, 0, 3) for i in range(64)]
    c = [O.normal(1, i, 1, 0, 2) for i in range(64)]
    d = [O.normal(2, i, 0, 0, 2) for i in range(64)]
    for other in (b, c, d):
        assert abs(np.corrcoef(a, other)[0, 1]) < 0.5
        assert not np.allclose(a, other)
