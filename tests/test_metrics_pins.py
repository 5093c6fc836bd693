"""Pins of the Schrijver et al. (2006) field-comparison metrics used for the paper's Table 1
(Sect. 2.3), on hand-computed three-point cases whose metrics are exact fractions.

Orientation (reading): b is the reference (analytic) field and B the reconstruction; E'_n, E'_m
are normalised by the reference field and eps is the reconstruction's energy over the
reference's.  Each case is chosen so that normalising by the wrong field, swapping eps, or
taking E'_m as a ratio of sums instead of a mean of ratios gives a different number."""
import math

import numpy as np
import pytest

from oracle.metrics import field_metrics


def test_scaled_copy():
    # B = 2 b at three points: every angle is 0, every error equals the reference vector.
    b = np.array([[1.0, 0, 0], [0, 2.0, 0], [0, 0, 2.0]])
    m = field_metrics(2.0 * b, b)
    assert m["C_vec"] == pytest.approx(1.0, abs=1e-15)
    assert m["C_cs"] == pytest.approx(1.0, abs=1e-15)
    assert m["E_n"] == pytest.approx(0.0, abs=1e-15)     # 1 - sum|b| / sum|b|; by |B|: 0.5
    assert m["E_m"] == pytest.approx(0.0, abs=1e-15)     # by |B|: 0.5
    assert m["eps"] == pytest.approx(4.0, abs=1e-15)     # swapped: 0.25


def test_mixed_errors_hand_computed():
    # reference b and reconstruction B:
    #   b1 = (2, 0, 0), B1 = (1, 0, 0): B.b = 2, |B|^2 = 1, |b|^2 = 4, |B - b| = 1
    #   b2 = (0, 1, 0), B2 = (0, 1, 1): B.b = 1, |B|^2 = 2, |b|^2 = 1, |B - b| = 1
    #   b3 = (0, 0, 4), B3 = (0, 0, 2): B.b = 8, |B|^2 = 4, |b|^2 = 16, |B - b| = 2
    b = np.array([[2.0, 0, 0], [0, 1.0, 0], [0, 0, 4.0]])
    B = np.array([[1.0, 0, 0], [0, 1.0, 1.0], [0, 0, 2.0]])
    m = field_metrics(B, b)
    # C_vec = 11 / sqrt(7 * 21) = 11 / (7 sqrt 3)
    assert m["C_vec"] == pytest.approx(11.0 / (7.0 * math.sqrt(3.0)), abs=1e-15)
    # C_cs = (2 / 2 + 1 / sqrt 2 + 8 / 8) / 3
    assert m["C_cs"] == pytest.approx((2.0 + 1.0 / math.sqrt(2.0)) / 3.0, abs=1e-15)
    # E'_n = 1 - (1 + 1 + 2) / (2 + 1 + 4) = 3/7  (by |B|: 1 - 4 / (3 + sqrt 2) = 0.0938)
    assert m["E_n"] == pytest.approx(3.0 / 7.0, abs=1e-15)
    # E'_m = 1 - (1/2 + 1/1 + 2/4) / 3 = 1/3  (by |B|: 0.0976; ratio of sums: 3/7)
    assert m["E_m"] == pytest.approx(1.0 / 3.0, abs=1e-15)
    # eps = 7 / 21 = 1/3  (swapped: 3)
    assert m["eps"] == pytest.approx(1.0 / 3.0, abs=1e-15)


def test_orthogonal_and_opposite():
    # B1 perpendicular to b1, B2 = -b2: C_cs = (0 - 1) / 2, E'_n = 1 - (sqrt 2 + 2) / 2.
    b = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    B = np.array([[0, 1.0, 0], [0, -1.0, 0]])
    m = field_metrics(B, b)
    assert m["C_vec"] == pytest.approx(-0.5, abs=1e-15)
    assert m["C_cs"] == pytest.approx(-0.5, abs=1e-15)
    assert m["E_n"] == pytest.approx(1.0 - (math.sqrt(2.0) + 2.0) / 2.0, abs=1e-15)
    assert m["E_m"] == pytest.approx(1.0 - (math.sqrt(2.0) + 2.0) / 2.0, abs=1e-15)
    assert m["eps"] == pytest.approx(1.0, abs=1e-15)


def test_invariant_to_point_order_and_common_rotation():
    rng = np.random.default_rng(3)
    b = rng.normal(size=(50, 3))
    B = b + 0.3 * rng.normal(size=(50, 3))
    m0 = field_metrics(B, b)
    perm = rng.permutation(50)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    m1 = field_metrics(B[perm] @ q.T, b[perm] @ q.T)
    for k in m0:
        assert m1[k] == pytest.approx(m0[k], rel=1e-12, abs=1e-14)
