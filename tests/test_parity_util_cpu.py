"""The comparison helpers of the parity tests on hand-built cases (no GPU):
the polyline point at an arc length, and the Frenet rule that accepts an s
far from the oracle's only at a projection near-tie."""
import numpy as np
import pytest

from tests.parity_util import FRENET_ABS, assert_frenet_close, polyline_point

SQUARE = np.float32([[0, 0, 0, 0], [10, 0, 0, 0], [10, 10, 0, 0], [0, 10, 0, 0]])


def test_polyline_point_on_a_square():
    pts = polyline_point(SQUARE, [0.0, 5.0, 10.0, 15.0, 25.0, 39.0, 40.0, 45.0])
    np.testing.assert_allclose(pts, [[0, 0], [5, 0], [10, 0], [10, 5], [5, 10], [0, 1], [0, 0], [5, 0]], atol=1e-12)


def test_frenet_rule_accepts_only_nearest_feet():
    # centre of the square: equidistant (5 m) from all four sides
    state = np.float64([[5.0, 5.0, 0.0, 0.0]])
    ref = np.float64([[5.0, -5.0]])                     # oracle: foot (5, 0), s = 5, d = -5
    tie = np.float64([[25.0, -5.0]])                    # GPU: foot (5, 10), equally near
    assert assert_frenet_close(tie, ref, state, SQUARE)[2] == 1
    wrong = np.float64([[12.0, -5.0]])                  # foot (10, 2): 5.39 m away
    with pytest.raises(AssertionError, match="not nearest"):
        assert_frenet_close(wrong, ref, state, SQUARE)
    with pytest.raises(AssertionError, match=r"\|d\| error"):
        assert_frenet_close(np.float64([[5.0, -5.0 - 2 * FRENET_ABS]]), ref, state, SQUARE)
