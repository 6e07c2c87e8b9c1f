"""Pins for the Hausdorff helper -- CPU only."""
import numpy as np
import pytest

from oracle.hausdorff import hausdorff


def test_parallel_segments():
    a = np.array([[0.0, 0.0], [1.0, 0.0]])
    b = np.array([[0.0, 0.3], [1.0, 0.3]])
    assert hausdorff(a, b, 0.01) == pytest.approx(0.3, abs=1e-12)


def test_subset_is_one_sided():
    a = np.array([[0.0, 0.0], [1.0, 0.0]])
    b = np.array([[0.0, 0.0], [0.5, 0.0]])
    assert hausdorff(a, b, 0.01) == pytest.approx(0.5, abs=1e-12)


def test_identical_and_point():
    a = np.array([[0.0, 0.0], [0.2, 0.7], [1.0, 1.0]])
    assert hausdorff(a, a, 0.01) < 1e-12
    assert hausdorff(a[:1], np.array([[3.0, 4.0]]), 0.1) == pytest.approx(5.0)
