"""Host-side helpers of the screening pipeline (no GPU): the travelling-wave
phase field, the coefficient of determination and the top-fraction
selection, each against a definition computed another way."""
import numpy as np
import pytest

from paper_2207_09334_gb300 import screen


def test_phase_field_is_a_wave_along_x():
    ph = screen.phase_field(8)
    assert ph.shape == (8, 8, 8) and ph.dtype == np.float32
    # constant over z and y, 2 pi x / 8 along x (the last axis)
    assert np.all(ph == ph[:1, :1, :])
    np.testing.assert_allclose(ph[0, 0], 2 * np.pi * np.arange(8) / 8, rtol=0, atol=1e-6)


def test_r2_special_values_and_library():
    rng = np.random.default_rng(0)
    y = rng.standard_normal(500)
    assert screen.r2(y, y) == 1.0                                   # perfect prediction
    assert abs(screen.r2(np.full_like(y, y.mean()), y)) < 1e-12     # the mean predicts nothing
    p = y + 0.5 * rng.standard_normal(500)
    metrics = pytest.importorskip("sklearn.metrics")
    assert abs(screen.r2(p, y) - metrics.r2_score(y, p)) < 1e-12


def test_top_indices_selects_the_largest_in_order():
    rng = np.random.default_rng(1)
    pred = rng.standard_normal(1000)
    top = screen.top_indices(pred, 0.01)
    assert len(top) == 10
    np.testing.assert_array_equal(top, np.argsort(-pred)[:10])      # a full sort gives the same
    assert len(screen.top_indices(pred[:20], 0.01)) == 1            # at least one
    # ties keep a valid order: every chosen value is at least every value left out
    ties = np.repeat(np.arange(10.0), 10)
    t = screen.top_indices(ties, 0.15)
    assert len(t) == 15 and ties[t].min() >= np.delete(ties, t).max()
    assert np.all(np.diff(ties[t]) <= 0)
