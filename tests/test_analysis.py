"""Host-side statistics of the long-run analysis: time averages and their standard
error, the power-law fit, the compensated spectrum (checked on data with known answers)."""
import numpy as np
import pytest

from paper_2205_04658_gb300 import analysis as A


def test_time_average_mean_and_standard_error():
    rng = np.random.default_rng(0)
    true = np.array([1.0, 0.5, 0.25])
    sig = np.array([0.1, 0.05, 0.01])
    M = 4000
    s = true + sig * rng.standard_normal((M, 3))
    mean, err = A.time_average(s)
    assert np.allclose(mean, s.mean(axis=0), rtol=1e-14)
    assert np.allclose(err, s.std(axis=0) / np.sqrt(M), rtol=1e-9)
    assert np.all(np.abs(mean - true) < 5 * err)
    # constant samples: no error
    m2, e2 = A.time_average(np.ones((10, 4)) * 3.0)
    assert np.all(m2 == 3.0) and np.all(e2 == 0.0)


def test_power_law_slope_recovers_kolmogorov():
    k = np.arange(1, 20, dtype=float)
    E = 7.0 * k ** (-5.0 / 3.0)
    assert A.power_law_slope(k, E) == pytest.approx(-5.0 / 3.0, abs=1e-12)
    assert np.allclose(A.compensated(k, E), 7.0, rtol=1e-12)
    # zero bins are ignored
    E2 = E.copy()
    E2[[0, 5]] = 0.0
    assert A.power_law_slope(k, E2) == pytest.approx(-5.0 / 3.0, abs=1e-12)
    with pytest.raises(ValueError):
        A.power_law_slope([1.0], [1.0])


def test_decorrelation_and_settling_constants():
    assert A.DECORRELATION_STEPS * 0.05 == pytest.approx(0.9)
    assert A.SETTLE_STEP * 0.05 == pytest.approx(32.0)


def test_fluctuation_spectrum_of_a_single_frequency():
    t = np.arange(64)
    s = 0.3 + 0.01 * np.cos(2 * np.pi * 5 * t / 64)
    P = A.fluctuation_spectrum(s)
    assert np.argmax(P) == 5
    assert P[0] < 1e-20
    assert P[5] == pytest.approx((0.01 * 64 / 2) ** 2, rel=1e-12)


def test_channel_impurities():
    from paper_2205_04658_gb300 import inputs
    one = inputs.channel_impurities(256, 128, 13)
    assert one.sum() == sum(1 for dy in range(-6, 7) for dx in range(-6, 7) if dx * dx + dy * dy <= 36)
    two = inputs.channel_impurities(256, 128, 13, count=2)
    assert two.sum() == 2 * one.sum()
