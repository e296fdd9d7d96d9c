"""Host-side Nusselt-history analysis (mean, amplitude, period in Fourier units)."""
import math

import numpy as np
import pytest

from paper_1601_04633_gb300 import analysis as A


def test_fourier_number_eq20():
    # Fo = alpha t / H^2; 122880 steps of a 64-row cavity at alpha = 0.1 is Fo = 3.
    assert A.fourier_number(122880, 0.1, 64) == pytest.approx(3.0, rel=1e-15)


@pytest.mark.parametrize("period,amp,mean", [(0.092, 0.01, 2.80), (0.093, 0.05, 2.65), (0.073, 0.2, 3.1)])
def test_sinusoid_statistics(period, amp, mean):
    fo_per_step = 0.1 / 128 ** 2
    n = int(round(1.0 / fo_per_step))
    fo = (np.arange(n) + 1) * fo_per_step
    nu = mean + amp * np.sin(2 * math.pi * fo / period + 0.3)
    s = A.nu_statistics(nu, fo_per_step, window_fo=0.6)
    assert not s.steady
    assert s.mean == pytest.approx(mean, abs=0.05 * amp)
    assert s.amplitude == pytest.approx(amp, rel=1e-3)
    assert s.crossing_period_fo == pytest.approx(period, rel=1e-4)
    assert s.period_fo == pytest.approx(period, rel=0.02)  # spectral estimate
    assert s.cycles >= int(0.6 / period) - 2  # the moving average trims one period


def test_noisy_and_drifting_signal():
    rng = np.random.default_rng(0)
    fo_per_step = 1e-5
    fo = (np.arange(200000) + 1) * fo_per_step
    nu = 2.0 + 0.05 * np.sin(2 * math.pi * fo / 0.1) + 1e-4 * rng.standard_normal(fo.size)
    s = A.nu_statistics(nu, fo_per_step, window_fo=1.0)
    assert s.period_fo == pytest.approx(0.1, rel=0.01)
    drifting = 2.0 + 0.3 * fo + 0.05 * np.sin(2 * math.pi * fo / 0.1)
    s2 = A.nu_statistics(drifting, fo_per_step, window_fo=1.0)
    assert s2.drift == pytest.approx(0.3 * 0.8, rel=0.05)
    assert s2.crossing_period_fo == pytest.approx(0.1, rel=1e-3)
    assert s2.period_fo == pytest.approx(0.1, rel=0.01)


def test_steady_detection():
    nu = 1.95 + 1e-6 * np.exp(-np.arange(10000) / 100.0)
    s = A.nu_statistics(nu, 1e-4)
    assert s.steady and s.period_fo is None and s.mean == pytest.approx(1.95, abs=1e-9)
    # converging without oscillation (slow drift) also counts as steady
    drift = 1.9 + 0.01 * (1 - np.exp(-np.arange(20000) / 30000.0))
    s = A.nu_statistics(drift, 1e-4)
    assert s.steady and s.drift > 0


def test_two_frequency_signal_dominant_period():
    fo_per_step = 1e-5
    fo = (np.arange(300000) + 1) * fo_per_step
    nu = 2.7 + 0.04 * np.sin(2 * math.pi * fo / 0.038) + 0.015 * np.sin(2 * math.pi * fo / 0.11)
    s = A.nu_statistics(nu, fo_per_step, window_fo=2.0)
    assert s.period_fo == pytest.approx(0.038, rel=0.01)
