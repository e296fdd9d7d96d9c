"""The seeded input generators (shared by both sides, no method arithmetic)."""
import numpy as np

from paper_1601_04633_gb300 import inputs


def test_splitmix64_reference_value():
    # First output of SplitMix64 from state 0 (Steele, Lea & Flood 2014; Vigna's splitmix64.c).
    assert int(inputs.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF


def test_uniform_and_noise_ranges():
    u = inputs.uniform01(5, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    n = inputs.uniform_noise(1, (64, 64), 1e-6)
    assert n.shape == (64, 64) and np.abs(n).max() <= 1e-6
    assert np.array_equal(n, inputs.uniform_noise(1, (64, 64), 1e-6))
    assert not np.array_equal(n, inputs.uniform_noise(2, (64, 64), 1e-6))


def test_normal_moments():
    z = inputs.normal(4, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_batch_sweep_distribution():
    b = inputs.batch_sweep()
    assert len(b) == 64
    assert {c.nx for c in b} <= {128, 192, 256, 384} and len({c.nx for c in b}) == 4
    assert all(1e4 <= c.Ra <= 1e6 for c in b)
    assert {c.Pr for c in b} <= {0.001, 0.005, 0.01}
    assert all(c.nx == c.ny and c.alpha == 0.1 for c in b)


def test_workload_shapes():
    assert (inputs.cavity_64().nx, inputs.cavity_64().Ra) == (64, 1e4)
    c = inputs.cavity_128_adjoint()
    assert c.theta_hot_profile.shape == (128,) and abs(c.theta_hot_profile.mean() - 0.5) < 0.01
    assert inputs.cavity_4096().nx == 4096
