"""Pins for the seeded geometry generators against the paper's printed slopes."""
import numpy as np
import pytest

from paper_2107_03550_gb300.workloads import (element_x, gaussian_seamount, rough_profile,
                                              rough_profile_fast)
from tests.golden.paper import paper_numbers


@pytest.mark.parametrize("A_km,key", [(0.03, "seamount_slope_A30"), (0.1, "seamount_slope_A100"),
                                      (0.3, "seamount_slope_A300")])
def test_seamount_max_slope_matches_sec_4_1(A_km, key):
    # Sec. 4.1: y2 = A exp(-(y1 - 7)^2) in km, i.e. a Gaussian of width 1/sqrt(2) km.
    x = np.linspace(-3000.0, 3000.0, 600001)
    h, _ = gaussian_seamount(x, A_km * 1e3, 1e3 / np.sqrt(2.0))
    slope = np.abs(np.gradient(h, x)).max()
    assert slope == pytest.approx(paper_numbers()[key], abs=0.0006 if A_km < 0.3 else 0.003)


def test_seamount_curvature_is_second_derivative():
    x = np.linspace(-2000.0, 2000.0, 40001)
    h, k = gaussian_seamount(x, 20.0, 500.0)
    num = np.gradient(np.gradient(h, x), x)
    assert np.abs(num - k)[100:-100].max() < 1e-3 * np.abs(k).max()


@pytest.mark.parametrize("alpha,key", [(1e-4, "rough_slope_1e-4"), (3e-4, "rough_slope_3e-4"),
                                       (1e-3, "rough_slope_1e-3"), (3e-3, "rough_slope_3e-3")])
def test_rough_profile_max_slope_distribution_contains_sec_4_2(alpha, key):
    # Sec. 4.2: L = 10.24 km, ds = 10 m, lambda_min = 200 m; the printed max
    # slope of one realization must sit inside our seed distribution, and the
    # slope must scale linearly with alpha.
    slopes = []
    for seed in range(40):
        h, _ = rough_profile(1024, 10.0, alpha, 200.0, 10240.0, seed)
        slopes.append(np.abs(np.gradient(h, 10.0)).max())
    slopes = np.array(slopes)
    lo, hi = np.quantile(slopes, [0.025, 0.975])
    assert lo <= paper_numbers()[key] <= hi
    h1, _ = rough_profile(1024, 10.0, 1.0, 200.0, 10240.0, 7)
    h2, _ = rough_profile(1024, 10.0, alpha, 200.0, 10240.0, 7)
    assert np.allclose(h2, alpha * h1, rtol=1e-12, atol=0)


def test_rough_profile_fft_synthesis_equals_direct_sum():
    h1, k1 = rough_profile(2048, 10.0, 5e-3, 20.0, 20480.0, 11)
    h2, k2 = rough_profile_fast(2048, 10.0, 5e-3, 20.0, 20480.0, 11)
    assert np.abs(h1 - h2).max() < 1e-10 * np.abs(h1).max()
    assert np.abs(k1 - k2).max() < 1e-10 * np.abs(k1).max()


def test_rough_profile_curvature_is_second_derivative():
    N, dx = 4096, 10.0
    h, k = rough_profile(N, dx, 1e-3, 200.0, N * dx, 3)
    # spectral second derivative of the periodic samples
    kk = 2 * np.pi * np.fft.rfftfreq(N, dx)
    k_num = np.fft.irfft(-(kk ** 2) * np.fft.rfft(h), n=N)
    assert np.abs(k_num - k).max() < 1e-9 * np.abs(k).max()
    assert element_x(N, dx)[0] == pytest.approx(-N * dx / 2 + dx / 2)


def test_sinusoidal_cycle_follows_table1_and_the_domain_of_the_comparison():
    from paper_2107_03550_gb300.workloads import sinusoidal_cycle
    w = sinusoidal_cycle()
    # Table 1
    assert (w.mu, w.cs, w.cp, w.f0, w.V0) == (40e9, 3464.0, 6000.0, 0.6, 1e-9)
    assert np.all(w.a == 0.012) and np.all(w.b == 0.015) and np.all(w.Dc == 1e-2)
    assert np.all(w.sigma_load == 100e6) and w.dx == 10.0
    fault = w.extra["fault"]
    # fault length 10.24 km in a 4L periodic domain, 1.5L held at null slip rate each side
    assert fault.sum() * w.dx == 10240.0 and w.N * w.dx == 4 * 10240.0
    assert np.all(w.prescribed == ~fault) and np.all(w.V_presc[~fault] == 0.0)
    x = element_x(w.N, w.dx)
    assert np.all(np.abs(x[~fault]) > 10240.0 / 2 - w.dx)
    assert np.all(w.tau_load_rate[fault] == 0.01)
    # curvature is h'' (periodic second difference, O(dx^2)); flat at the middle
    d2 = (np.roll(w.h, -1) - 2 * w.h + np.roll(w.h, 1)) / w.dx ** 2
    assert np.abs(d2 - w.kappa).max() < 1e-3 * np.abs(w.kappa).max()
    mid = w.N // 2  # elements -dx/2 and +dx/2 straddle x = 0, where kappa changes sign
    assert w.kappa[mid - 1] * w.kappa[mid] < 0 and x[mid - 1] < 0 < x[mid]
