"""Pins for the oracle's kernel functions W, C^T_II, C^N_II (Sec. 2.3, 2.4, App. A).

Each test checks the oracle against something other than itself:
  * W against a high-precision evaluation of its defining integral and
    against the Struve-function form (Sec. 2.3);
  * C(0) = -(1 - c_s^2/c_p^2), the cancellation stated in Sec. 2.3 / 2.4;
  * dC^T/ds against the integrand printed in App. A (shear primitive);
  * the Laplace transform in time of both kernels against the closed-form
    elastodynamic responses of a periodic slip (mode II) and opening (mode I)
    distribution on a plane -- an independent derivation from the
    Green's function;
  * the normal kernel against the Fourier-transform pairs of App. B.
"""
import numpy as np
import pytest
from scipy import integrate, special

from oracle.kernels import G_N, G_T, W

R_SQRT3 = 1.0 / np.sqrt(3.0)
R_TABLE1 = 3464.0 / 6000.0


def test_W_at_zero_and_limit():
    assert W(np.array([0.0]))[0] == pytest.approx(1.0, abs=1e-16)
    # int_0^inf J1(t)/t dt = 1  ->  W -> 0 slowly (x^-3/2 envelope)
    x = np.linspace(900.0, 1000.0, 201)
    assert np.abs(W(x)).max() < 3.0 * 900.0 ** -1.5


def test_W_against_high_precision_tail_integral():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 30
    for x in [0.5, 3.0, 17.0, 60.0, 200.0, 346.0]:
        ref = mpmath.quadosc(lambda t: mpmath.besselj(1, t) / t, [x, mpmath.inf], omega=1)
        assert abs(W(np.array([x]))[0] - float(ref)) < 2e-16, x


def test_W_against_struve_form():
    # Sec. 2.3: W = 1 - x J0 + J1 - psi,  psi = (pi/2) x (J1 H0 - J0 H1)
    x = np.linspace(0.01, 40.0, 400)
    psi = 0.5 * np.pi * x * (special.j1(x) * special.struve(0, x) - special.j0(x) * special.struve(1, x))
    ref = 1.0 - x * special.j0(x) + special.j1(x) - psi
    # scipy's Struve route itself cancels to ~1e-12 for x in 20..40
    assert np.abs(W(x) - ref).max() < 5e-12


@pytest.mark.parametrize("r", [R_SQRT3, R_TABLE1])
def test_kernels_cancel_static_term_at_t0(r):
    # Sec. 2.3 / 2.4: static and dynamic terms cancel at t = 0.
    s0 = np.array([0.0, 1e-14])
    assert np.allclose(G_T(s0, r), -(1.0 - r * r), atol=1e-12, rtol=0)
    assert np.allclose(G_N(s0, r), -(1.0 - r * r), atol=1e-12, rtol=0)


@pytest.mark.parametrize("r", [R_SQRT3, R_TABLE1])
def test_shear_kernel_derivative_matches_appendix_A(r):
    # App. A prints the shear integrand; per unit s it is twice dC^T/ds:
    # J1(s)/s + 4 s [W(s/r) - W(s)] - 4 r J0(s/r) + 3 J0(s).
    s = np.array([0.5, 3.0, 7.7, 20.0, 55.0, 100.0, 180.0])
    h = 1e-4
    num = (G_T(s + h, r) - G_T(s - h, r)) / (2 * h)
    integrand = (special.j1(s) / s + 4 * s * (W(s / r) - W(s))
                 - 4 * r * special.j0(s / r) + 3 * special.j0(s))
    assert np.allclose(num, 0.5 * integrand, atol=2e-7, rtol=0)


def _laplace(G, p, r, T=3000.0):
    val, _ = integrate.quad(lambda s: np.exp(-p * s) * G(np.array([s]), r)[0], 0.0, T,
                            limit=4000, epsabs=1e-13, epsrel=1e-12)
    return val


def _elastodynamic(p, r):
    """Closed-form Laplace-domain responses (k = 1, c_s = 1, mu = 1).

    alpha = sqrt(1 + r^2 p^2), beta = sqrt(1 + p^2), R = (2 + p^2)^2 - 4 alpha beta
    (Rayleigh function).  Traction per unit slip of a mode-II distribution:
    K_II = R / (2 beta p^2); per unit opening (mode I): K_I = R / (2 alpha p^2).
    The inertia term of the opening (rho (lambda+2mu) p^2 G_22 on the plane)
    is (1/r^2) [p^2/(2 beta) - (beta - alpha)/2].
    """
    al = np.sqrt(1.0 + r * r * p * p)
    be = np.sqrt(1.0 + p * p)
    R = (2.0 + p * p) ** 2 - 4.0 * al * be
    return R / (2 * be * p * p), R / (2 * al * p * p), (p * p / (2 * be) - 0.5 * (be - al)) / (r * r)


@pytest.mark.parametrize("r", [R_SQRT3, R_TABLE1])
@pytest.mark.parametrize("p", [0.3, 1.0, 3.0])
def test_shear_kernel_laplace_transform_is_mode_II_response(p, r):
    # tau(k,p) = -[eta p + S|k| + mu |k| p L[C^T]] delta(k,p) must equal -K_II delta:
    # L[C^T](p) = (K_II - 1/2 p - S) / p  with S = 1 - r^2, eta = 1/2.
    K2, _, _ = _elastodynamic(p, r)
    expect = (K2 - 0.5 * p - (1.0 - r * r)) / p
    assert _laplace(G_T, p, r) == pytest.approx(expect, abs=2e-10)


@pytest.mark.parametrize("r", [R_SQRT3, R_TABLE1])
@pytest.mark.parametrize("p", [0.3, 1.0, 3.0])
def test_normal_kernel_laplace_transform_is_mode_I_without_inertia(p, r):
    # The curvature x slip term acts as an opening gradient; the inertia term of
    # main_eq carries only the shear slip, so the normal kernel is the mode-I
    # response with its inertia part removed: S + p L[C^N] = K_I - inertia.
    _, K1, inert = _elastodynamic(p, r)
    expect = (K1 - inert - (1.0 - r * r)) / p
    assert _laplace(G_N, p, r) == pytest.approx(expect, abs=2e-10)


@pytest.mark.parametrize("r", [R_SQRT3, R_TABLE1])
def test_normal_kernel_matches_appendix_B_transform_pairs(r):
    # App. B: with b = c t, the space-time kernel transforms through
    # F[b^3/x^3 sqrt(1-x^2/b^2) rect] = (i pi b/2)(bk J0 + J1 + 1 + b^2k^2 - (1+b^2k^2) W)
    # F[rect / ((x/b) sqrt(1-x^2/b^2))] = -i pi b (1 + J1 - W); with the Lame
    # identities the sum over the P and S parts divided by i mu must equal
    # (1 - r^2) + C^N.
    s = np.linspace(0.05, 150.0, 301)
    sp_ = s / r
    A = (1.0 / r ** 2 - 2.0) ** 2 * r * r / 2.0

    def big(z):
        return z * special.j0(z) + special.j1(z) + 1 + z * z - (1 + z * z) * W(z)

    def small(z):
        return 1 + special.j1(z) - W(z)

    total = r * r * big(sp_) - A * small(sp_) - big(s) + small(s) / (2 * r * r)
    assert np.abs(total - ((1 - r * r) + G_N(s, r))).max() < 1e-9


def test_kernels_decay_at_large_argument():
    # Sec. 3.1: both kernels go to zero as the argument grows.
    r = R_SQRT3
    s_lo = np.linspace(50.0, 60.0, 400)
    s_hi = np.linspace(5000.0, 5010.0, 400)
    for G in (G_T, G_N):
        assert np.abs(G(s_hi, r)).max() < 0.2 * np.abs(G(s_lo, r)).max()
