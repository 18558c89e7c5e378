"""Seeded synthetic inputs: fault geometry, friction parameters, initial state.

This module feeds both the CUDA path and the CPU oracle, so it holds none of
the method's arithmetic: it only lays out grids, draws seeded random numbers
and builds the geometry families the paper uses (Gaussian seamount, Sec. 4.1;
self-similar rough profile, Sec. 4.2).  Loading in equilibrium with the
initial state is left to each side (``tau_load=None``).

Workloads
---------
seamount_rupture  N=256, dx=25 m, 20 m Gaussian seamount, single rupture.
rough_cycle       N=4096, dx=10 m, Hurst-1 roughness, central 70% frictional,
                  outer 30% at plate rate.
rough_fault       one rough-fault realization of any N (ensemble member).
large_fault       N=262144, dx=1 m, Hurst-1 roughness (alpha=0.003) plus a
                  200 m Gaussian seamount, friction layout of rough_cycle.
sinusoidal_cycle  the earthquake cycle of Sec. "Seismic cycles": Table 1, a
                  sinusoidal fault of length L in a periodic domain of 4L
                  with null slip rate on 1.5L each side, uniform loading
                  rate 0.01 Pa/s.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = ["Workload", "gaussian_seamount", "seamount_rupture", "rough_profile", "rough_cycle", "rough_fault",
           "sinusoidal_cycle", "large_fault", "random_history", "random_history_device", "element_x"]


@dataclass
class Workload:
    name: str
    N: int
    dx: float
    mu: float
    cs: float
    cp: float
    dt_min: float
    h: np.ndarray
    kappa: np.ndarray
    a: np.ndarray
    b: np.ndarray
    Dc: np.ndarray
    f0: float
    V0: float
    sigma_load: np.ndarray
    V_init: np.ndarray
    theta_init: np.ndarray
    prescribed: np.ndarray
    V_presc: np.ndarray
    tau_load: np.ndarray | None = None
    tau_load_rate: np.ndarray | None = None
    steps: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def L(self) -> float:
        return self.N * self.dx


def element_x(N: int, dx: float) -> np.ndarray:
    """Element centres x_i = -L/2 + (i + 1/2) dx of the periodic fault."""
    return -0.5 * N * dx + (np.arange(N) + 0.5) * dx


def gaussian_seamount(x, amp, width):
    """h = amp exp(-x^2/(2 w^2)) and its analytic second derivative."""
    g = np.exp(-x * x / (2.0 * width * width))
    h = amp * g
    h2 = amp * g * (x * x / width ** 4 - 1.0 / width ** 2)
    return h, h2


def seamount_rupture(N: int = 256, dx: float = 25.0, amp: float = 20.0,
                     width: float = 500.0, steps: int = 2000) -> Workload:
    """Single dynamic rupture across a Gaussian seamount (mildly non-planar).

    mu=30 GPa, cs=3464 m/s, cp=sqrt(3) cs; aging law a=0.010, b=0.015 in the
    central 4 km, a-b=+0.004 outside; Dc=1 mm, sigma=50 MPa, V0=1e-6 m/s,
    f0=0.6.  V=1e-9 m/s with a log-Gaussian nucleation patch up to 1e-3 m/s
    centred at x=-1.5 km (w=150 m); theta=Dc/1e-9 everywhere.
    dt_min = 0.25 dx / cs.
    """
    cs = 3464.0
    x = element_x(N, dx)
    h, kappa = gaussian_seamount(x, amp, width)
    central = np.abs(x) < 2000.0
    a = np.where(central, 0.010, 0.019)
    b = np.full(N, 0.015)
    Dc = np.full(N, 1e-3)
    lnV = np.log(1e-9) + np.log(1e6) * np.exp(-(x + 1500.0) ** 2 / (2.0 * 150.0 ** 2))
    return Workload(
        name=f"seamount_rupture N={N} dx={dx:g}m h={amp:g}m*exp(-x^2/(2*{width:g}^2))",
        N=N, dx=dx, mu=30e9, cs=cs, cp=np.sqrt(3.0) * cs, dt_min=0.25 * dx / cs,
        h=h, kappa=kappa, a=a, b=b, Dc=Dc, f0=0.6, V0=1e-6,
        sigma_load=np.full(N, 50e6), V_init=np.exp(lnV), theta_init=np.full(N, 1e-3 / 1e-9),
        prescribed=np.zeros(N, dtype=bool), V_presc=np.zeros(N), steps=steps)


def rough_profile(N: int, dx: float, alpha: float, lam_min: float, lam_max: float,
                  seed: int):
    """Self-similar (Hurst 1) profile by spectral synthesis with random phases.

    Power spectral density P(k) = (2 pi)^3 alpha^2 |k|^-3 (Dunham et al. 2011),
    band-limited to wavelengths in [lam_min, lam_max], zero outside.  On the
    periodic grid, |h_n|^2 = P(k_n)/L for each signed mode, phases uniform from
    numpy's PCG64 seeded with ``seed``.  Returns (h, kappa) with kappa = h''
    taken mode by mode from the same spectrum (exact for the synthesized
    trigonometric sum).
    """
    L = N * dx
    n = np.arange(N // 2 + 1)
    k = 2.0 * np.pi * n / L
    rng = np.random.default_rng(seed)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n.size)
    band = np.zeros(n.size, dtype=bool)
    band[1:] = (2.0 * np.pi / k[1:] >= lam_min * (1 - 1e-12)) & (2.0 * np.pi / k[1:] <= lam_max * (1 + 1e-12))
    band[-1] = False                       # keep the Nyquist mode out (no phase freedom)
    amp = np.zeros(n.size)
    amp[band] = np.sqrt((2.0 * np.pi) ** 3 * alpha ** 2 * k[band] ** -3.0 / L)
    x = element_x(N, dx)
    # h(x) = sum_{n in band} 2 |h_n| cos(k_n x + phi_n)
    arg = np.outer(x, k[band]) + phase[band]
    h = (np.cos(arg) @ (2.0 * amp[band])) if band.any() else np.zeros(N)
    kappa = (np.cos(arg) @ (-2.0 * amp[band] * k[band] ** 2)) if band.any() else np.zeros(N)
    return h, kappa


def rough_profile_fast(N: int, dx: float, alpha: float, lam_min: float, lam_max: float,
                       seed: int):
    """Same profile as :func:`rough_profile`, synthesized with an inverse FFT (large N)."""
    L = N * dx
    n = np.arange(N // 2 + 1)
    k = 2.0 * np.pi * n / L
    rng = np.random.default_rng(seed)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=n.size)
    band = np.zeros(n.size, dtype=bool)
    band[1:] = (2.0 * np.pi / k[1:] >= lam_min * (1 - 1e-12)) & (2.0 * np.pi / k[1:] <= lam_max * (1 + 1e-12))
    band[-1] = False
    amp = np.zeros(n.size)
    amp[band] = np.sqrt((2.0 * np.pi) ** 3 * alpha ** 2 * k[band] ** -3.0 / L)
    x0 = element_x(N, dx)[0]
    # coefficient of exp(i k_n (x - x0)) such that the sum equals the cosine series
    c = amp * np.exp(1j * (phase + k * x0))
    h = np.fft.irfft(c * N, n=N)
    kap = np.fft.irfft(-(k ** 2) * c * N, n=N)
    return h, kap


def _central_friction(x, L, frac, a_vw=0.010, b=0.015, a_vs=0.019):
    central = np.abs(x) < 0.5 * frac * L
    return np.where(central, a_vw, a_vs), np.full(x.size, b), central


def rough_cycle(N: int = 4096, dx: float = 10.0, alpha: float = 0.005, seed: int = 1,
                lam_min: float = 20.0, lam_max: float = 40e3) -> Workload:
    """Rough-fault earthquake cycle: Hurst-1 roughness, central 70% frictional.

    Friction of :func:`seamount_rupture` over the central 70% of the fault; the
    outer 30% slides at the plate rate V_pl = 1e-9 m/s (prescribed elements).
    Initial V = 1e-9 m/s and steady state theta = Dc/V.
    """
    cs = 3464.0
    x = element_x(N, dx)
    gen = rough_profile if N <= 8192 else rough_profile_fast
    h, kappa = gen(N, dx, alpha, lam_min, min(lam_max, N * dx), seed)
    a, b, central = _central_friction(x, N * dx, 0.7)
    Vpl = 1e-9
    return Workload(
        name=f"rough_cycle N={N} dx={dx:g}m Hurst=1 alpha={alpha:g} lambda=[{lam_min:g},{lam_max:g}]m seed={seed}",
        N=N, dx=dx, mu=30e9, cs=cs, cp=np.sqrt(3.0) * cs, dt_min=0.25 * dx / cs,
        h=h, kappa=kappa, a=a, b=b, Dc=np.full(N, 1e-3), f0=0.6, V0=1e-6,
        sigma_load=np.full(N, 50e6), V_init=np.full(N, Vpl), theta_init=np.full(N, 1e-3 / Vpl),
        prescribed=~central, V_presc=np.where(central, 0.0, Vpl))


def sinusoidal_cycle(N: int = 4096, dx: float = 10.0, amp: float = 5.0, wavelength: float = 1280.0) -> Workload:
    """Earthquake cycle on a sinusoidal fault (Sec. "Seismic cycles", Table 1).

    Table 1: f0 = 0.6, V0 = 1e-9 m/s, Dc = 1 cm, a = 0.012, b = 0.015,
    sigma = 100 MPa, mu = 40 GPa, cs = 3464 m/s, cp = 6000 m/s, fault length
    L = 10.24 km, ds = 10 m.  As in the paper's comparison setup (Sec.
    "Comparison with ..."), the periodic domain is 4L and 1.5L on each side of
    the fault is held at a null slip rate (prescribed V = 0); the fault is
    loaded by a uniform shear-traction rate of 0.01 Pa/s.  The profile
    h = amp sin(2 pi x / wavelength) is centred so that the fault's middle is
    locally flat (kappa = 0 at x = 0); the text gives neither amplitude nor
    wavelength (they are drawn in a figure), so the defaults, 5 m over
    1.28 km (eight wavelengths on the fault, so the geometric modulation of
    slip is distinct from the rupture-scale profile; slope at most 0.025;
    32 wavelengths over the domain, so kappa is periodic), are this
    generator's choice.  Initial V = V0 on the fault with steady state
    theta = Dc / V0.
    """
    x = element_x(N, dx)
    Lf = N * dx / 4.0
    q = 2.0 * np.pi / wavelength
    h = amp * np.sin(q * x)
    kappa = -amp * q * q * np.sin(q * x)
    fault = np.abs(x) < 0.5 * Lf
    V0 = 1e-9
    Dc = 1e-2
    return Workload(
        name=f"sinusoidal_cycle N={N} dx={dx:g}m fault L={Lf / 1e3:g}km amp={amp:g}m wavelength={wavelength:g}m",
        N=N, dx=dx, mu=40e9, cs=3464.0, cp=6000.0, dt_min=0.25 * dx / 3464.0,
        h=h, kappa=kappa, a=np.full(N, 0.012), b=np.full(N, 0.015), Dc=np.full(N, Dc), f0=0.6, V0=V0,
        sigma_load=np.full(N, 100e6), V_init=np.full(N, V0), theta_init=np.full(N, Dc / V0),
        prescribed=~fault, V_presc=np.zeros(N), tau_load_rate=np.where(fault, 0.01, 0.0),
        extra={"fault": fault, "fault_length": Lf, "amp": amp, "wavelength": wavelength})


def rough_fault(N: int, dx: float, alpha: float, seed: int, lam_min: float | None = None,
                lam_max: float | None = None) -> Workload:
    """One rough-fault rupture realization (ensemble member).

    Hurst-1 profile with wavelengths in [2 dx, L]; friction and nucleation as
    :func:`seamount_rupture`, scaled to the fault length (velocity-weakening
    over the central 60%, nucleation patch at -L/4).
    """
    cs = 3464.0
    L = N * dx
    x = element_x(N, dx)
    gen = rough_profile if N <= 8192 else rough_profile_fast
    h, kappa = gen(N, dx, alpha, lam_min or 2.0 * dx, lam_max or L, seed)
    a, b, _ = _central_friction(x, L, 0.6)
    lnV = np.log(1e-9) + np.log(1e6) * np.exp(-(x + 0.25 * L) ** 2 / (2.0 * 150.0 ** 2))
    return Workload(
        name=f"rough_fault N={N} dx={dx:g}m alpha={alpha:g} seed={seed}",
        N=N, dx=dx, mu=30e9, cs=cs, cp=np.sqrt(3.0) * cs, dt_min=0.25 * dx / cs,
        h=h, kappa=kappa, a=a, b=b, Dc=np.full(N, 1e-3), f0=0.6, V0=1e-6,
        sigma_load=np.full(N, 50e6), V_init=np.exp(lnV), theta_init=np.full(N, 1e-3 / 1e-9),
        prescribed=np.zeros(N, dtype=bool), V_presc=np.zeros(N))


def random_history_device(R: np.ndarray, seed: int, scale: float, torch, dtype=None, device="cuda"):
    """Seeded complex history drawn on the device (for rings too large to draw on the host).

    Same layout as :func:`random_history` (flat, modes in order, newest
    first); values N(0, scale^2) per part from PyTorch's generator on
    ``device`` seeded with ``seed``.  Returns two complex tensors.
    """
    tot = int(np.maximum(np.asarray(R, dtype=np.int64), 0).sum())
    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = []
    for _ in range(2):
        v = torch.randn(tot, 2, generator=g, dtype=dtype, device=device)
        v.mul_(scale)
        out.append(torch.view_as_complex(v))
    return out[0], out[1]


def large_fault(N: int = 262144, dx: float = 1.0, alpha: float = 0.003, seed: int = 4,
                lam_min: float = 20.0, lam_max: float = 40e3, sea_amp: float = 200.0,
                sea_sigma: float = 1000.0) -> Workload:
    """A large rough fault with a seamount: Hurst-1 roughness (ratio alpha,
    wavelengths in [lam_min, min(lam_max, L)]) plus a Gaussian seamount of
    height sea_amp and standard deviation sea_sigma (2 sigma = 2 km wide, max
    slope ~0.12) at the centre; friction and plate-rate loading of
    :func:`rough_cycle` (central 70% rate-and-state, outer 30% at V_pl).
    """
    cs = 3464.0
    x = element_x(N, dx)
    h, kappa = rough_profile_fast(N, dx, alpha, lam_min, min(lam_max, N * dx), seed)
    hs, ks = gaussian_seamount(x, sea_amp, sea_sigma)
    h = h + hs
    kappa = kappa + ks
    a, b, central = _central_friction(x, N * dx, 0.7)
    Vpl = 1e-9
    return Workload(
        name=(f"large_fault N={N} dx={dx:g}m Hurst=1 alpha={alpha:g} lambda=[{lam_min:g},{min(lam_max, N * dx):g}]m "
              f"seed={seed} + seamount {sea_amp:g}m sigma={sea_sigma:g}m"),
        N=N, dx=dx, mu=30e9, cs=cs, cp=np.sqrt(3.0) * cs, dt_min=0.25 * dx / cs,
        h=h, kappa=kappa, a=a, b=b, Dc=np.full(N, 1e-3), f0=0.6, V0=1e-6,
        sigma_load=np.full(N, 50e6), V_init=np.full(N, Vpl), theta_init=np.full(N, 1e-3 / Vpl),
        prescribed=~central, V_presc=np.where(central, 0.0, Vpl),
        extra={"alpha": alpha, "lam_min": lam_min, "lam_max": min(lam_max, N * dx), "seamount": (sea_amp, sea_sigma)})


def random_history(R: np.ndarray, seed: int, scale: float = 1e-9):
    """Seeded complex history values for pre-filled rings.

    R[n] is the number of past slots of mode n.  Returns two flat complex128
    arrays (shear and normal fields), mode n occupying [off[n], off[n+1]),
    newest slot first, and the offsets.  Values are N(0, scale^2) per part.
    """
    R = np.asarray(R, dtype=np.int64)
    off = np.zeros(R.size + 1, dtype=np.int64)
    off[1:] = np.cumsum(R)
    rng = np.random.default_rng(seed)
    tot = int(off[-1])
    HT = scale * (rng.standard_normal(tot) + 1j * rng.standard_normal(tot))
    HN = scale * (rng.standard_normal(tot) + 1j * rng.standard_normal(tot))
    return HT, HN, off
