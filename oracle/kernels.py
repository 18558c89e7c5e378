"""Oracle: the spectral convolution kernels C^T_II and C^N_II in plain FP64.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.

Everything here is written straight from the paper's formulas, in the
dimensionless variable s = c_s |k| t and with r = c_s / c_p:

* W(x) = int_x^inf J1(t)/t dt = 1 - int_0^x J1(t)/t dt            (App. A, Eq. A.1)
  The integral is a composite Gauss-Legendre rule on panels of width 1/2
  with compensated (Neumaier) accumulation of the panel sums.
* G_T(s) = C^T_II(k, t)                                             (Eq. Ct, Sec. 2.3)
* G_N(s) = C^N_II(k, t)                                             (Sec. 2.4)

Bessel J0, J1 come from scipy.special (a library primitive).
"""
from __future__ import annotations

import numpy as np
from scipy import special

__all__ = ["W", "G_T", "G_N", "kernel_pair"]

_PANEL = 0.5          # panel width of the composite Gauss-Legendre rule
_GL_ORDER = 16        # points per panel; J1(t)/t is entire, 16 points on 1/2 is exact to rounding
_gl_x, _gl_w = np.polynomial.legendre.leggauss(_GL_ORDER)


def _j1_over_t(t: np.ndarray) -> np.ndarray:
    """J1(t)/t with its limit 1/2 at t = 0."""
    out = np.empty_like(t)
    small = np.abs(t) < 1e-8
    out[~small] = special.j1(t[~small]) / t[~small]
    out[small] = 0.5 - t[small] ** 2 / 16.0
    return out


def _panel_integral(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Gauss-Legendre value of int_a^b J1(t)/t dt, elementwise."""
    half = 0.5 * (b - a)
    mid = 0.5 * (b + a)
    t = mid[..., None] + half[..., None] * _gl_x
    return half * (_j1_over_t(t) @ _gl_w)


class _CumulativeJ1t:
    """Running integral I(m) = int_0^{m*h} J1(t)/t dt at panel ends m*h.

    Accumulated with Neumaier compensation so the rounding error of the
    partial sums stays at a few ulps of the sum itself.
    """

    def __init__(self) -> None:
        self.cum = np.zeros(1)

    def ensure(self, xmax: float) -> None:
        m_needed = int(np.floor(xmax / _PANEL)) + 2
        if m_needed < self.cum.size:
            return
        m_needed = max(m_needed, 2 * self.cum.size)
        edges = _PANEL * np.arange(m_needed + 1, dtype=np.float64)
        panels = _panel_integral(edges[:-1], edges[1:])
        cum = np.empty(m_needed + 1)
        s = 0.0
        c = 0.0
        cum[0] = 0.0
        for i, v in enumerate(panels.tolist()):
            t = s + v
            if abs(s) >= abs(v):
                c += (s - t) + v
            else:
                c += (v - t) + s
            s = t
            cum[i + 1] = s + c
        self.cum = cum


_cum = _CumulativeJ1t()


def W(x) -> np.ndarray:
    """W(x) = 1 - int_0^x J1(t)/t dt for x >= 0 (App. A, Eq. A.1; Sec. 2.3)."""
    x = np.asarray(x, dtype=np.float64)
    if np.any(x < 0):
        raise ValueError("W is evaluated for x >= 0 only")
    flat = x.ravel()
    if flat.size == 0:
        return x.copy()
    _cum.ensure(float(flat.max()))
    m = np.floor(flat / _PANEL).astype(np.int64)
    base = _cum.cum[m]
    rest = _panel_integral(m * _PANEL, flat)
    return (1.0 - (base + rest)).reshape(x.shape)


def _parts(s, r: float):
    """W, J0, J1 at the S-wave argument s and the P-wave argument s/r."""
    s = np.asarray(s, dtype=np.float64)
    sp_ = s / r
    return (s, sp_, W(s), W(sp_), special.j0(s), special.j1(s), special.j0(sp_), special.j1(sp_))


def _gt(parts, r):
    s, sp_, Ws, Wp, J0s, J1s, J0p, J1p = parts
    return ((s * s + r * r) * Wp - (s * s + 1.0) * Ws
            - r * r * J1p + 0.5 * J1s - r * s * J0p + s * J0s)


def _gn(parts, r):
    s, sp_, Ws, Wp, J0s, J1s, J0p, J1p = parts
    A = (1.0 / (r * r) - 2.0) ** 2 * r * r / 2.0
    return ((A - r * r - s * s) * Wp + (1.0 + s * s - 1.0 / (2.0 * r * r)) * Ws
            + (r * r - A) * J1p + (1.0 / (2.0 * r * r) - 1.0) * J1s + r * s * J0p - s * J0s)


def G_T(s, r: float) -> np.ndarray:
    """Shear kernel C^T_II as a function of s = c_s k t (Eq. Ct).

    C^T = (s^2 + r^2) W(s/r) - (s^2 + 1) W(s) - r^2 J1(s/r) + J1(s)/2
          - r s J0(s/r) + s J0(s),   with c_p k t = s/r and (c_s^2/c_p) k t = r s.
    """
    return _gt(_parts(s, r), r)


def G_N(s, r: float) -> np.ndarray:
    """Normal kernel C^N_II as a function of s = c_s k t (Sec. 2.4).

    With A = (c_p^2/c_s^2 - 2)^2 c_s^2 / (2 c_p^2) = (1/r^2 - 2)^2 r^2 / 2:
    C^N = (A - r^2 - s^2) W(s/r) + (1 + s^2 - 1/(2 r^2)) W(s)
          + (r^2 - A) J1(s/r) + (1/(2 r^2) - 1) J1(s) + r s J0(s/r) - s J0(s).
    """
    return _gn(_parts(s, r), r)


def kernel_pair(s, r: float):
    """(G_T(s), G_N(s)) from one evaluation of W, J0, J1 at s and s/r."""
    parts = _parts(s, r)
    return _gt(parts, r), _gn(parts, r)
