"""Oracle: one time step of the non-planar spectral BIEM, plain FP64 on the CPU.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.

The step follows Sec. 3.3 in the paper's order (after Lapusta et al. 2000):

  (1) slip and state prediction with the pass velocity Vbar,
  (2) tractions from the spectral formulas of Sec. 3.1 with the history
      integral over [dt, T_w] and the current interval [0, dt],
      midpoint quadrature of the kernels,
  (3) rate-and-state momentum balance (Eq. momentum) solved per element for V,
  then the same three steps again with Vbar = (V + V1)/2, and the history of
  the slip rate spectrum is extended with that averaged value.

Readings taken where the paper is silent or garbled (each is listed, with its
reason, in the design notes of the repository):

* radiation damping -mu/(2 c_s) V is added to the shear traction explicitly
  (Sec. 2.3 states that the kernel contains it; the spectral form has none);
* the normal traction is compression-positive and carries the odd factor
  -i sgn(k) under F[f]_n = sum_i f_i exp(-i k_n x_i); it is zero at k = 0 and
  at the Nyquist mode;
* k_c = 200/(eta L) in rad/m by default; windows M_n = ceil(T_w(k_n)/dt_min);
* quadrature weights w_{n,j} = dt_min * C(k_n, (j+1/2) dt_min), j = 0..M_n-1
  (the midpoint rule Sec. 3.3 names); the option ``quadrature="exact"``
  takes the integral of C(k_n, tau) over [j dt_min, (j+1) dt_min] instead;
* the state variable follows the aging law integrated exactly at constant
  Vbar over the step (Lapusta et al. 2000); the explicit form of Sec. 3.3
  (theta + thetadot dt) is an option;
* a step of length dt = m dt_min (m >= 1 integer) advances the history by m
  slots; its current interval takes the sum of the first m weights.

FFTs are numpy's (a library primitive); the operators applied per mode are
translation invariant, so the index-based DFT equals the one over x_i.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .kernels import kernel_pair

__all__ = ["Params", "windows", "weights", "Oracle", "newton_lnV", "state_update", "mode_history_sum",
           "history_sums_sampled",
           "STATUS_OK", "STATUS_NEWTON", "STATUS_OPENING", "STATUS_STATE"]

STATUS_OK = 0
STATUS_NEWTON = 1      # Newton did not converge within the cap
STATUS_OPENING = 2     # sigma_load + sigma_el <= 0 (Sec. 3.2, failure conditions)
STATUS_STATE = 4       # theta <= 0 (explicit state update only)


@dataclass
class Params:
    """Material, grid and truncation parameters (Table 1 names)."""
    N: int
    dx: float
    mu: float
    cs: float
    cp: float
    dt_min: float                 # beta_min * dx / cs (Sec. 3.2)
    eta_w: float = 1.0            # truncation parameter eta (Sec. 3.1)
    kc_L: float = 200.0           # k_c * (eta * L) (Sec. 3.1)
    kcN_L: float = 0.0            # k_c of the normal-traction kernel, same units; 0: kc_L
    kc_units: str = "rad"         # "rad": k_c in rad/m; "cycles": k_c in cycles/m
    quadrature: str = "midpoint"  # "midpoint" (Sec. 3.3) or "exact": the integral over each interval
    state_law: str = "analytic"   # "analytic" aging at constant Vbar, or "explicit"
    newton_tol: float = 1e-13
    newton_maxit: int = 200

    @property
    def L(self) -> float:
        return self.N * self.dx

    @property
    def r(self) -> float:
        return self.cs / self.cp

    @property
    def S(self) -> float:
        """Static mode-II stiffness factor mu (1 - c_s^2/c_p^2) (Sec. 2.3)."""
        return self.mu * (1.0 - self.r ** 2)

    @property
    def eta_rd(self) -> float:
        """Radiation damping coefficient mu / (2 c_s) (Sec. 2.3)."""
        return self.mu / (2.0 * self.cs)


def wavenumbers(p: Params) -> np.ndarray:
    """k_n = 2 pi n / L for n = 0..N/2 (rad/m)."""
    return 2.0 * np.pi * np.arange(p.N // 2 + 1) / p.L


def field_windows(p: Params):
    """Windows (M^T_n, M^N_n) of the shear and normal kernels (Sec. 3.1).

    M^X_n is the number of dt_min intervals covering the truncation window
    T_w(k_n): T_w = eta L / c_s for k <= k_c and (eta L / c_s)(k_c / k)
    above, M^X_n the ceiling of T_w / dt_min, taken with a relative slack of
    1e-12 so that an exact integer ratio is not pushed up by rounding.  Mode
    0 has no traction (|k| = 0) and gets M_0 = 0.  The shear kernel is cut at
    k_c = kc_L / (eta L); the normal kernel at kcN_L / (eta L) when kcN_L > 0,
    the two cutting planes Sec. 3.1 proposes for the slower-converging normal
    traction, else at the same k_c (the paper's single plane).

    eta_w = 0 selects the quasi-dynamic limit (Appendix, Quasi-dynamic BIEM):
    the past slip rate acts only through the radiation damping of
    Eq. (momentum), so every window is empty, and with it the history sums
    and the current-interval kernel term; the elastic response is the static
    stiffness alone.
    """
    if p.eta_w == 0:
        z = np.zeros(p.N // 2 + 1, dtype=np.int64)
        return z, z.copy()
    if p.kc_units not in ("rad", "cycles"):
        raise ValueError("kc_units must be 'rad' or 'cycles'")
    k = wavenumbers(p)
    Omega = p.L

    def one(kc_L):
        kc = kc_L / (p.eta_w * Omega)
        if p.kc_units == "cycles":
            kc = 2.0 * np.pi * kc
        Tw = np.where(k <= kc, p.eta_w * Omega / p.cs, 0.0)
        above = k > kc
        Tw[above] = (p.eta_w * Omega / p.cs) * (kc / k[above])
        M = np.ceil(Tw / p.dt_min * (1.0 - 1e-12)).astype(np.int64)
        M[0] = 0
        return M

    MT = one(p.kc_L)
    MN = one(p.kcN_L) if p.kcN_L > 0 else MT.copy()
    return MT, MN


def windows(p: Params) -> np.ndarray:
    """Lags kept per mode: M_n = max(M^T_n, M^N_n) (field_windows; one window with one plane)."""
    MT, MN = field_windows(p)
    return np.maximum(MT, MN)


_CHUNK = 1 << 20   # kernel points evaluated per call (bounds the quadrature's temporaries)


def _kernel_pair_chunk(args):
    s, r = args
    return kernel_pair(s, r)


def _kernel_pair_all(s: np.ndarray, r: float, workers: int = 1):
    """kernel_pair over s in chunks of _CHUNK points, optionally in worker processes.

    The kernels are evaluated point by point, so chunking and the worker
    count change only the schedule, never a value.  Workers are started with
    the 'spawn' method (safe beside an initialized CUDA context).
    """
    if s.size <= _CHUNK or workers <= 1:
        parts = [kernel_pair(s[i:i + _CHUNK], r) for i in range(0, max(s.size, 1), _CHUNK)]
    else:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        jobs = [(s[i:i + _CHUNK], r) for i in range(0, s.size, _CHUNK)]
        with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_kernel_pair_chunk, jobs))
    return np.concatenate([a for a, _ in parts]), np.concatenate([b for _, b in parts])


# Gauss-Legendre rule of the "exact" interval weights: 8 points integrate a
# kernel oscillating at most at c_p |k| (s/r, r = c_s/c_p) over an interval
# of at most pi/4 in s to rounding (error term (8!)^4/(17 (16!)^3) (h w/2)^16
# < 1e-25 relative).
_IV_X, _IV_W = np.polynomial.legendre.leggauss(8)


def weights(p: Params, M: np.ndarray | None = None, modes=None, workers: int = 1):
    """Kernel weights of the history and current-interval sums (Sec. 3.3).

    Midpoint rule (the paper's, default): w_{n,j} = dt_min C(k_n, (j + 1/2) dt_min).
    quadrature="exact": w_{n,j} = integral of C(k_n, tau) over
    [j dt_min, (j + 1) dt_min], by the Gauss-Legendre rule _IV_X/_IV_W on
    the interval in s = c_s |k| tau (d tau = dt_min ds / ds_n).
    j = 0..M_n-1.  Returns (wT, wN, offsets): flat arrays with mode n
    occupying [offsets[n], offsets[n+1]).  With two cutting planes a field's
    weights are zero past its own window M^X_n (the kernel truncated there).
    ``modes`` (optional) restricts the evaluation to those modes: the other
    modes then get empty ranges.  ``workers`` > 1 evaluates the kernels in
    that many processes.
    """
    if M is None:
        M = windows(p)
    M = np.asarray(M, dtype=np.int64)
    Mk = M
    if modes is not None:
        keep = np.zeros(M.size, dtype=bool)
        keep[np.asarray(modes, dtype=np.int64)] = True
        Mk = np.where(keep, M, 0)
    k = wavenumbers(p)
    offsets = np.zeros(Mk.size + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(Mk)
    mode = np.repeat(np.arange(Mk.size), Mk)
    j = np.arange(offsets[-1]) - offsets[mode]
    if p.quadrature == "midpoint":
        s = p.cs * k[mode] * (j + 0.5) * p.dt_min
        GT, GN = _kernel_pair_all(s, p.r, workers)
    elif p.quadrature == "exact":
        ds = p.cs * k[mode] * p.dt_min                    # interval width in s
        s = (p.cs * k[mode] * j * p.dt_min)[:, None] + ds[:, None] * 0.5 * (1.0 + _IV_X)[None, :]
        gT, gN = _kernel_pair_all(s.ravel(), p.r, workers)
        GT = 0.5 * (gT.reshape(s.shape) @ _IV_W)         # mean of C over the interval
        GN = 0.5 * (gN.reshape(s.shape) @ _IV_W)
    else:
        raise ValueError("quadrature must be 'midpoint' or 'exact'")
    wT, wN = p.dt_min * GT, p.dt_min * GN
    MT, MN = field_windows(p)
    if Mk.size == MT.size:
        wT = np.where(j < MT[mode], wT, 0.0)
        wN = np.where(j < MN[mode], wN, 0.0)
    return wT, wN, offsets


def mode_history_sum(wT, wN, HT, HN, m: int):
    """One mode's history sums A^X = sum_{j=m}^{M-1} w^X_j H^X[j-m] (Sec. 3.3 step (2)).

    wT, wN: the mode's M weights (lag order); HT, HN: its past spectra,
    newest first (at least M - m of them).  The sum runs over j ascending.
    """
    M = len(wT)
    if M <= m:
        return 0j, 0j
    j = np.arange(m, M)
    return np.sum(wT[j] * HT[j - m]), np.sum(wN[j] * HN[j - m])


def history_sums_sampled(p: Params, modes, HT, HN, m: int = 1, workers: int = 1):
    """The history sums of the listed modes alone, from their own histories.

    HT[i], HN[i]: the past spectra of modes[i], newest first.  The same
    windows, weights and sums as Oracle.history_sums, with the weights
    evaluated only for these modes (for faults too large to tabulate whole).
    """
    M = windows(p)
    wT, wN, woff = weights(p, M, modes=modes, workers=workers)
    AT = np.zeros(len(modes), dtype=np.complex128)
    AN = np.zeros(len(modes), dtype=np.complex128)
    for i, n in enumerate(modes):
        w = slice(woff[n], woff[n + 1])
        AT[i], AN[i] = mode_history_sum(wT[w], wN[w], np.asarray(HT[i]), np.asarray(HN[i]), m)
    return AT, AN


def state_update(theta0, Vbar, thetadot_bar, Dc, dt, law: str):
    """Predicted state theta_p over one step (Sec. 3.3 step (1)).

    analytic: aging law d theta/dt = 1 - theta V / Dc integrated exactly at
              constant V = Vbar (Lapusta et al. 2000);
    explicit: theta0 + thetadot_bar * dt, as printed in Sec. 3.3.
    """
    if law == "analytic":
        # theta0 e^{-u} + (Dc/Vbar)(1 - e^{-u}), u = Vbar dt / Dc, written as
        # theta0 e^{-u} + dt (1 - e^{-u})/u so that Vbar -> 0 gives theta0 + dt
        u = np.asarray(Vbar * dt / Dc, dtype=np.float64)
        phi = np.ones_like(u)
        nz = u > 0
        phi[nz] = -np.expm1(-u[nz]) / u[nz]
        return theta0 * np.exp(-u) + dt * phi
    if law == "explicit":
        return theta0 + thetadot_bar * dt
    raise ValueError("state law must be 'analytic' or 'explicit'")


def newton_lnV(tau, sigma, theta, a, b, Dc, f0, V0, eta, x_start, tol, maxit):
    """Solve Eq. (momentum) with radiation damping for x = ln V, per element.

    g(x) = tau - eta e^x - sigma [f0 + a (x - ln V0) + b ln(theta V0 / Dc)] = 0.
    For sigma > 0 and a > 0, g is strictly decreasing, so the root is unique.
    The quasi-static root x_qs (eta = 0) bounds it from above; a lower bound is
    found by stepping down until g >= 0.  Newton steps that leave the bracket
    are replaced by bisection.  Returns (x, iterations, converged mask).
    """
    psi_term = b * (np.log(theta) + np.log(V0 / Dc))
    lnV0 = np.log(V0)

    def g(x):
        return tau - eta * np.exp(x) - sigma * (f0 + a * (x - lnV0) + psi_term)

    hi = lnV0 + (tau / sigma - f0 - psi_term) / a
    hi = np.minimum(hi, 700.0)
    lo = hi - 1.0
    step = 1.0
    for _ in range(80):
        bad = g(lo) < 0
        if not bad.any():
            break
        step *= 2.0
        lo = np.where(bad, hi - step, lo)
    x = np.clip(x_start, lo, hi)
    conv = np.zeros(x.shape, dtype=bool)
    iters = np.zeros(x.shape, dtype=np.int64)
    for it in range(maxit):
        gx = g(x)
        lo = np.where(gx > 0, x, lo)
        hi = np.where(gx <= 0, x, hi)
        e = eta * np.exp(x)
        q = gx + e                      # tau - sigma F(x), linear in x
        # Newton on g where friction dominates; where radiation damping
        # dominates (q > sigma a, so that h' lies in (1, 2)) Newton on
        # h(x) = x - ln(q(x)/eta), which has the same root and is nearly
        # linear there.
        rad = q > sigma * a
        xg = x - gx / (-e - sigma * a)
        with np.errstate(divide="ignore", invalid="ignore"):
            xh = x - (x - np.log(np.where(rad, q, 1.0) / eta)) / (1.0 + sigma * a / np.where(rad, q, 1.0))
        xn = np.where(rad, xh, xg)
        # a step below the tolerance is accepted as converged, and a Newton
        # point within tol of the bracket is kept (roots next to the
        # quasi-static bound land there up to rounding)
        small = np.abs(xn - x) <= tol
        outside = ((xn < lo - tol) | (xn > hi + tol)) & ~small
        xn = np.where(outside, 0.5 * (lo + hi), xn)
        dx = np.abs(xn - x)
        iters = np.where(conv, iters, it + 1)
        x = np.where(conv, x, xn)
        conv = conv | (dx <= tol)
        if conv.all():
            break
    return x, iters, conv


@dataclass
class Oracle:
    """Fault state and history of the plain FP64 spectral BIEM (Sec. 3)."""
    p: Params
    kappa: np.ndarray
    a: np.ndarray
    b: np.ndarray
    Dc: np.ndarray
    f0: float
    V0: float
    sigma_load: np.ndarray
    tau_load: np.ndarray
    V: np.ndarray
    theta: np.ndarray
    tau_load_rate: np.ndarray | None = None
    prescribed: np.ndarray | None = None
    V_presc: np.ndarray | None = None
    delta: np.ndarray | None = None
    t: float = 0.0
    steps: int = 0
    thetadot: np.ndarray | None = field(default=None)
    workers: int = 1              # processes evaluating the weight tables (values do not depend on it)

    def __post_init__(self):
        p = self.p
        N = p.N
        if N % 2:
            raise ValueError("N must be even")
        f = lambda v, fill: (np.full(N, fill, dtype=np.float64) if v is None
                             else np.array(v, dtype=np.float64).reshape(N))
        self.kappa = f(self.kappa, 0.0)
        self.a, self.b, self.Dc = f(self.a, 0), f(self.b, 0), f(self.Dc, 1)
        self.sigma_load = f(self.sigma_load, 0)
        equilibrium = self.tau_load is None
        self.tau_load = f(self.tau_load, 0)
        self.tau_load_rate = f(self.tau_load_rate, 0.0)
        self.V, self.theta = f(self.V, 0), f(self.theta, 1)
        self.delta = f(self.delta, 0.0)
        self.prescribed = (np.zeros(N, dtype=bool) if self.prescribed is None
                           else np.asarray(self.prescribed, dtype=bool).reshape(N))
        self.V_presc = f(self.V_presc, 0.0)
        self.V = np.where(self.prescribed, self.V_presc, self.V)
        if self.thetadot is None:
            self.thetadot = 1.0 - self.theta * self.V / self.Dc
        if equilibrium:
            # loading in equilibrium with the initial state (Eq. momentum with
            # radiation damping and zero elastic change at t = 0)
            # (prescribed elements may hold V = 0; their load is set to 0 below)
            with np.errstate(divide="ignore"):
                fr = (self.f0 + self.a * np.log(self.V / self.V0)
                      + self.b * np.log(self.theta * self.V0 / self.Dc))
            self.tau_load = np.where(self.prescribed, 0.0,
                                     self.sigma_load * fr + p.eta_rd * self.V)
        self.k = wavenumbers(p)
        self.M = windows(p)
        self.wT, self.wN, self.woff = weights(p, self.M, workers=self.workers)
        # history: mode n keeps R_n = M_n - 1 past spectra; lag j (>= 1) of
        # mode n sits at ring slot (head_n + j - 1) mod R_n.
        self.R = np.maximum(self.M - 1, 0)
        self.hoff = np.zeros(self.R.size + 1, dtype=np.int64)
        self.hoff[1:] = np.cumsum(self.R)
        self.hist_T = np.zeros(self.hoff[-1], dtype=np.complex128)
        self.hist_N = np.zeros(self.hoff[-1], dtype=np.complex128)
        self.head = np.zeros(self.R.size, dtype=np.int64)
        self.last = {}

    # ------------------------------------------------------------------ history
    def history_slot(self, n: int, lag: int) -> int:
        """Flat index of lag ``lag`` (>= 1) of mode n."""
        return int(self.hoff[n] + (self.head[n] + lag - 1) % self.R[n])

    def set_history(self, HT: list, HN: list) -> None:
        """Load history: HT[n][i] is the spectrum of lag i+1 (newest first)."""
        for n in range(self.R.size):
            Rn = int(self.R[n])
            self.head[n] = 0
            self.hist_T[self.hoff[n]:self.hoff[n] + Rn] = np.asarray(HT[n], np.complex128)[:Rn]
            self.hist_N[self.hoff[n]:self.hoff[n] + Rn] = np.asarray(HN[n], np.complex128)[:Rn]

    def get_history(self):
        """History as lists of per-mode arrays, newest first."""
        HT, HN = [], []
        for n in range(self.R.size):
            Rn = int(self.R[n])
            idx = self.hoff[n] + (self.head[n] + np.arange(Rn)) % max(Rn, 1)
            HT.append(self.hist_T[idx].copy())
            HN.append(self.hist_N[idx].copy())
        return HT, HN

    def history_sums(self, m: int = 1):
        """A^X_n = sum_{j=m}^{M_n-1} w^X_{n,j} H^X_n[j-m]: the integral over [m dt_min, T_w].

        Sums run over j in ascending order, mode by mode.
        """
        nm = self.R.size
        AT = np.zeros(nm, dtype=np.complex128)
        AN = np.zeros(nm, dtype=np.complex128)
        for n in range(1, nm):
            Mn, Rn = int(self.M[n]), int(self.R[n])
            if Mn <= m:
                continue
            idx = self.hoff[n] + (self.head[n] + np.arange(Mn - m)) % Rn
            w = slice(self.woff[n], self.woff[n] + Mn)
            AT[n], AN[n] = mode_history_sum(self.wT[w], self.wN[w], self.hist_T[idx], self.hist_N[idx], m)
        return AT, AN

    def current_weights(self, m: int = 1):
        """Weight of the current interval [0, m dt_min]: sum of the first m weights."""
        nm = self.R.size
        w0T = np.zeros(nm)
        w0N = np.zeros(nm)
        for n in range(1, nm):
            Mn = int(self.M[n])
            j = np.arange(min(m, Mn))
            w0T[n] = np.sum(self.wT[self.woff[n] + j])
            w0N[n] = np.sum(self.wN[self.woff[n] + j])
        return w0T, w0N

    def push(self, UT: np.ndarray, UN: np.ndarray, m: int = 1) -> None:
        """Extend every ring by m copies of this step's spectra (Sec. 3.3, last paragraph)."""
        for n in range(1, self.R.size):
            Rn = int(self.R[n])
            if Rn == 0:
                continue
            for _ in range(min(m, Rn)):
                self.head[n] = (self.head[n] - 1) % Rn
                self.hist_T[self.hoff[n] + self.head[n]] = UT[n]
                self.hist_N[self.hoff[n] + self.head[n]] = UN[n]
            if m > Rn:
                # the ring now holds Rn copies; the head position is still
                # defined as m pushes from the start
                self.head[n] = (self.head[n] - (m - Rn)) % Rn

    # -------------------------------------------------------------- tractions
    def tractions(self, delta_p, Vbar, AT, AN, w0T, w0N):
        """Elastic shear and normal traction changes (Sec. 3.1 and Sec. 3.3 step (2))."""
        p = self.p
        kap = self.kappa
        U = np.fft.rfft(Vbar)              # F[Vbar]
        Q = np.fft.rfft(kap * Vbar)        # F[kappa Vbar]
        D = np.fft.rfft(delta_p)           # F[delta_p]
        K = np.fft.rfft(kap * delta_p)     # F[kappa delta_p]
        absk = self.k
        tau_hat = -p.S * absk * D - p.mu * absk * (AT + w0T * U)
        sgn = np.ones_like(absk)
        sgn[0] = 0.0
        sgn[-1] = 0.0                      # Nyquist: odd operator has no real representation
        sig_hat = -1j * sgn * (p.S * K + p.mu * (AN + w0N * Q))
        tau_el = np.fft.irfft(tau_hat, n=p.N)
        sig_el = np.fft.irfft(sig_hat, n=p.N)
        return tau_el, sig_el, U, Q

    # ---------------------------------------------------------------- the step
    def _pass(self, Vbar, thetadot_bar, dt, t_end, AT, AN, w0T, w0N):
        p = self.p
        delta_p = self.delta + Vbar * dt
        theta_p = state_update(self.theta, Vbar, thetadot_bar, self.Dc, dt, p.state_law)
        status = STATUS_OK
        if np.any(theta_p <= 0):
            status |= STATUS_STATE
        tau_el, sig_el, U, Q = self.tractions(delta_p, Vbar, AT, AN, w0T, w0N)
        tau = self.tau_load + self.tau_load_rate * t_end + tau_el
        sigma = self.sigma_load + sig_el
        free = ~self.prescribed
        if np.any(sigma[free] <= 0):
            status |= STATUS_OPENING
        Vnew = self.V_presc.copy()
        iters = np.zeros(p.N, dtype=np.int64)
        if free.any() and not (status & (STATUS_OPENING | STATUS_STATE)):
            x, it, conv = newton_lnV(tau[free], sigma[free], theta_p[free], self.a[free],
                                     self.b[free], self.Dc[free], self.f0, self.V0, p.eta_rd,
                                     np.log(self.V[free]), p.newton_tol, p.newton_maxit)
            if not conv.all():
                status |= STATUS_NEWTON
            Vnew[free] = np.exp(x)
            iters[free] = it
        thetadot_new = 1.0 - theta_p * Vnew / self.Dc
        return dict(V=Vnew, theta=theta_p, thetadot=thetadot_new, delta=delta_p,
                    tau_el=tau_el, sig_el=sig_el, U=U, Q=Q, status=status, iters=iters)

    def step(self, m: int = 1) -> int:
        """Advance by dt = m * dt_min; returns a status bitmask (0 on success).

        On failure the state is left unchanged.
        """
        if m < 1:
            raise ValueError("m >= 1")
        dt = m * self.p.dt_min
        t_end = self.t + dt
        AT, AN = self.history_sums(m)
        w0T, w0N = self.current_weights(m)
        r1 = self._pass(self.V, self.thetadot, dt, t_end, AT, AN, w0T, w0N)
        if r1["status"]:
            self.last = r1
            return r1["status"]
        Vbar = 0.5 * (self.V + r1["V"])
        thd_bar = 0.5 * (self.thetadot + r1["thetadot"])
        r2 = self._pass(Vbar, thd_bar, dt, t_end, AT, AN, w0T, w0N)
        if r2["status"]:
            self.last = r2
            return r2["status"]
        self.delta = r2["delta"]
        self.V = r2["V"]
        self.theta = r2["theta"]
        self.thetadot = r2["thetadot"]
        self.push(r2["U"], r2["Q"], m)
        self.t = t_end
        self.steps += 1
        r2["pass1"] = r1
        self.last = r2
        return STATUS_OK


# ---------------------------------------------------------------- adaptive dt
def _snapshot(o: Oracle) -> dict:
    keys = ("delta", "V", "theta", "thetadot", "hist_T", "hist_N", "head")
    snap = {k: getattr(o, k).copy() for k in keys}
    snap["t"], snap["steps"] = o.t, o.steps
    return snap


def _restore(o: Oracle, snap: dict) -> None:
    for k, v in snap.items():
        setattr(o, k, v.copy() if isinstance(v, np.ndarray) else v)


def adaptive_run(o: Oracle, t_end: float, eps0: float, m0: int = 1, m_max: int = 1 << 40,
                 max_steps: int = 10 ** 9):
    """Step-doubling time integration (Sec. 3.2) with dt = m dt_min, m a power of two.

    A trial from state S advances once by dt and twice by dt/2; the error is
    eps = max_i |delta_full - delta_halves| (slip, Sec. 3.2 with u read as the
    slip).  eps <= eps0: the two-half-step state is kept and the next m is the
    largest power of two <= 0.9 (eps0/eps)^(1/3) m, at most doubling.  eps >
    eps0 or any failure (Newton, opening, state): S is restored and m is the
    largest power of two <= min(m/2, 0.9 (eps0/eps)^(1/3) m).  At m = 1
    (dt_min) a single step is taken and its error is ignored; a failure there
    stops the run (status returned with the DTMIN flag 8).

    Returns (status, list of accepted m).
    """
    m = max(1, int(m0))
    accepted = []
    while o.t < t_end * (1 - 1e-15) and len(accepted) < max_steps:
        if m == 1:
            st = o.step(1)
            if st:
                return st | 8, accepted
            accepted.append(1)
            m = 2
            continue
        snap = _snapshot(o)
        st = o.step(m)
        if st:
            _restore(o, snap)
            m //= 2
            continue
        delta_full = o.delta.copy()
        _restore(o, snap)
        st = o.step(m // 2)
        if not st:
            st = o.step(m // 2)
        if st:
            _restore(o, snap)
            m //= 2
            continue
        eps = float(np.abs(o.delta - delta_full).max())
        factor = 0.9 * (eps0 / eps) ** (1.0 / 3.0) if eps > 0 else np.inf
        if eps > eps0:
            _restore(o, snap)
            m_new = m // 2
            while m_new > 1 and m_new > factor * m:
                m_new //= 2
            m = max(1, m_new)
            continue
        accepted.append(m)
        m_new = m
        while m_new * 2 <= factor * m and m_new < 2 * m:
            m_new *= 2
        while m_new > 1 and m_new > factor * m:
            m_new //= 2
        m = max(1, min(m_new, m_max))
    return 0, accepted
