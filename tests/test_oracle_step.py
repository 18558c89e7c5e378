"""Pins for the oracle's time step (Sec. 3), each against an independent fact.

* static stiffness vs the textbook mu/(2(1-nu)) and Table 1's nucleation lengths;
* uniform slip rate: no elastic shear change (only k = 0 is excited);
* flat fault: the normal traction change vanishes bitwise;
* a single Fourier mode of prescribed slip rate: closed form of the
  static + truncated dynamic response, which fixes the lag/weight indexing;
  in the quasi-dynamic limit (eta_w = 0) the static response alone; with
  two cutting planes (Sec. 3.1) each field truncated at its own window;
* the normal cutting plane: shear unchanged bitwise, normal traction
  converging monotonically to the long-window result;
* truncation: a slip pulse is forgotten after the window;
* tiny N: a brute-force space-time double sum with real-space kernels equals
  the spectral step (FFT plumbing, sgn(k), Nyquist);
* Newton vs plain bisection on the same residual;
* aging law: steady state is a fixed point; explicit and exact updates agree
  to second order;
* the sign of the normal traction: the slip/curvature scaling law of Sec. 5.
"""
import numpy as np
import pytest

from oracle import Oracle, Params, newton_lnV, state_update
from oracle.kernels import G_N, G_T
from oracle.sbiem import windows
from paper_2107_03550_gb300.workloads import element_x, rough_fault, seamount_rupture
from tests.golden.paper import paper_numbers


def _params(N=64, dx=25.0, kc_L=200.0, mu=30e9, cs=3464.0, cp=None, eta_w=1.0):
    cp = cp or np.sqrt(3.0) * cs
    return Params(N=N, dx=dx, mu=mu, cs=cs, cp=cp, dt_min=0.25 * dx / cs, kc_L=kc_L, eta_w=eta_w)


def _prescribed_oracle(p, kappa, V):
    N = p.N
    return Oracle(p, kappa, np.full(N, 0.01), np.full(N, 0.015), np.full(N, 1e-3), 0.6, 1e-6,
                  np.full(N, 50e6), np.zeros(N), V.copy(), np.full(N, 1.0),
                  prescribed=np.ones(N, dtype=bool), V_presc=V.copy())


def test_static_stiffness_and_table1_lengths():
    pn = paper_numbers()
    mu, cs, cp = pn["table1_mu"], pn["table1_cs"], pn["table1_cp"]
    p = Params(N=8, dx=pn["table1_ds"], mu=mu, cs=cs, cp=cp, dt_min=1.0)
    nu = (cp ** 2 - 2 * cs ** 2) / (2 * (cp ** 2 - cs ** 2))
    assert p.S == pytest.approx(mu / (2 * (1 - nu)), rel=1e-14)
    # Table 1: with mu' = mu/(1-nu) = 2 S the printed nucleation lengths follow.
    mup = 2 * p.S
    a, b, Dc, sig = pn["table1_a"], pn["table1_b"], pn["table1_Dc"], pn["table1_sigma_n"]
    assert mup * Dc / (b * sig) == pytest.approx(pn["table1_L_b"], rel=2e-3)
    assert 2 * mup * b * Dc / (np.pi * sig * (b - a) ** 2) == pytest.approx(pn["table1_L_inf"], rel=1e-3)


# pi to 40 digits as an exact rational: the window counts below are ceilings
# of irrational numbers, so 40 digits decide every one of them exactly
_PI = __import__("fractions").Fraction("3.141592653589793238462643383279502884197")


def _exact_windows(N: int, kc_L, beta=__import__("fractions").Fraction(1, 4), cycles=False):
    """M_n of Sec. 3.1 in exact arithmetic, written from the window's definition.

    dt_min = beta dx / c_s and the full window eta L / c_s (eta = 1) give
    T_w / dt_min = N / beta below the cutting plane.  Above it the window
    shrinks by k_c / k_n with k_n = 2 pi n / L and k_c = kc_L / L rad/m
    (kc_L / L cycles/m, i.e. 2 pi kc_L / L rad/m, with cycles=True), so
    T_w / dt_min = (N / beta) kc_L / (2 pi n)  (rad)  or  (N / beta) kc_L / n
    (cycles).  The window is continuous at k = k_c, so either side of the
    plane gives the same count there.  M_0 = 0.
    """
    from fractions import Fraction
    import math
    full = Fraction(N) / beta
    out = [0]
    for n in range(1, N // 2 + 1):
        ratio = Fraction(kc_L) / (n if cycles else 2 * _PI * n)
        out.append(math.ceil(full * min(Fraction(1), ratio)))
    return np.array(out, dtype=np.int64)


def test_windows_exact_counts():
    # The seamount rupture (N = 256, dx = 25 m, k_c L = 200 rad): 31 modes
    # below the plane (n_c = 100/pi = 31.83) keep the full 4N = 1024 lags,
    # mode 32 keeps ceil(102400/(32 pi)) = 1019, mode 33 988, the Nyquist
    # mode 255; in all 77,616 lags per field.
    p = _params(N=256, dx=25.0)
    M = windows(p)
    ref = _exact_windows(256, 200)
    assert np.array_equal(M, ref)
    assert M[31] == 1024 and M[32] == 1019 and M[33] == 988 and M[128] == 255
    assert int(M.sum()) == 77616
    # The rough-fault cycle (N = 4096, dx = 10 m): 2,684,079 ring slots
    # (M_n - 1 per mode with history)
    p = _params(N=4096, dx=10.0)
    M = windows(p)
    assert np.array_equal(M, _exact_windows(4096, 200))
    assert int(np.maximum(M - 1, 0).sum()) == 2684079
    # cycles/m with an exact integer ratio above the plane: n = 16 of N = 64
    # at k_c L = 10 cycles has T_w / dt_min = 256 * 10 / 16 = 160 exactly,
    # which the ceiling must not push to 161; n = 10 sits on the plane
    p = Params(N=64, dx=25.0, mu=30e9, cs=3464.0, cp=np.sqrt(3.0) * 3464.0, dt_min=0.25 * 25.0 / 3464.0,
               kc_L=10.0, kc_units="cycles")
    M = windows(p)
    assert np.array_equal(M, _exact_windows(64, 10, cycles=True))
    assert M[16] == 160 and M[10] == 256 and M[11] == 233
    # two planes: each field's window from its own k_c
    p = Params(N=256, dx=25.0, mu=30e9, cs=3464.0, cp=np.sqrt(3.0) * 3464.0, dt_min=0.25 * 25.0 / 3464.0,
               kc_L=100.0, kcN_L=300.0)
    from oracle.sbiem import field_windows
    MT, MN = field_windows(p)
    assert np.array_equal(MT, _exact_windows(256, 100))
    assert np.array_equal(MN, _exact_windows(256, 300))
    assert np.array_equal(windows(p), np.maximum(MT, MN))


def test_uniform_slip_rate_gives_no_elastic_shear_change():
    w = rough_fault(128, 25.0, 3e-3, seed=2, lam_min=100.0)
    p = _params(N=128, dx=25.0)
    V = np.full(p.N, 2e-3)
    o = Oracle(p, w.kappa, w.a, w.b, w.Dc, w.f0, w.V0, w.sigma_load, None, V, np.full(p.N, 0.5))
    assert o.step() == 0
    r1 = o.last["pass1"]
    assert np.abs(r1["tau_el"]).max() < 1e-18 * p.S
    # with tau_el = 0 the pass-1 Newton balances tau_load - eta V against friction alone
    assert np.abs(r1["sig_el"]).max() > 0.0   # curvature still loads the normal traction


def test_flat_fault_has_zero_normal_traction_change():
    w = seamount_rupture(N=128, dx=25.0)
    p = _params(N=128, dx=25.0)
    o = Oracle(p, np.zeros(p.N), w.a, w.b, w.Dc, w.f0, w.V0, w.sigma_load, None,
               w.V_init, w.theta_init)
    for _ in range(5):
        assert o.step() == 0
        assert not np.any(o.last["sig_el"])
        assert not np.any(o.last["pass1"]["sig_el"])


@pytest.mark.parametrize("steps", [1, 7, 60])
def test_single_mode_closed_form(steps):
    # Prescribed V = Va cos(q x) from t = 0 on a fault of constant curvature k0.
    # Shear: -|k| acts on cos as -q cos; normal: -i sgn(k) acts on cos as sin.
    # After s steps of dt = dt_min (V constant so Vbar = V every pass):
    #   tau = -q cos(qx) Va [S s dt + mu sum_{j < min(s, M)} wT_j]
    #   sig = sin(qx) k0 Va [S s dt + mu sum_{j < min(s, M)} wN_j]
    p = _params(N=64, kc_L=20.0)
    m = 16
    q = 2 * np.pi * m / p.L
    x = element_x(p.N, p.dx)
    Va, k0 = 1e-3, 3e-4
    V = Va * np.cos(q * x)
    o = _prescribed_oracle(p, np.full(p.N, k0), V)
    M = windows(p)[m]
    assert 10 < M < 60
    for _ in range(steps):
        assert o.step() == 0
    dt = p.dt_min
    j = np.arange(min(steps, M))
    sT = dt * G_T(p.cs * q * (j + 0.5) * dt, p.r).sum()
    sN = dt * G_N(p.cs * q * (j + 0.5) * dt, p.r).sum()
    tau = -q * np.cos(q * x) * Va * (p.S * steps * dt + p.mu * sT)
    sig = np.sin(q * x) * k0 * Va * (p.S * steps * dt + p.mu * sN)
    scale = q * Va * p.S * steps * dt
    assert np.abs(o.last["tau_el"] - tau).max() < 1e-12 * scale
    assert np.abs(o.last["sig_el"] - sig).max() < 1e-12 * scale


@pytest.mark.parametrize("steps", [1, 7])
def test_quasi_dynamic_single_mode_closed_form(steps):
    # eta_w = 0 (Appendix, Quasi-dynamic BIEM): no window, so no history and no
    # current-interval kernel term; prescribed V = Va cos(q x) on a fault of
    # constant curvature k0 gives after s steps the static responses alone:
    #   tau = -q cos(qx) Va S s dt,  sig = sin(qx) k0 Va S s dt
    p = _params(N=64, eta_w=0.0)
    assert not windows(p).any()
    m = 16
    q = 2 * np.pi * m / p.L
    x = element_x(p.N, p.dx)
    Va, k0 = 1e-3, 3e-4
    V = Va * np.cos(q * x)
    o = _prescribed_oracle(p, np.full(p.N, k0), V)
    for _ in range(steps):
        assert o.step() == 0
    dt = p.dt_min
    tau = -q * np.cos(q * x) * Va * p.S * steps * dt
    sig = np.sin(q * x) * k0 * Va * p.S * steps * dt
    scale = q * Va * p.S * steps * dt
    assert np.abs(o.last["tau_el"] - tau).max() < 1e-12 * scale
    assert np.abs(o.last["sig_el"] - sig).max() < 1e-12 * scale


def test_two_cutting_planes_single_mode_closed_form():
    # Sec. 3.1's two cutting planes: the shear kernel cut at k_c, the normal
    # kernel at kcN.  Prescribed V = Va cos(q x), constant curvature k0; after
    # s steps with M^T <= s <= M^N each field's dynamic term is its own
    # truncated sum:
    #   tau = -q cos(qx) Va [S s dt + mu sum_{j < M^T} wT_j]
    #   sig = sin(qx) k0 Va [S s dt + mu sum_{j < s} wN_j]
    from oracle.sbiem import field_windows
    p = _params(N=64, kc_L=20.0)
    p.kcN_L = 40.0
    m = 16
    MT, MN = field_windows(p)
    assert MT[m] + 5 < MN[m]
    q = 2 * np.pi * m / p.L
    x = element_x(p.N, p.dx)
    Va, k0 = 1e-3, 3e-4
    V = Va * np.cos(q * x)
    o = _prescribed_oracle(p, np.full(p.N, k0), V)
    steps = (MT[m] + MN[m]) // 2
    for _ in range(steps):
        assert o.step() == 0
    dt = p.dt_min
    sT = dt * G_T(p.cs * q * (np.arange(MT[m]) + 0.5) * dt, p.r).sum()
    sN = dt * G_N(p.cs * q * (np.arange(steps) + 0.5) * dt, p.r).sum()
    tau = -q * np.cos(q * x) * Va * (p.S * steps * dt + p.mu * sT)
    sig = np.sin(q * x) * k0 * Va * (p.S * steps * dt + p.mu * sN)
    scale = q * Va * p.S * steps * dt
    assert np.abs(o.last["tau_el"] - tau).max() < 1e-12 * scale
    assert np.abs(o.last["sig_el"] - sig).max() < 1e-12 * scale


def test_quasi_dynamic_limit_empties_both_planes():
    from oracle.sbiem import field_windows
    p = _params(N=64, eta_w=0.0)
    p.kcN_L = 400.0
    MT, MN = field_windows(p)
    assert not MT.any() and not MN.any() and not windows(p).any()


def test_normal_cutting_plane_convergence():
    # Truncation study (Sec. 3.1): with the shear plane fixed, raising the
    # normal plane leaves the shear traction bitwise unchanged and brings
    # the normal traction monotonically to the long-window result; at equal
    # planes the normal error exceeds the shear error (the slower-converging
    # normal kernel the paper gives as the reason for a second plane).
    def run(kc, kcN, steps=600):
        p = _params(N=64, kc_L=kc)
        p.kcN_L = kcN
        x = element_x(p.N, p.dx)
        rng = np.random.default_rng(3)
        V = 1e-3 * (1 + 0.5 * sum(np.cos(2 * np.pi * m * x / p.L + rng.uniform(0, 2 * np.pi))
                                  for m in (3, 7, 12, 21)))
        o = _prescribed_oracle(p, 1e-4 * np.cos(2 * np.pi * 5 * x / p.L), V)
        for _ in range(steps):
            assert o.step() == 0
        return o.last["tau_el"], o.last["sig_el"]

    tau_ref, sig_ref = run(1e4, 1e4)
    err = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    taus, sig_err = [], []
    for kcN in (10.0, 20.0, 40.0, 80.0, 160.0):
        t, sg = run(10.0, kcN)
        taus.append(t)
        sig_err.append(err(sg, sig_ref))
    assert all(np.array_equal(t, taus[0]) for t in taus)
    assert all(b < a for a, b in zip(sig_err, sig_err[1:])), sig_err
    assert sig_err[-1] < 0.02 * sig_err[0]
    assert sig_err[0] > 3 * err(taus[0], tau_ref)


def test_truncation_forgets_a_pulse():
    p = _params(N=32, kc_L=20.0)
    rng = np.random.default_rng(0)
    kappa = 1e-4 * rng.standard_normal(p.N)
    o = _prescribed_oracle(p, kappa, np.zeros(p.N))
    for V in (rng.standard_normal(p.N) * 1e-2, rng.standard_normal(p.N) * 1e-2, np.zeros(p.N)):
        o.V_presc = V
        assert o.step() == 0
    Mmax = int(windows(p).max())
    for _ in range(Mmax + 1):
        assert o.step() == 0
    k = 2 * np.pi * np.arange(p.N // 2 + 1) / p.L
    tau_static = np.fft.irfft(-p.S * k * np.fft.rfft(o.delta), n=p.N)
    assert np.allclose(o.last["tau_el"], tau_static, rtol=0, atol=1e-12 * np.abs(tau_static).max())


def _real_space_kernels(p, wT, wN, woff, M):
    """Even (shear) and odd (normal) real-space kernels by explicit sums over all N modes."""
    N = p.N
    k = 2 * np.pi * np.arange(N // 2 + 1) / p.L
    Jmax = int(M.max())
    d = np.arange(N)
    KsT = np.zeros(N)
    KsN = np.zeros(N)
    KT = np.zeros((Jmax, N))
    KN = np.zeros((Jmax, N))
    for n in range(N):
        nn = min(n, N - n)
        ph = 2 * np.pi * n * d / N
        # even operator c(|n|): c cos(2 pi n d / N) / N from every n
        KsT += -p.S * k[nn] * np.cos(ph) / N
        # odd operator -i sgn(k) c: the pair (n, N-n) adds 2 c sin(2 pi nn d / N) / N,
        # one half from each member; n = 0 and n = N/2 add nothing
        odd = (0 < n < N // 2) or (n > N // 2)
        sin_nn = np.sin(2 * np.pi * nn * d / N)
        if odd:
            KsN += p.S * sin_nn / N
        for j in range(int(M[nn])):
            KT[j] += -p.mu * k[nn] * wT[woff[nn] + j] * np.cos(ph) / N
            if odd:
                KN[j] += p.mu * wN[woff[nn] + j] * sin_nn / N
    return KsT, KsN, KT, KN


@pytest.mark.parametrize("N", [8, 16, 32])
def test_tiny_N_space_time_double_sum_equals_spectral(N):
    p = _params(N=N, kc_L=20.0)
    rng = np.random.default_rng(N)
    kappa = 1e-4 * rng.standard_normal(N)
    o = _prescribed_oracle(p, kappa, np.zeros(N))
    Vbars = []                       # real-space pass-2 Vbar per step, oldest first
    Vold = np.zeros(N)
    for s in range(int(o.M.max()) + 5):
        Vn = 1e-2 * rng.standard_normal(N)
        o.V_presc = Vn
        assert o.step() == 0
        Vbars.append(0.5 * (Vold + Vn))
        Vold = Vn
    KsT, KsN, KT, KN = _real_space_kernels(p, o.wT, o.wN, o.woff, o.M)
    delta = o.delta
    tau = np.zeros(N)
    sig = np.zeros(N)
    for i in range(N):
        for l in range(N):
            dd = (i - l) % N
            tau[i] += KsT[dd] * delta[l]
            sig[i] += KsN[dd] * kappa[l] * delta[l]
            for j in range(KT.shape[0]):
                if j < len(Vbars):
                    Vl = Vbars[-1 - j][l]
                    tau[i] += KT[j, dd] * Vl
                    sig[i] += KN[j, dd] * kappa[l] * Vl
    st = np.abs(tau).max()
    assert np.abs(o.last["tau_el"] - tau).max() < 1e-12 * st
    assert np.abs(o.last["sig_el"] - sig).max() < 1e-12 * max(np.abs(sig).max(), 1e-30)


def _bisect(tau, sig, theta, a, b, Dc, f0, V0, eta):
    g = lambda x: tau - eta * np.exp(x) - sig * (f0 + a * (x - np.log(V0)) + b * np.log(theta * V0 / Dc))
    lo, hi = -400.0, 50.0
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_newton_matches_bisection():
    rng = np.random.default_rng(3)
    n = 200
    sig = rng.uniform(1e6, 1e8, n)
    a = rng.uniform(0.005, 0.03, n)
    b = rng.uniform(0.005, 0.03, n)
    Dc = rng.uniform(1e-4, 1e-1, n)
    theta = np.exp(rng.uniform(-5, 25, n))
    f = rng.uniform(0.3, 0.9, n)
    eta = 4.33e6
    tau = sig * f
    # a quarter of the cases sit far below steady sliding (V ~ 1e-30 m/s): the
    # root then lies next to the quasi-static bound
    tau[: n // 4] = sig[: n // 4] * rng.uniform(0.0, 0.05, n // 4)
    x, it, conv = newton_lnV(tau, sig, theta, a, b, Dc, 0.6, 1e-6, eta,
                             np.log(1e-9) * np.ones(n), 1e-13, 200)
    assert conv.all()
    ref = np.array([_bisect(tau[i], sig[i], theta[i], a[i], b[i], Dc[i], 0.6, 1e-6, eta) for i in range(n)])
    assert np.abs(x - ref).max() < 1e-11
    assert it.max() <= 12


def test_aging_law_fixed_point_and_explicit_agreement():
    V = np.array([1e-9, 1e-3, 1.0])
    Dc = np.full(3, 1e-3)
    th_ss = Dc / V
    out = state_update(th_ss, V, np.zeros(3), Dc, 0.3, "analytic")
    assert np.allclose(out, th_ss, rtol=1e-14)
    # small V dt / Dc: explicit trapezoid-free Euler and exact agree to O((V dt/Dc)^2)
    th0 = np.full(3, 7.0)
    for dt in (1e-4, 1e-5):
        u = V * dt / Dc
        ex = state_update(th0, V, 1 - th0 * V / Dc, Dc, dt, "explicit")
        an = state_update(th0, V, None, Dc, dt, "analytic")
        assert np.all(np.abs(ex - an) <= 2 * (u ** 2) * np.maximum(th0, Dc / V) + 1e-15)


@pytest.mark.slow
def test_normal_traction_sign_follows_scaling_law():
    # Sec. 5: (1/(f delta)) d delta/dx = -kappa.  A rough-fault rupture must
    # show a positive correlation of the two sides, and a regression slope near 1.
    w = rough_fault(256, 25.0, 3e-3, seed=5, lam_min=200.0)
    p = _params(N=256, dx=25.0)
    o = Oracle(p, w.kappa, w.a, w.b, w.Dc, w.f0, w.V0, w.sigma_load, None, w.V_init, w.theta_init)
    for _ in range(2000):
        assert o.step() == 0
    d = o.delta
    lhs = np.gradient(d, p.dx) / (0.6 * d)
    rhs = -w.kappa
    assert d.min() > 0.3 * d.max()
    c = np.corrcoef(lhs, rhs)[0, 1]
    slope = np.polyfit(rhs, lhs, 1)[0]
    assert c > 0.4
    assert 0.5 < slope < 1.5


@pytest.mark.slow
def test_seamount_rupture_nucleates_and_crosses():
    w = seamount_rupture()
    p = Params(N=w.N, dx=w.dx, mu=w.mu, cs=w.cs, cp=w.cp, dt_min=w.dt_min)
    o = Oracle(p, w.kappa, w.a, w.b, w.Dc, w.f0, w.V0, w.sigma_load, None, w.V_init, w.theta_init)
    x = element_x(w.N, w.dx)
    crossed = False
    vmax = 0.0
    for _ in range(1300):
        assert o.step() == 0
        vmax = max(vmax, o.V.max())
        crossed = crossed or (o.V[np.argmin(np.abs(x - 1000.0))] > 1e-1)
    assert vmax > 0.1
    assert crossed


def test_weight_evaluation_schedule_changes_no_value():
    # restricting the weights to some modes, chunking them and evaluating them
    # in worker processes only reschedules a pointwise evaluation: the values
    # are bitwise those of the full table, and the sampled history sums those
    # of Oracle.history_sums
    import oracle.sbiem as osb
    from oracle.sbiem import history_sums_sampled, weights
    from paper_2107_03550_gb300.workloads import random_history
    p = _params(N=256, dx=25.0)
    wT, wN, off = weights(p)
    modes = [1, 31, 32, 100, 128]
    sT, sN, soff = weights(p, modes=modes)
    for n in modes:
        assert np.array_equal(sT[soff[n]:soff[n + 1]], wT[off[n]:off[n + 1]])
        assert np.array_equal(sN[soff[n]:soff[n + 1]], wN[off[n]:off[n + 1]])
    assert soff[-1] == sum(off[n + 1] - off[n] for n in modes)
    old = osb._CHUNK
    try:
        osb._CHUNK = 4096
        cT, cN, _ = weights(p, workers=2)
    finally:
        osb._CHUNK = old
    assert np.array_equal(cT, wT) and np.array_equal(cN, wN)
    w = seamount_rupture(N=256)
    o = Oracle(p, w.kappa, w.a, w.b, w.Dc, w.f0, w.V0, w.sigma_load, None, w.V_init, w.theta_init)
    R = np.maximum(o.M - 1, 0)
    HT, HN, hoff = random_history(R, 3, 1e-3)
    o.set_history([HT[hoff[n]:hoff[n + 1]] for n in range(R.size)], [HN[hoff[n]:hoff[n + 1]] for n in range(R.size)])
    for m in (1, 3):
        AT, AN = o.history_sums(m)
        sAT, sAN = history_sums_sampled(p, modes, [HT[hoff[n]:hoff[n + 1]] for n in modes],
                                        [HN[hoff[n]:hoff[n + 1]] for n in modes], m)
        assert np.array_equal(sAT, AT[modes]) and np.array_equal(sAN, AN[modes])


def _primitives(s, r):
    """Antiderivatives P_T, P_N of the kernels in s (P(0) = 0), written here in
    closed form from int W = x W - J0, int x^2 W = x^3 W / 3 + x^2 J2 / 3,
    int J1 = -J0, int x J0 = x J1 (W' = -J1/x), term by term over the
    kernels of Eq. Ct and Sec. 2.4; the P-wave terms in x = s/r."""
    from scipy import special
    from oracle.kernels import W
    s = np.asarray(s, dtype=np.float64)
    x = s / r
    J0s, J1s, J0x, J1x = special.j0(s), special.j1(s), special.j0(x), special.j1(x)
    J2s, J2x = special.jv(2, s), special.jv(2, x)
    Ws, Wx = W(s), W(x)
    r2, r3 = r * r, r ** 3
    A = (1.0 / r2 - 2.0) ** 2 * r2 / 2.0
    x2W = lambda z, Wz, J2z: z ** 3 * Wz / 3.0 + z * z * J2z / 3.0   # int z^2 W dz
    xW = lambda z, Wz, J0z: z * Wz - J0z                               # int W dz
    FT = (r3 * x2W(x, Wx, J2x) + r3 * xW(x, Wx, J0x) - x2W(s, Ws, J2s) - xW(s, Ws, J0s)
          + r3 * J0x - 0.5 * J0s - r3 * x * J1x + s * J1s)
    FN = ((A - r2) * r * xW(x, Wx, J0x) - r3 * x2W(x, Wx, J2x) + (1.0 - 1.0 / (2.0 * r2)) * xW(s, Ws, J0s)
          + x2W(s, Ws, J2s) - (r2 - A) * r * J0x - (1.0 / (2.0 * r2) - 1.0) * J0s + r3 * x * J1x - s * J1s)
    return FT - 0.5, FN


def test_exact_interval_weights():
    # quadrature="exact": each weight is the integral of C over its interval.
    # (i) the closed-form primitives are antiderivatives of the kernels and
    #     vanish at 0; (ii) the running sums of the exact weights equal the
    #     primitive at the interval ends (a mode whose window ends at s = 31);
    # (iii) exact minus midpoint is dt ds^2 C''(s_mid)/24 to leading order:
    #     the O(dt^2) difference of the two rules.
    from oracle.sbiem import weights
    r = 1.0 / np.sqrt(3.0)
    PT0, PN0 = _primitives(np.array([0.0]), r)
    assert abs(PT0[0]) < 1e-15 and abs(PN0[0]) < 1e-15
    for s0 in (0.3, 2.7, 11.0, 25.0):
        h = 1e-4
        pT, pN = _primitives(np.array([s0 - h, s0 + h]), r)
        assert abs((pT[1] - pT[0]) / (2 * h) - G_T(s0, r)) < 1e-7
        assert abs((pN[1] - pN[0]) / (2 * h) - G_N(s0, r)) < 1e-7
    p = _params(N=64, dx=25.0)
    pe = Params(**{**p.__dict__, "quadrature": "exact"})
    wT, wN, off = weights(pe)
    mT, mN, _ = weights(p)
    n = 5                                   # 2 pi n = 31.4: window ends at s = 31.4
    k = 2 * np.pi * n / p.L
    ds = p.cs * k * p.dt_min
    M = off[n + 1] - off[n]
    PT, PN = _primitives(ds * np.arange(M + 1), r)
    cT = np.cumsum(wT[off[n]:off[n + 1]])
    cN = np.cumsum(wN[off[n]:off[n + 1]])
    scale = p.dt_min / ds                   # d tau = dt_min ds / ds_n
    assert np.abs(cT - scale * PT[1:]).max() < 1e-10 * np.abs(scale * PT).max()
    assert np.abs(cN - scale * PN[1:]).max() < 1e-10 * np.abs(scale * PN).max()
    j = np.arange(M)
    sm = ds * (j + 0.5)
    h = 1e-3
    d2T = (G_T(sm + h, r) - 2 * G_T(sm, r) + G_T(sm - h, r)) / h ** 2
    lead = p.dt_min * ds ** 2 * d2T / 24.0
    diff = wT[off[n]:off[n + 1]] - mT[off[n]:off[n + 1]]
    assert np.abs(diff - lead).max() < 1e-2 * np.abs(lead).max()
    assert np.abs(diff).max() > 0
