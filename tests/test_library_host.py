"""CPU tests of the C-ABI library: it loads, exports every declared symbol,
rejects bad arguments on the host, and its own FP64 kernel route agrees with
the oracle's.  No GPU compute is issued here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_03550_gb300 import sbiem
    try:
        return sbiem.load_library()
    except ImportError:
        import __graft_entry__
        __graft_entry__.build()
        return sbiem.load_library()


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(sbiem_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "sbiem_create" in names and "sbiem_step" in names and "sbiem_destroy" in names
    for name in names:
        assert hasattr(lib, name), name


def test_header_and_binding_agree():
    from paper_2107_03550_gb300 import sbiem
    declared = set(_declared_functions())
    bound = set(sbiem._SIGS)
    assert bound <= declared
    missing = declared - bound
    assert not missing, f"binding lacks {missing}"


def test_kernel_route_matches_oracle(lib):
    from oracle.kernels import G_N, G_T
    from paper_2107_03550_gb300.sbiem import kernel_values
    for r in (1 / np.sqrt(3.0), 3464.0 / 6000.0):
        s = np.concatenate([np.linspace(0.0, 5.0, 501), np.linspace(5.0, 60.0, 1101),
                            np.linspace(60.0, 210.0, 3001)])
        cT, cN = kernel_values(s, r)
        # the oracle's W = 1 - int_0^x carries a few ulps of 1, times s^2 in the kernels
        tol = 1e-13 + 6e-16 * s * s
        assert np.all(np.abs(cT - G_T(s, r)) <= tol)
        assert np.all(np.abs(cN - G_N(s, r)) <= tol)


def test_kernel_values_rejects_bad_input(lib):
    from paper_2107_03550_gb300.sbiem import SbiemError, kernel_values
    with pytest.raises(SbiemError):
        kernel_values(np.array([-1.0]), 0.5)
    with pytest.raises(SbiemError):
        kernel_values(np.array([1.0]), 1.5)


def test_read_probe_rejects_bad_arguments(lib):
    # host-side checks only: none of these reaches a CUDA call
    from paper_2107_03550_gb300.sbiem import SbiemError, read_probe
    for data, nbytes, sink in ((0, 1024, 16), (16, 1000, 16), (8, 1024, 16), (16, 0, 16), (16, 1024, 0)):
        with pytest.raises(SbiemError):
            read_probe(data, nbytes, sink)


def test_strerror_covers_codes(lib):
    for code in range(0, -9, -1):
        assert lib.sbiem_strerror(code)


def test_kernel_route_against_high_precision(lib):
    mpmath = pytest.importorskip("mpmath")
    from paper_2107_03550_gb300.sbiem import kernel_values
    mpmath.mp.dps = 30
    r = 1 / mpmath.sqrt(3)

    def Wm(x):
        return mpmath.quadosc(lambda t: mpmath.besselj(1, t) / t, [x, mpmath.inf], omega=1)

    def GTm(s):
        s = mpmath.mpf(s)
        sp = s / r
        return ((s * s + r * r) * Wm(sp) - (s * s + 1) * Wm(s) - r * r * mpmath.besselj(1, sp)
                + mpmath.besselj(1, s) / 2 - r * s * mpmath.besselj(0, sp) + s * mpmath.besselj(0, s))

    for s in (0.7, 11.9, 19.35, 39.95, 99.6, 198.9):
        cT, _ = kernel_values(np.array([s]), float(r))
        assert abs(cT[0] - float(GTm(s))) < 5e-14, s


def test_truncation_parameters_are_validated_before_any_device_work(lib):
    # eta_w >= 0 (0: quasi-dynamic limit) and kcN_L >= 0 (0: one cutting
    # plane); negative values are rejected by the host checks, no GPU needed
    from paper_2107_03550_gb300.sbiem import ERR, Fault, SbiemError
    from paper_2107_03550_gb300.workloads import seamount_rupture
    w = seamount_rupture(N=64)
    for kw in ({"eta_w": -1.0}, {"kcN_L": -5.0}, {"kc_L": 0.0}):
        with pytest.raises(SbiemError) as e:
            Fault.from_workload(w, use_torch=False, **kw)
        assert ERR.get(e.value.code) == "INVALID"
