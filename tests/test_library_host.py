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
    # every SBIEM_ERR_* code of the header has a message and a binding name
    import re
    from paper_2107_03550_gb300.sbiem import ERR
    hdr = open(os.path.join(ROOT, "include", "sbiem.h")).read()
    codes = {int(v) for v in re.findall(r"#define SBIEM_(?:OK|ERR_\w+)\s+(-?\d+)", hdr)}
    assert codes == set(range(0, -10, -1))
    unknown = lib.sbiem_strerror(-1000)
    for code in codes:
        assert lib.sbiem_strerror(code) and lib.sbiem_strerror(code) != unknown
        assert code in ERR


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


def _write_checkpoint(path, N, heads=None, total_slots=None, head_delta=None):
    """A checkpoint file in the library's format, written by hand (no GPU):
    header (magic, N, total_slots, six int32, eleven doubles), 14 element
    arrays, the prescribed mask, F[delta] and F[kappa delta], the ring heads,
    the FP64 ring (32 bytes per slot), the time and the step count."""
    import struct
    from oracle.sbiem import Params, windows
    dx, mu, cs = 25.0, 30e9, 3464.0
    cp = np.sqrt(3.0) * cs
    p = Params(N=N, dx=dx, mu=mu, cs=cs, cp=cp, dt_min=0.25 * dx / cs)
    R = np.maximum(windows(p) - 1, 0)
    slots = int(R.sum()) if total_slots is None else total_slots
    hd = b"SBIEMCK3" + struct.pack("<qq6i11d", N, slots, 0, 0, 0, 50, 0, 0, dx, mu, cs, cp, 0.25, 1.0, 200.0,
                                   1e-12, 0.6, 1e-6, 0.0)
    el = np.ones(14 * N)
    h = np.zeros(R.size, dtype=np.int32) if heads is None else np.asarray(heads, np.int32)
    with open(path, "wb") as fh:
        fh.write(hd)
        fh.write(el.tobytes())
        fh.write(np.zeros(N, np.uint8).tobytes())
        fh.write(np.zeros(4 * (N // 2 + 1)).tobytes())
        fh.write(h.tobytes())
        fh.write(np.zeros(4 * int(R.sum())).tobytes())
        fh.write(struct.pack("<dq", 0.0, 0))
    return R


def test_checkpoint_load_rejects_bad_heads_and_sizes_on_the_host(lib, tmp_path):
    # a corrupt checkpoint must fail with SBIEM_ERR_INVALID before any device
    # work: a ring head at or past R_n would steer the sweep's bulk copies
    # outside the ring, and a forged history size would size host buffers
    # from the file
    out = ctypes.c_void_p()
    path = str(tmp_path / "ck.bin")
    R = _write_checkpoint(path, 64)
    n = int(np.argmax(R))
    heads = np.zeros(R.size, np.int32)
    heads[n] = R[n]
    _write_checkpoint(path, 64, heads=heads)
    assert lib.sbiem_load(ctypes.byref(out), path.encode(), None) == -1
    assert b"ring head" in lib.sbiem_last_error()
    heads[n] = -1
    _write_checkpoint(path, 64, heads=heads)
    assert lib.sbiem_load(ctypes.byref(out), path.encode(), None) == -1
    heads[n] = 0
    heads[0] = 1                      # mode 0 has no history
    _write_checkpoint(path, 64, heads=heads)
    assert lib.sbiem_load(ctypes.byref(out), path.encode(), None) == -1
    _write_checkpoint(path, 64, total_slots=1 << 40)
    assert lib.sbiem_load(ctypes.byref(out), path.encode(), None) == -1
    assert b"history size" in lib.sbiem_last_error()
    with open(path, "r+b") as fh:      # truncated file
        fh.truncate(200)
    assert lib.sbiem_load(ctypes.byref(out), path.encode(), None) == -1
    assert not out.value
