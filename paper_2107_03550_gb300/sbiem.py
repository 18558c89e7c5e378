"""Python binding of libsbiem (ctypes): argument marshalling only.

Every step of the time integration runs in the library's CUDA kernels; this
module converts numpy arrays to pointers, maps return codes to exceptions
and, when PyTorch is present, routes the library's device allocations
through PyTorch's caching allocator and its launches onto a PyTorch stream.
There is no CPU fallback: if ``libsbiem.so`` is missing the import of
:class:`Fault` fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Fault", "Batch", "SbiemError", "mlp_predict", "mlp_grad", "mlp_train", "kernel_values", "history_sums_noalloc", "load_library", "library_path", "FLAG_NEWTON", "FLAG_OPENING",
           "FLAG_STATE", "FLAG_WAIT", "ERR"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

FLAG_NEWTON, FLAG_OPENING, FLAG_STATE, FLAG_WAIT = 1, 2, 4, 8
ERR = {0: "OK", -1: "INVALID", -2: "NOMEM", -3: "CUDA", -4: "NEWTON", -5: "OPENING", -6: "STATE",
       -7: "DTMIN", -8: "UNSUPPORTED", -9: "WAIT"}

_alloc_t = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_output_t = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int64,
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), ctypes.c_int64)
_free_t = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("dx", ctypes.c_double), ("mu", ctypes.c_double),
                ("cs", ctypes.c_double), ("cp", ctypes.c_double), ("beta_min", ctypes.c_double),
                ("eta_w", ctypes.c_double), ("kc_L", ctypes.c_double), ("kcN_L", ctypes.c_double),
                ("kc_units", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("state_law", ctypes.c_int32),
                ("newton_maxit", ctypes.c_int32), ("quadrature", ctypes.c_int32), ("newton_tol", ctypes.c_double),
                ("f0", ctypes.c_double), ("V0", ctypes.c_double),
                ("alloc_fn", _alloc_t), ("free_fn", _free_t), ("alloc_user", ctypes.c_void_p)]


class SbiemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sbiem error {code} ({ERR.get(code, '?')}): {msg}")
        self.code = code


def library_path() -> str:
    return os.environ.get("SBIEM_LIB", os.path.join(_HERE, "_lib", "libsbiem.so"))


_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_VP = ctypes.c_void_p

_SIGS = {
    "sbiem_default_params": (None, [ctypes.POINTER(Params)]),
    "sbiem_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(Params), _D, _D, _D, _D, _D, _D, _D,
                                    _D, _U8, _D, _D, _D]),
    "sbiem_destroy": (None, [_VP]),
    "sbiem_set_stream": (ctypes.c_int, [_VP, _VP]),
    "sbiem_step": (ctypes.c_int, [_VP, ctypes.c_double]),
    "sbiem_enqueue": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int64]),
    "sbiem_status": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint32), _I64, ctypes.c_int]),
    "sbiem_step_kernels": (ctypes.c_int, [_VP, ctypes.c_double, _I64]),
    "sbiem_step_host": (ctypes.c_int, [_VP, ctypes.c_double, _D, _D]),
    "sbiem_run": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                 ctypes.c_int64, _I64, _I64, _D, _I64]),
    "sbiem_get_state": (ctypes.c_int, [_VP, _D, _D, _D, _D, _D, _D]),
    "sbiem_set_state": (ctypes.c_int, [_VP, _D, _D, _D]),
    "sbiem_windows": (ctypes.c_int, [_VP, _I64]),
    "sbiem_set_history": (ctypes.c_int, [_VP, _D, _D]),
    "sbiem_get_history": (ctypes.c_int, [_VP, _D, _D]),
    "sbiem_set_history_device": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32]),
    "sbiem_newton_stats": (ctypes.c_int, [_VP, _I64, ctypes.POINTER(ctypes.c_int32)]),
    "sbiem_newton_totals": (ctypes.c_int, [_VP, _I64, _I64, ctypes.c_int]),
    "sbiem_probe_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "sbiem_history_sums": (ctypes.c_int, [_VP, ctypes.c_int64, _D, _D]),
    "sbiem_history_enqueue": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "sbiem_history_enqueue_marked": (ctypes.c_int, [_VP, ctypes.c_int64, _VP]),
    "sbiem_read_probe": (ctypes.c_int, [_VP, ctypes.c_int64, _VP, _VP]),
    "sbiem_save": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "sbiem_get_params": (ctypes.c_int, [_VP, ctypes.c_void_p]),
    "sbiem_load": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_char_p, ctypes.c_void_p]),
    "sbiem_probe_read": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_float)]),
    "sbiem_footprint": (ctypes.c_int, [_VP, _I64, _I64]),
    "sbiem_get_sweep": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), _D, ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32), _D]),
    "sbiem_set_sweep": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_double, ctypes.c_int32]),
    "sbiem_set_lag_sweep": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "sbiem_set_wait_limit": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "sbiem_set_output": (ctypes.c_int, [_VP, _output_t, _VP, ctypes.c_int64]),
    "sbiem_tune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), _D,
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]),
    "sbiem_history_sums_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _VP, _VP, _VP,
                                                  _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "sbiem_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP), ctypes.c_int64]),
    "sbiem_batch_destroy": (None, [_VP]),
    "sbiem_batch_set_stream": (ctypes.c_int, [_VP, _VP]),
    "sbiem_batch_enqueue": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "sbiem_batch_status": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint32), _I64]),
    "sbiem_batch_tune": (ctypes.c_int, [_VP, ctypes.c_int, _I64, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_float)]),
    "sbiem_batch_set_overlap": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "sbiem_batch_set_wait_limit": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "sbiem_batch_get_sweep": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "sbiem_batch_set_persistent": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "sbiem_set_mlp": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "sbiem_harvest_enable": (ctypes.c_int, [_VP, ctypes.c_int64]),
    "sbiem_harvest_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_int64, _I64, ctypes.c_int]),
    "sbiem_mlp_predict": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                         ctypes.c_int64, ctypes.POINTER(ctypes.c_float)]),
    "sbiem_mlp_grad": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_float), ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "sbiem_mlp_train": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_float)]),
    "sbiem_kernel_values": (ctypes.c_int, [_D, ctypes.c_int64, ctypes.c_double, _D, _D]),
    "sbiem_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sbiem_last_error": (ctypes.c_char_p, []),
}


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libsbiem.so and declare its signatures; raises if it is missing."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or library_path()
    if not os.path.exists(p):
        raise ImportError(f"libsbiem.so not found at {p}; build it with "
                          f"`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = lib
    return lib


def _ptr(a, dtype=np.float64, n=None):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    if n is not None and arr.size != n:
        raise ValueError(f"expected {n} values, got {arr.size}")
    ct = ctypes.c_uint8 if dtype == np.uint8 else ctypes.c_double
    return arr, arr.ctypes.data_as(ctypes.POINTER(ct))


def _torch_allocator():
    """(alloc, free) callbacks backed by torch's CUDA caching allocator, or None."""
    try:
        import torch
    except ImportError:
        return None
    if not torch.cuda.is_available():
        return None
    dev = torch.cuda.current_device()

    def _alloc(nbytes, _user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev))
        except Exception:  # out of memory: the library reports SBIEM_ERR_NOMEM
            return None

    def _free(ptr, _user):
        if ptr:
            torch.cuda.caching_allocator_delete(int(ptr))

    return _alloc_t(_alloc), _free_t(_free)


def kernel_values(s, r: float):
    """Library route of (C^T_II, C^N_II) at points s = c_s |k| t (host FP64, no GPU)."""
    lib = load_library()
    sa = np.ascontiguousarray(np.asarray(s, np.float64).ravel())
    cT = np.empty_like(sa)
    cN = np.empty_like(sa)
    rc = lib.sbiem_kernel_values(sa.ctypes.data_as(_D), sa.size, float(r), cT.ctypes.data_as(_D),
                                 cN.ctypes.data_as(_D))
    if rc != 0:
        raise SbiemError(rc, "kernel_values: invalid argument")
    return cT, cN


def history_sums_noalloc(nmodes: int, precision: int, m: int, ring: int, weights: int, ring_off: int,
                         w_off: int, R: int, M: int, head: int, AT: int, AN: int, stream=None) -> None:
    """History convolution on caller-owned device buffers (raw device pointers), no allocation.

    For callers that cannot allocate device memory; see the C header for the
    buffer layouts, the size limits and the one-stream rule.
    """
    lib = load_library()
    raw = getattr(stream, "cuda_stream", stream)
    rc = lib.sbiem_history_sums_noalloc(int(nmodes), int(precision), int(m), ring, weights, ring_off, w_off, R, M,
                                        head, AT, AN, raw or None)
    if rc != 0:
        raise SbiemError(rc, "history_sums_noalloc: invalid sizes or CUDA failure")


def read_probe(data: int, nbytes: int, sink: int, stream=None) -> None:
    """Enqueue one plain streaming read of nbytes at device pointer data (a measurement helper;
    see sbiem_read_probe in the C header).  sink: device pointer to one float."""
    lib = load_library()
    raw = getattr(stream, "cuda_stream", stream)
    rc = lib.sbiem_read_probe(data, int(nbytes), sink, raw or None)
    if rc != 0:
        raise SbiemError(rc, "read_probe: null or misaligned pointer or size, or CUDA failure")


MLP_PARAMS, MLP_NORM = 4609, 12
_F = ctypes.POINTER(ctypes.c_float)


def _f32(a, n=None):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if n is not None and arr.size != n:
        raise ValueError(f"expected {n} values, got {arr.size}")
    return arr, arr.ctypes.data_as(_F)


def mlp_predict(params, X) -> np.ndarray:
    """Evaluate the Newton-guess network on the GPU: X [n, 5] raw features -> residuals [n]."""
    lib = load_library()
    p, pp = _f32(params, MLP_PARAMS + MLP_NORM)
    x, xp = _f32(X)
    n = x.size // 5
    out = np.empty(n, dtype=np.float32)
    rc = lib.sbiem_mlp_predict(pp, xp, n, out.ctypes.data_as(_F))
    if rc != 0:
        raise SbiemError(rc, "mlp_predict failed")
    return out


def mlp_grad(params, X, t):
    """(loss, gradient) of the mean squared error on normalized X [n, 5], targets t [n]."""
    lib = load_library()
    p, pp = _f32(params)
    x, xp = _f32(X)
    tt, tp = _f32(t)
    g = np.empty(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    rc = lib.sbiem_mlp_grad(pp, xp, tp, tt.size, g.ctypes.data_as(_F), ctypes.byref(loss))
    if rc != 0:
        raise SbiemError(rc, "mlp_grad failed")
    return float(loss.value), g


def mlp_train(samples, epochs=5, batch=8192, lr=1e-3, seed=0):
    """Train on harvested rows [n, 6]; returns (params [4621], final batch loss)."""
    lib = load_library()
    s, sp = _f32(samples)
    n = s.size // 6
    params = np.empty(MLP_PARAMS + MLP_NORM, dtype=np.float32)
    loss = ctypes.c_float()
    rc = lib.sbiem_mlp_train(sp, n, int(epochs), int(batch), float(lr), int(seed), params.ctypes.data_as(_F),
                             ctypes.byref(loss))
    if rc != 0:
        raise SbiemError(rc, "mlp_train failed")
    return params, float(loss.value)


class Fault:
    """One periodic non-planar fault on the GPU (a libsbiem handle).

    Arguments mirror ``sbiem_params`` and ``sbiem_create`` in the C header:
    ``eta_w`` is the truncation parameter of Sec. 3.1 (0: the quasi-dynamic
    limit, no history); ``kc_L`` the cutting plane k_c eta L of both kernels,
    ``kcN_L`` (> 0) a second plane for the normal-traction kernel;
    ``precision`` 0 (FP64) or 1 (FP32 history and FFTs, FP64 state).
    """

    def __init__(self, N, dx, mu, cs, cp, f0, V0, a, b, Dc, sigma_load, V_init, theta_init,
                 kappa=None, h=None, tau_load=None, tau_load_rate=None, prescribed=None,
                 V_presc=None, beta_min=0.25, eta_w=1.0, kc_L=200.0, kcN_L=0.0, kc_units=0, precision=0,
                 state_law=0, newton_maxit=50, newton_tol=1e-12, quadrature=0, use_torch=True, allocator=None,
                 lib=None):
        self.lib = lib or load_library()
        self.N = int(N)
        p = Params()
        self.lib.sbiem_default_params(ctypes.byref(p))
        p.N, p.dx, p.mu, p.cs, p.cp = self.N, dx, mu, cs, cp
        p.beta_min, p.eta_w, p.kc_L, p.kcN_L, p.kc_units = beta_min, eta_w, kc_L, kcN_L, kc_units
        p.precision, p.state_law = precision, state_law
        p.newton_maxit, p.newton_tol, p.f0, p.V0 = newton_maxit, newton_tol, f0, V0
        p.quadrature = quadrature
        if allocator is not None:
            # caller's device memory: alloc(nbytes) -> device pointer or 0, free(ptr)
            a_fn, f_fn = allocator
            self._cb = (_alloc_t(lambda n, _u: a_fn(int(n)) or None), _free_t(lambda q, _u: f_fn(q)))
        else:
            self._cb = _torch_allocator() if use_torch else None
        if self._cb is not None:
            p.alloc_fn, p.free_fn = self._cb
        self.params = p
        n = self.N
        keep = []

        def P(x, dtype=np.float64):
            arr, ptr = _ptr(x, dtype, n)
            keep.append(arr)
            return ptr

        handle = _VP()
        rc = self.lib.sbiem_create(ctypes.byref(handle), ctypes.byref(p), P(h), P(kappa), P(a), P(b), P(Dc),
                                   P(sigma_load), P(tau_load), P(tau_load_rate),
                                   P(None if prescribed is None else np.asarray(prescribed).astype(np.uint8),
                                     np.uint8),
                                   P(V_presc), P(V_init), P(theta_init))
        self._check(rc)
        self.h = handle
        self.dt_min = beta_min * dx / cs
        self._stream = None

    @classmethod
    def from_workload(cls, w, **kw):
        """Handle for a :class:`paper_2107_03550_gb300.workloads.Workload`."""
        args = dict(N=w.N, dx=w.dx, mu=w.mu, cs=w.cs, cp=w.cp, f0=w.f0, V0=w.V0, a=w.a, b=w.b, Dc=w.Dc,
                    sigma_load=w.sigma_load, V_init=w.V_init, theta_init=w.theta_init, kappa=w.kappa,
                    tau_load=w.tau_load, tau_load_rate=w.tau_load_rate,
                    prescribed=w.prescribed if np.any(w.prescribed) else None,
                    V_presc=w.V_presc if np.any(w.prescribed) else None,
                    beta_min=w.dt_min * w.cs / w.dx)
        args.update(kw)
        return cls(**args)

    # ------------------------------------------------------------ checkpoint
    def save(self, path) -> None:
        """Write a checkpoint (parameters, inputs, state, time, history)."""
        self._check(self.lib.sbiem_save(self.h, os.fsencode(path)))

    @classmethod
    def load(cls, path, use_torch=True, lib=None):
        """New handle continuing a checkpoint written by :meth:`save`."""
        self = cls.__new__(cls)
        self.lib = lib or load_library()
        p = Params()
        self.lib.sbiem_default_params(ctypes.byref(p))
        self._cb = _torch_allocator() if use_torch else None
        if self._cb is not None:
            p.alloc_fn, p.free_fn = self._cb
        handle = _VP()
        self._check(self.lib.sbiem_load(ctypes.byref(handle), os.fsencode(path), ctypes.cast(ctypes.byref(p),
                                                                                              ctypes.c_void_p)))
        self.h = handle
        q = Params()
        self._check(self.lib.sbiem_get_params(self.h, ctypes.cast(ctypes.byref(q), ctypes.c_void_p)))
        self.params = q
        self.N = int(q.N)
        self.dt_min = q.beta_min * q.dx / q.cs
        self._stream = None
        return self

    # ---------------------------------------------------------------- errors
    def _check(self, rc):
        if rc != 0:
            raise SbiemError(rc, self.lib.sbiem_last_error().decode())

    # ------------------------------------------------------------------ steps
    def set_stream(self, stream) -> None:
        """Bind to a CUDA stream: a torch.cuda.Stream or a raw handle (int); 0 / None is the
        legacy default stream (torch's default stream)."""
        raw = getattr(stream, "cuda_stream", stream)
        self._stream = stream
        self._check(self.lib.sbiem_set_stream(self.h, _VP(raw or None)))

    def history_enqueue(self, m: int = 1, sweep_done=None) -> None:
        """Enqueue the history convolution alone (no synchronization), for timing.

        sweep_done: a torch.cuda.Event recorded between the sweep kernel and
        the per-mode finish (None: not recorded)."""
        ev = None if sweep_done is None else ctypes.c_void_p(sweep_done.cuda_event)
        self._check(self.lib.sbiem_history_enqueue_marked(self.h, int(m), ev))

    def step(self, dt=None) -> None:
        self._check(self.lib.sbiem_step(self.h, float(dt or self.dt_min)))

    def try_step(self, dt=None) -> int:
        """One step; returns the SBIEM code instead of raising on a rejected step."""
        return int(self.lib.sbiem_step(self.h, float(dt or self.dt_min)))

    def enqueue(self, nsteps: int, dt=None) -> None:
        self._check(self.lib.sbiem_enqueue(self.h, float(dt or self.dt_min), int(nsteps)))

    def step_kernels(self, dt=None) -> int:
        """Kernel launches in one replay of the step graph of :meth:`enqueue`."""
        k = ctypes.c_int64()
        self._check(self.lib.sbiem_step_kernels(self.h, float(dt or self.dt_min), ctypes.byref(k)))
        return k.value

    def status(self, clear: bool = False):
        fl = ctypes.c_uint32()
        st = ctypes.c_int64()
        self._check(self.lib.sbiem_status(self.h, ctypes.byref(fl), ctypes.byref(st), int(clear)))
        return int(fl.value), int(st.value)

    def run(self, t_end: float, eps0: float, m0: int = 1, m_max: int = 1 << 30, max_steps: int = 10 ** 6):
        """Adaptive step-doubling run (Sec. 3.2).  Returns (accepted m list, next m, t reached, code)."""
        hist = np.zeros(max(int(max_steps), 1), dtype=np.int64)
        n = ctypes.c_int64()
        mn = ctypes.c_int64()
        t = ctypes.c_double()
        rc = self.lib.sbiem_run(self.h, float(t_end), float(eps0), int(m0), int(m_max), int(max_steps),
                                ctypes.byref(n), ctypes.byref(mn), ctypes.byref(t), hist.ctypes.data_as(_I64))
        if rc not in (0, -7):
            self._check(rc)
        return hist[:n.value].tolist(), int(mn.value), float(t.value), int(rc)

    def set_output(self, fn, every: int = 1) -> None:
        """Call fn(step, t, m, delta, V) during :meth:`run` after every `every`-th accepted step and the
        last (delta, V: numpy copies); fn returning True stops the run.  fn=None removes it."""
        if fn is None:
            self._out = None
            self._check(self.lib.sbiem_set_output(self.h, _output_t(), None, 0))
            return
        n = self.N

        def _cb(_user, step, t, m, d, v, _n):
            try:
                return 1 if fn(int(step), float(t), int(m), np.ctypeslib.as_array(d, (n,)).copy(),
                               np.ctypeslib.as_array(v, (n,)).copy()) else 0
            except Exception:       # an exception cannot cross the C ABI: stop the run
                return 1
        self._out = _output_t(_cb)  # kept alive with the handle
        self._check(self.lib.sbiem_set_output(self.h, self._out, None, int(every)))

    def step_host(self, dt=None, tau_load=None, V_out=None) -> None:
        ta, tp = _ptr(tau_load, np.float64, self.N)
        vp = None
        if V_out is not None:
            assert V_out.dtype == np.float64 and V_out.flags.c_contiguous and V_out.size == self.N
            vp = V_out.ctypes.data_as(_D)
        self._check(self.lib.sbiem_step_host(self.h, float(dt or self.dt_min), tp, vp))

    # ------------------------------------------------------------------ state
    def get_state(self) -> dict:
        n = self.N
        out = {k: np.empty(n) for k in ("delta", "V", "theta", "tau_el", "sigma_el")}
        t = ctypes.c_double()
        self._check(self.lib.sbiem_get_state(self.h, *(out[k].ctypes.data_as(_D) for k in
                                                       ("delta", "V", "theta", "tau_el", "sigma_el")),
                                             ctypes.byref(t)))
        out["t"] = t.value
        return out

    def set_state(self, delta=None, V=None, theta=None) -> None:
        a1, p1 = _ptr(delta, np.float64, self.N)
        a2, p2 = _ptr(V, np.float64, self.N)
        a3, p3 = _ptr(theta, np.float64, self.N)
        self._check(self.lib.sbiem_set_state(self.h, p1, p2, p3))

    def windows(self) -> np.ndarray:
        M = np.empty(self.N // 2 + 1, dtype=np.int64)
        self._check(self.lib.sbiem_windows(self.h, M.ctypes.data_as(_I64)))
        return M

    def history_size(self) -> int:
        return int(np.maximum(self.windows() - 1, 0).sum())

    def set_history(self, HT: np.ndarray, HN: np.ndarray) -> None:
        """Flat complex128 arrays, modes in order, newest slot first per mode."""
        tot = self.history_size()
        a = np.ascontiguousarray(np.asarray(HT, np.complex128).reshape(tot)).view(np.float64)
        b = np.ascontiguousarray(np.asarray(HN, np.complex128).reshape(tot)).view(np.float64)
        self._check(self.lib.sbiem_set_history(self.h, a.ctypes.data_as(_D), b.ctypes.data_as(_D)))

    def set_history_device(self, HT, HN) -> None:
        """The same from device tensors: complex64/complex128 (or float pairs), flat, contiguous."""
        import torch
        tot = self.history_size()
        ts = []
        for h in (HT, HN):
            t = torch.view_as_real(h) if h.is_complex() else h
            if t.numel() != 2 * tot or not t.is_contiguous() or t.dtype not in (torch.float32, torch.float64):
                raise ValueError("expected contiguous FP32/FP64 history of the handle's size on the device")
            ts.append(t)
        if ts[0].dtype != ts[1].dtype:
            raise ValueError("both fields must have the same precision")
        f32 = 1 if ts[0].dtype == torch.float32 else 0
        self._check(self.lib.sbiem_set_history_device(self.h, ts[0].data_ptr(), ts[1].data_ptr(), f32))

    def get_history(self):
        tot = self.history_size()
        a = np.empty(2 * tot)
        b = np.empty(2 * tot)
        self._check(self.lib.sbiem_get_history(self.h, a.ctypes.data_as(_D), b.ctypes.data_as(_D)))
        return a.view(np.complex128), b.view(np.complex128)

    def history_sums(self, m: int = 1):
        """(A^T_n, A^N_n) of the current rings for a step of m dt_min (complex arrays)."""
        nm = self.N // 2 + 1
        at = np.empty(2 * nm)
        an = np.empty(2 * nm)
        self._check(self.lib.sbiem_history_sums(self.h, int(m), at.ctypes.data_as(_D), an.ctypes.data_as(_D)))
        return at.view(np.complex128), an.view(np.complex128)

    def probe_enable(self, nslots: int = 1) -> None:
        """Record step / history-convolution events into a ring of nslots slots (0: off)."""
        self._check(self.lib.sbiem_probe_enable(self.h, int(nslots)))

    def probe_read(self, slot: int = 0):
        """(ms of the step in this slot, ms of its history convolution), device events."""
        a = ctypes.c_float()
        b = ctypes.c_float()
        self._check(self.lib.sbiem_probe_read(self.h, int(slot), ctypes.byref(a), ctypes.byref(b)))
        return float(a.value), float(b.value)

    def set_mlp(self, params) -> None:
        """Deploy a Newton initial-guess network (None: plain Newton)."""
        if params is None:
            self._check(self.lib.sbiem_set_mlp(self.h, None))
            return
        p, pp = _f32(params, MLP_PARAMS + MLP_NORM)
        self._check(self.lib.sbiem_set_mlp(self.h, pp))

    def harvest_enable(self, capacity: int) -> None:
        self._check(self.lib.sbiem_harvest_enable(self.h, int(capacity)))

    def harvest_read(self, reset: bool = False) -> np.ndarray:
        n = ctypes.c_int64()
        self._check(self.lib.sbiem_harvest_read(self.h, None, 0, ctypes.byref(n), 0))
        out = np.empty((n.value, 6), dtype=np.float32)
        m = ctypes.c_int64()
        self._check(self.lib.sbiem_harvest_read(self.h, out.ctypes.data_as(_F), n.value, ctypes.byref(m),
                                                int(reset)))
        return out

    def newton_stats(self):
        s = ctypes.c_int64()
        m = ctypes.c_int32()
        self._check(self.lib.sbiem_newton_stats(self.h, ctypes.byref(s), ctypes.byref(m)))
        return int(s.value), int(m.value)

    def get_sweep(self) -> dict:
        """History sweep configuration: shape, on-chip weight threshold, CTAs per SM, weight-table error."""
        sh, ct, lc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        th, err = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.sbiem_get_sweep(self.h, ctypes.byref(sh), ctypes.byref(th), ctypes.byref(ct),
                                             ctypes.byref(lc), ctypes.byref(err)))
        return {"shape": sh.value, "gen_ds_max": th.value, "ctas_per_sm": ct.value, "lag_ctas_per_sm": lc.value,
                "table_err": err.value}

    def set_sweep(self, shape: int = 3, gen_ds_max: float = 0.0625, ctas_per_sm: int = 0) -> None:
        """gen_ds_max: modes with s step c_s k dt_min at most this evaluate their weights on chip (0: none)."""
        self._check(self.lib.sbiem_set_sweep(self.h, int(shape), float(gen_ds_max), int(ctas_per_sm)))

    def set_lag_sweep(self, lag_ctas_per_sm: int = 0) -> None:
        """Resident CTAs per SM of the next step's sweep run beside the passes (0: the built-in rule)."""
        self._check(self.lib.sbiem_set_lag_sweep(self.h, int(lag_ctas_per_sm)))

    def set_wait_limit(self, polls: int = 4194304) -> None:
        """Polls of the history sweep's copy waits before it gives up (0: at once)."""
        self._check(self.lib.sbiem_set_wait_limit(self.h, int(polls)))

    def tune(self, reps: int = 5) -> dict:
        """Autotune the history sweep (shape, on-chip weight threshold, CTAs per SM); returns the choice."""
        sh, ct = ctypes.c_int32(), ctypes.c_int32()
        th = ctypes.c_double()
        ms = ctypes.c_float()
        self._check(self.lib.sbiem_tune(self.h, int(reps), ctypes.byref(sh), ctypes.byref(th), ctypes.byref(ct),
                                        ctypes.byref(ms)))
        return {"shape": sh.value, "gen_ds_max": th.value, "ctas_per_sm": ct.value, "ms": ms.value}

    def newton_totals(self, reset: bool = False):
        """(iterations, solves) of every Newton solve since creation or the last reset."""
        it, so = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.sbiem_newton_totals(self.h, ctypes.byref(it), ctypes.byref(so), 1 if reset else 0))
        return int(it.value), int(so.value)

    def footprint(self):
        hb = ctypes.c_int64()
        db = ctypes.c_int64()
        self._check(self.lib.sbiem_footprint(self.h, ctypes.byref(hb), ctypes.byref(db)))
        return int(hb.value), int(db.value)

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.sbiem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """An ensemble of Fault handles advanced together (batched launches, one graph per step)."""

    def __init__(self, members, chunk_slots: int = 0, lib=None):
        self.lib = lib or load_library()
        self.members = list(members)
        arr = (_VP * len(self.members))(*[m.h for m in self.members])
        h = _VP()
        rc = self.lib.sbiem_batch_create(ctypes.byref(h), len(self.members), arr, int(chunk_slots))
        if rc != 0:
            raise SbiemError(rc, self.lib.sbiem_last_error().decode())
        self.h = h

    def _check(self, rc):
        if rc != 0:
            raise SbiemError(rc, self.lib.sbiem_last_error().decode())

    def set_stream(self, stream) -> None:
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.sbiem_batch_set_stream(self.h, _VP(raw or None)))

    def enqueue(self, nsteps: int) -> None:
        self._check(self.lib.sbiem_batch_enqueue(self.h, int(nsteps)))

    def set_wait_limit(self, polls: int = 4194304) -> None:
        """Polls of the persistent history launch's grid barrier before a CTA gives up (0: at once)."""
        self._check(self.lib.sbiem_batch_set_wait_limit(self.h, int(polls)))

    def get_sweep(self) -> dict:
        """History-convolution configuration: shape, weight form, CTAs per SM, overlap, shared weights, form."""
        sh, thr, ctas, ov, dw, pe = (ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32(), ctypes.c_int32(),
                                     ctypes.c_int32(), ctypes.c_int32())
        self._check(self.lib.sbiem_batch_get_sweep(self.h, ctypes.byref(sh), ctypes.byref(thr), ctypes.byref(ctas),
                                                   ctypes.byref(ov), ctypes.byref(dw), ctypes.byref(pe)))
        return {"shape": sh.value, "gen_ds_max": thr.value, "ctas_per_sm": ctas.value, "overlap": bool(ov.value),
                "distinct_weights": dw.value, "persistent": bool(pe.value)}

    def set_persistent(self, on: bool) -> bool:
        """One persistent launch (True, the default) or a sweep launch plus a sum launch; returns the old form."""
        old = ctypes.c_int()
        self._check(self.lib.sbiem_batch_set_persistent(self.h, 1 if on else 0, ctypes.byref(old)))
        return bool(old.value)

    def set_overlap(self, on: bool) -> bool:
        """Sweep the next step's history beside the passes (True) or not; returns the old setting."""
        old = ctypes.c_int()
        self._check(self.lib.sbiem_batch_set_overlap(self.h, 1 if on else 0, ctypes.byref(old)))
        return bool(old.value)

    def status(self):
        n = len(self.members)
        fl = (ctypes.c_uint32 * n)()
        sd = np.zeros(n, dtype=np.int64)
        self._check(self.lib.sbiem_batch_status(self.h, fl, sd.ctypes.data_as(_I64)))
        return np.array(list(fl), dtype=np.uint32), sd

    def tune(self, reps: int = 5):
        """Autotune the batched history convolution (shape, weight form, resident CTAs per SM) and the
        overlap; returns (chunk length, CTAs per SM, ms)."""
        c = ctypes.c_int64()
        b = ctypes.c_int()
        ms = ctypes.c_float()
        self._check(self.lib.sbiem_batch_tune(self.h, int(reps), ctypes.byref(c), ctypes.byref(b), ctypes.byref(ms)))
        return int(c.value), int(b.value), float(ms.value)

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.sbiem_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
