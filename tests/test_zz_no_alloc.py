"""The history convolution for callers that cannot allocate device memory.

Some callers must not allocate device memory, themselves or through a
library: an application that hands out every byte of the GPU from its own
fixed arena or runs under a hard device-memory budget, or a real-time loop
that cannot take cudaMalloc's latency and synchronization mid-step.  They
keep the history in their own buffers and call sbiem_history_sums_noalloc,
whose scratch lives in a static device array of the library.

This test builds those buffers with PyTorch (the test's own allocation),
with every mode's ring rotated to a random head as a caller's ring is after
many steps, calls the entry point twice in a row through the C ABI and
checks both results against the handle's sbiem_history_sums on the same
history and against the FP64 oracle.  It runs last (file name) so that a
run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _caller_buffers(torch, g, w, HT, HN, precision, rng):
    from paper_2107_03550_gb300.sbiem import kernel_values
    M = g.windows()
    R = np.maximum(M - 1, 0)
    ring_off = np.concatenate([[0], np.cumsum(R)[:-1]]).astype(np.int64)
    w_off = np.concatenate([[0], np.cumsum(M)[:-1]]).astype(np.int64)
    # weights w_{n,j} = dt C(k_n, (j + 1/2) dt) from the library's kernel route
    dt = w.dt_min
    L = w.N * w.dx
    mode = np.repeat(np.arange(M.size), M)
    j = np.arange(M.sum()) - np.repeat(w_off, M)
    s = w.cs * (2 * np.pi * mode / L) * (j + 0.5) * dt
    cT, cN = kernel_values(s, w.cs / w.cp)
    wts = np.stack([dt * cT, dt * cN], axis=1)
    # each mode's ring rotated: the i-th newest value at slot (head + i) mod R
    head = np.where(R > 0, rng.integers(0, np.maximum(R, 1)), 0).astype(np.int32)
    slots = np.empty((int(R.sum()), 4))
    hoff = np.concatenate([[0], np.cumsum(R)])
    for n in range(M.size):
        r = int(R[n])
        if r == 0:
            continue
        pos = ring_off[n] + (head[n] + np.arange(r)) % r
        h = slice(hoff[n], hoff[n + 1])
        slots[pos] = np.stack([HT[h].real, HT[h].imag, HN[h].real, HN[h].imag], axis=1)
    ft = torch.float64 if precision == 0 else torch.float32
    dev = torch.device("cuda")
    bufs = dict(
        ring=torch.tensor(slots, dtype=ft, device=dev).contiguous(),
        weights=torch.tensor(wts, dtype=ft, device=dev).contiguous(),
        ring_off=torch.tensor(ring_off, dtype=torch.int64, device=dev),
        w_off=torch.tensor(w_off, dtype=torch.int64, device=dev),
        R=torch.tensor(R, dtype=torch.int32, device=dev),
        M=torch.tensor(M, dtype=torch.int32, device=dev),
        head=torch.tensor(head, dtype=torch.int32, device=dev),
        AT=torch.full((M.size, 2), np.nan, dtype=torch.float64, device=dev),
        AN=torch.full((M.size, 2), np.nan, dtype=torch.float64, device=dev),
    )
    assert int(head.max()) > 0
    return bufs


# tolerances: against the handle's sums (same weights route, another
# summation order) and against the oracle (its own kernel route; FP32
# values and weights rounded once), as in the handle's own parity tests
@pytest.mark.parametrize("precision,tol_handle,tol_oracle", [(0, 1e-12, 1e-10), (1, 1e-6, 2e-6)])
def test_noalloc_history_sums_match_handle_and_oracle(torch_cuda, precision, tol_handle, tol_oracle):
    torch = torch_cuda
    from paper_2107_03550_gb300.sbiem import Fault, history_sums_noalloc
    from paper_2107_03550_gb300.workloads import random_history, rough_fault
    from tests.gpu_helpers import oracle_for, rel
    w = rough_fault(2048, 10.0, 3e-3, seed=21)
    g = Fault.from_workload(w, precision=precision)
    o = oracle_for(w)
    R = np.maximum(g.windows() - 1, 0)
    assert np.array_equal(g.windows(), o.M)
    HT, HN, off = random_history(R, 5, 1e-3)
    g.set_history(HT, HN)
    o.set_history([HT[off[n]:off[n + 1]] for n in range(R.size)], [HN[off[n]:off[n + 1]] for n in range(R.size)])
    b = _caller_buffers(torch, g, w, HT, HN, precision, np.random.default_rng(3))
    stream = torch.cuda.current_stream()
    for m in (1, 2):   # two calls in a row share the static scratch
        ref_T, ref_N = g.history_sums(m)
        o_T, o_N = o.history_sums(m)
        history_sums_noalloc(R.size, precision, m, b["ring"].data_ptr(), b["weights"].data_ptr(),
                             b["ring_off"].data_ptr(), b["w_off"].data_ptr(), b["R"].data_ptr(),
                             b["M"].data_ptr(), b["head"].data_ptr(), b["AT"].data_ptr(), b["AN"].data_ptr(),
                             stream)
        torch.cuda.synchronize()
        at = b["AT"].cpu().numpy()
        an = b["AN"].cpu().numpy()
        at = at[:, 0] + 1j * at[:, 1]
        an = an[:, 0] + 1j * an[:, 1]
        assert np.all(np.isfinite(at)) and np.all(np.isfinite(an))
        assert rel(at, ref_T) <= tol_handle and rel(an, ref_N) <= tol_handle, m
        assert rel(at, o_T) <= tol_oracle and rel(an, o_N) <= tol_oracle, m
    g.close()


def test_noalloc_rejects_oversized_input(torch_cuda):
    from paper_2107_03550_gb300.sbiem import SbiemError, history_sums_noalloc
    with pytest.raises(SbiemError) as ei:
        history_sums_noalloc(10 ** 6, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1)
    assert ei.value.code == -1
