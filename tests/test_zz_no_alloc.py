"""The history convolution for callers that cannot allocate device memory.

Some callers must not call cudaMalloc: code recorded into their own CUDA
graph, real-time loops, frameworks with a fixed device arena.  They keep the
history in their own buffers and call sbiem_history_sums_noalloc, whose
scratch lives in a static device array.  This test builds those buffers with
PyTorch (the test's own allocation), calls the entry point twice in a row
through the C ABI and checks both results against the handle-based
sbiem_history_sums on the same history.  It runs last (file name) so that a
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


def _caller_buffers(torch, g, w, HT, HN, precision):
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
    slots = np.stack([HT.real, HT.imag, HN.real, HN.imag], axis=1)
    ft = torch.float64 if precision == 0 else torch.float32
    dev = torch.device("cuda")
    bufs = dict(
        ring=torch.tensor(slots, dtype=ft, device=dev).contiguous(),
        weights=torch.tensor(wts, dtype=ft, device=dev).contiguous(),
        ring_off=torch.tensor(ring_off, dtype=torch.int64, device=dev),
        w_off=torch.tensor(w_off, dtype=torch.int64, device=dev),
        R=torch.tensor(R, dtype=torch.int32, device=dev),
        M=torch.tensor(M, dtype=torch.int32, device=dev),
        head=torch.zeros(M.size, dtype=torch.int32, device=dev),
        AT=torch.full((M.size, 2), np.nan, dtype=torch.float64, device=dev),
        AN=torch.full((M.size, 2), np.nan, dtype=torch.float64, device=dev),
    )
    return bufs


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)])
def test_noalloc_history_sums_match_handle(torch_cuda, precision, tol):
    torch = torch_cuda
    from paper_2107_03550_gb300.sbiem import Fault, history_sums_noalloc
    from paper_2107_03550_gb300.workloads import random_history, rough_fault
    w = rough_fault(2048, 10.0, 3e-3, seed=21)
    g = Fault.from_workload(w, precision=precision)
    R = np.maximum(g.windows() - 1, 0)
    HT, HN, _ = random_history(R, 5, 1e-3)
    g.set_history(HT, HN)
    b = _caller_buffers(torch, g, w, HT, HN, precision)
    stream = torch.cuda.current_stream()
    for m in (1, 2):   # two calls in a row share the static scratch
        ref_T, ref_N = g.history_sums(m)
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
        assert np.abs(at - ref_T).max() <= tol * np.abs(ref_T).max(), m
        assert np.abs(an - ref_N).max() <= tol * np.abs(ref_N).max(), m
    g.close()


def test_noalloc_rejects_oversized_input(torch_cuda):
    from paper_2107_03550_gb300.sbiem import SbiemError, history_sums_noalloc
    with pytest.raises(SbiemError) as ei:
        history_sums_noalloc(10 ** 6, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1)
    assert ei.value.code == -1
