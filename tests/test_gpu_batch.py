"""Ensembles (uneven N) in batched launches vs the same faults stepped one by
one, and vs the FP64 oracle for one member."""
import numpy as np
import pytest

from paper_2107_03550_gb300.workloads import rough_fault
from tests.gpu_helpers import compare, gpu_for, oracle_for, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ensemble(seed0=100):
    rng = np.random.default_rng(seed0)
    out = []
    for k, N in enumerate((256, 512, 256, 1024, 512, 256)):
        out.append(rough_fault(N, 10.0, float(rng.uniform(1e-3, 1e-2)), seed=seed0 + k))
    return out


@pytest.mark.parametrize("precision,tol,overlap", [(0, 1e-12, False), (1, 1e-5, False), (0, 1e-12, True),
                                                   (1, 1e-5, True)])
def test_batch_equals_individual_steps(precision, tol, overlap):
    from paper_2107_03550_gb300.sbiem import Batch
    ws = _ensemble()
    solo = [gpu_for(w, precision=precision) for w in ws]
    mem = [gpu_for(w, precision=precision) for w in ws]
    b = Batch(mem)
    assert b.set_overlap(overlap) is False  # a new batch steps without overlap
    steps = 40
    b.enqueue(steps)
    fl, sd = b.status()
    assert np.all(fl == 0) and np.all(sd == steps)
    for g in solo:
        g.enqueue(steps)
        assert g.status()[0] == 0
    for g1, g2 in zip(solo, mem):
        s1, s2 = g1.get_state(), g2.get_state()
        for k in ("delta", "V", "theta", "tau_el", "sigma_el"):
            assert rel(s2[k], s1[k]) <= tol, k
    b.close()


def test_batch_member_matches_oracle_and_tuner_keeps_results():
    from paper_2107_03550_gb300.sbiem import Batch
    ws = _ensemble(200)
    mem = [gpu_for(w) for w in ws]
    o = oracle_for(ws[3])
    b = Batch(mem)
    chunk, blocks, ms = b.tune(reps=3)
    assert chunk in (256, 512, 1024, 2048, 4096, 8192) and blocks >= 1 and ms > 0
    b.enqueue(30)
    for _ in range(30):
        assert o.step() == 0
    assert np.all(b.status()[0] == 0)
    err = compare(o, mem[3])
    for k in ("delta", "tau_el", "sigma_el"):
        assert err[k] < 1e-10, (k, err)
    b.close()


def test_failed_member_stops_alone():
    from paper_2107_03550_gb300.sbiem import Batch
    ws = _ensemble(300)
    mem = [gpu_for(w, newton_maxit=(1 if k == 2 else 50)) for k, w in enumerate(ws)]
    b = Batch(mem)
    b.enqueue(5)
    fl, sd = b.status()
    assert fl[2] != 0 and sd[2] == 0
    assert np.all(np.delete(fl, 2) == 0) and np.all(np.delete(sd, 2) == 5)
    b.close()


def test_persistent_barrier_limit_rejects_the_step_and_recovers():
    # The ensemble's history convolution runs as one persistent cooperative
    # launch with a grid barrier between the sweep and the per-mode sums.
    # With a barrier limit of zero polls every CTA but the last to arrive
    # gives up at once (no fault involved) and flags every member: the step
    # is rejected for all of them with nothing committed.  With the default
    # limit back the batch steps bitwise like an untouched one.
    from paper_2107_03550_gb300.sbiem import FLAG_WAIT, Batch
    ws = _ensemble(400)
    mem = [gpu_for(w, precision=1) for w in ws]
    ref = [gpu_for(w, precision=1) for w in ws]
    b, bref = Batch(mem), Batch(ref)
    before = [g.get_state() for g in mem]
    b.set_wait_limit(0)
    b.enqueue(2)
    fl, sd = b.status()
    assert np.all(fl & FLAG_WAIT) and np.all(sd == 0)
    for g, s0 in zip(mem, before):
        s1 = g.get_state()
        for k in ("delta", "V", "theta"):
            assert np.array_equal(s0[k], s1[k]), k
        g.status(clear=True)
    b.set_wait_limit()
    b.enqueue(10)
    bref.enqueue(10)
    fl, sd = b.status()
    assert np.all(fl == 0) and np.all(sd == 10)
    for g1, g2 in zip(mem, ref):
        s1, s2 = g1.get_state(), g2.get_state()
        for k in ("delta", "V", "theta", "tau_el", "sigma_el"):
            assert np.array_equal(s1[k], s2[k]), k
    b.close()
    bref.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_two_launch_form_equals_persistent_and_weights_shared(precision):
    # The members share their weights: equal dx, material and dt_min give
    # mode n of N the wavenumber of mode 4n of 4N, and every window of the
    # smaller members is no longer than the N = 1024 member's, so all read
    # that member's weight array (a prefix of each mode's run).  The two-launch form (sweep,
    # then the per-(member, mode) sums in a second launch) partitions the chunks
    # the same way and adds in the same order as the persistent launch, so the
    # two step bitwise alike.
    from paper_2107_03550_gb300.sbiem import Batch
    ws = _ensemble(500)
    a = [gpu_for(w, precision=precision) for w in ws]
    c = [gpu_for(w, precision=precision) for w in ws]
    ba, bc = Batch(a), Batch(c)
    info = ba.get_sweep()
    assert info["persistent"] and info["distinct_weights"] == 1
    assert bc.set_persistent(False) is True
    assert bc.get_sweep()["persistent"] is False
    ba.enqueue(12)
    bc.enqueue(12)
    for b in (ba, bc):
        fl, sd = b.status()
        assert np.all(fl == 0) and np.all(sd == 12)
    for g1, g2 in zip(a, c):
        s1, s2 = g1.get_state(), g2.get_state()
        for k in ("delta", "V", "theta", "tau_el", "sigma_el"):
            assert np.array_equal(s1[k], s2[k]), k
    ba.close()
    bc.close()


def test_batch_tuner_choice_is_reported_and_keeps_results():
    # the tuner picks the sweep shape with its chunk length (the ensemble
    # builds a chunk table per length), the weight form and the CTAs per SM;
    # the step stays that of the solo handles to FP32 rounding
    from paper_2107_03550_gb300.sbiem import Batch
    ws = _ensemble(600)
    solo = [gpu_for(w, precision=1) for w in ws]
    mem = [gpu_for(w, precision=1) for w in ws]
    b = Batch(mem)
    chunk, blocks, ms = b.tune(reps=3)
    info = b.get_sweep()
    # the chunk length goes with the shape (FP32: 512 lags for shapes 0 and
    # 2, 1024 for shape 1, 2048 for shapes 3 and 4)
    assert info["ctas_per_sm"] == blocks
    assert chunk == {0: 512, 1: 1024, 2: 512, 3: 2048, 4: 2048}[info["shape"]]
    assert info["gen_ds_max"] in (0.0, 1.0 / 256, 1.0 / 64, 1.0 / 32)
    b.enqueue(20)
    assert np.all(b.status()[0] == 0)
    for g in solo:
        g.enqueue(20)
    for g1, g2 in zip(solo, mem):
        s1, s2 = g1.get_state(), g2.get_state()
        for k in ("delta", "V", "theta", "tau_el", "sigma_el"):
            assert rel(s2[k], s1[k]) <= 1e-5, k
    b.close()


def test_weight_sharing_only_where_the_weights_agree():
    # Sharing needs equal dx (equal wavenumbers for modes n and 2^p n) and one
    # cutting plane (each field's window the mode's): members with another dx
    # or a second plane keep their own weights, and every member still steps
    # as it does alone.
    from paper_2107_03550_gb300.sbiem import Batch
    base = [rough_fault(N, 10.0, 3e-3, seed=700 + k) for k, N in enumerate((256, 512, 1024))]
    other_dx = rough_fault(512, 5.0, 3e-3, seed=710)
    ws = base + [other_dx]
    kw = [{}, {}, {}, {}]
    kw.append({"kcN_L": 400.0})
    ws.append(rough_fault(512, 10.0, 3e-3, seed=711))
    solo = [gpu_for(w, precision=1, **k) for w, k in zip(ws, kw)]
    mem = [gpu_for(w, precision=1, **k) for w, k in zip(ws, kw)]
    b = Batch(mem)
    # the three of dx = 10 m share the N = 1024 member's weights; the dx = 5 m
    # member and the two-plane member read their own
    assert b.get_sweep()["distinct_weights"] == 3
    b.enqueue(15)
    assert np.all(b.status()[0] == 0)
    for g in solo:
        g.enqueue(15)
    for g1, g2 in zip(solo, mem):
        s1, s2 = g1.get_state(), g2.get_state()
        for k in ("delta", "V", "theta", "tau_el", "sigma_el"):
            assert rel(s2[k], s1[k]) <= 1e-5, k
    b.close()


@pytest.mark.parametrize("chunk_slots", [512, 1024])
def test_batch_with_another_chunk_length_equals_solo(chunk_slots):
    # a batch cut into shorter chunks than its members' (its own chunk table)
    # steps like the solo handles
    from paper_2107_03550_gb300.sbiem import Batch
    ws = _ensemble(800)
    solo = [gpu_for(w, precision=1) for w in ws]
    mem = [gpu_for(w, precision=1) for w in ws]
    b = Batch(mem, chunk_slots=chunk_slots)
    b.enqueue(12)
    assert np.all(b.status()[0] == 0)
    for g in solo:
        g.enqueue(12)
    for g1, g2 in zip(solo, mem):
        s1, s2 = g1.get_state(), g2.get_state()
        for k in ("delta", "V", "theta", "tau_el", "sigma_el"):
            assert rel(s2[k], s1[k]) <= 1e-5, k
    b.close()
