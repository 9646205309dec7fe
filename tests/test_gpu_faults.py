"""Failure handling: allocation failures injected through the allocator
hook, memory routed through a caller's pool, and a bounded device-side wait
made to run out (a wait target nothing reaches, with a short limit), which
the plan's error word reports.  Nothing here faults, traps or hangs a GPU."""
import numpy as np
import pytest

import oracle as O
import paper_0803_2386_gb300 as M
import workloads as W
from parity_check import err_one, err_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    M.build()
    yield
    M.fft_set_allocator(None, None)


@pytest.mark.parametrize("fail_at", [0, 1, 2])
def test_injected_allocation_failure(fail_at):
    """The k-th device allocation of plan creation fails: the plan reports
    FFT_ERR_ALLOC and releases everything it had allocated."""
    live = {}
    calls = {"n": 0}

    def alloc(nbytes):
        k = calls["n"]
        calls["n"] += 1
        if k == fail_at:
            return 0
        ptr = torch.cuda.caching_allocator_alloc(nbytes)
        live[ptr] = nbytes
        return ptr

    def release(ptr):
        torch.cuda.caching_allocator_delete(ptr)
        live.pop(ptr)

    M.fft_set_allocator(alloc, release)
    try:
        with pytest.raises(M.MoaFFTError) as e:
            M.fft_plan(1 << 16, 8, M.FFT_C64, M.FFT_FORWARD)  # two passes: workspace, error word, tables
        assert e.value.status == M.FFT_ERR_ALLOC
        assert "allocator returned NULL" in str(e.value)
        assert live == {}
    finally:
        M.fft_set_allocator(None, None)


def test_plan_memory_from_callers_pool():
    seen = []

    def alloc(nbytes):
        ptr = torch.cuda.caching_allocator_alloc(nbytes)
        seen.append(ptr)
        return ptr

    M.fft_set_allocator(alloc, torch.cuda.caching_allocator_delete)
    try:
        n = 1 << 14
        x = W.uniform_complex(n, 3, seed=1)
        d = torch.from_numpy(x).cuda()
        out = torch.empty_like(d)
        p = M.fft_plan(n, 3, M.FFT_C128, M.FFT_FORWARD)
        M.fft_exec(p, d, out)
        M.fft_plan_check(p)
        M.fft_destroy(p)
        assert len(seen) >= 2
        ref = O.fft(x, "forward", c=64)
        assert err_rows(out.cpu().numpy(), ref).max() <= 1e-12
    finally:
        M.fft_set_allocator(None, None)


def test_allocator_hook_needs_both_functions():
    with pytest.raises(M.MoaFFTError) as e:
        M._check(M.lib().fft_set_allocator(M.ALLOC_FN(lambda n, c: 0), M.FREE_FN(), None))
    assert e.value.status == M.FFT_ERR_ARG


def test_persistent_wait_runs_out_and_recovers(monkeypatch):
    """A bounded device-side wait that runs out, made on purpose without any
    fault: the persistent uneven-batch kernel's second-pass tiles wait on a
    round counter; fft_plan_set_wait raises every wait's target by one (a
    count no tile reaches -- a flag that nothing sets) and limits the wait to
    1e5 SM cycles (about 50 us).  Every such wait gives up, the kernel
    records FFT_ERR_TIMEOUT, skips those tiles and finishes; fft_plan_check
    reports the timeout and clears it; with the default waits restored the
    same plan runs again and matches the oracle."""
    monkeypatch.setenv("MOAFFT_PERSIST", "1")
    sizes, data = W.uneven_batch(count=200, seed=8, lo_exp=13, hi_exp=15)  # two-pass lengths only
    d_in = torch.from_numpy(data).to(torch.complex64).cuda()
    d_out = torch.empty_like(d_in)
    p = M.fft_plan_many(sizes, M.FFT_C64, M.FFT_FORWARD)
    try:
        assert '"persistent": true' in M.fft_plan_describe(p)
        M.fft_plan_set_wait(p, 100000, 1)
        M.fft_exec(p, d_in, d_out)
        with pytest.raises(M.MoaFFTError) as e:
            M.fft_plan_check(p)
        assert e.value.status == M.FFT_ERR_TIMEOUT
        M.fft_plan_check(p)  # the flag was cleared; the context still answers
        M.fft_plan_set_wait(p)  # default limit, reachable targets
        M.fft_exec(p, d_in, d_out)
        M.fft_plan_check(p)
        y = d_out.cpu().numpy().astype(np.complex128)
    finally:
        M.fft_destroy(p)
    xr = data.astype(np.complex64).astype(np.complex128)
    at = 0
    for n in sizes.tolist():
        ref = O.fft(xr[None, at:at + n], "forward", c=1024)[0]
        err = err_one(y[at:at + n], ref)
        assert err <= 1e-6 * np.log2(n), (n, err)
        at += n


def test_set_wait_rejects_plans_without_a_persistent_launch():
    p = M.fft_plan(1 << 14, 2, M.FFT_C64, M.FFT_FORWARD)
    try:
        with pytest.raises(M.MoaFFTError) as e:
            M.fft_plan_set_wait(p, 1000, 0)
        assert e.value.status == M.FFT_ERR_UNSUPPORTED
    finally:
        M.fft_destroy(p)
