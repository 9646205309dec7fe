"""Failure handling made on the host: allocation failures injected through
the allocator hook, memory routed through a caller's pool, and the plan's
device-side error word in its healthy state.  Nothing here faults, traps or
hangs a GPU."""
import numpy as np
import pytest

import oracle as O
import paper_0803_2386_gb300 as M
import workloads as W

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
        err = np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-12
    finally:
        M.fft_set_allocator(None, None)


def test_allocator_hook_needs_both_functions():
    with pytest.raises(M.MoaFFTError) as e:
        M._check(M.lib().fft_set_allocator(M.ALLOC_FN(lambda n, c: 0), M.FREE_FN(), None))
    assert e.value.status == M.FFT_ERR_ARG
