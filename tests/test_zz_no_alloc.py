"""fft_exec_noalloc, the transform that allocates no device memory.

It exists for callers that cannot call cudaMalloc (inside another framework's
allocator callback, in real-time loops that must not block on allocation, or
with device memory owned by someone else's pool); it keeps its tables and
inter-pass buffer in a fixed 32 MiB array inside the library.  These checks
compare it with a plan's fft_exec on the same input, for two calls in a row
(the second call finds the first call's leftovers in the shared array).

The file's name makes pytest collect it last, so a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

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


def tol(dt, n):
    return 1e-12 if dt == M.FFT_C128 else 1e-6 * max(1, int(np.log2(n)))


def plan_result(x, n, batch, dt, direction):
    out = torch.empty_like(x)
    p = M.fft_plan(n, batch, dt, direction)
    try:
        M.fft_exec(p, x, out)
        torch.cuda.synchronize()
    finally:
        M.fft_destroy(p)
    return out


@pytest.mark.parametrize("direction", [M.FFT_FORWARD, M.FFT_INVERSE])
@pytest.mark.parametrize("dt,n,batch", [(M.FFT_C128, 1 << 20, 3), (M.FFT_C64, 1 << 21, 2),
                                        (M.FFT_C64, 1 << 16, 9), (M.FFT_C128, 1 << 13, 7),
                                        (M.FFT_C128, 1024, 5), (M.FFT_C64, 64, 33)])
def test_noalloc_matches_plan_two_calls(dt, n, batch, direction):
    tdt = torch.complex128 if dt == M.FFT_C128 else torch.complex64
    for call, seed in enumerate((11, 12)):
        x = torch.from_numpy(W.uniform_complex(n, batch, seed=seed)).to(tdt).cuda()
        ref = plan_result(x, n, batch, dt, direction)
        got = torch.empty_like(x)
        M.fft_exec_noalloc(x, got, n, batch, dt, direction)
        torch.cuda.synchronize()
        err = (torch.linalg.vector_norm(got - ref, dim=-1) /
               torch.linalg.vector_norm(ref, dim=-1)).max().item()
        assert err <= tol(dt, n), (call, err)


def test_noalloc_in_place():
    n, batch = 1 << 15, 4
    x = torch.from_numpy(W.uniform_complex(n, batch, seed=5)).cuda()
    ref = plan_result(x, n, batch, M.FFT_C128, M.FFT_FORWARD)
    M.fft_exec_noalloc(x, x, n, batch, M.FFT_C128, M.FFT_FORWARD)
    torch.cuda.synchronize()
    err = (torch.linalg.vector_norm(x - ref, dim=-1) / torch.linalg.vector_norm(ref, dim=-1)).max()
    assert err.item() <= 1e-12


@pytest.mark.parametrize("dt,n", [(M.FFT_C128, 1 << 21), (M.FFT_C64, 1 << 22)])
def test_noalloc_rejects_sizes_beyond_the_array(dt, n):
    tdt = torch.complex128 if dt == M.FFT_C128 else torch.complex64
    x = torch.zeros(n, dtype=tdt, device="cuda")
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_exec_noalloc(x, x, n, 1, dt, M.FFT_FORWARD)
    assert e.value.status == M.FFT_ERR_UNSUPPORTED
    assert "32 MiB" in str(e.value)
