"""fft_exec_noalloc, the transform that allocates no device memory.

It exists for callers that cannot call cudaMalloc (inside another framework's
allocator callback, in real-time loops that must not block on allocation, or
with device memory owned by someone else's pool); it keeps its tables and
inter-pass buffer in a fixed 32 MiB array inside the library.  These checks
compare it with the FP64 oracle and with a plan's fft_exec on the same input,
for two calls in a row (the second call finds the first call's leftovers in
the shared array), check that a call leaves the device's free memory
unchanged, and that the array's error word reads clean afterwards.

The file's name makes pytest collect it last, so a run that stops at the
first failure has already run every other test.
"""
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


def oracle_result(x, direction, rows):
    """The FP64 oracle on the (rounded) input rows."""
    xr = x[rows].cpu().numpy().astype(np.complex128)
    op = "forward" if direction == M.FFT_FORWARD else "inverse"
    return O.fft(xr, op, c=1024, threads=len(rows))


def rel_rows(a, b):
    a = np.atleast_2d(a)
    b = np.atleast_2d(b)
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


@pytest.mark.parametrize("direction", [M.FFT_FORWARD, M.FFT_INVERSE])
@pytest.mark.parametrize("dt,n,batch", [(M.FFT_C128, 1 << 20, 3), (M.FFT_C64, 1 << 21, 2),
                                        (M.FFT_C64, 1 << 16, 9), (M.FFT_C128, 1 << 13, 7),
                                        (M.FFT_C128, 1024, 5), (M.FFT_C64, 64, 33)])
def test_noalloc_matches_oracle_and_plan_two_calls(dt, n, batch, direction):
    tdt = torch.complex128 if dt == M.FFT_C128 else torch.complex64
    rows = sorted({0, batch // 2, batch - 1})
    for call, seed in enumerate((11, 12)):
        x = torch.from_numpy(W.uniform_complex(n, batch, seed=seed)).to(tdt).cuda()
        ref = plan_result(x, n, batch, dt, direction)
        got = torch.empty_like(x)
        M.fft_exec_noalloc(x, got, n, batch, dt, direction)
        torch.cuda.synchronize()
        M.fft_noalloc_check()
        # against the FP64 oracle, sampled rows: relative L2 and element-wise
        y = got[rows].cpu().numpy().astype(np.complex128)
        want = oracle_result(x, direction, rows)
        assert rel_rows(y, want).max() <= tol(dt, n), call
        assert np.abs(y - want).max() <= tol(dt, n) * np.abs(want).max(), call
        # against the plan on every row
        err = (torch.linalg.vector_norm(got - ref, dim=-1) /
               torch.linalg.vector_norm(ref, dim=-1)).max().item()
        assert err <= tol(dt, n), (call, err)


@pytest.mark.parametrize("dt,n,batch", [(M.FFT_C128, 1 << 15, 4), (M.FFT_C64, 1024, 5)])
def test_noalloc_in_place(dt, n, batch):
    """In place, for a two-pass length and for a one-pass length."""
    tdt = torch.complex128 if dt == M.FFT_C128 else torch.complex64
    x = torch.from_numpy(W.uniform_complex(n, batch, seed=5)).to(tdt).cuda()
    want = oracle_result(x, M.FFT_FORWARD, list(range(batch)))
    ref = plan_result(x, n, batch, dt, M.FFT_FORWARD)
    M.fft_exec_noalloc(x, x, n, batch, dt, M.FFT_FORWARD)
    torch.cuda.synchronize()
    M.fft_noalloc_check()
    assert rel_rows(x.cpu().numpy().astype(np.complex128), want).max() <= tol(dt, n)
    err = (torch.linalg.vector_norm(x - ref, dim=-1) / torch.linalg.vector_norm(ref, dim=-1)).max()
    assert err.item() <= tol(dt, n)


@pytest.mark.parametrize("dt,n,batch", [(M.FFT_C128, 1 << 20, 2), (M.FFT_C64, 1 << 12, 16)])
def test_noalloc_leaves_free_memory_unchanged(dt, n, batch):
    """The property the entry point exists for: after a first call on this
    device, a call allocates no device memory at all."""
    tdt = torch.complex128 if dt == M.FFT_C128 else torch.complex64
    x = torch.from_numpy(W.uniform_complex(n, batch, seed=21)).to(tdt).cuda()
    y = torch.empty_like(x)
    M.fft_exec_noalloc(x, y, n, batch, dt, M.FFT_FORWARD)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    M.fft_exec_noalloc(x, y, n, batch, dt, M.FFT_FORWARD)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    M.fft_noalloc_check()


@pytest.mark.parametrize("dt,n", [(M.FFT_C128, 1 << 21), (M.FFT_C64, 1 << 22)])
def test_noalloc_rejects_sizes_beyond_the_array(dt, n):
    tdt = torch.complex128 if dt == M.FFT_C128 else torch.complex64
    x = torch.zeros(n, dtype=tdt, device="cuda")
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_exec_noalloc(x, x, n, 1, dt, M.FFT_FORWARD)
    assert e.value.status == M.FFT_ERR_UNSUPPORTED
    assert "32 MiB" in str(e.value)
