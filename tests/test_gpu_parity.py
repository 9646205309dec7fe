"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.  Tolerances (relative L2 per transform): FP64 path
1e-12; FP32 path 1e-6 * log2 n."""
import json

import numpy as np
import pytest

import oracle as O
import paper_0803_2386_gb300 as M
import workloads as W
from parity_check import err_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    M.build()
    yield


def tol(dt, n):
    t = max(1, int(np.log2(max(n, 1))))
    return 1e-12 if dt == M.FFT_C128 else 1e-6 * t



def to_dev(x, dt):
    t = torch.from_numpy(np.ascontiguousarray(x))
    t = t.to(torch.complex128 if dt == M.FFT_C128 else torch.complex64)
    return t.cuda()


def run_plan(x, dt, direction=M.FFT_FORWARD, adjoint=False, schedule=None, inplace=False):
    """x: batch x n complex128 numpy.  Returns numpy complex128."""
    batch, n = x.shape
    d_in = to_dev(x, dt)
    d_out = d_in if inplace else torch.empty_like(d_in)
    p = M.fft_plan_ex(n, batch, dt, direction, M.FFT_FORM_PLAIN, schedule)
    try:
        if adjoint:
            M.fft_exec_adjoint(p, d_in, d_out)
        else:
            M.fft_exec(p, d_in, d_out)
        torch.cuda.synchronize()
    finally:
        M.fft_destroy(p)
    return d_out.cpu().numpy().astype(np.complex128)


def oracle_op(x, direction, adjoint):
    if direction == M.FFT_FORWARD:
        op = "adjoint_forward" if adjoint else "forward"
    else:
        op = "adjoint_inverse" if adjoint else "inverse"
    return O.fft(x, op, c=64, threads=4)


def rounded(x, dt):
    return x if dt == M.FFT_C128 else x.astype(np.complex64).astype(np.complex128)


# ---------------------------------------------------------------- config 1

def test_c1_uniform_n1024():
    x = W.uniform_complex(1024, 1, seed=0)
    y = run_plan(x, M.FFT_C128)
    assert err_rows(y, O.fft(x, "forward"))[0] <= 1e-12


def test_c1_closed_forms():
    n = 1024
    k = np.arange(n)
    cf = W.closed_form_inputs(n)
    X = np.stack([cf[key] for key in ("delta0", "delta5", "const", "cos37", "sin37")])
    Y = run_plan(X, M.FFT_C128)
    exact = np.zeros((5, n), complex)
    exact[0] = 1.0
    exact[1] = np.exp(-2j * np.pi * ((5 * k) % n) / n)
    exact[2, 0] = n
    exact[3, 37] = exact[3, n - 37] = n / 2
    exact[4, 37], exact[4, n - 37] = -0.5j * n, 0.5j * n
    assert np.abs(Y - exact).max() < 1e-11 * n


# ------------------------------------------------------- sizes and forms

@pytest.mark.parametrize("dt", [M.FFT_C128, M.FFT_C64])
@pytest.mark.parametrize("t", list(range(0, 17)))
def test_sizes_forward_inverse(dt, t):
    n = 1 << t
    batch = 3 if t > 12 else 5  # odd batches leave a ragged last tile
    x = W.uniform_complex(n, batch, seed=100 + t)
    xr = rounded(x, dt)
    for direction in (M.FFT_FORWARD, M.FFT_INVERSE):
        y = run_plan(x, dt, direction)
        err = err_rows(y, oracle_op(xr, direction, False))
        assert err.max() <= tol(dt, n), (t, direction, err.max())


@pytest.mark.parametrize("dt", [M.FFT_C128, M.FFT_C64])
@pytest.mark.parametrize("direction", [M.FFT_FORWARD, M.FFT_INVERSE])
@pytest.mark.parametrize("t", [1, 5, 10, 13])
def test_adjoint(dt, direction, t):
    n = 1 << t
    x = W.gaussian_complex(n, 3, seed=7 + t)
    xr = rounded(x, dt)
    y = run_plan(x, dt, direction, adjoint=True)
    err = err_rows(y, oracle_op(xr, direction, True))
    assert err.max() <= tol(dt, n)


@pytest.mark.parametrize("dt", [M.FFT_C128, M.FFT_C64])
@pytest.mark.parametrize("schedule", ["4,4,4", "6,6", "2,3,3,4", "1,11", "12@2", "4@16,4@2,4@4",
                                      "3,3,3,3;chunk=2", "11,1", "5,7;chunk=3",
                                      "6/1,6/1", "6/2,6/3", "7/3,5/2", "12/2"])
def test_forced_schedules(dt, schedule):
    n = 1 << 12
    x = W.uniform_complex(n, 7, seed=3)
    xr = rounded(x, dt)
    y = run_plan(x, dt, M.FFT_FORWARD, schedule=schedule)
    assert err_rows(y, O.fft(xr, "forward", c=64)).max() <= tol(dt, n)
    yi = run_plan(x, dt, M.FFT_INVERSE, schedule=schedule)
    assert err_rows(yi, O.fft(xr, "inverse", c=64)).max() <= tol(dt, n)


def test_two_level_twiddles_large_first_pass():
    # n = 2^22 with a 2-pass schedule puts w_{2^22} on a two-level table (c128)
    n = 1 << 22
    x = W.uniform_complex(n, 1, seed=44)
    y = run_plan(x, M.FFT_C128, schedule="11,11")
    assert err_rows(y, O.fft(x, "forward", c=1024))[0] <= 1e-12


@pytest.mark.parametrize("dt", [M.FFT_C128, M.FFT_C64])
def test_in_place(dt):
    n = 1 << 14
    x = W.uniform_complex(n, 4, seed=5)
    y = run_plan(x, dt, inplace=True)
    assert err_rows(y, O.fft(rounded(x, dt), "forward", c=64)).max() <= tol(dt, n)


# --------------------------------------------------------------- errors

def test_alias_and_pointer_errors():
    n = 1024
    buf = torch.zeros(2 * n + 16, dtype=torch.complex128, device="cuda")
    p = M.fft_plan(n, 1, M.FFT_C128, M.FFT_FORWARD)
    try:
        with pytest.raises(M.MoaFFTError) as e:
            M.fft_exec(p, buf.data_ptr(), buf.data_ptr() + 16 * 8)
        assert e.value.status == M.FFT_ERR_ALIAS
        host = np.zeros(n, np.complex128)
        with pytest.raises(M.MoaFFTError) as e:
            M.fft_exec(p, host.ctypes.data, buf.data_ptr())
        assert e.value.status == M.FFT_ERR_ARG
        with pytest.raises(M.MoaFFTError) as e:
            M.fft_exec(p, buf.data_ptr() + 8, buf.data_ptr() + 16 * 1040)
        assert e.value.status == M.FFT_ERR_ARG
    finally:
        M.fft_destroy(p)


# --------------------------------------------------- full benchmark sizes

@pytest.mark.parametrize("t", [20, 24])
def test_full_size_c128_sampled(t):
    """N * batch = 2^26 (1 GiB per buffer), the benchmark's launch
    configuration; the oracle recomputes sampled transforms in full."""
    n = 1 << t
    batch = (1 << 26) // n
    x = W.uniform_complex(n, batch, seed=0)
    d_in = to_dev(x, M.FFT_C128)
    d_out = torch.empty_like(d_in)
    p = M.fft_plan(n, batch, M.FFT_C128, M.FFT_FORWARD)
    try:
        M.fft_exec(p, d_in, d_out)
        torch.cuda.synchronize()
    finally:
        M.fft_destroy(p)
    picks = sorted({0, batch // 2, batch - 1})
    y = d_out[picks].cpu().numpy()
    ref = O.fft(x[picks], "forward", c=1024, threads=len(picks))
    assert err_rows(y, ref).max() <= 1e-12
    # every transform: Parseval, sum |X|^2 = n sum |x|^2
    ex = torch.sum(torch.abs(d_in) ** 2, dim=-1)
    eX = torch.sum(torch.abs(d_out) ** 2, dim=-1)
    assert torch.max(torch.abs(eX - n * ex) / (n * ex)).item() < 1e-12
    # the inverse plan (in place, as the benchmark's step runs it out of
    # place) against the oracle's inverse of the same sampled rows
    pi = M.fft_plan(n, batch, M.FFT_C128, M.FFT_INVERSE)
    try:
        M.fft_exec(pi, d_out, d_out)
        torch.cuda.synchronize()
    finally:
        M.fft_destroy(pi)
    yi = d_out[picks].cpu().numpy()
    refi = O.fft(y, "inverse", c=1024, threads=len(picks))
    assert err_rows(yi, refi).max() <= 1e-12
    # ... and it brings every transform back
    err = torch.linalg.vector_norm(d_out - d_in, dim=-1) / torch.linalg.vector_norm(d_in, dim=-1)
    assert err.max().item() <= 1e-12


def test_full_size_c64_sampled():
    """complex64 n = 2^16, batch 4096 (the precision-form configuration)."""
    n, batch = 1 << 16, 4096
    x = W.gaussian_complex(n, batch, seed=0)
    d_in = to_dev(x, M.FFT_C64)
    d_out = torch.empty_like(d_in)
    p = M.fft_plan(n, batch, M.FFT_C64, M.FFT_FORWARD)
    try:
        M.fft_exec(p, d_in, d_out)
        torch.cuda.synchronize()
    finally:
        M.fft_destroy(p)
    picks = [0, 1234, batch - 1]
    y = d_out[picks].cpu().numpy().astype(np.complex128)
    ref = O.fft(rounded(x[picks], M.FFT_C64), "forward", c=1024, threads=3)
    assert err_rows(y, ref).max() <= 1e-6 * 16


# ------------------------------------- unblocked routine (one pass per stage)

@pytest.mark.parametrize("order", ["stages", "stages_stride"])
@pytest.mark.parametrize("dt", [M.FFT_C128, M.FFT_C64])
@pytest.mark.parametrize("t", [0, 1, 2, 5, 10, 13])
def test_unblocked_stages(dt, t, order):
    """Schedules "stages" / "stages_stride": bit reversal, then one HBM pass
    per radix-2 stage with the hyper-cube ONF pairs, taken in unit-stride or
    in power-of-two stepping order (the paper's fftpsirad2 on the GPU)."""
    n = 1 << t
    x = W.uniform_complex(n, 3, seed=200 + t)
    xr = rounded(x, dt)
    for direction in (M.FFT_FORWARD, M.FFT_INVERSE):
        y = run_plan(x, dt, direction, schedule=order)
        assert err_rows(y, oracle_op(xr, direction, False)).max() <= tol(dt, n)
    y = run_plan(x, dt, M.FFT_FORWARD, adjoint=True, schedule=order)
    assert err_rows(y, oracle_op(xr, M.FFT_FORWARD, True)).max() <= tol(dt, n)
    y = run_plan(x, dt, M.FFT_FORWARD, schedule=order, inplace=True)
    assert err_rows(y, oracle_op(xr, M.FFT_FORWARD, False)).max() <= tol(dt, n)


def plan_passes(n, batch, dt):
    p = M.fft_plan(n, batch, dt, M.FFT_FORWARD)
    try:
        s = json.loads(M.fft_plan_describe(p))["schedule"]
    finally:
        M.fft_destroy(p)
    return [(q["log_r"], q["width"]) for q in s["passes"]]


def test_latency_schedule_for_tiny_batches():
    """A few small complex128 transforms take two passes of narrow tiles
    (many thread blocks instead of one tile with idle rows; at most 512 tiles
    in the first pass); larger batches and complex64 keep the tile passes."""
    assert plan_passes(1 << 10, 1, M.FFT_C128) == [(5, 1), (5, 1)]
    assert plan_passes(1 << 10, 32, M.FFT_C128) == [(5, 2), (5, 2)]
    assert plan_passes(1 << 6, 512, M.FFT_C128) == [(3, 8), (3, 8)]
    assert plan_passes(1 << 10, 64, M.FFT_C128) == [(10, 4)]
    assert plan_passes(1 << 10, 1, M.FFT_C64) == [(10, 4)]
    for n, batch in ((1 << 10, 32), (1 << 6, 512), (1 << 13, 3)):
        x = W.uniform_complex(n, batch, seed=5)
        for direction in (M.FFT_FORWARD, M.FFT_INVERSE):
            y = run_plan(x, M.FFT_C128, direction)
            assert err_rows(y, oracle_op(x, direction, False)).max() <= 1e-12


@pytest.mark.parametrize("t", [22, 24])
def test_large_complex64_three_passes(t):
    """Large complex64 transforms (2^22: passes of 2^7, 2^7, 2^8; 2^24:
    three of 2^8; pass weights split by the digits of k), every transform
    against the oracle."""
    n = 1 << t
    batch = 2
    x = W.uniform_complex(n, batch, seed=60 + t)
    y = run_plan(x, M.FFT_C64)
    ref = O.fft(rounded(x, M.FFT_C64), "forward", c=4096, threads=2)
    assert err_rows(y, ref).max() <= 1e-6 * t


@pytest.mark.parametrize("t,split", [(17, [8, 9]), (18, [8, 10]), (19, [9, 10]), (20, [10, 10]), (21, [7, 7, 7])])
def test_complex64_default_splits(t, split):
    """The measured complex64 default splits between 2^16 and 2^22 points,
    forward and inverse, with an odd batch (a ragged last column group),
    every transform against the oracle."""
    n = 1 << t
    s = json.loads(M.fft_describe_schedule(n, M.FFT_C64))
    assert [q["log_r"] for q in s["passes"]] == split
    x = W.uniform_complex(n, 3, seed=80 + t)
    xr = rounded(x, M.FFT_C64)
    for direction in (M.FFT_FORWARD, M.FFT_INVERSE):
        y = run_plan(x, M.FFT_C64, direction)
        err = err_rows(y, oracle_op(xr, direction, False))
        assert err.max() <= tol(M.FFT_C64, n), (t, direction, err.max())
