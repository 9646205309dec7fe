"""The end-to-end entry point fft_exec_host (host buffers streamed through
the plan's device staging slots) against the FP64 oracle: pageable and
pinned buffers, batches that span several 64 MiB slots, in place, and the
plans it refuses."""
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



def test_pageable_complex128_every_row():
    n, batch = 1 << 12, 37
    x = W.uniform_complex(n, batch, seed=70)
    y = np.zeros_like(x)
    p = M.fft_plan(n, batch, M.FFT_C128, M.FFT_FORWARD)
    try:
        M.fft_exec_host(p, x, y)
        torch.cuda.synchronize()
    finally:
        M.fft_destroy(p)
    assert err_rows(y, O.fft(x, "forward", c=64, threads=4)).max() <= 1e-12


def test_pinned_complex64_several_slots():
    """n = 2^16 x 300 complex64 (157 MB): three staging slices overlap copy
    in, transform and copy out."""
    n, batch = 1 << 16, 300
    x = W.uniform_complex(n, batch, seed=71).astype(np.complex64)
    xin = torch.from_numpy(x).pin_memory()
    yout = torch.empty_like(xin).pin_memory()
    p = M.fft_plan(n, batch, M.FFT_C64, M.FFT_FORWARD)
    try:
        M.fft_exec_host(p, xin, yout)
        torch.cuda.synchronize()
    finally:
        M.fft_destroy(p)
    y = yout.numpy().astype(np.complex128)
    xr = x.astype(np.complex128)
    # both sides of every multiple of 16 rows (the slices, ramped at both
    # ends, start at multiples of 16 here)
    rows = sorted({0, batch - 1} | {r for b in range(16, batch, 16) for r in (b - 1, b)})
    assert err_rows(y[rows], O.fft(xr[rows], "forward", c=256, threads=4)).max() <= 1.6e-5
    ex = np.sum(np.abs(xr) ** 2, axis=-1)
    assert np.max(np.abs(np.sum(np.abs(y) ** 2, axis=-1) - n * ex) / (n * ex)) <= 1e-5


def test_in_place_inverse():
    n, batch = 1 << 10, 5
    x = W.uniform_complex(n, batch, seed=72)
    buf = x.copy()
    p = M.fft_plan(n, batch, M.FFT_C128, M.FFT_INVERSE)
    try:
        M.fft_exec_host(p, buf, buf)
        torch.cuda.synchronize()
    finally:
        M.fft_destroy(p)
    assert err_rows(buf, O.fft(x, "inverse", c=64)).max() <= 1e-12


def test_rejects_uneven_plans_and_device_pointers():
    p = M.fft_plan_many([16, 32], M.FFT_C64)
    try:
        buf = np.zeros(48, dtype=np.complex64)
        with pytest.raises(M.MoaFFTError) as e:
            M.fft_exec_host(p, buf, buf)
        assert e.value.status == M.FFT_ERR_UNSUPPORTED
    finally:
        M.fft_destroy(p)
    p = M.fft_plan(16, 1, M.FFT_C64, M.FFT_FORWARD)
    try:
        d = torch.zeros(16, dtype=torch.complex64, device="cuda")
        with pytest.raises(M.MoaFFTError) as e:
            M.fft_exec_host(p, d, d)
        assert e.value.status == M.FFT_ERR_ARG
    finally:
        M.fft_destroy(p)


def test_chained_calls_are_stream_ordered():
    """Forward then inverse through host buffers on one stream, the second
    call reading the first call's output, with no synchronisation between
    them: the second call's copies start after the first call's work."""
    n, batch = 1 << 16, 512
    x = W.uniform_complex(n, batch, seed=73).astype(np.complex64)
    xin = torch.from_numpy(x).pin_memory()
    mid = torch.empty_like(xin).pin_memory()
    back = torch.empty_like(xin).pin_memory()
    pf = M.fft_plan(n, batch, M.FFT_C64, M.FFT_FORWARD)
    pi = M.fft_plan(n, batch, M.FFT_C64, M.FFT_INVERSE)
    try:
        s = torch.cuda.Stream()
        M.fft_exec_host(pf, xin, mid, s)
        M.fft_exec_host(pi, mid, back, s)
        s.synchronize()
    finally:
        M.fft_destroy(pf)
        M.fft_destroy(pi)
    err = err_rows(back.numpy().astype(np.complex128), x.astype(np.complex128))
    assert err.max() <= 1e-6 * 16


def test_pinned_complex128_ramped_slices():
    """complex128 n = 2^20 x 9 through 64 MiB slots of 4 transforms: the
    slices ramp up and down (1, 2, 3, 2, 1 transforms), every transform
    against the oracle."""
    n, batch = 1 << 20, 9
    x = W.uniform_complex(n, batch, seed=72)
    xin = torch.from_numpy(x).pin_memory()
    yout = torch.empty_like(xin).pin_memory()
    p = M.fft_plan(n, batch, M.FFT_C128, M.FFT_FORWARD)
    try:
        M.fft_exec_host(p, xin, yout)
        torch.cuda.synchronize()
    finally:
        M.fft_destroy(p)
    assert err_rows(yout.numpy(), O.fft(x, "forward", c=1024, threads=4)).max() <= 1e-12
