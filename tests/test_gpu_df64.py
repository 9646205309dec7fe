"""Double-float form: complex128 transforms whose butterflies run in
double-float arithmetic (pairs of floats, ~48 significant bits) on the FP32
pipes.  Same tolerance as the FP64 path: relative L2 <= 1e-12 against the
FP64 oracle."""
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



def run(x, direction=M.FFT_FORWARD, adjoint=False, inplace=False, rows=None, schedule=None):
    batch, n = x.shape
    d_in = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    d_out = d_in if inplace else torch.empty_like(d_in)
    p = M.fft_plan_ex(n, batch, M.FFT_C128, direction, M.FFT_FORM_DF64, schedule)
    try:
        (M.fft_exec_adjoint if adjoint else M.fft_exec)(p, d_in, d_out)
        M.fft_plan_check(p)
        assert '"form": "df64"' in M.fft_plan_describe(p)
    finally:
        M.fft_destroy(p)
    out = d_out if rows is None else d_out[rows]
    return out.cpu().numpy()


@pytest.mark.parametrize("t", [4, 5, 8, 10, 11, 12, 13, 16])
def test_df64_sizes(t):
    n = 1 << t
    x = W.uniform_complex(n, 3, seed=300 + t)
    for direction, op in ((M.FFT_FORWARD, "forward"), (M.FFT_INVERSE, "inverse")):
        err = err_rows(run(x, direction), O.fft(x, op, c=64))
        assert err.max() <= 1e-12, (t, op, err.max())
    err = err_rows(run(x, M.FFT_INVERSE, adjoint=True), O.fft(x, "adjoint_inverse", c=64))
    assert err.max() <= 1e-12
    err = err_rows(run(x, inplace=True), O.fft(x, "forward", c=64))
    assert err.max() <= 1e-12


@pytest.mark.parametrize("t,sched", [(13, "4,4,5"), (16, "8,8"), (16, "4,12"), (20, "12,8"), (22, None),
                                     (24, "8,8,8")])
def test_df64_pass_boundaries(t, sched):
    """Every pass boundary of the double-float form: the first pass reads
    complex128 and leaves (hi, lo) float pairs in the workspace, middle
    passes read and write pairs, the last reads pairs and writes complex128
    -- through the generic tiles (a shorter first digit, then radix-16
    digits) and the one-loop tiles of 2^8 / 2^12 points, in either order,
    forward and inverse."""
    n = 1 << t
    x = W.uniform_complex(n, 2, seed=400 + t)
    for direction, op in ((M.FFT_FORWARD, "forward"), (M.FFT_INVERSE, "inverse")):
        err = err_rows(run(x, direction, schedule=sched), O.fft(x, op, c=1024, threads=2))
        assert err.max() <= 1e-12, (t, sched, op, err.max())


def test_df64_closed_forms_n1024():
    n = 1024
    k = np.arange(n)
    cf = W.closed_form_inputs(n)
    X = np.stack([cf[key] for key in ("delta0", "delta5", "const", "cos37")])
    Y = run(X)
    exact = np.zeros((4, n), complex)
    exact[0] = 1.0
    exact[1] = np.exp(-2j * np.pi * ((5 * k) % n) / n)
    exact[2, 0] = n
    exact[3, 37] = exact[3, n - 37] = n / 2
    assert np.abs(Y - exact).max() < 1e-11 * n


def test_df64_full_size_sampled():
    n, batch = 1 << 20, 64
    x = W.uniform_complex(n, batch, seed=0)
    picks = [0, 33, 63]
    y = run(x, rows=picks)
    ref = O.fft(x[picks], "forward", c=1024, threads=3)
    assert err_rows(y, ref).max() <= 1e-12


def test_df64_rejects_small_and_c64():
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_plan_ex(8, 1, M.FFT_C128, M.FFT_FORWARD, M.FFT_FORM_DF64)
    assert e.value.status == M.FFT_ERR_UNSUPPORTED
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_plan_ex(1024, 1, M.FFT_C64, M.FFT_FORWARD, M.FFT_FORM_DF64)
    assert e.value.status == M.FFT_ERR_UNSUPPORTED


def test_df64_dynamic_range_input():
    """Amplitudes log-uniform over 1e-4..1e4 (the precision-form input):
    the double-float form keeps the FP64 tolerance."""
    n = 1 << 16
    x = W.dynamic_range_complex(n, 4, seed=0)
    assert err_rows(run(x), O.fft(x, "forward", c=1024, threads=4)).max() <= 1e-12


@pytest.mark.parametrize("scale", [1e-25, 1e30])
def test_df64_inside_the_fp32_exponent_range(scale):
    """Inputs scaled far from 1 but inside the range the header states
    (every value and partial sum between about 2e-31 and 3.4e38): the FP64
    tolerance holds."""
    n = 1024
    x = W.uniform_complex(n, 3, seed=31) * scale
    for direction, op in ((M.FFT_FORWARD, "forward"), (M.FFT_INVERSE, "inverse")):
        assert err_rows(run(x, direction), O.fft(x, op, c=64)).max() <= 1e-12


def test_df64_outside_the_fp32_exponent_range():
    """What the header documents beyond that range, checked as stated: near
    1e-35 the low float falls into FP32's subnormals and the result is only
    about single-precision accurate (still within the FP32 form's tolerance);
    a result beyond 3.4e38 is infinite (n times a constant 1e36)."""
    n = 1024
    x = W.uniform_complex(n, 2, seed=32) * 1e-35
    err = err_rows(run(x), O.fft(x, "forward", c=64))
    assert err.max() <= 1e-6 * 10
    big = np.full((1, n), 1e36, dtype=np.complex128)
    y = run(big)
    assert np.isinf(y[0, 0].real)
