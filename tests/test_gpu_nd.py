"""Multi-dimensional transforms (fft_plan_nd) against the oracle's fftn on
the same seeded inputs: the last axis as 1-D transforms, every other axis as
one column pass without pass weights or, for long axes, two passes (the
axis's 1-D schedule over its strided lines).  Tolerances as the 1-D parity
tests, with log2 of the points per array: relative L2 per array <= 1e-12
(complex128), 1e-6 * log2 N (complex64)."""
import json
import math

import numpy as np
import pytest

import oracle as O
import paper_0803_2386_gb300 as M
import workloads as W
from parity_check import err_arrays, err_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    M.build()
    yield


def tol(dt, n):
    return 1e-12 if dt == M.FFT_C128 else 1e-6 * max(1, int(math.log2(n)))



def seeded(batch, dims, seed):
    n = math.prod(dims)
    return W.uniform_complex(n, batch, seed=seed).reshape((batch,) + tuple(dims))


def rounded(x, dt):
    return x if dt == M.FFT_C128 else x.astype(np.complex64).astype(np.complex128)


def run_nd(x, dims, dt, direction=M.FFT_FORWARD, adjoint=False, inplace=False):
    batch = x.shape[0]
    d_in = torch.from_numpy(np.ascontiguousarray(x)).to(
        torch.complex128 if dt == M.FFT_C128 else torch.complex64).cuda()
    d_out = d_in if inplace else torch.empty_like(d_in)
    p = M.fft_plan_nd(dims, batch, dt, direction)
    try:
        (M.fft_exec_adjoint if adjoint else M.fft_exec)(p, d_in, d_out)
        M.fft_plan_check(p)
    finally:
        M.fft_destroy(p)
    return d_out.cpu().numpy().astype(np.complex128)


SHAPES = [(16, 64), (64, 16), (8, 4, 32), (2, 2, 2, 8), (4096, 16), (16, 4096), (32, 1 << 14),
          (2, 1 << 17), (4, 1, 32), (1, 256), (8, 8, 8, 8), (1 << 12, 1 << 10), (512, 64),
          (1 << 14, 8), (1 << 16, 4), (2, 1024, 32), (1024, 2, 8), (1 << 20, 2)]


@pytest.mark.parametrize("dt", [M.FFT_C128, M.FFT_C64])
@pytest.mark.parametrize("dims", SHAPES)
def test_nd_forward_inverse(dt, dims):
    n = math.prod(dims)
    batch = 3 if n <= (1 << 16) else 1
    x = seeded(batch, dims, 400 + len(dims) + n % 97)
    xr = rounded(x, dt)
    ops = (("forward", M.FFT_FORWARD, False), ("inverse", M.FFT_INVERSE, False),
           ("adjoint_forward", M.FFT_FORWARD, True))
    for op, direction, adjoint in ops:
        y = run_nd(x, dims, dt, direction, adjoint)
        ref = O.fftn(xr, ndim=len(dims), op=op, c=64, threads=4)
        err = err_arrays(y, ref)
        assert err.max() <= tol(dt, n), (dims, op, err.max())


@pytest.mark.parametrize("dt", [M.FFT_C128, M.FFT_C64])
def test_nd_in_place_and_roundtrip(dt):
    dims = (32, 8, 64)
    x = seeded(2, dims, 77)
    y = run_nd(x, dims, dt, inplace=True)
    assert err_arrays(y, O.fftn(rounded(x, dt), ndim=3, c=64)).max() <= tol(dt, 32 * 8 * 64)
    back = run_nd(y, dims, dt, M.FFT_INVERSE, inplace=True)
    assert err_arrays(back, rounded(x, dt)).max() <= 2 * tol(dt, 32 * 8 * 64)


def test_nd_closed_forms_c128():
    dims = (64, 32, 16)
    n = math.prod(dims)
    delta = np.zeros((1,) + dims, complex)
    delta[0, 0, 0, 0] = 1
    assert np.abs(run_nd(delta, dims, M.FFT_C128) - 1).max() < 1e-14
    f = (5, 31, 3)
    grids = np.meshgrid(*[np.arange(s) for s in dims], indexing="ij")
    wave = np.exp(2j * np.pi * sum(fj * g / s for fj, g, s in zip(f, grids, dims)))[None]
    X = run_nd(wave, dims, M.FFT_C128)
    expect = np.zeros_like(X)
    expect[(0,) + f] = n
    assert np.abs(X - expect).max() < 1e-9


def test_nd_plan_structure_and_wrappers():
    dims = (8, 16, 1024)
    p = M.fft_plan_nd(dims, 4, M.FFT_C64, M.FFT_FORWARD)
    try:
        d = json.loads(M.fft_plan_describe(p))
        assert d["dims"] == list(dims) and d["n"] == 8 * 16 * 1024 and d["batch"] == 4
        assert [[(q["log_r"], q["A"], q["B"]) for q in ax] for ax in d["axes"]] == [[(3, 1, 16 * 1024)],
                                                                                   [(4, 8, 1024)]]
        assert M.fft_plan_launches(p) == 1 + 2  # one pass of the last axis, one per other axis
        host = np.zeros((4,) + dims, np.complex64)
        with pytest.raises(M.MoaFFTError, match="UNSUPPORTED"):
            M.fft_exec_host(p, host, host)
    finally:
        M.fft_destroy(p)
    # the torch wrapper over the last axes, leading axes as the batch
    x = torch.from_numpy(seeded(3, (16, 32), 5)).cuda()
    X = M.fftn(x, ndim=2)
    ref = O.fftn(seeded(3, (16, 32), 5), ndim=2)
    assert err_arrays(X.cpu().numpy(), ref).max() <= 1e-12
    assert err_arrays(M.ifftn(X, ndim=2).cpu().numpy(), seeded(3, (16, 32), 5)).max() <= 1e-12


def test_nd_long_axis_takes_two_passes():
    """A 4096-point leading axis of complex64 runs as two column passes of 64
    (weights w_4096^(b k) on the first, split by the digits of k; the axis's
    final transpose on the second) instead of one pass with tiles one column
    wide."""
    p = M.fft_plan_nd((4096, 16), 2, M.FFT_C64, M.FFT_FORWARD)
    try:
        d = json.loads(M.fft_plan_describe(p))
        (ax,) = d["axes"]
        assert [(q["log_r"], q["A"], q["B"], q["tw_mode"]) for q in ax] == [(6, 1, 64 * 16, 3), (6, 64, 16, 4)]
        assert M.fft_plan_launches(p) == 1 + 2
    finally:
        M.fft_destroy(p)


def test_nd_full_size_c64_4096_squared():
    """The bench's 2-D complex64 shape (4096 x 4096), one array against the
    oracle."""
    dims = (4096, 4096)
    x = seeded(1, dims, 9)
    y = run_nd(x, dims, M.FFT_C64)
    ref = O.fftn(rounded(x, M.FFT_C64), ndim=2, c=4096, threads=4)
    assert err_arrays(y, ref).max() <= tol(M.FFT_C64, 1 << 24)


@pytest.mark.parametrize("inverse", [False, True])
def test_nd_autograd_gradcheck_c128(inverse):
    """fftn_autograd: backward through the hand-written adjoint of the
    multi-dimensional plan, against torch's numerical Jacobian."""
    x = torch.from_numpy(seeded(2, (8, 4, 16), 21)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: M.fftn_autograd(t, ndim=3, inverse=inverse), (x,),
                                    eps=1e-6, atol=1e-9, rtol=1e-7)


def test_nd_autograd_gradient_vs_oracle_adjoint():
    """loss = ||FFTn(x) H - y||^2 on complex128 2-D arrays: the gradient is
    F^H (2 (F x H - y) conj(H)) with F^H the oracle's adjoint transform."""
    dims = (64, 128)
    rng = np.random.default_rng(5)
    xn = seeded(2, dims, 31)
    Hn = rng.standard_normal((2,) + dims) + 1j * rng.standard_normal((2,) + dims)
    yn = rng.standard_normal((2,) + dims) + 1j * rng.standard_normal((2,) + dims)
    x = torch.from_numpy(xn).cuda().requires_grad_(True)
    H = torch.from_numpy(Hn).cuda()
    y = torch.from_numpy(yn).cuda()
    loss = torch.sum(torch.abs(M.fftn_autograd(x, ndim=2) * H - y) ** 2)
    loss.backward()
    Xn = O.fftn(xn, ndim=2)
    expect = O.fftn(2 * (Xn * Hn - yn) * np.conj(Hn), ndim=2, op="adjoint_forward")
    got = x.grad.cpu().numpy()
    assert err_arrays(got[None], expect[None]).max() <= 1e-12
