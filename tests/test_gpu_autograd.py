"""Differentiation form: y = FFT(x) through torch.autograd.Function whose
backward is the library's hand-written adjoint (fft_exec_adjoint).

Workload: loss = ||FFT(x) * H - y||^2, x complex64 n = 2^18, batch 256,
H and y seeded complex Gaussian.  The gradient is checked against central
finite differences (eps = 1e-3, loss in FP64; the loss is quadratic, so the
central difference is exact up to rounding) on 64 sampled coordinates, real
and imaginary parts, and against the FP64 oracle's adjoint on sampled rows."""
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


@pytest.mark.parametrize("inverse", [False, True])
def test_gradcheck_complex128(inverse):
    x = torch.from_numpy(W.gaussian_complex(16, 2, seed=1)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: M.fft_autograd(t, inverse=inverse), (x,),
                                    eps=1e-6, atol=1e-9, rtol=1e-7)


@pytest.fixture(scope="module")
def problem():
    n, batch = 1 << 18, 256
    xn, Hn, yn = W.loss_problem(n, batch)
    x = torch.from_numpy(xn).to(torch.complex64).cuda().requires_grad_(True)
    H = torch.from_numpy(Hn).to(torch.complex64).cuda()
    y = torch.from_numpy(yn).to(torch.complex64).cuda()
    X = M.fft_autograd(x)
    loss = torch.sum(torch.abs(X * H - y) ** 2)
    loss.backward()
    return n, batch, x, H, y, x.grad.detach().clone()


def loss_row_fp64(xrow, Hrow, yrow, plan, buf_in, buf_out):
    buf_in.copy_(xrow)
    M.fft_exec(plan, buf_in, buf_out)
    return torch.sum(torch.abs(buf_out * Hrow - yrow) ** 2).item()


def test_gradient_vs_central_differences(problem):
    n, batch, x, H, y, g = problem
    rng = np.random.default_rng(7)
    rows = rng.integers(0, batch, 64)
    cols = rng.integers(0, n, 64)
    plan = M.fft_plan(n, 1, M.FFT_C128, M.FFT_FORWARD)
    bi = torch.empty(n, dtype=torch.complex128, device="cuda")
    bo = torch.empty_like(bi)
    eps = 1e-3
    fd, an = [], []
    try:
        for b, j in zip(rows, cols):
            x64 = x[b].detach().to(torch.complex128)
            H64, y64 = H[b].to(torch.complex128), y[b].to(torch.complex128)
            for part, unit in (("re", 1.0), ("im", 1j)):
                xp = x64.clone()
                xp[j] += eps * unit
                lp = loss_row_fp64(xp, H64, y64, plan, bi, bo)
                xm = x64.clone()
                xm[j] -= eps * unit
                lm = loss_row_fp64(xm, H64, y64, plan, bi, bo)
                fd.append((lp - lm) / (2 * eps))
                gv = g[b, j].item()
                an.append(gv.real if part == "re" else gv.imag)
    finally:
        M.fft_destroy(plan)
    fd, an = np.array(fd), np.array(an)
    rel = np.linalg.norm(an - fd) / np.linalg.norm(fd)
    assert rel <= 2e-5, rel


def test_gradient_vs_oracle_adjoint(problem):
    n, batch, x, H, y, g = problem
    picks = [0, 137, batch - 1]
    xs = x.detach()[picks].cpu().numpy().astype(np.complex128)
    Hs = H[picks].cpu().numpy().astype(np.complex128)
    ys = y[picks].cpu().numpy().astype(np.complex128)
    X = O.fft(xs, "forward", c=1024, threads=3)
    G = 2.0 * np.conj(Hs) * (X * Hs - ys)  # grad w.r.t. X in PyTorch's convention
    ref = O.fft(G, "adjoint_forward", c=1024, threads=3)
    got = g[picks].cpu().numpy().astype(np.complex128)
    err = err_rows(got, ref)
    assert err.max() <= 2e-6 * 18, err
