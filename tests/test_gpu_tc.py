"""Precision form: radix-16 DFT digits as tensor-core (tcgen05) products with
split FP16 / BF16 operands and FP32 accumulation, complex64 data.
Tolerance (relative L2 per transform against the FP64 oracle): 1e-5 * log2 n."""
import numpy as np
import pytest

import oracle as O
import paper_0803_2386_gb300 as M
import workloads as W
from parity_check import err_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FORMS = [M.FFT_FORM_TC_FP16, M.FFT_FORM_TC_BF16]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    M.build()
    yield



def run(x, form, direction=M.FFT_FORWARD, adjoint=False, rows=None):
    batch, n = x.shape
    d_in = torch.from_numpy(x).to(torch.complex64).cuda()
    d_out = torch.empty_like(d_in)
    p = M.fft_plan_ex(n, batch, M.FFT_C64, direction, form)
    try:
        (M.fft_exec_adjoint if adjoint else M.fft_exec)(p, d_in, d_out)
        M.fft_plan_check(p)  # raises on a recorded mbarrier timeout
        desc = M.fft_plan_describe(p)
    finally:
        M.fft_destroy(p)
    assert '"form": "tc_' in desc
    out = d_out if rows is None else d_out[rows]
    return out.cpu().numpy().astype(np.complex128)


def c64(x):
    return x.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("t", [6, 7, 8, 9, 10, 11, 12, 13, 14, 16])
def test_tc_sizes(form, t):
    n = 1 << t
    x = W.gaussian_complex(n, 3, seed=t)
    ref_in = c64(x)
    for direction, op in ((M.FFT_FORWARD, "forward"), (M.FFT_INVERSE, "inverse")):
        y = run(x, form, direction)
        err = err_rows(y, O.fft(ref_in, op, c=256))
        assert err.max() <= 1e-5 * t, (t, op, err.max())


@pytest.mark.parametrize("form", FORMS)
def test_tc_adjoint(form):
    n = 1 << 12
    x = W.gaussian_complex(n, 2, seed=5)
    y = run(x, form, M.FFT_FORWARD, adjoint=True)
    assert err_rows(y, O.fft(c64(x), "adjoint_forward", c=256)).max() <= 1e-5 * 12


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("kind", ["gaussian", "dynamic_range"])
def test_tc_precision_config(form, kind):
    """complex64 n = 2^16, batch 4096; Gaussian sigma = 1 and amplitudes
    log-uniform over 1e-4 .. 1e4; sampled transforms against the oracle."""
    n, batch = 1 << 16, 4096
    gen = W.gaussian_complex if kind == "gaussian" else W.dynamic_range_complex
    x = gen(n, batch, seed=0)
    picks = [0, 2049, batch - 1]
    y = run(x, form, rows=picks)
    ref = O.fft(c64(x[picks]), "forward", c=1024, threads=3)
    err = err_rows(y, ref)
    assert err.max() <= 1e-5 * 16, err


def describe_schedule(p):
    import json
    return json.loads(M.fft_plan_describe(p))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("t,schedule,batch", [
    (8, None, 5), (8, None, 19),          # one 16 x 16 pass, whole transforms as rows (ragged last tile)
    (10, None, 3), (10, None, 6),         # one 32 x 32 pass
    (16, None, 3),                        # 8, 8: a column pass and a row pass of 16 x 16
    (18, None, 2),                        # 8, 10
    (20, None, 2),                        # 10, 10
    (16, "10,6", 2), (16, "6,10", 2),     # a 32 x 32 pass beside a per-tile pass
    (24, "8,8,8", 1),                     # three passes: the middle one reads the last pass's digit order
    (24, "10,10,4", 1),                   # 32 x 32 passes first and in the middle (the radix sweep's schedule)
])
def test_tc_two_digit_passes(form, t, schedule, batch):
    """Passes of 2^8 = 16 x 16 and 2^10 = 32 x 32 points, whose two DFT
    digits both run as tensor-core products (persistent, TMA-staged), in
    every position (first, middle, last pass, single pass), both directions
    and the adjoint, against the oracle."""
    n = 1 << t
    x = W.gaussian_complex(n, batch, seed=40 + t)
    ref_in = c64(x)
    d_in = torch.from_numpy(x).to(torch.complex64).cuda()
    for direction, op in ((M.FFT_FORWARD, "forward"), (M.FFT_INVERSE, "inverse")):
        for adjoint in (False, True):
            d_out = torch.empty_like(d_in)
            p = M.fft_plan_ex(n, batch, M.FFT_C64, direction, form, schedule)
            try:
                (M.fft_exec_adjoint if adjoint else M.fft_exec)(p, d_in, d_out)
                M.fft_plan_check(p)
            finally:
                M.fft_destroy(p)
            y = d_out.cpu().numpy().astype(np.complex128)
            opx = ("adjoint_" + op) if adjoint else op
            err = err_rows(y, O.fft(ref_in, opx, c=1024, threads=min(4, batch)))
            assert err.max() <= 1e-5 * t, (t, schedule, opx, err.max())


@pytest.mark.parametrize("form", FORMS)
def test_tc_in_place_and_dynamic_range_two_digit(form):
    """In place, on amplitudes 10^U(-4, 4) (the per-column FP16 scale must
    keep every vector of a column in range), n = 2^20 (two 32 x 32 passes)."""
    n, batch = 1 << 20, 2
    x = W.dynamic_range_complex(n, batch, seed=3)
    d = torch.from_numpy(x).to(torch.complex64).cuda()
    p = M.fft_plan_ex(n, batch, M.FFT_C64, M.FFT_FORWARD, form)
    try:
        M.fft_exec(p, d, d)
        M.fft_plan_check(p)
    finally:
        M.fft_destroy(p)
    err = err_rows(d.cpu().numpy().astype(np.complex128), O.fft(c64(x), "forward", c=1024, threads=2))
    assert err.max() <= 1e-5 * 20, err.max()
