"""Batching form: many transforms of uneven power-of-two lengths, packed back
to back, in one plan (fft_plan_many) replayed as one captured graph."""
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


def split(flat, sizes):
    out, at = [], 0
    for s in sizes:
        out.append(flat[at:at + s])
        at += s
    return out


def run_many(sizes, data, dt, direction=M.FFT_FORWARD, adjoint=False, reps=1):
    tdt = torch.complex128 if dt == M.FFT_C128 else torch.complex64
    d_in = torch.from_numpy(data).to(tdt).cuda()
    d_out = torch.empty_like(d_in)
    p = M.fft_plan_many(sizes, dt, direction)
    try:
        for _ in range(reps):
            (M.fft_exec_adjoint if adjoint else M.fft_exec)(p, d_in, d_out)
        torch.cuda.synchronize()
        M.fft_plan_check(p)  # raises if a persistent-kernel wait timed out
        desc = M.fft_plan_describe(p)
    finally:
        M.fft_destroy(p)
    return d_out.cpu().numpy().astype(np.complex128), desc


@pytest.mark.parametrize("dt", [M.FFT_C64, M.FFT_C128])
@pytest.mark.parametrize("direction", [M.FFT_FORWARD, M.FFT_INVERSE])
def test_uneven_small(dt, direction):
    sizes, data = W.uneven_batch(count=300, seed=4, lo_exp=0, hi_exp=14)
    xr = data if dt == M.FFT_C128 else data.astype(np.complex64).astype(np.complex128)
    y, _ = run_many(sizes, data, dt, direction, reps=2)  # second run replays the graph
    op = "forward" if direction == M.FFT_FORWARD else "inverse"
    tol_of = (lambda n: 1e-12) if dt == M.FFT_C128 else (lambda n: 1e-6 * max(1, np.log2(n)))
    for yi, xi in zip(split(y, sizes), split(xr, sizes)):
        ref = O.fft(xi[None, :], op, c=64)[0]
        err = err_one(yi, ref)
        assert err <= tol_of(len(xi)), (len(xi), err)


def test_uneven_adjoint():
    sizes, data = W.uneven_batch(count=60, seed=9, lo_exp=1, hi_exp=13)
    y, _ = run_many(sizes, data, M.FFT_C128, M.FFT_FORWARD, adjoint=True)
    for yi, xi in zip(split(y, sizes), split(data, sizes)):
        ref = O.fft(xi[None, :], "adjoint_forward", c=64)[0]
        assert err_one(yi, ref) <= 1e-12


@pytest.mark.parametrize("persistent", [False, True])
def test_uneven_full_config_sampled(persistent, monkeypatch):
    """20,000 complex64 transforms, n log-uniform over 2^6..2^16 (seed 1),
    as the default graph of per-length launches and as the one persistent
    launch, each against the oracle."""
    sizes, data = W.uneven_batch()
    if persistent:
        monkeypatch.setenv("MOAFFT_PERSIST", "1")
    y, desc = run_many(sizes, data, M.FFT_C64)
    assert ('"persistent": true' in desc) == persistent
    xs = split(data.astype(np.complex64).astype(np.complex128), sizes)
    ys = split(y, sizes)
    rng = np.random.default_rng(3)
    picks = sorted(set(rng.integers(0, len(sizes), 40).tolist()) | {0, len(sizes) - 1})
    for i in picks:
        ref = O.fft(xs[i][None, :], "forward", c=1024)[0]
        err = err_one(ys[i], ref)
        assert err <= 1e-6 * np.log2(len(xs[i])), (i, len(xs[i]), err)
    # Parseval on every transform
    for xi, yi in zip(xs, ys):
        n = len(xi)
        ex = np.vdot(xi, xi).real
        assert abs(np.vdot(yi, yi).real - n * ex) <= 1e-5 * n * ex


def test_many_rejects_bad_sizes():
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_plan_many([16, 12, 8], M.FFT_C64)
    assert e.value.status == M.FFT_ERR_NOT_POW2
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_plan_many([], M.FFT_C64)
    assert e.value.status == M.FFT_ERR_ARG


def test_persistent_matches_per_class_graph(monkeypatch):
    """One persistent launch (atomic ticket queue over every class and pass,
    round counters for the pass dependencies) gives the same transforms as
    the graph of per-class launches."""
    sizes, data = W.uneven_batch(count=2000, seed=6)
    monkeypatch.setenv("MOAFFT_PERSIST", "1")
    y_p, desc_p = run_many(sizes, data, M.FFT_C64, reps=2)
    monkeypatch.delenv("MOAFFT_PERSIST")
    y_g, desc_g = run_many(sizes, data, M.FFT_C64)
    assert '"persistent": true' in desc_p and '"launches": 1' in desc_p
    assert '"persistent": false' in desc_g
    for a, b in zip(split(y_p, sizes), split(y_g, sizes)):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b)


@pytest.mark.parametrize("dt", [M.FFT_C64, M.FFT_C128])
def test_persistent_inverse_and_adjoint(dt, monkeypatch):
    monkeypatch.setenv("MOAFFT_PERSIST", "1")
    sizes, data = W.uneven_batch(count=400, seed=2, lo_exp=4, hi_exp=15)
    xr = data if dt == M.FFT_C128 else data.astype(np.complex64).astype(np.complex128)
    tol_of = (lambda n: 1e-12) if dt == M.FFT_C128 else (lambda n: 1e-6 * np.log2(n))
    y, desc = run_many(sizes, data, dt, M.FFT_INVERSE)
    assert '"persistent": true' in desc
    for yi, xi in zip(split(y, sizes), split(xr, sizes)):
        ref = O.fft(xi[None, :], "inverse", c=64)[0]
        assert err_one(yi, ref) <= tol_of(len(xi))
    y, _ = run_many(sizes, data, dt, M.FFT_FORWARD, adjoint=True)
    for yi, xi in zip(split(y, sizes), split(xr, sizes)):
        ref = O.fft(xi[None, :], "adjoint_forward", c=64)[0]
        assert err_one(yi, ref) <= tol_of(len(xi))
