"""Autotuner: schedule "auto" times the candidate schedules, caches the
fastest, and later plans of the same shape pick it up."""
import json
import os

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


def test_auto_schedule_is_cached_and_reused(tmp_path, monkeypatch):
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("MOAFFT_TUNE_CACHE", str(cache))
    n, batch = 1 << 14, 64
    x = W.uniform_complex(n, batch, seed=8)
    d = torch.from_numpy(x).to(torch.complex64).cuda()
    out = torch.empty_like(d)
    p = M.fft_plan_ex(n, batch, M.FFT_C64, M.FFT_FORWARD, M.FFT_FORM_PLAIN, "auto")
    tuned = json.loads(M.fft_plan_describe(p))["schedule"]
    M.fft_exec(p, d, out)
    torch.cuda.synchronize()
    M.fft_destroy(p)
    ref = O.fft(x.astype(np.complex64).astype(np.complex128), "forward", c=256)
    err = err_rows(out.cpu().numpy(), ref)
    assert err.max() <= 1e-6 * 14
    lines = [json.loads(l) for l in cache.read_text().splitlines()]
    assert len(lines) == 1 and lines[0]["schedule"] in M.fft_tune_candidates(n, M.FFT_C64)
    # a default plan of the same shape now uses the cached schedule
    p2 = M.fft_plan(n, batch, M.FFT_C64, M.FFT_FORWARD)
    again = json.loads(M.fft_plan_describe(p2))["schedule"]
    M.fft_destroy(p2)
    assert [q["log_r"] for q in again["passes"]] == [q["log_r"] for q in tuned["passes"]]
