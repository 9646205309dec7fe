"""One-round-trip complex64 transforms of n = 2^16 through thread-block
clusters (schedule "cluster"): parity against the FP64 oracle, in place,
adjoint, both cluster sizes, and the two-pass fallback for buffers the
tensor map cannot describe."""
import json

import numpy as np
import pytest

import oracle as O
import paper_0803_2386_gb300 as M
import workloads as W
from parity_check import err_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 1 << 16
TOL = 1e-6 * 16


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    M.build()
    yield



def run(x, direction=M.FFT_FORWARD, schedule=None, adjoint=False, inplace=False, offset=0):
    batch = x.shape[0]
    flat = torch.zeros(batch * N + offset, dtype=torch.complex64, device="cuda")
    d_in = flat[offset:].view(batch, N)
    d_in.copy_(torch.from_numpy(x.astype(np.complex64)))
    d_out = d_in if inplace else torch.empty_like(d_in)
    p = M.fft_plan_ex(N, batch, M.FFT_C64, direction, M.FFT_FORM_PLAIN, schedule)
    try:
        desc = json.loads(M.fft_plan_describe(p))
        (M.fft_exec_adjoint if adjoint else M.fft_exec)(p, d_in, d_out)
        torch.cuda.synchronize()
        M.fft_plan_check(p)
    finally:
        M.fft_destroy(p)
    return d_out.cpu().numpy().astype(np.complex128), desc


def ref(x, op, rows=None):
    xr = x.astype(np.complex64).astype(np.complex128)
    if rows is not None:
        xr = xr[rows]
    return O.fft(xr, op, c=256, threads=8)


def test_cluster_plan_is_one_launch():
    x = W.uniform_complex(N, 2, seed=11)
    y, desc = run(x, schedule="cluster")
    assert desc["schedule"]["cluster"] is True and desc["launches"] == 1
    assert desc["cluster_ctas"] in (8, 16) and desc["resident_clusters"] >= 1
    assert err_rows(y, ref(x, "forward")).max() <= TOL


@pytest.mark.parametrize("batch", [1, 3, 41])
@pytest.mark.parametrize("direction", [M.FFT_FORWARD, M.FFT_INVERSE])
def test_cluster_parity(batch, direction):
    """Batches smaller and larger than the number of resident clusters: each
    cluster runs 0..3 transforms through both signal buffers."""
    x = W.uniform_complex(N, batch, seed=300 + batch)
    y, _ = run(x, direction, schedule="cluster")
    op = "forward" if direction == M.FFT_FORWARD else "inverse"
    assert err_rows(y, ref(x, op)).max() <= TOL


def test_cluster_adjoint_and_in_place():
    x = W.uniform_complex(N, 5, seed=21)
    y, _ = run(x, M.FFT_FORWARD, schedule="cluster", adjoint=True)
    assert err_rows(y, ref(x, "adjoint_forward")).max() <= TOL
    y, _ = run(x, M.FFT_INVERSE, schedule="cluster", adjoint=True)
    assert err_rows(y, ref(x, "adjoint_inverse")).max() <= TOL
    y, _ = run(x, M.FFT_FORWARD, schedule="cluster", inplace=True)
    assert err_rows(y, ref(x, "forward")).max() <= TOL


def test_cluster_many_rounds_sampled():
    """300 transforms: every cluster cycles its two buffers many times (the
    mbarrier parity alternates); sampled rows against the oracle, Parseval on
    every row."""
    batch = 300
    x = W.gaussian_complex(N, batch, seed=5)
    y, _ = run(x, schedule="cluster")
    rows = [0, 1, 17, 18, 19, 150, 298, 299]
    assert err_rows(y[rows], ref(x, "forward", rows)).max() <= TOL
    xr = x.astype(np.complex64).astype(np.complex128)
    ex = np.sum(np.abs(xr) ** 2, axis=-1)
    ey = np.sum(np.abs(y) ** 2, axis=-1)
    assert np.max(np.abs(ey - N * ex) / (N * ex)) <= 1e-5


def test_misaligned_buffer_takes_two_pass_path():
    """An input 8 bytes off a 16-byte boundary cannot be a TMA source: the
    plan falls back to its two passes and gives the same transform."""
    x = W.uniform_complex(N, 3, seed=8)
    y, desc = run(x, schedule="cluster", offset=1)
    assert desc["schedule"]["cluster"] is True
    assert err_rows(y, ref(x, "forward")).max() <= TOL


def test_cluster_matches_two_pass():
    x = W.uniform_complex(N, 4, seed=9)
    a, _ = run(x, schedule="cluster")
    b, desc = run(x, schedule="8,8")
    assert "cluster" not in desc["schedule"]
    assert err_rows(a, b).max() <= 1e-6


def test_eight_cta_clusters_in_a_child_process():
    """MOAFFT_CLUSTER=8 selects clusters of 8 CTAs (one per SM); the choice is
    made once per process, so the check runs in a child."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import json, numpy as np, torch, oracle as O, paper_0803_2386_gb300 as M, workloads as W\n"
        "n = 1 << 16\n"
        "x = W.uniform_complex(n, 5, seed=77)\n"
        "d = torch.from_numpy(x.astype(np.complex64)).cuda()\n"
        "y = torch.empty_like(d)\n"
        "p = M.fft_plan_ex(n, 5, M.FFT_C64, M.FFT_INVERSE, M.FFT_FORM_PLAIN, 'cluster')\n"
        "desc = json.loads(M.fft_plan_describe(p))\n"
        "M.fft_exec(p, d, y); torch.cuda.synchronize(); M.fft_plan_check(p); M.fft_destroy(p)\n"
        "ref = O.fft(x.astype(np.complex64).astype(np.complex128), 'inverse', c=256, threads=4)\n"
        "yy = y.cpu().numpy().astype(np.complex128)\n"
        "err = (np.linalg.norm(yy - ref, axis=-1) / np.linalg.norm(ref, axis=-1)).max()\n"
        "assert desc['cluster_ctas'] == 8, desc\n"
        "assert err <= 1.6e-5, err\n"
        "print('ok', err)\n")
    env = dict(os.environ, MOAFFT_CLUSTER="8", PYTHONPATH=root)
    r = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
