"""The 256-point single-pass complex64 tiles exchange between their two
radix-16 digits by warp shuffles by default; MOAFFT_NO_SHFL selects the
shared-memory (TMA-staged) tiles instead.  Both against the FP64 oracle,
forward and inverse, with a batch that leaves a partial CTA, and an uneven
batch whose 256-point transforms sit at ragged offsets.  Run in child
processes: the switch is read once per process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import oracle as O, paper_0803_2386_gb300 as M, workloads as W
from parity_check import err_one, err_rows
n, batch = 256, 37
x = W.uniform_complex(n, batch, seed=90)
xr = x.astype(np.complex64).astype(np.complex128)
d = torch.from_numpy(x).to(torch.complex64).cuda()
for direction, op in ((M.FFT_FORWARD, "forward"), (M.FFT_INVERSE, "inverse")):
    out = torch.empty_like(d)
    p = M.fft_plan(n, batch, M.FFT_C64, direction)
    M.fft_exec(p, d, out)
    M.fft_plan_check(p)
    M.fft_destroy(p)
    err = err_rows(out.cpu().numpy().astype(np.complex128), O.fft(xr, op, c=64)).max()
    assert err <= 1e-6 * 8, (op, err)
# an uneven batch: lengths 2^5..2^9, so 256-point transforms at ragged offsets
sizes, data = W.uneven_batch(count=200, seed=91, lo_exp=5, hi_exp=9)
du = torch.from_numpy(data).to(torch.complex64).cuda()
ou = torch.empty_like(du)
pm = M.fft_plan_many(sizes, M.FFT_C64, M.FFT_FORWARD)
M.fft_exec(pm, du, ou)
M.fft_plan_check(pm)
M.fft_destroy(pm)
y = ou.cpu().numpy().astype(np.complex128)
dr = data.astype(np.complex64).astype(np.complex128)
at = 0
for s_ in sizes.tolist():
    e = err_one(y[at:at + s_], O.fft(dr[None, at:at + s_], "forward", c=64)[0])
    assert e <= 1e-6 * 9, (s_, e)
    at += s_
print("ok")
"""


@pytest.mark.parametrize("no_shfl", [False, True])
def test_256_point_tiles_match_oracle(no_shfl):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    env = {k: v for k, v in os.environ.items() if k != "MOAFFT_NO_SHFL"}
    if no_shfl:
        env["MOAFFT_NO_SHFL"] = "1"
    env["PYTHONPATH"] = os.pathsep.join([ROOT, os.path.join(ROOT, "tests"), env.get("PYTHONPATH", "")])
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
