"""Pins of the oracle's multi-dimensional transform (oracle.fftn) against
the definition of the multi-dimensional DFT, written out as one sum over all
index tuples (not as 1-D transforms along the axes), closed forms and
invariants."""
import itertools

import numpy as np
import pytest

import oracle as O


def dft_nd_direct(x, sign=-1, scale=1.0):
    """X[k] = scale * sum_n x[n] exp(sign 2 pi i sum_j n_j k_j / N_j) over the
    whole shape, as one dense matrix over flattened index tuples."""
    shape = x.shape
    idx = np.array(list(itertools.product(*[range(s) for s in shape])), dtype=np.int64)
    phase = np.zeros((len(idx), len(idx)))
    for j, nj in enumerate(shape):
        phase += np.mod(np.outer(idx[:, j], idx[:, j]), nj) / nj
    M = np.exp(sign * 2j * np.pi * phase)
    return (scale * (M @ x.reshape(-1))).reshape(shape)


SHAPES = [(4, 8), (8, 4), (2, 4, 8), (16, 2), (8, 1, 4), (2, 2, 2, 4)]


@pytest.mark.parametrize("shape", SHAPES)
def test_fftn_matches_direct_sum(shape):
    rng = np.random.default_rng(11)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    n = int(np.prod(shape))
    cases = {"forward": (-1, 1.0), "inverse": (1, 1.0 / n), "adjoint_forward": (1, 1.0),
             "adjoint_inverse": (-1, 1.0 / n)}
    for op, (sign, scale) in cases.items():
        ref = dft_nd_direct(x, sign, scale)
        got = O.fftn(x, op=op, c=2)
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max()), op


def test_fftn_closed_forms():
    shape = (8, 16, 32)
    n = int(np.prod(shape))
    delta = np.zeros(shape, complex)
    delta[0, 0, 0] = 1
    assert np.array_equal(O.fftn(delta), np.ones(shape, complex))
    const = np.ones(shape, complex)
    X = O.fftn(const)
    expect = np.zeros(shape, complex)
    expect[0, 0, 0] = n
    assert np.abs(X - expect).max() < 1e-10
    # plane wave exp(+2 pi i f . n / N) -> n at k = f
    f = (3, 5, 17)
    grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    wave = np.exp(2j * np.pi * sum(fj * g / s for fj, g, s in zip(f, grids, shape)))
    X = O.fftn(wave)
    expect = np.zeros(shape, complex)
    expect[f] = n
    assert np.abs(X - expect).max() < 1e-9


def test_fftn_parseval_roundtrip_and_batch_axes():
    rng = np.random.default_rng(12)
    x = rng.uniform(-1, 1, (3, 16, 8, 32)) + 1j * rng.uniform(-1, 1, (3, 16, 8, 32))
    X = O.fftn(x, ndim=3)
    n = 16 * 8 * 32
    for b in range(3):
        assert abs(np.sum(np.abs(X[b]) ** 2) - n * np.sum(np.abs(x[b]) ** 2)) < 1e-9 * n * np.sum(np.abs(x[b]) ** 2)
        assert np.abs(X[b] - O.fftn(x[b])).max() == 0.0  # the leading axis is a batch
    back = O.fftn(X, ndim=3, op="inverse")
    assert np.abs(back - x).max() < 1e-14 * 12
    # one axis: the 1-D transform
    assert np.abs(O.fftn(x, ndim=1) - O.fft(x)).max() == 0.0
