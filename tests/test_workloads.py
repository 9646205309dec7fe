"""The seeded input generators (workloads.py): the recipes of the workloads,
deterministic, with the sizes and value ranges they state.  Host only."""
import numpy as np

import workloads as W


def test_uniform_and_gaussian_are_seeded_and_shaped():
    a = W.uniform_complex(64, 3, seed=5)
    assert a.shape == (3, 64) and a.dtype == np.complex128
    assert np.array_equal(a, W.uniform_complex(64, 3, seed=5))
    assert not np.array_equal(a, W.uniform_complex(64, 3, seed=6))
    assert np.abs(a.real).max() <= 1 and np.abs(a.imag).max() <= 1
    # re then im drawn as two arrays of n * batch values
    rng = np.random.default_rng(5)
    re = rng.uniform(-1, 1, 192)
    assert np.array_equal(a.real.reshape(-1), re)
    g = W.gaussian_complex(4096, 4, seed=1)
    assert abs(g.real.std() - 1) < 0.05 and abs(g.imag.mean()) < 0.05


def test_dynamic_range_amplitudes():
    x = W.dynamic_range_complex(1 << 14, 1, seed=0)
    amp = np.log10(np.abs(x))
    assert amp.min() >= -4 - 1e-12 and amp.max() <= 4 + 1e-12
    assert amp.min() < -3.9 and amp.max() > 3.9


def test_uneven_batch_recipe():
    """20,000 lengths 2^6..2^16 with uniform exponents from default_rng(1):
    mean length about (2^17 - 2^6) / 11, about 2.4e8 points in all."""
    sizes, data = W.uneven_batch()
    assert len(sizes) == 20000
    assert set(np.unique(sizes).tolist()) == {1 << k for k in range(6, 17)}
    assert abs(sizes.mean() - ((1 << 17) - (1 << 6)) / 11) < 0.03 * sizes.mean()
    assert data.shape == (int(sizes.sum()),) and np.abs(data.real).max() <= 1
    s2, rng = W.uneven_sizes()
    assert np.array_equal(sizes, s2)
    assert np.array_equal(data[:1000].real, rng.uniform(-1.0, 1.0, 1000))  # data drawn next


def test_closed_form_inputs_and_loss_problem():
    cf = W.closed_form_inputs(1024)
    assert set(cf) == {"delta0", "delta5", "const", "cos37", "sin37"}
    assert cf["delta5"][5] == 1 and cf["delta5"].sum() == 1
    x, H, y = W.loss_problem(256, 3)
    assert x.shape == H.shape == y.shape == (3, 256)
    assert np.array_equal(x, W.uniform_complex(256, 3, 0))
    assert np.array_equal(H, W.gaussian_complex(256, 3, 2))
