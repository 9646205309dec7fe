"""Pins for the oracle's transforms against what mathematics fixes:
brute-force DFT, closed forms, invariants, library cross-checks, and the
paper's claim that the blocked routine with c >= n is the unblocked one."""
import numpy as np
import pytest

import oracle as O
import workloads as W

EPS = 2.0 ** -53


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def fft_tol(n):
    return 8.0 * EPS * max(1, int(np.log2(max(n, 1))))


# ------------------------------------------------------ the direct DFT itself

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 256])
def test_dft_direct_closed_forms(n):
    k = np.arange(n)
    cf = W.closed_form_inputs(n)
    f = 37 % n
    X = O.dft_direct(cf["delta0"])
    assert np.allclose(X, np.ones(n), rtol=0, atol=4 * EPS)
    m = 5 % n
    X = O.dft_direct(cf["delta5"])
    assert np.allclose(X, np.exp(-2j * np.pi * ((m * k) % n) / n), rtol=0, atol=8 * EPS)
    X = O.dft_direct(cf["const"])
    expect = np.zeros(n, complex)
    expect[0] = n
    assert np.allclose(X, expect, rtol=0, atol=4 * n * EPS)
    X = O.dft_direct(cf["cos37"])
    expect = np.zeros(n, complex)
    expect[f] += n / 2
    expect[(n - f) % n] += n / 2
    assert np.allclose(X, expect, rtol=0, atol=16 * n * EPS)
    if n > 2 and f not in (0, n // 2):
        X = O.dft_direct(cf["sin37"])
        expect = np.zeros(n, complex)
        expect[f] = -0.5j * n
        expect[n - f] = 0.5j * n
        assert np.allclose(X, expect, rtol=0, atol=16 * n * EPS)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 64, 100, 256])
def test_dft_direct_matches_numpy(n):
    x = W.uniform_complex(n, 1, seed=n)[0]
    assert rel(O.dft_direct(x), np.fft.fft(x)) < 16 * EPS * max(1, np.log2(n))
    assert rel(O.dft_direct(x, sign=+1), n * np.fft.ifft(x)) < 16 * EPS * max(1, np.log2(n))


def test_dft_bins_match_direct():
    x = W.uniform_complex(512, 1, seed=3)[0]
    full = O.dft_direct(x)
    ks = np.array([0, 1, 7, 255, 256, 511])
    assert np.array_equal(O.dft_bins(x, ks), full[ks])


# ----------------------------------------------------------- the FFT routines

@pytest.mark.parametrize("t", range(0, 13))
def test_moa_fft_vs_direct_dft_all_blockings(t):
    n = 1 << t
    x = W.uniform_complex(n, 1, seed=t)[0]
    ref = O.dft_direct(x)
    unblocked = O.fftpsirad2(x)
    assert rel(unblocked, ref) < fft_tol(n)
    # "the non-optimised code is the same code with c >= n": every blocking
    # performs the same butterflies on the same values, so bit-identical.
    for g in range(1, t + 2):
        for reading in (0, 1):
            y = O.moa_fft(x, 1 << g, reading=reading)
            assert np.array_equal(y, unblocked), (n, 1 << g, reading)


@pytest.mark.parametrize("sign", [-1, 1])
def test_moa_fft_sign(sign):
    n = 256
    x = W.uniform_complex(n, 1, seed=11)[0]
    ref = O.dft_direct(x, sign=sign)
    assert rel(O.moa_fft(x, 16, sign=sign), ref) < fft_tol(n)


def test_closed_forms_n1024():
    n = 1024
    k = np.arange(n)
    cf = W.closed_form_inputs(n)
    tol = 64 * EPS * np.log2(n)
    assert np.abs(O.moa_fft(cf["delta0"], 32) - 1).max() < tol
    assert np.abs(O.moa_fft(cf["delta5"], 32) - np.exp(-2j * np.pi * ((5 * k) % n) / n)).max() < tol
    X = O.moa_fft(cf["const"], 32)
    assert abs(X[0] - n) < n * tol and np.abs(X[1:]).max() < n * tol
    X = O.moa_fft(cf["cos37"], 32)
    spikes = np.zeros(n, complex)
    spikes[37] = spikes[n - 37] = n / 2
    assert np.abs(X - spikes).max() < n * tol
    X = O.moa_fft(cf["sin37"], 32)
    spikes = np.zeros(n, complex)
    spikes[37], spikes[n - 37] = -0.5j * n, 0.5j * n
    assert np.abs(X - spikes).max() < n * tol


def test_invariants():
    n = 4096
    x = W.uniform_complex(n, 1, seed=5)[0]
    y = W.gaussian_complex(n, 1, seed=6)[0]
    X = O.moa_fft(x, 64)
    # Parseval
    assert abs(np.vdot(X, X).real - n * np.vdot(x, x).real) < 1e-12 * n * np.vdot(x, x).real
    # linearity
    a, b = 0.3 - 1.2j, 2.5 + 0.1j
    L = O.moa_fft(a * x + b * y, 64)
    R = a * X + b * O.moa_fft(y, 64)
    assert rel(L, R) < 1e-14
    # shift theorem: x[(j - s) mod n] -> X_k w^(k s)
    s = 123
    k = np.arange(n)
    assert rel(O.moa_fft(np.roll(x, s), 64), X * np.exp(-2j * np.pi * k * s / n)) < 1e-13
    # modulation: x_j w^(-j m) -> X_(k - m)
    m = 77
    xm = x * np.exp(2j * np.pi * k * m / n)
    assert rel(O.moa_fft(xm, 64), np.roll(X, m)) < 1e-13
    # conjugate symmetry of a real input
    r = x.real.astype(complex)
    R = O.moa_fft(r, 64)
    assert np.abs(R[1:] - np.conj(R[1:][::-1])).max() < 1e-12 * np.abs(R).max()


@pytest.mark.parametrize("n", [1, 2, 16, 1024, 1 << 14])
def test_batched_ops(n):
    x = W.uniform_complex(n, 3, seed=9)
    f = O.fft(x, "forward", c=64)
    assert rel(f, np.fft.fft(x, axis=-1)) < fft_tol(n)
    inv = O.fft(x, "inverse", c=64)
    assert rel(inv, np.fft.ifft(x, axis=-1)) < fft_tol(n)
    # inverse(forward(x)) = x
    assert rel(O.fft(f, "inverse", c=64), x) < 2 * fft_tol(n)
    # adjoint of forward = unscaled +i transform; adjoint of inverse =
    # (1/N)-scaled -i transform
    assert rel(O.fft(x, "adjoint_forward", c=64), n * np.fft.ifft(x, axis=-1)) < fft_tol(n)
    assert rel(O.fft(x, "adjoint_inverse", c=64), np.fft.fft(x, axis=-1) / n) < fft_tol(n)
    # threads over the batch give the same bits
    assert np.array_equal(O.fft(x, "forward", c=64, threads=3), f)


@pytest.mark.parametrize("op,adj", [("forward", "adjoint_forward"),
                                    ("inverse", "adjoint_inverse")])
def test_adjoint_dot_product(op, adj):
    """<F x, y> = <x, F^H y> for the operator and its adjoint."""
    n = 2048
    x = W.uniform_complex(n, 1, seed=21)[0]
    y = W.gaussian_complex(n, 1, seed=22)[0]
    lhs = np.vdot(y, O.fft(x, op, c=32))
    rhs = np.vdot(O.fft(y, adj, c=32), x)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_errors():
    with pytest.raises(O.OracleError):
        O.moa_fft(np.zeros(12, complex), 4)
    with pytest.raises(O.OracleError):
        O.dft_direct(np.zeros(0, complex))


# ---- general radix (Fig. radnbutterfly) ------------------------------------

@pytest.mark.parametrize("base,n", [(2, 1), (2, 2), (4, 4), (4, 256), (8, 512), (16, 4096), (64, 4096),
                                    (4, 1024), (2, 2048), (256, 256)])
def test_fftpsiradn_matches_direct_dft(base, n):
    """The general-radix routine against the definition (long double
    accumulation), both exponent signs."""
    rng = np.random.default_rng(base + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        got = O.fftpsiradn(x, base, sign)
        ref = O.dft_direct(x, sign)
        assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.log2(n)) * np.abs(ref).max()


@pytest.mark.parametrize("t", range(0, 13))
def test_fftpsiradn_base2_is_fftpsirad2_bitwise(t):
    """Radix 2 of the general routine performs the butterflies of
    fftpsirad2 exactly (same weights, w_2 = -1 exact)."""
    x = W.uniform_complex(1 << t, 1, seed=t)[0]
    for sign in (-1, 1):
        assert np.array_equal(O.fftpsiradn(x, 2, sign), O.fftpsirad2(x, sign))


def test_fftpsiradn_rejects_lengths_that_are_not_powers_of_the_base():
    x = np.ones(32, complex)
    with pytest.raises(RuntimeError):
        O.fftpsiradn(x, 4)   # 32 = 2^5 is not a power of 4
    with pytest.raises(RuntimeError):
        O.fftpsiradn(x, 3)   # radix 3 is outside the routine's domain (powers of two)
