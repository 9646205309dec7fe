"""FP64 CPU oracle for the MoA / psi-calculus radix-2 FFT.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA path (the package
``paper_0803_2386_gb300``) and imports nothing from it.

Every routine is a thin ctypes wrapper over ``moa_oracle.c`` (plain C,
binary64, no fused multiply-add).  What each one follows in the paper
(Mullin & Raynolds, "Conformal Computing"):

* :func:`dft_direct`, :func:`dft_bins` -- the definition of the DFT
  (Fig. vanloan_fft: "Output: the FFT of x"), brute force in long double.
* :func:`fftpsirad2` -- Fig. fftpsirad2 / rad2_fft, preceded by the
  bit-reversal P_n of Fig. vanloan_fft line (1).
* :func:`fftpsiradn` -- the general-radix routine (Fig. radnbutterfly):
  base-digit reversal, then stages of direct base-point DFTs of weighted
  inputs.
* :func:`fftn` -- multi-dimensional transforms as 1-D transforms along
  every axis (Sec. "Conclusions for the General Radix Approach", footnote).
* :func:`moa_fft` -- the cache-optimised algorithm of Ch.3 (Sec. butter-order
  steps (1)-(5)): stages inside rows of length c, reshape-transposes
  (Eqs. reshape1-3, xdeqn), weights carried like the data (Eqs. xi1, xi2),
  final transpose (Eq. xihyper, Fig. final_trans_code).
* index machinery: :func:`gamma_row` (Def. gammadef), :func:`rotate`,
  :func:`tvec` (Eq. tvec), :func:`hyper_transpose` (Eqs. b_vs_a, zj),
  :func:`reshape_transpose` (Eq. trans), :func:`final_trans`,
  :func:`bit_reverse`, :func:`xi` (Sec. trans-weights), :func:`schedule`
  (Sec. "The Number of Reshape-Transpose Operations" and "Number of
  Different Weight Matrices").
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

FORWARD, INVERSE, ADJOINT_FORWARD, ADJOINT_INVERSE = 0, 1, 2, 3
_OPS = {"forward": FORWARD, "inverse": INVERSE,
        "adjoint_forward": ADJOINT_FORWARD, "adjoint_inverse": ADJOINT_INVERSE}

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_intp = ctypes.POINTER(ctypes.c_int)


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        sig = {
            "moa_gamma_row": (ctypes.c_int64, [ctypes.c_int, _i64p, _i64p]),
            "moa_rotate": (None, [ctypes.c_int, ctypes.c_int, _i64p, _i64p]),
            "moa_tvec": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _i64p]),
            "moa_hyper_transpose": (ctypes.c_int, [ctypes.c_int, _i64p, _i64p, _i64p]),
            "moa_reshape_transpose_i64": (ctypes.c_int, [_i64p, _i64p, ctypes.c_int64,
                                                         ctypes.c_int64]),
            "moa_final_trans_i64": (ctypes.c_int, [_i64p, _i64p, ctypes.c_int64, ctypes.c_int]),
            "moa_bit_reverse_i64": (ctypes.c_int, [_i64p, _i64p, ctypes.c_int64]),
            "moa_schedule": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int)]),
            "moa_xi_i64": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int, _i64p]),
            "dft_direct_c128": (ctypes.c_int, [_f64p, _f64p, ctypes.c_int64, ctypes.c_int]),
            "dft_bins_c128": (ctypes.c_int, [_f64p, ctypes.c_int64, ctypes.c_int, _i64p,
                                             ctypes.c_int64, _f64p]),
            "fftpsirad2_c128": (ctypes.c_int, [_f64p, _f64p, ctypes.c_int64, ctypes.c_int]),
            "fftpsiradn_c128": (ctypes.c_int, [_f64p, _f64p, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_int]),
            "moa_fft_c128": (ctypes.c_int, [_f64p, _f64p, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_int, ctypes.c_int]),
            "oracle_fft_many": (ctypes.c_int, [_f64p, _f64p, ctypes.c_int64, ctypes.c_int64,
                                               ctypes.c_int, ctypes.c_int64, ctypes.c_int]),
            "moa_dm_perm": (ctypes.c_int, [ctypes.c_int, _intp, ctypes.c_int, _i64p]),
            "moa_dm_gate_c128": (ctypes.c_int, [_f64p, ctypes.c_int, _intp, ctypes.c_int, _f64p]),
            "moa_dm_gate_block_c128": (ctypes.c_int, [_f64p, ctypes.c_int, _intp, ctypes.c_int, _f64p,
                                                      ctypes.c_int64, ctypes.c_int64, _f64p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


class OracleError(RuntimeError):
    pass


def _check(status: int, what: str):
    if status != 0:
        raise OracleError(f"{what} failed with status {status}")


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_i64p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _fp(a: np.ndarray):
    return a.ctypes.data_as(_f64p)


# ----------------------------------------------------------------- indices --

def gamma_row(shape, idx) -> int:
    """gamma(s, p): row-major offset of index p in shape s (Def. gammadef)."""
    s, p = _i64(shape), _i64(idx)
    return int(lib().moa_gamma_row(len(s), _ip(s), _ip(p)))


def rotate(v, s: int) -> np.ndarray:
    """s phi v (rotate left by s; negative s rotates right)."""
    v = _i64(v)
    out = np.empty_like(v)
    lib().moa_rotate(len(v), int(s), _ip(v), _ip(out))
    return out


def tvec(l: int, j: int) -> np.ndarray:
    """Permutation vector t_j of the hyper-cube FFT (Eq. tvec)."""
    out = np.empty(l, dtype=np.int64)
    _check(lib().moa_tvec(int(l), int(j), _ip(out)), "tvec")
    return out


def hyper_transpose(perm, A) -> np.ndarray:
    """perm transpose A on a rank-d 2x...x2 hyper-cube given by its ravel."""
    perm, A = _i64(perm), _i64(A)
    d = len(perm)
    assert len(A) == 1 << d
    B = np.empty_like(A)
    _check(lib().moa_hyper_transpose(d, _ip(perm), _ip(A), _ip(B)), "hyper_transpose")
    return B


def reshape_transpose(x, c: int) -> np.ndarray:
    """<r c> rho-hat (transpose (<r c> rho-hat x)) of an index vector."""
    x = _i64(x)
    y = np.empty_like(x)
    _check(lib().moa_reshape_transpose_i64(_ip(x), _ip(y), len(x), int(c)),
           "reshape_transpose")
    return y


def final_trans(x, sigma: int) -> np.ndarray:
    """Final transpose by sigma bits (Eq. xihyper) of an index vector."""
    x = _i64(x)
    y = np.empty_like(x)
    _check(lib().moa_final_trans_i64(_ip(x), _ip(y), len(x), int(sigma)), "final_trans")
    return y


def bit_reverse(x) -> np.ndarray:
    """P_n x, the bit-reversal permutation of an index vector."""
    x = _i64(x)
    y = np.empty_like(x)
    _check(lib().moa_bit_reverse_i64(_ip(x), _ip(y), len(x)), "bit_reverse")
    return y


def schedule(n: int, c: int, reading: int = 0):
    """(gamma, l_max, p_max) of the blocked algorithm for length n, row c."""
    g, lm, pm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().moa_schedule(int(n), int(c), int(reading), ctypes.byref(g),
                              ctypes.byref(lm), ctypes.byref(pm)), "schedule")
    return g.value, lm.value, pm.value


def xi(n: int, c: int, L: int, l: int) -> np.ndarray:
    """Weight vector of stage L after l reshape-transposes: -1 encodes unity,
    e >= 0 encodes w_L^e (Sec. trans-weights)."""
    out = np.empty(n, dtype=np.int64)
    _check(lib().moa_xi_i64(int(n), int(c), int(L), int(l), _ip(out)), "xi")
    return out


# -------------------------------------------------------------- transforms --

def dft_direct(x, sign: int = -1) -> np.ndarray:
    """Direct O(N^2) DFT (long double accumulation)."""
    x = _c128(x)
    y = np.empty_like(x)
    _check(lib().dft_direct_c128(_fp(x), _fp(y), len(x), int(sign)), "dft_direct")
    return y


def dft_bins(x, ks, sign: int = -1) -> np.ndarray:
    """Selected bins X_k of the direct DFT, O(N) each (long double)."""
    x = _c128(x)
    ks = _i64(ks)
    y = np.empty(len(ks), dtype=np.complex128)
    _check(lib().dft_bins_c128(_fp(x), len(x), int(sign), _ip(ks), len(ks), _fp(y)),
           "dft_bins")
    return y


def fftpsirad2(x, sign: int = -1) -> np.ndarray:
    """Unblocked radix-2 FFT (bit-reversal then Fig. fftpsirad2)."""
    x = _c128(x)
    y = np.empty_like(x)
    _check(lib().fftpsirad2_c128(_fp(x), _fp(y), len(x), int(sign)), "fftpsirad2")
    return y


def fftpsiradn(x, base: int, sign: int = -1) -> np.ndarray:
    """General-radix FFT (Fig. radnbutterfly): len(x) a power of `base`."""
    x = _c128(x)
    y = np.empty_like(x)
    _check(lib().fftpsiradn_c128(_fp(x), _fp(y), len(x), int(base), int(sign)), "fftpsiradn")
    return y


def moa_fft(x, c: int | None = None, sign: int = -1, reading: int = 0) -> np.ndarray:
    """Cache-optimised MoA FFT with row length c (c >= len(x): unblocked)."""
    x = _c128(x)
    n = len(x)
    if c is None:
        c = max(2, n)
    y = np.empty_like(x)
    _check(lib().moa_fft_c128(_fp(x), _fp(y), n, int(c), int(sign), int(reading)), "moa_fft")
    return y


def fft(x, op: str = "forward", c: int = 1024, threads: int = 1) -> np.ndarray:
    """Batched transform over the last axis.

    op: "forward" (exp(-i..), unscaled), "inverse" (exp(+i..), x 1/N),
    "adjoint_forward" (exp(+i..), unscaled), "adjoint_inverse"
    (exp(-i..), x 1/N).  c is the blocking row length."""
    x = _c128(x)
    shape = x.shape
    n = shape[-1]
    batch = int(np.prod(shape[:-1])) if len(shape) > 1 else 1
    y = np.empty_like(x)
    _check(lib().oracle_fft_many(_fp(x), _fp(y), n, batch, _OPS[op], int(c), int(threads)),
           "oracle_fft_many")
    return y


def fftn(x, ndim: int | None = None, op: str = "forward", c: int = 1024, threads: int = 1) -> np.ndarray:
    """Multi-dimensional transform of the last `ndim` axes (default: all):
    the multi-dimensional DFT kernel is a product of one 1-D kernel per
    axis, so it is the 1-D transform (:func:`fft`, same `op`) applied along
    each axis in turn, as the paper builds multi-dimensional FFTs from its
    1-D one (Sec. "Conclusions for the General Radix Approach").  An inverse
    is scaled by 1/n_i on every axis, 1/prod(n_i) in all."""
    y = _c128(x)
    ndim = y.ndim if ndim is None else ndim
    for axis in range(y.ndim - ndim, y.ndim):
        moved = np.ascontiguousarray(np.moveaxis(y, axis, -1))
        y = np.moveaxis(fft(moved, op, c=c, threads=threads), -1, axis)
    return np.ascontiguousarray(y)


def library_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "liboracle.so")


# ------------------------------------------------- density-matrix gating --

def _qubits(qubits) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(qubits, dtype=np.int32))


def dm_perm(n: int, qubits) -> np.ndarray:
    """Transpose vector t (length 2n) that moves the gated qubits' axes of the
    2^(2n) hyper-cube behind the others in both halves (Ch. "Density Matrix
    Operations", Sec. "The Algorithm")."""
    qb = _qubits(qubits)
    t = np.zeros(2 * n, dtype=np.int64)
    _check(lib().moa_dm_perm(n, qb.ctypes.data_as(_intp), len(qb), _ip(t)), "moa_dm_perm")
    return t


def dm_gate(rho, qubits, u) -> np.ndarray:
    """rho' = G rho G^H, G = u on the gated qubits (the highest gated qubit is
    the most significant bit of u's index), computed block by block in the
    transposed view.  rho: 2^n x 2^n complex; returns a new array."""
    r = _c128(rho).copy()
    N = r.shape[0]
    n = int(N).bit_length() - 1
    qb = _qubits(qubits)
    uu = _c128(u)
    _check(lib().moa_dm_gate_c128(_fp(r), n, qb.ctypes.data_as(_intp), len(qb), _fp(uu)), "moa_dm_gate_c128")
    return r


def dm_gate_block(rho, qubits, u, I: int, J: int) -> np.ndarray:
    """Block (I, J) of the transposed view after the gate: U B_IJ U^H."""
    r = _c128(rho)
    N = r.shape[0]
    n = int(N).bit_length() - 1
    qb = _qubits(qubits)
    m = 1 << len(qb)
    out = np.zeros((m, m), dtype=np.complex128)
    _check(lib().moa_dm_gate_block_c128(_fp(r), n, qb.ctypes.data_as(_intp), len(qb), _fp(_c128(u)), I, J,
                                        _fp(out)), "moa_dm_gate_block_c128")
    return out

