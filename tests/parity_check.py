"""The parity measure of the GPU tests: for each transform (row), the larger
of two errors against the oracle's result r,
    relative L2         ||y - r||_2 / ||r||_2, and
    element-wise        max_k |y_k - r_k| / max_k |r_k|,
so one tolerance bounds both the overall error and the worst single bin (a
bad bin in a large-amplitude spectrum shows in the second even when the
first stays small)."""
import numpy as np


def err_rows(y, r):
    """Per-row parity error (see the module docstring); rows of zeros in r
    are measured absolutely."""
    y = np.atleast_2d(np.asarray(y))
    r = np.atleast_2d(np.asarray(r))
    d = y - r
    den2 = np.linalg.norm(r, axis=-1)
    den2[den2 == 0] = 1.0
    deni = np.abs(r).max(axis=-1)
    deni[deni == 0] = 1.0
    return np.maximum(np.linalg.norm(d, axis=-1) / den2, np.abs(d).max(axis=-1) / deni)


def err_arrays(y, r):
    """err_rows over whole arrays: one value per leading index."""
    y = np.asarray(y)
    r = np.asarray(r)
    return err_rows(y.reshape(y.shape[0], -1), r.reshape(r.shape[0], -1))


def err_one(y, r):
    """The parity error of one transform."""
    return float(err_rows(np.ravel(y), np.ravel(r))[0])
