"""Pins of the oracle's density-matrix gating (Ch. "Density Matrix Operations
for a Quantum Computer"): the printed transpose vectors, a brute-force dense
gate matrix built from the definition of a gate on chosen qubits, the
hyper-cube transpose of Ch.4, and invariants of rho -> G rho G^H."""
import itertools

import numpy as np
import pytest

import oracle as O
from conftest import read_golden


def test_transpose_vectors_match_the_paper():
    g = read_golden("dm_transpose_vectors.txt")
    n = int(g["n"][0])
    assert list(O.dm_perm(n, [0, 2])) == [int(v) for v in g["bits_0_2"]]
    assert list(O.dm_perm(n, [1, 2])) == [int(v) for v in g["bits_1_2"]]


def test_transpose_vector_rejects_bad_qubits():
    for n, qb in [(4, [4]), (4, [1, 1]), (4, [-1]), (3, [0, 1, 2, 0])]:
        with pytest.raises(O.OracleError):
            O.dm_perm(n, qb)


def dense_gate(n, qubits, u):
    """G as a 2^n x 2^n matrix from the definition: G|x> = sum_y U[y_g][x_g]
    |y> over the y that agree with x outside the gated qubits; x_g packs the
    gated bits of x, the highest gated qubit most significant."""
    N = 1 << n
    order = sorted(qubits, reverse=True)
    mask = sum(1 << b for b in qubits)
    G = np.zeros((N, N), dtype=np.complex128)
    for x in range(N):
        xg = 0
        for b in order:
            xg = (xg << 1) | ((x >> b) & 1)
        for yg in range(1 << len(qubits)):
            y = x & ~mask
            for k, b in enumerate(order):
                if (yg >> (len(order) - 1 - k)) & 1:
                    y |= 1 << b
            G[y, x] += u[yg, xg]
    return G


def random_unitary(m, rng):
    z = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    qm, r = np.linalg.qr(z)
    return qm * (np.diag(r) / np.abs(np.diag(r)))


def random_rho(n, rng):
    a = rng.standard_normal((1 << n, 1 << n)) + 1j * rng.standard_normal((1 << n, 1 << n))
    rho = a @ a.conj().T
    return rho / np.trace(rho).real


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gate_matches_dense_definition(n):
    rng = np.random.default_rng(100 + n)
    for q in range(1, min(n, 3) + 1):
        for qubits in itertools.combinations(range(n), q):
            qb = list(qubits)
            rng.shuffle(qb)  # the set, not the listing order, matters
            u = random_unitary(1 << q, rng)
            rho = rng.standard_normal((1 << n, 1 << n)) + 1j * rng.standard_normal((1 << n, 1 << n))
            G = dense_gate(n, list(qubits), u)
            ref = G @ rho @ G.conj().T
            got = O.dm_gate(rho, qb, u)
            assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max()), (n, qubits)


def test_transposed_view_is_the_chapter4_hyper_transpose():
    """The element addresses of the transposed view (direct indexing through
    gamma) agree with materialising the transpose with the Ch.4 hyper-cube
    transpose (whose convention lists, for each axis of D_h, its new
    position: the inverse of t)."""
    n = 4
    for qubits in ([0, 2], [1, 2], [3], [0, 1, 3]):
        t = O.dm_perm(n, qubits)
        inv = np.argsort(t)
        idx = np.arange(1 << (2 * n), dtype=np.int64)
        view = O.hyper_transpose(inv, idx).reshape(1 << n, 1 << n)
        # an identity 'gate' leaves rho alone; a gate that scales the gated
        # block index g by (g + 1) exposes which elements form each block
        q = len(qubits)
        m = 1 << q
        u = np.diag(np.arange(1, m + 1)).astype(np.complex128)
        rho = np.ones((1 << n, 1 << n), dtype=np.complex128)
        got = O.dm_gate(rho, qubits, u)
        for rp in range(1 << n):
            for cp in range(1 << n):
                addr = view[rp, cp]
                g, h = rp % m, cp % m
                assert got.reshape(-1)[addr] == (g + 1) * (h + 1)


def test_invariants():
    rng = np.random.default_rng(7)
    n = 5
    rho = random_rho(n, rng)
    for qb in ([0], [4], [1, 3], [0, 2, 4]):
        u = random_unitary(1 << len(qb), rng)
        out = O.dm_gate(rho, qb, u)
        assert abs(np.trace(out) - np.trace(rho)) <= 1e-13  # trace
        assert np.abs(out - out.conj().T).max() <= 1e-13  # Hermitian
        assert np.linalg.eigvalsh(out).min() >= -1e-12  # positive semidefinite
        back = O.dm_gate(out, qb, u.conj().T)  # the inverse gate undoes it
        assert np.abs(back - rho).max() <= 1e-13
        same = O.dm_gate(rho, qb, np.eye(1 << len(qb)))
        assert np.array_equal(same, rho)  # identity: bitwise unchanged


def test_single_block_matches_full_gate():
    rng = np.random.default_rng(11)
    n, qb = 6, [1, 4]
    rho = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    u = random_unitary(4, rng)
    full = O.dm_gate(rho, qb, u)
    t = O.dm_perm(n, qb)
    for I, J in [(0, 0), (3, 7), (15, 2)]:
        blk = O.dm_gate_block(rho, qb, u, I, J)
        for g in range(4):
            for h in range(4):
                rp, cp = I * 4 + g, J * 4 + h
                bits = [(rp >> (n - 1 - j)) & 1 for j in range(n)] + [(cp >> (n - 1 - j)) & 1 for j in range(n)]
                old = [0] * (2 * n)
                for j in range(2 * n):
                    old[t[j]] = bits[j]
                addr = int("".join(map(str, old)), 2)
                assert blk[g, h] == full.reshape(-1)[addr]
