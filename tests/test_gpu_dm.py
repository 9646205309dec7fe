"""Density-matrix gating on the GPU (dm_gate through the C ABI) against the
FP64 oracle (Ch. "Density Matrix Operations for a Quantum Computer"): every
qubit set of one, two and three qubits of small matrices, both dtypes, and
sampled blocks of a large matrix.  Tolerances: complex128 1e-13, complex64
2e-6 (relative to the largest element; each output element is a sum of
2^(2q) products)."""
import itertools

import numpy as np
import pytest

import oracle as O
import paper_0803_2386_gb300 as M

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    M.build()
    yield


def unitary(m, rng):
    z = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    qm, r = np.linalg.qr(z)
    return qm * (np.diag(r) / np.abs(np.diag(r)))


def run(rho, qubits, u, f64):
    t = torch.from_numpy(rho.astype(np.complex128 if f64 else np.complex64)).cuda()
    M.dm_gate(t, qubits, u)
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("f64", [True, False])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_every_qubit_set(n, f64):
    rng = np.random.default_rng(40 + n)
    N = 1 << n
    for q in (1, 2, 3):
        for qubits in itertools.combinations(range(n), q):
            rho = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
            u = unitary(1 << q, rng)
            if not f64:
                rho = rho.astype(np.complex64).astype(np.complex128)
                u = u.astype(np.complex64).astype(np.complex128)
            ref = O.dm_gate(rho, list(qubits), u)
            got = run(rho, list(reversed(qubits)), u, f64)
            tol = 1e-13 if f64 else 2e-6
            assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (n, qubits)


def test_paper_patterns_on_sixteen_by_sixteen():
    """The chapter's 16 x 16 example: gate bits {0, 2} (xaxb) and {1, 2}
    (xabx) of four qubits."""
    rng = np.random.default_rng(5)
    for qubits in ([0, 2], [1, 2]):
        rho = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
        u = unitary(4, rng)
        assert np.abs(run(rho, qubits, u, True) - O.dm_gate(rho, qubits, u)).max() <= 1e-13


def test_large_matrix_sampled_blocks():
    """n = 13 (8192 x 8192, complex128, 1 GiB): blocks sampled across the
    view against the oracle's single-block routine; trace preserved."""
    n = 13
    N = 1 << n
    rng = np.random.default_rng(9)
    rho = (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))).astype(np.complex128)
    for qubits in ([0], [12], [3, 9], [1, 6, 11]):
        u = unitary(1 << len(qubits), rng)
        t = torch.from_numpy(rho).cuda()
        M.dm_gate(t, qubits, u)
        got = t.cpu().numpy()
        perm = O.dm_perm(n, qubits)
        q = len(qubits)
        m = 1 << q
        nb = 1 << (n - q)
        for I, J in [(0, 0), (nb - 1, nb - 1), (17, 4000 % nb), (nb // 2, 3)]:
            ref = O.dm_gate_block(rho, qubits, u, I, J)
            for g in range(m):
                for h in range(m):
                    rp, cp = I * m + g, J * m + h
                    bits = [(rp >> (n - 1 - j)) & 1 for j in range(n)] + \
                           [(cp >> (n - 1 - j)) & 1 for j in range(n)]
                    old = [0] * (2 * n)
                    for j in range(2 * n):
                        old[perm[j]] = bits[j]
                    addr = int("".join(map(str, old)), 2)
                    assert abs(got.reshape(-1)[addr] - ref[g, h]) <= 1e-12 * max(1.0, abs(ref[g, h]))
        assert abs(np.trace(got) - np.trace(rho)) <= 1e-9 * abs(np.trace(rho))
        del t


def test_gate_errors():
    t = torch.zeros(16, 16, dtype=torch.complex64, device="cuda")
    for qubits, status in [([0, 1, 2, 3], M.FFT_ERR_UNSUPPORTED), ([4], M.FFT_ERR_ARG), ([1, 1], M.FFT_ERR_ARG)]:
        with pytest.raises(M.MoaFFTError) as e:
            M.dm_gate(t, qubits, np.eye(1 << len(qubits)))
        assert e.value.status == status
    with pytest.raises(M.MoaFFTError) as e:
        M.dm_gate(t.cpu(), [0], np.eye(2))  # host memory
    assert e.value.status == M.FFT_ERR_ARG
