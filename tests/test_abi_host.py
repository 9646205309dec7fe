"""Host-side checks of the C ABI: the library loads, exports every symbol
include/moafft.h declares, and rejects bad arguments before touching a GPU.
No compute call runs here."""
import json
import os
import re

import pytest

import paper_0803_2386_gb300 as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    M.build()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b((?:fft|dm)_[a-z_0-9]+)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_what_binding_lists():
    assert set(declared_functions()) == set(M.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = M.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_version_and_no_error():
    assert M.fft_version() >= 100


@pytest.mark.parametrize("n,bad", [(0, M.FFT_ERR_ARG), (-4, M.FFT_ERR_ARG), (12, M.FFT_ERR_NOT_POW2),
                                   (1000, M.FFT_ERR_NOT_POW2), (1 << 31, M.FFT_ERR_UNSUPPORTED)])
def test_plan_rejects_bad_length(n, bad):
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_plan(n, 1, M.FFT_C128, M.FFT_FORWARD)
    assert e.value.status == bad
    assert M.fft_last_error()


def test_plan_rejects_bad_batch_dtype_dir_form():
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_plan(16, 0)
    assert e.value.status == M.FFT_ERR_ARG
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_plan(16, 1, 7)
    assert e.value.status == M.FFT_ERR_DTYPE
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_plan(16, 1, M.FFT_C64, 0)
    assert e.value.status == M.FFT_ERR_DTYPE
    with pytest.raises(M.MoaFFTError) as e:
        M.fft_plan_ex(16, 1, M.FFT_C64, M.FFT_FORWARD, 9)
    assert e.value.status == M.FFT_ERR_ARG


def test_bad_schedules():
    for text in ["3,3", "x", "5,5,", "5@3,5", "10@0", "4,4,4,4,4,4,4,4,4", "5/5,5", "5/0,5", "5/,5"]:
        with pytest.raises(M.MoaFFTError) as e:
            M.fft_describe_schedule(1 << 10, M.FFT_C128, M.FFT_FORM_PLAIN, text)
        assert e.value.status == M.FFT_ERR_ARG, text


def test_null_handles():
    L = M.lib()
    assert L.fft_destroy(None) == 0
    assert L.fft_exec(None, None, None, None) == M.FFT_ERR_ARG
    assert L.fft_exec_adjoint(None, None, None, None) == M.FFT_ERR_ARG
    assert L.fft_plan(None, 16, 1, 0, -1) == M.FFT_ERR_ARG
    assert L.fft_plan_launches(None) == 0


@pytest.mark.parametrize("t", range(0, 25))
@pytest.mark.parametrize("dt", [M.FFT_C64, M.FFT_C128])
def test_default_schedule_covers_all_stages(t, dt):
    """The passes' radices add up to log2 n (every radix-2 stage once, Fig.
    vanloan_fft) and each pass lifts n to A x R x B consistently."""
    n = 1 << t
    s = json.loads(M.fft_describe_schedule(n, dt))
    assert s["n"] == n
    A = 1
    total = 0
    for i, p in enumerate(s["passes"]):
        R = 1 << p["log_r"]
        assert p["A"] == A and p["A"] * R * p["B"] == n
        assert sum(p["sub_log"]) == p["log_r"] and all(1 <= x <= 4 for x in p["sub_log"])
        assert R * p["width"] <= (4096 if dt == M.FFT_C128 else 8192) * 2
        if i < len(s["passes"]) - 1:
            assert p["B"] % p["width"] == 0 and p["tw_m"] == R * p["B"]
        A *= R
        total += p["log_r"]
    assert total == t
    assert s["passes"][-1]["B"] == 1


def test_default_schedule_splits():
    """One pass up to 2^12 points; complex64 beyond takes the split measured
    fastest on GB300 (column tiles of at least 4 columns, a third pass from
    2^21); complex128 from 2^16 to 2^22 a first pass of t - 12 and a last of
    12, otherwise balanced passes of at most 2^11."""
    c64 = {13: [7, 6], 14: [7, 7], 15: [7, 8], 16: [8, 8], 17: [8, 9], 18: [8, 10], 19: [9, 10],
           20: [10, 10], 21: [7, 7, 7], 22: [7, 7, 8], 23: [7, 8, 8], 24: [8, 8, 8]}
    for t in range(0, 31):
        for dt in (M.FFT_C64, M.FFT_C128):
            radices = [p["log_r"] for p in json.loads(M.fft_describe_schedule(1 << t, dt))["passes"]]
            if t <= 12:
                assert radices == [t], (t, dt)
            elif dt == M.FFT_C64 and t in c64:
                assert radices == c64[t], t
            elif dt == M.FFT_C128 and 16 <= t <= 22:
                assert radices == [t - 12, 12], t
            else:
                cap = 11 if dt == M.FFT_C128 else 10
                g = -(-t // cap)
                assert len(radices) == g and max(radices) - min(radices) <= 1 and max(radices) <= cap


def test_explicit_schedule_parse():
    s = json.loads(M.fft_describe_schedule(1 << 12, M.FFT_C64, M.FFT_FORM_PLAIN, "4@8,4,4"))
    assert [p["log_r"] for p in s["passes"]] == [4, 4, 4]
    assert s["passes"][0]["width"] == 8
    assert [p["B"] for p in s["passes"]] == [256, 16, 1]


def test_allocator_hook_arguments():
    with pytest.raises(M.MoaFFTError):
        M.lib().fft_set_allocator(M.ALLOC_FN(lambda n, c: 0), M.FREE_FN(), None) and None
        _ = M._check(M.lib().fft_set_allocator(M.ALLOC_FN(lambda n, c: 0), M.FREE_FN(), None))
    M.fft_set_allocator(None, None)


@pytest.mark.parametrize("t", [0, 3, 6, 10, 12, 13, 16, 20, 24])
@pytest.mark.parametrize("dt", [M.FFT_C64, M.FFT_C128])
def test_tune_candidates_are_valid_schedules(t, dt):
    """Every schedule the autotuner may time covers all log2 n stages."""
    cands = M.fft_tune_candidates(1 << t, dt)
    assert cands and len(set(cands)) == len(cands)
    for c in cands:
        s = json.loads(M.fft_describe_schedule(1 << t, dt, M.FFT_FORM_PLAIN, c))
        assert sum(p["log_r"] for p in s["passes"]) == t


def test_unblocked_schedule_describes_stages():
    s = json.loads(M.fft_describe_schedule(1 << 12, M.FFT_C64, M.FFT_FORM_PLAIN, "stages"))
    assert s["unblocked"] and s["stages"] == 12 and s["passes"] == [] and s["order"] == "onf"
    s = json.loads(M.fft_describe_schedule(1 << 12, M.FFT_C64, M.FFT_FORM_PLAIN, "stages_stride"))
    assert s["unblocked"] and s["order"] == "stride"


def test_cluster_schedule_describes_two_groups():
    """Schedule "cluster" (complex64, n = 2^16): the 8,8 split whose
    reshape-transpose goes through distributed shared memory."""
    s = json.loads(M.fft_describe_schedule(1 << 16, M.FFT_C64, M.FFT_FORM_PLAIN, "cluster"))
    assert s["cluster"] is True and [p["log_r"] for p in s["passes"]] == [8, 8]
    for n, dt in [(1 << 15, M.FFT_C64), (1 << 16, M.FFT_C128), (1 << 17, M.FFT_C64)]:
        with pytest.raises(M.MoaFFTError) as e:
            M.fft_describe_schedule(n, dt, M.FFT_FORM_PLAIN, "cluster")
        assert e.value.status == M.FFT_ERR_UNSUPPORTED
    assert "cluster" in M.fft_tune_candidates(1 << 16, M.FFT_C64)
    assert "cluster" not in M.fft_tune_candidates(1 << 16, M.FFT_C128)


def test_dm_transpose_vector_matches_the_paper_and_the_oracle():
    """Host-side transpose vector of the gating entry point: the printed
    worked examples, and the oracle's construction for other qubit sets."""
    import oracle as O
    assert M.dm_transpose_vector(4, [0, 2]) == [0, 2, 1, 3, 4, 6, 5, 7]
    assert M.dm_transpose_vector(4, [2, 1]) == [0, 3, 1, 2, 4, 7, 5, 6]
    for n, qb in [(1, [0]), (5, [4]), (6, [0, 5]), (7, [3, 1, 6])]:
        assert M.dm_transpose_vector(n, qb) == list(O.dm_perm(n, qb))


def test_dm_gate_argument_errors():
    L = M.lib()
    for n, qb in [(4, [4]), (4, [1, 1]), (0, [0]), (3, [-1])]:
        with pytest.raises(M.MoaFFTError) as e:
            M.dm_transpose_vector(n, qb)
        assert e.value.status == M.FFT_ERR_ARG
    assert L.dm_gate(None, 4, None, 1, None, M.FFT_C64, None) == M.FFT_ERR_ARG


def test_register_digit_schedules():
    """'/k' limits the register digits of a pass to 2^k points (the general
    radix of fftpsiradn as a schedule dimension); the default split is a
    first digit of log_r mod 4 bits, then radix-16 digits."""
    s = json.loads(M.fft_describe_schedule(1 << 16, M.FFT_C64, M.FFT_FORM_PLAIN, "10/2,6/3"))
    assert [p["sub_log"] for p in s["passes"]] == [[2, 2, 2, 2, 2], [3, 3]]
    s = json.loads(M.fft_describe_schedule(1 << 16, M.FFT_C64, M.FFT_FORM_PLAIN, "10,6"))
    assert [p["sub_log"] for p in s["passes"]] == [[2, 4, 4], [2, 4]]
    s = json.loads(M.fft_describe_schedule(1 << 13, M.FFT_C64, M.FFT_FORM_PLAIN, "7/1,6/1"))
    assert [sum(p["sub_log"]) for p in s["passes"]] == [7, 6] and s["passes"][0]["sub_log"] == [1] * 7
    assert "8/1,8/1" in M.fft_tune_candidates(1 << 16, M.FFT_C64)



def test_plan_nd_argument_errors():
    """fft_plan_nd validates its shape before touching the GPU."""
    cases = [
        (([64, 5000], 1), "NOT_POW2"),
        (([1 << 25, 2], 1), "UNSUPPORTED"),         # an axis before the last above 2^24
        (([4096, 4096, 8192], 1), "UNSUPPORTED"),   # 2^37 points per array
        (([], 1), "FFT_ERR_ARG"),
        (([2] * 9, 1), "FFT_ERR_ARG"),
        (([16, 16], 0), "FFT_ERR_ARG"),
        (([16, 0], 1), "FFT_ERR_ARG"),
    ]
    for (dims, batch), code in cases:
        with pytest.raises(M.MoaFFTError, match=code):
            M.fft_plan_nd(dims, batch, M.FFT_C64, M.FFT_FORWARD)
    with pytest.raises(M.MoaFFTError, match="FFT_ERR_DTYPE"):
        M.fft_plan_nd([16, 16], 1, 7, M.FFT_FORWARD)


def test_fftn_wrapper_rejects_bad_axis_counts():
    torch = pytest.importorskip("torch")
    x = torch.zeros(2, 4, 8, dtype=torch.complex64)
    for nd in (0, 4, 9):
        with pytest.raises(ValueError):
            M.fftn(x, ndim=nd)
        with pytest.raises(ValueError):
            M.fftn_autograd(x, ndim=nd)
