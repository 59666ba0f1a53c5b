"""weno_sums_noalloc: the conservation sums for callers that cannot allocate
device memory (their scratch is a fixed array inside the library), checked
through the C ABI against the allocating entry point weno_sums.  This file is
collected last so that a stop at the first failure has already run every other
test."""
import ctypes

import numpy as np
import pytest

from paper_2405_12301_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12301_gb300 import build, weno
    build.build()
    return weno, weno.lib()


def _call(L, U, nf, out, stream):
    return L.weno_sums_noalloc(ctypes.c_void_p(U.data_ptr()), nf, U.numel() // nf, ctypes.c_void_p(out.data_ptr()),
                               stream)


def _ref(weno, dim, n, U):
    s = weno.Solver(dim, n)
    ref = np.array(s.sums(U))
    s.close()
    return ref


def test_sums_noalloc_matches_weno_sums_on_two_calls_in_a_row():
    """Two calls in a row, each synchronised, with other nf, sizes and data; the
    second grid has more than 1024 x 4096 cells, so its reduction fills all 1024
    partial-sum slots of the scratch array.  Both results are bitwise those of
    weno_sums (the same fixed-order reduction)."""
    weno, L = _lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(3, (40, 30, 20), 1), (2, (2100, 2100), 2)]
    assert 2100 * 2100 > 1024 * 4096
    for dim, n, seed in cases:
        U = torch.from_numpy(I.random_state(dim, n, seed=seed, jumps=True)).cuda()
        nf = dim + 2
        out = torch.full((nf,), float("nan"), dtype=torch.float64, device="cuda")
        code = _call(L, U, nf, out, stream)
        assert code == weno.OK, L.weno_last_error(None)
        torch.cuda.synchronize()
        ref = _ref(weno, dim, n, U)
        np.testing.assert_array_equal(out.cpu().numpy(), ref)


def test_sums_noalloc_two_calls_queued_on_one_stream():
    """Two calls queued back to back on one stream with no synchronisation
    between them (stream order keeps the second call's use of the shared scratch
    after the first's): both equal weno_sums bitwise."""
    weno, L = _lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = (2100, 2100)
    A = torch.from_numpy(I.random_state(2, n, seed=3, jumps=True)).cuda()
    B = torch.from_numpy(I.random_state(2, n, seed=4)).cuda()
    oa = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    ob = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(L, A, 4, oa, stream) == weno.OK
    assert _call(L, B, 4, ob, stream) == weno.OK
    torch.cuda.synchronize()
    np.testing.assert_array_equal(oa.cpu().numpy(), _ref(weno, 2, n, A))
    np.testing.assert_array_equal(ob.cpu().numpy(), _ref(weno, 2, n, B))


def test_sums_noalloc_rejects_sizes_beyond_its_scratch():
    weno, L = _lib()
    U = torch.zeros((6, 10), dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    code = L.weno_sums_noalloc(ctypes.c_void_p(U.data_ptr()), 6, 10, ctypes.c_void_p(out.data_ptr()), None)
    assert code == weno.ERR_ARG
    assert b"nf must be 1..5" in L.weno_last_error(None)
