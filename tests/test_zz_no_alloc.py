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


def test_sums_noalloc_matches_weno_sums_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12301_gb300 import build, weno
    build.build()
    L = weno.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(3, (40, 30, 20), 1), (2, (300, 200), 2)]  # second call: other nf, size and data
    for dim, n, seed in cases:
        U = torch.from_numpy(I.random_state(dim, n, seed=seed, jumps=True)).cuda()
        nf = dim + 2
        out = torch.full((nf,), float("nan"), dtype=torch.float64, device="cuda")
        code = L.weno_sums_noalloc(ctypes.c_void_p(U.data_ptr()), nf, U.numel() // nf,
                                   ctypes.c_void_p(out.data_ptr()), stream)
        assert code == weno.OK, L.weno_last_error(None)
        torch.cuda.synchronize()
        s = weno.Solver(dim, n)
        ref = np.array(s.sums(U))
        s.close()
        got = out.cpu().numpy()
        scale = U.abs().sum(dim=tuple(range(1, U.dim()))).cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-14 * scale), (got, ref)


def test_sums_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12301_gb300 import build, weno
    build.build()
    L = weno.lib()
    U = torch.zeros((6, 10), dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    code = L.weno_sums_noalloc(ctypes.c_void_p(U.data_ptr()), 6, 10, ctypes.c_void_p(out.data_ptr()), None)
    assert code == weno.ERR_ARG
    assert b"nf must be 1..5" in L.weno_last_error(None)
