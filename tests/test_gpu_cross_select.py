"""Cross-index selection on the GPU: batched maxvol (weno_maxvol) and the
fixed-rank TT-cross driver (weno_tt_cross) against the oracle (oracle/cross.py).
GPU only.

maxvol returns indices, so they are compared exactly; the decisions are
argmaxes of FP64 values computed in a different order on the two sides, so
the inputs are random matrices without near-ties, and the GPU result is also
checked for what defines it (a dominant submatrix: |A A[I]^{-1}| <= 1 + delta,
recomputed in numpy from the GPU's indices)."""
import itertools

import numpy as np
import pytest

from oracle import cross as X

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_12301_gb300 import build, weno
    build.build()
    weno.lib()
    return weno


@pytest.fixture(scope="module")
def H(W):
    h = W.weno_init(None)
    yield h
    W.weno_destroy(h)


SIZES = [(1, 1), (40, 1), (5, 4), (64, 16), (300, 12), (1000, 32), (2560, 32), (700, 64)]


def test_maxvol_matches_oracle(W, H):
    rng = np.random.default_rng(1)
    mats = [rng.standard_normal(s) for s in SIZES]
    outs = W.weno_maxvol(H, [torch.from_numpy(A).cuda() for A in mats], delta=1e-2)
    for A, (idx, B, swaps) in zip(mats, outs):
        I = idx.cpu().numpy()
        Io, Bo, so = X.maxvol(A, delta=1e-2)
        assert I.tolist() == Io.tolist()
        assert swaps == so
        assert np.abs(B.cpu().numpy() - Bo).max() <= 1e-9 * max(1.0, np.abs(Bo).max())
        Bn = A @ np.linalg.inv(A[I])
        assert np.abs(Bn).max() <= 1.0 + 1e-2 + 1e-10


def test_maxvol_with_one_spare_row_finds_the_maximum_volume(W, H):
    rng = np.random.default_rng(2)
    mats = [rng.standard_normal((r + 1, r)) for r in (2, 3, 4, 5) for _ in range(5)]
    outs = W.weno_maxvol(H, [torch.from_numpy(A).cuda() for A in mats], delta=0.0)
    for A, (idx, _, _) in zip(mats, outs):
        r = A.shape[1]
        I = idx.cpu().numpy()
        best = max(abs(np.linalg.det(A[list(s)])) for s in itertools.combinations(range(r + 1), r))
        assert abs(np.linalg.det(A[I])) >= best * (1 - 1e-12)


def test_maxvol_rejects_rank_deficient_matrices(W, H):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((50, 4))
    A[:, 3] = A[:, 1]
    with pytest.raises(W.WenoError) as e:
        W.weno_maxvol(H, [torch.from_numpy(A).cuda()])
    assert e.value.code == W.ERR_ARG
