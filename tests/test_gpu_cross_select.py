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


def test_maxvol_large_and_mixed_batch_matches_oracle(W, H):
    """Row counts from fewer rows than a cluster has CTAs up to the 65536-row
    limit, orthonormal inputs as the TT-cross passes them, in one batch (the
    batch is launched largest first; results keep the caller's order)."""
    rng = np.random.default_rng(4)
    sizes = [(3, 3), (65536, 8), (17, 16), (15360, 32), (4097, 64), (9, 2)]
    mats = []
    for k, s in enumerate(sizes):
        A = rng.standard_normal(s)
        mats.append(np.linalg.qr(A)[0] if k % 2 else A)
    outs = W.weno_maxvol(H, [torch.from_numpy(A).cuda() for A in mats], delta=1e-2)
    for A, (idx, B, swaps) in zip(mats, outs):
        Io, Bo, so = X.maxvol(A, delta=1e-2)
        assert idx.cpu().numpy().tolist() == Io.tolist()
        assert swaps == so
        assert np.abs(B.cpu().numpy() - Bo).max() <= 1e-9 * max(1.0, np.abs(Bo).max())


def test_maxvol_stops_at_max_iters(W, H):
    rng = np.random.default_rng(5)
    mats = [rng.standard_normal((3000, 24)) for _ in range(3)]
    outs = W.weno_maxvol(H, [torch.from_numpy(A).cuda() for A in mats], delta=1e-2, max_iters=2)
    for A, (idx, B, swaps) in zip(mats, outs):
        Io, Bo, so = X.maxvol(A, delta=1e-2, max_iters=2)
        assert so == 2 and swaps == 2
        assert idx.cpu().numpy().tolist() == Io.tolist()
        assert np.abs(B.cpu().numpy() - Bo).max() <= 1e-9 * max(1.0, np.abs(Bo).max())


def test_maxvol_of_an_ill_conditioned_matrix_equals_that_of_its_q_factor(W, H):
    """maxvol's pivots and B = A A[I]^{-1} depend only on A's column space when
    A = Q R with R upper triangular (the Schur-complement residual of Q's column
    j is a multiple of A's), which is why the TT-cross path skips the QR: the
    GPU's rows for A equal the oracle's rows for Q, and B agrees to about
    eps cond(A)."""
    rng = np.random.default_rng(7)
    for n, r, c, tol in [(3000, 32, 1e-4, 1e-8), (500, 12, 1e-8, None)]:
        G = rng.standard_normal((n, r)) * np.geomspace(1, c, r)
        A = G @ (np.eye(r) + 0.5 * np.triu(rng.standard_normal((r, r)), 1))
        (idx, B, swaps), = W.weno_maxvol(H, [torch.from_numpy(A).cuda()], delta=1e-2)
        Io, Bo, so = X.maxvol(np.linalg.qr(A)[0], delta=1e-2)
        assert idx.cpu().numpy().tolist() == Io.tolist()
        assert swaps == so
        if tol is not None:
            assert np.abs(B.cpu().numpy() - Bo).max() <= tol


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


# ------------------------------------------------------------ TT-cross driver
import oracle as O  # noqa: E402
from paper_2405_12301_gb300 import inputs as I  # noqa: E402


def _instance(seed, n, r):
    inst = I.tt_instance(seed=seed, n=n, r=r, device="cpu")
    n, r, cores = inst["n"], inst["r"], inst["cores"]
    U = np.stack([O.tt_full(n, r, cores[f]) for f in range(5)])
    cfg = O.Cfg(dim=3, n=tuple(n), hi=(1.0, 1.0, 1.0), bc=((O.PERIODIC, O.PERIODIC),) * 3)
    return dict(n=n, r=r, cores=cores, h=[1.0 / n[0], 1.0 / n[1], 1.0 / n[2]], bc=((0, 0),) * 3,
                alpha=1.05 * O.alpha_max(cfg, U))


def _dev(inst):
    d = dict(inst)
    d["cores"] = [[torch.from_numpy(c).cuda() for c in fc] for fc in inst["cores"]]
    return d


def _oracle_fun(inst, fd):
    def fun(mode, left, right):
        return O.cross_eval(inst["n"], inst["r"], inst["cores"], inst["h"], inst["alpha"], 1.4, 1e-6, inst["bc"],
                            mode, fd, left, right)
    return fun


def _initial_sets(rng, n, r1, r2):
    J1 = np.stack([rng.choice(n[1], r1), rng.choice(n[2], r1), rng.integers(0, 5, r1)], 1).astype(np.int32)
    J2 = np.stack([rng.choice(n[2], r2, replace=False), rng.integers(0, 5, r2)], 1).astype(np.int32)
    return J1, J2


@pytest.mark.parametrize("fd,sweeps", [(0, 1), (1, 1), (2, 0), (2, 2)])
def test_tt_cross_matches_oracle_fp64(W, H, fd, sweeps):
    """Same function (the FP64 pointwise residual), same initial sets: the GPU
    sweep selects the same index sets as the oracle and builds the same cores."""
    rng = np.random.default_rng(10 + fd)
    insts = [_instance(40 + k, [12, 16, 10], [3, 4]) for k in range(2)]
    ranks = [(4, 6), (3, 5)]
    sets = [_initial_sets(rng, insts[k]["n"], *ranks[k]) for k in range(2)]
    outs = W.weno_tt_cross(H, [_dev(d) for d in insts], fd, ranks,
                           [torch.from_numpy(s[0].copy()).cuda() for s in sets],
                           [torch.from_numpy(s[1].copy()).cuda() for s in sets], sweeps=sweeps, fp64_check=True)
    torch.cuda.synchronize()
    for k in range(2):
        G, I1, I2, J1, J2 = X.cross_sweeps(_oracle_fun(insts[k], fd), insts[k]["n"], ranks[k], sets[k][0], sets[k][1],
                                           sweeps=sweeps)
        o = outs[k]
        assert o["I1"].cpu().numpy().tolist() == I1.tolist()
        assert o["I2"].cpu().numpy().tolist() == I2.tolist()
        assert o["J1"].cpu().numpy().tolist() == J1.tolist()
        assert o["J2"].cpu().numpy().tolist() == J2.tolist()
        T, To = X.tt4_full([c.cpu().numpy() for c in o["cores"]]), X.tt4_full(G)
        assert np.abs(T - To).max() <= 1e-10 * np.abs(To).max()


def test_tt_cross_fp32_interpolates_the_residual_on_its_sets(W, H):
    """FP32 fiber evaluation: the TT equals the (FP64 oracle) residual on the
    final cross to FP32 accuracy, and the first core is the identity on I1."""
    rng = np.random.default_rng(20)
    inst = _instance(50, [16, 12, 14], [4, 3])
    r1, r2 = 5, 7
    J1, J2 = _initial_sets(rng, inst["n"], r1, r2)
    o, = W.weno_tt_cross(H, [_dev(inst)], 1, [(r1, r2)], [torch.from_numpy(J1).cuda()],
                         [torch.from_numpy(J2).cuda()], sweeps=1)
    torch.cuda.synchronize()
    G = [c.cpu().numpy() for c in o["cores"]]
    I1, I2, J2o = o["I1"].cpu().numpy(), o["I2"].cpu().numpy(), o["J2"].cpu().numpy()
    assert np.allclose(G[0][I1, 0, :], np.eye(r1), atol=1e-12)
    T = X.tt4_full(G)
    fun = _oracle_fun(inst, 1)
    A2 = fun(2, I2, np.zeros((1, 0), np.int32))           # A(I2, :, f)
    scale = np.abs(A2).max()
    for b in range(r2):
        i, j = I2[b]
        assert np.abs(T[i, j] - A2[:, b, :, 0].T).max() <= 1e-5 * scale
    A1 = fun(1, I1[:, None].astype(np.int32), J2o[:, :1].astype(np.int32))   # A(I1, :, J2)
    for b in range(r2):
        k, f = J2o[b]
        assert np.abs(T[I1][:, :, k, f] - A1[f, :, :, b]).max() <= 1e-5 * scale
