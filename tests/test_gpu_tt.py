"""GPU TT-rounding and TT-SSPRK3 stage combination (weno_tt_round) against the
FP64 oracle (oracle/tt.py).  GPU only.

TT cores are not unique (any invertible matrix between two cores gives the
same tensor), so the comparison is on what is unique: the full tensor, the
ranks chosen (cases with clear singular-value gaps), the norm, the error bound,
and the left-orthogonality of the output cores.  Tolerance: both sides run
the same two-pass algorithm in FP64 with Householder QR; a backward-stable QR
and SVD give a relative error of a few hundred ulp of the sum's scale, so the
full tensors agree to 1e-12 relative to sum_t |c_t| ||X_t||."""
import math

import numpy as np
import pytest

from oracle import tt as OT

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


def rand_tt(rng, n, r, scale=1.0):
    r0 = (1, r[0], r[1], 1)
    return [scale * rng.standard_normal((n[m], r0[m], r0[m + 1])) for m in range(3)]


def dev_terms(terms):
    return [(c, [torch.from_numpy(np.ascontiguousarray(g)).cuda() for g in cores]) for c, cores in terms]


def host(cores):
    torch.cuda.synchronize()
    return [g.cpu().numpy() for g in cores]


def scale(terms):
    return sum(abs(c) * np.linalg.norm(OT.tt_full(cores)) for c, cores in terms)


def left_orth_err(cores):
    M1 = cores[0][:, 0, :]
    M2 = cores[1].transpose(1, 0, 2).reshape(-1, cores[1].shape[2])
    return max(np.abs(M1.T @ M1 - np.eye(M1.shape[1])).max(), np.abs(M2.T @ M2 - np.eye(M2.shape[1])).max())


def compare(W, H, problems, eps):
    outs = W.weno_tt_round(H, [dev_terms(t) for t in problems], eps)
    for terms, (cores, norm) in zip(problems, outs):
        G = host(cores)
        Y, s, no = OT.tt_round(OT.tt_add(terms), eps)
        S = scale(terms)
        F = OT.tt_full(OT.tt_add(terms))
        assert (G[0].shape[2], G[1].shape[2]) == (Y[0].shape[2], Y[1].shape[2])
        assert np.linalg.norm(OT.tt_full(G) - OT.tt_full(Y)) <= 1e-12 * S
        assert abs(norm - no) <= 1e-12 * S
        assert np.linalg.norm(OT.tt_full(G) - F) <= eps * np.linalg.norm(F) + 1e-12 * S
        assert left_orth_err(G) <= 1e-12
    return outs


SHAPES = [
    ((5, 4, 6), [(2, 3)]),
    ((12, 10, 9), [(3, 2), (2, 4), (1, 1)]),
    ((40, 3, 7), [(5, 6), (4, 3)]),            # n3 < R2: the last QR is short and wide
    ((3, 30, 4), [(2, 5), (3, 2)]),            # tiny first and last modes
    ((64, 60, 50), [(12, 14), (10, 9)]),       # several row chunks in the middle QRs
    ((20, 120, 20), [(8, 8), (8, 8)]),
    ((33, 17, 65), [(32, 32), (32, 32), (32, 32)]),  # summed ranks at the 96 limit
]


@pytest.mark.parametrize("n,ranks", SHAPES)
def test_round_of_full_rank_sums_matches_oracle(W, H, n, ranks):
    rng = np.random.default_rng(sum(n))
    terms = [(rng.uniform(-2, 2), rand_tt(rng, n, r)) for r in ranks]
    compare(W, H, [terms], 1e-12)


def test_redundant_sum_rounds_to_the_exact_rank(W, H):
    rng = np.random.default_rng(11)
    X = rand_tt(rng, (30, 25, 20), (3, 4))
    (G, _), = compare(W, H, [[(1.0, X), (1.0, X), (-1.0, X)]], 1e-12)
    assert (G[0].shape[2], G[1].shape[2]) == (3, 4)


def test_cancelling_sum_is_zero_to_rounding(W, H):
    rng = np.random.default_rng(12)
    X = rand_tt(rng, (16, 15, 14), (4, 5))
    outs = W.weno_tt_round(H, [dev_terms([(1.0, X), (-1.0, X)])], 1e-10)
    G = host(outs[0][0])
    assert np.linalg.norm(OT.tt_full(G)) <= 1e-13 * 2 * np.linalg.norm(OT.tt_full(X))


def _decaying(rng, n, decay, terms=12):
    F = np.zeros(n)
    for p in range(terms):
        u, v, w = rng.standard_normal(n[0]), rng.standard_normal(n[1]), rng.standard_normal(n[2])
        F += decay ** p * np.einsum("i,j,k->ijk", u, v, w)
    U1, s1, V1 = np.linalg.svd(F.reshape(n[0], -1), full_matrices=False)
    rest = (s1[:, None] * V1).reshape(len(s1) * n[1], n[2])
    U2, s2, V2 = np.linalg.svd(rest, full_matrices=False)
    return [U1[:, None, :], U2.reshape(len(s1), n[1], len(s2)).transpose(1, 0, 2), (s2[:, None] * V2).T[:, :, None]]


@pytest.mark.parametrize("eps", [1e-2, 1e-5, 1e-9])
def test_truncation_meets_the_bound_with_the_oracle_ranks(W, H, eps):
    rng = np.random.default_rng(13)
    X = _decaying(rng, (20, 18, 16), 0.25)
    Y = _decaying(rng, (20, 18, 16), 0.25)
    compare(W, H, [[(1.0, X)], [(0.7, X), (0.3, Y)]], eps)


def test_batch_of_uneven_problems_in_one_call(W, H):
    rng = np.random.default_rng(14)
    probs = []
    for k in range(9):
        n = tuple(int(x) for x in rng.choice([8, 16, 33, 64], size=3))
        probs.append([(1.0, rand_tt(rng, n, (int(rng.integers(1, 9)), int(rng.integers(1, 9))))),
                      (0.01, rand_tt(rng, n, (int(rng.integers(1, 9)), int(rng.integers(1, 9)))))])
    compare(W, H, probs, 1e-10)


def _sample_full(cores, idx):
    G1, G2, G3 = cores
    return np.array([G1[i, 0] @ G2[j] @ G3[k, :, 0] for i, j, k in idx])


def test_full_size_modes_sampled(W, H):
    """n = 512 and 2 x 32 summed ranks (the largest TT-cross workload instance):
    sampled elements of the GPU result equal the oracle's, and the cores are
    orthogonal."""
    rng = np.random.default_rng(15)
    n = (512, 256, 512)
    terms = [(1.0, rand_tt(rng, n, (32, 32))), (0.05, rand_tt(rng, n, (32, 32)))]
    (G, norm), = W.weno_tt_round(H, [dev_terms(terms)], 1e-10)
    G = host(G)
    Y, s, no = OT.tt_round(OT.tt_add(terms), 1e-10)
    assert (G[0].shape[2], G[1].shape[2]) == (Y[0].shape[2], Y[1].shape[2]) == (64, 64)
    idx = rng.integers(0, [n[0], n[1], n[2]], size=(2000, 3))
    a, b = _sample_full(G, idx), _sample_full(Y, idx)
    S = max(np.abs(b).max(), 1.0)
    assert np.abs(a - b).max() <= 1e-11 * S
    assert norm == pytest.approx(no, rel=1e-12)
    assert left_orth_err(G) <= 1e-12


def test_ssprk3_stages_on_the_gpu_give_the_stability_polynomial(W, H):
    """The three stages of Eq. (tt-ssprk3), each the forward-Euler rounding and
    the stage combination (two weno_tt_round calls), for L(u) = c u: U^{n+1} =
    (1 + z + z^2/2 + z^3/6) U^n with z = c dt."""
    rng = np.random.default_rng(16)
    U = rand_tt(rng, (24, 20, 16), (3, 3))
    c, dt = -1.3, 0.31
    h = H
    Ud = dev_terms([(1.0, U)])[0][1]

    def rnd(terms):
        return W.weno_tt_round(h, [terms], 1e-13)[0][0]

    def L(V):
        return [c * V[0], V[1], V[2]]

    Uk = Ud
    for stage in range(3):
        F = rnd([(1.0, Uk), (dt, L(Uk))])
        if stage == 0:
            Uk = F
        else:
            a, b = ((0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))[stage - 1]
            Uk = rnd([(a, Ud), (b, F)])
        Uk = [g.contiguous() for g in Uk]
    z = c * dt
    want = (1 + z + z * z / 2 + z ** 3 / 6) * OT.tt_full(U)
    got = OT.tt_full(host(Uk))
    assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    assert (Uk[0].shape[2], Uk[1].shape[2]) == (3, 3)


def test_rejects_bad_batches(W, H):
    rng = np.random.default_rng(17)
    big = [(1.0, rand_tt(rng, (8, 8, 8), (40, 8))), (1.0, rand_tt(rng, (8, 8, 8), (40, 8))),
           (1.0, rand_tt(rng, (8, 8, 8), (20, 8)))]
    with pytest.raises(W.WenoError) as e:
        W.weno_tt_round(H, [dev_terms(big)], 1e-8)
    assert e.value.code == W.ERR_UNSUPPORTED
    mixed = [(1.0, rand_tt(rng, (8, 8, 8), (2, 2))), (1.0, rand_tt(rng, (8, 9, 8), (2, 2)))]
    with pytest.raises(W.WenoError) as e:
        W.weno_tt_round(H, [dev_terms(mixed)], 1e-8)
    assert e.value.code == W.ERR_ARG
    with pytest.raises(W.WenoError) as e:
        W.weno_tt_round(H, [dev_terms([(1.0, rand_tt(rng, (8, 8, 8), (2, 2)))])], -1.0)
    assert e.value.code == W.ERR_ARG
