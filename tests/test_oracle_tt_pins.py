"""Pins of the TT-algebra oracle (oracle/tt.py) against facts that do not come
from the oracle itself: brute-force element loops, singular values of the full
tensor's unfoldings (numpy SVD of the full tensor, the TT-SVD route), the
error bound of TT-rounding, orthogonality, and the stability polynomial of
SSP-RK3 for a linear operator."""
import math

import numpy as np
import pytest

from oracle import tt


def rand_tt(rng, n, r, scale=1.0):
    r0 = (1, r[0], r[1], 1)
    return [scale * rng.standard_normal((n[m], r0[m], r0[m + 1])) for m in range(3)]


def brute_full(cores):
    G1, G2, G3 = cores
    n = [c.shape[0] for c in cores]
    X = np.zeros(n)
    for i in range(n[0]):
        for j in range(n[1]):
            for k in range(n[2]):
                X[i, j, k] = float(G1[i, 0, :] @ G2[j] @ G3[k, :, 0])
    return X


def test_full_and_add_match_brute_force():
    rng = np.random.default_rng(1)
    A = rand_tt(rng, (4, 3, 5), (2, 3))
    B = rand_tt(rng, (4, 3, 5), (3, 1))
    assert np.allclose(tt.tt_full(A), brute_full(A), rtol=0, atol=1e-13)
    S = tt.tt_add([(0.7, A), (-2.0, B)])
    assert [c.shape for c in S] == [(4, 1, 5), (3, 5, 4), (5, 4, 1)]
    assert np.allclose(brute_full(S), 0.7 * brute_full(A) - 2.0 * brute_full(B), rtol=0, atol=1e-12)


def test_rounding_recovers_the_exact_rank_of_a_redundant_sum():
    """X + X - X is X with every rank tripled; rounding at eps = 1e-12 returns
    X's ranks and X itself."""
    rng = np.random.default_rng(2)
    X = rand_tt(rng, (9, 8, 7), (2, 3))
    Y, s, norm = tt.tt_round(tt.tt_add([(1.0, X), (1.0, X), (-1.0, X)]), 1e-12)
    assert (Y[0].shape[2], Y[1].shape[2]) == (2, 3)
    F = tt.tt_full(X)
    assert np.linalg.norm(tt.tt_full(Y) - F) <= 1e-12 * np.linalg.norm(F)
    assert norm == pytest.approx(np.linalg.norm(F), rel=1e-13)


def test_singular_values_equal_those_of_the_full_unfoldings():
    """Without truncation the SVDs of the rounding are those of the unfoldings
    X_(1) (n1 x n2 n3) and X_(2) (n1 n2 x n3) of the full tensor."""
    rng = np.random.default_rng(3)
    n = (6, 5, 7)
    X = tt.tt_add([(1.0, rand_tt(rng, n, (3, 4))), (0.5, rand_tt(rng, n, (2, 2)))])
    F = tt.tt_full(X)
    _, s, _ = tt.tt_round(X, 0.0)
    s1 = np.linalg.svd(F.reshape(n[0], -1), compute_uv=False)
    s2 = np.linalg.svd(F.reshape(n[0] * n[1], n[2]), compute_uv=False)
    k1, k2 = len(s[0]), len(s[1])
    assert np.allclose(s[0], s1[:k1], rtol=0, atol=1e-12 * s1[0])
    assert np.allclose(s[1], s2[:k2], rtol=0, atol=1e-12 * s2[0])


def _decaying_tensor(rng, n, decay):
    """Full tensor with geometrically decaying spectra in every unfolding."""
    F = np.zeros(n)
    for p in range(min(n)):
        u, v, w = (rng.standard_normal(n[0]), rng.standard_normal(n[1]), rng.standard_normal(n[2]))
        F += decay ** p * np.einsum("i,j,k->ijk", u, v, w)
    return F


def _tt_svd_exact(F):
    """TT of a full tensor without truncation (sequential SVDs of the unfoldings)."""
    n = F.shape
    U1, s1, V1 = np.linalg.svd(F.reshape(n[0], -1), full_matrices=False)
    G1 = U1[:, None, :]
    rest = (s1[:, None] * V1).reshape(len(s1) * n[1], n[2])
    U2, s2, V2 = np.linalg.svd(rest, full_matrices=False)
    G2 = U2.reshape(len(s1), n[1], len(s2)).transpose(1, 0, 2)
    G3 = (s2[:, None] * V2).T[:, :, None]
    return [G1, G2, G3]


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-7])
def test_rounding_meets_its_error_bound_and_the_tt_svd_ranks(eps):
    """||X - round(X)|| <= eps ||X|| (Sec. 3); the ranks are those the full
    tensor's TT-SVD picks at the same threshold (same sequential SVDs)."""
    rng = np.random.default_rng(4)
    n = (12, 10, 11)
    F = _decaying_tensor(rng, n, 0.3)
    X = _tt_svd_exact(F)
    Y, s, norm = tt.tt_round(X, eps)
    err = np.linalg.norm(tt.tt_full(Y) - F)
    assert err <= eps * np.linalg.norm(F)
    delta = eps / math.sqrt(2) * np.linalg.norm(F)
    s1 = np.linalg.svd(F.reshape(n[0], -1), compute_uv=False)
    r1 = next(r for r in range(1, len(s1) + 1) if np.sqrt((s1[r:] ** 2).sum()) <= delta)
    assert Y[0].shape[2] == r1
    # a smaller rank at the first unfolding would already break the bound there
    if r1 > 1:
        assert np.sqrt((s1[r1 - 1:] ** 2).sum()) > delta


def test_rounded_cores_are_left_orthogonal():
    rng = np.random.default_rng(5)
    X = tt.tt_add([(1.0, rand_tt(rng, (10, 9, 8), (4, 5))), (1e-3, rand_tt(rng, (10, 9, 8), (3, 3)))])
    Y, _, _ = tt.tt_round(X, 1e-6)
    M1 = Y[0][:, 0, :]
    M2 = Y[1].transpose(1, 0, 2).reshape(-1, Y[1].shape[2])
    assert np.allclose(M1.T @ M1, np.eye(M1.shape[1]), atol=1e-13)
    assert np.allclose(M2.T @ M2, np.eye(M2.shape[1]), atol=1e-13)


def test_ssprk3_stages_give_the_third_order_stability_polynomial():
    """For L(u) = c u the three TT stages (Eq. tt-ssprk3) multiply U^n by
    1 + z + z^2/2 + z^3/6 with z = c dt, the SSP-RK3 stability polynomial."""
    rng = np.random.default_rng(6)
    U = rand_tt(rng, (7, 6, 5), (2, 2))
    c, dt = -1.7, 0.23
    L = lambda V: [c * V[0], V[1], V[2]]
    U1 = tt.ssprk3_stage(0, dt, U, U, L(U), 1e-13)
    U2 = tt.ssprk3_stage(1, dt, U, U1, L(U1), 1e-13)
    U3 = tt.ssprk3_stage(2, dt, U, U2, L(U2), 1e-13)
    z = c * dt
    want = (1 + z + z * z / 2 + z ** 3 / 6) * brute_full(U)
    assert np.linalg.norm(brute_full(U3) - want) <= 1e-12 * np.linalg.norm(want)
    assert (U3[0].shape[2], U3[1].shape[2]) == (2, 2)
