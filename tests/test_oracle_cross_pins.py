"""Pins of the cross-index-selection oracle (oracle/cross.py): maxvol against
closed forms and brute-force volumes, and the TT-cross sweep against exact
recovery of tensors of known TT rank and the interpolation property."""
import itertools

import numpy as np
import pytest

from oracle import cross as X


def test_maxvol_of_one_column_is_the_largest_entry():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((50, 1))
    I, B, _ = X.maxvol(A, delta=0.0)
    assert I[0] == int(np.argmax(np.abs(A[:, 0])))


@pytest.mark.parametrize("r", [2, 3, 4])
def test_maxvol_with_one_spare_row_finds_the_maximum_volume(r):
    """n = r + 1 and delta = 0: every other subset is one swap away, and a swap
    multiplies the volume by |B[i, j]| <= 1, so the result has the largest
    |det| of all r-row subsets (brute force)."""
    rng = np.random.default_rng(r)
    for _ in range(20):
        A = rng.standard_normal((r + 1, r))
        I, B, _ = X.maxvol(A, delta=0.0)
        best = max(abs(np.linalg.det(A[list(s)])) for s in itertools.combinations(range(r + 1), r))
        assert abs(np.linalg.det(A[I])) >= best * (1 - 1e-12)


def test_maxvol_result_is_dominant_and_b_is_a_times_inverse():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((300, 12))
    I, B, swaps = X.maxvol(A, delta=1e-2)
    assert len(set(I.tolist())) == 12
    assert np.abs(B).max() <= 1.0 + 1e-2 + 1e-12
    assert np.allclose(B[I], np.eye(12), atol=1e-12)
    assert np.allclose(B, A @ np.linalg.inv(A[I]), atol=1e-10)


def test_maxvol_is_unchanged_by_upper_triangular_mixing_of_columns():
    """A and A R (R upper triangular, invertible) have the same maxvol rows,
    swaps and B: column j of A R mixes only columns 0..j of A, so every
    partial-pivoting residual of A R is a fixed multiple of A's, and
    B = A A[I]^{-1} depends on the column space only.  (This is why the rows
    maxvol picks from a fiber matrix and from its Householder Q agree.)"""
    rng = np.random.default_rng(9)
    for n, r in [(300, 12), (1000, 24), (40, 40)]:
        A = rng.standard_normal((n, r))
        R = np.triu(0.3 * rng.standard_normal((r, r)), 1) + np.diag(rng.uniform(0.5, 2.0, r) * rng.choice([-1, 1], r))
        I1, B1, s1 = X.maxvol(A, delta=1e-2)
        I2, B2, s2 = X.maxvol(A @ R, delta=1e-2)
        assert I1.tolist() == I2.tolist() and s1 == s2
        assert np.abs(B1 - B2).max() <= 1e-9 * max(1.0, np.abs(B1).max())


def test_maxvol_finds_planted_rows():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((100, 5)) * 0.01
    planted = [7, 23, 41, 66, 90]
    A[planted] = rng.standard_normal((5, 5)) + 3 * np.eye(5)
    I, _, _ = X.maxvol(A)
    assert sorted(I.tolist()) == planted


def _tt_fun(cores):
    """Fiber evaluator of A(i,j,k,f) = G1[i] G2[j] G3[k][:, f] in the fiber-set layout."""
    G1, G2, G3 = cores

    def fun(mode, left, right):
        n = [G1.shape[0], G2.shape[0], G3.shape[0]]
        nl = left.shape[0] if mode > 0 else 1
        nr = right.shape[0] if mode < 2 else 1
        out = np.zeros((5, nl, n[mode], nr))
        for a in range(nl):
            for b in range(nr):
                for t in range(n[mode]):
                    idx = list(left[a]) + [t] + list(right[b] if mode < 2 else [])
                    i, j, k = idx
                    out[:, a, t, b] = G1[i, 0] @ G2[j] @ G3[k]
        return out
    return fun


@pytest.mark.parametrize("sweeps", [0, 1])
def test_cross_recovers_a_tensor_of_the_same_ranks(sweeps):
    rng = np.random.default_rng(5)
    n, r = (9, 8, 7), (3, 4)
    cores = [rng.standard_normal((n[0], 1, r[0])), rng.standard_normal((n[1], r[0], r[1])),
             rng.standard_normal((n[2], r[1], 5))]
    J1 = np.stack([rng.integers(0, n[1], r[0]), rng.integers(0, n[2], r[0]), rng.integers(0, 5, r[0])], 1)
    J2 = np.stack([rng.integers(0, n[2], r[1]), rng.integers(0, 5, r[1])], 1)
    G, I1, I2, J1o, J2o = X.cross_sweeps(_tt_fun(cores), n, r, J1, J2, sweeps=sweeps)
    A = X.tt4_full(cores)
    assert np.linalg.norm(X.tt4_full(G) - A) <= 1e-10 * np.linalg.norm(A)


def test_cross_interpolates_on_its_index_sets():
    """A tensor of higher rank than the cross: the TT equals it at every sample
    (I1[a], j, J2[b]) and (I2[b], k, f) of the last pass, and the first core is
    the identity on I1."""
    rng = np.random.default_rng(6)
    n = (10, 9, 8)
    cores = [rng.standard_normal((n[0], 1, 6)), rng.standard_normal((n[1], 6, 6)), rng.standard_normal((n[2], 6, 5))]
    A = X.tt4_full(cores)
    r = (3, 4)
    J1 = np.stack([rng.integers(0, n[1], 3), rng.integers(0, n[2], 3), rng.integers(0, 5, 3)], 1)
    J2 = np.stack([rng.integers(0, n[2], 4), rng.integers(0, 5, 4)], 1)
    G, I1, I2, J1o, J2o = X.cross_sweeps(_tt_fun(cores), n, r, J1, J2, sweeps=1)
    T = X.tt4_full(G)
    assert np.allclose(G[0][I1, 0, :], np.eye(3), atol=1e-12)
    for b in range(4):
        k, f = J2o[b]
        assert np.allclose(T[I1][:, :, k, f], A[I1][:, :, k, f], atol=1e-10 * np.abs(A).max())
    for b in range(4):
        i, j = I2[b]
        assert np.allclose(T[i, j], A[i, j], atol=1e-10 * np.abs(A).max())
