"""Oracle for the TT time-step algebra of Sec. 3 and Sec. 4.4: TT addition,
TT-rounding and the TT-SSPRK3 stages, for 3D tensors, in FP64
numpy.  TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's
CPU legs may call it; the CUDA path never does).

Cores follow the layout of the TT cross evaluation: core m is an array
[n_m, r_{m-1}, r_m] with r_0 = r_3 = 1, so that
    X[i, j, k] = G1[i] @ G2[j] @ G3[k]            (Eq. TT_def)
with G1[i] a 1 x r1 row, G2[j] r1 x r2, G3[k] r2 x 1.

TT-rounding (Sec. 3, "TT-rounding", which defers to Oseledets 2011,
Algorithm 2): a right-to-left orthogonalisation pass (QR of every core's
transposed unfolding, the triangular factor pushed into the core on its
left), then a left-to-right pass that truncates the SVD of every core's
unfolding and pushes S V^T into the core on its right.  The threshold of each
truncation is delta = eps / sqrt(d - 1) * ||X||_F (d = 3), which gives
||X - Y||_F <= eps ||X||_F; the rank kept is the smallest r whose discarded
singular values have a 2-norm <= delta (at least 1).

numpy's QR and SVD are the library steps; nothing else is blocked or fused.
"""
import numpy as np


def tt_full(cores):
    """Full tensor X[i, j, k] of a 3-core TT (Eq. TT_def)."""
    G1, G2, G3 = cores
    return np.einsum("ia,jab,kb->ijk", G1[:, 0, :], G2, G3[:, :, 0])


def tt_norm(cores):
    return float(np.linalg.norm(tt_full(cores)))


def tt_add(terms):
    """Sum of c_t X_t for terms [(c_t, cores_t)] as one TT (Sec. 3 TT arithmetic):
    the first cores side by side (scaled by c_t), the middle cores block-diagonal,
    the last cores stacked."""
    n = [terms[0][1][m].shape[0] for m in range(3)]
    r1 = [t[1][0].shape[2] for t in terms]
    r2 = [t[1][1].shape[2] for t in terms]
    R1, R2 = sum(r1), sum(r2)
    G1 = np.zeros((n[0], 1, R1))
    G2 = np.zeros((n[1], R1, R2))
    G3 = np.zeros((n[2], R2, 1))
    a = b = 0
    for (c, cores), p, q in zip(terms, r1, r2):
        G1[:, :, a:a + p] = c * cores[0]
        G2[:, a:a + p, b:b + q] = cores[1]
        G3[:, b:b + q, :] = cores[2]
        a += p
        b += q
    return [G1, G2, G3]


def _trunc_rank(s, delta):
    """Smallest r >= 1 with sqrt(sum_{i >= r} s_i^2) <= delta (s descending)."""
    tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]  # tail[i] = ||s[i:]||
    r = len(s)
    while r > 1 and tail[r - 1] <= delta:
        r -= 1
    return r


def tt_round(cores, eps):
    """TT-rounding with relative accuracy eps; returns (cores, singular values of
    the two truncated unfoldings, ||X||_F)."""
    G = [np.array(c, dtype=np.float64) for c in cores]
    n = [g.shape[0] for g in G]
    # right-to-left orthogonalisation: core m unfolded as r_{m-1} x (n_m r_m)
    for m in (2, 1):
        r0, r1 = G[m].shape[1], G[m].shape[2]
        M = G[m].transpose(1, 0, 2).reshape(r0, n[m] * r1)        # rows a, columns (i, b)
        Q, T = np.linalg.qr(M.T)                                  # M^T = Q T, M = T^T Q^T
        k = Q.shape[1]
        G[m] = Q.T.reshape(k, n[m], r1).transpose(1, 0, 2)        # [n, k, r1]
        G[m - 1] = np.einsum("iab,cb->iac", G[m - 1], T)          # G_{m-1} times T^T on its right rank
    norm = float(np.linalg.norm(G[0]))
    delta = eps / np.sqrt(2.0) * norm
    svals = []
    # left-to-right truncation: core m unfolded as (r_{m-1} n_m) x r_m
    for m in (0, 1):
        r0, r1 = G[m].shape[1], G[m].shape[2]
        M = G[m].transpose(1, 0, 2).reshape(r0 * n[m], r1)        # rows (a, i), columns b
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        r = _trunc_rank(s, delta)
        svals.append(s)
        G[m] = U[:, :r].reshape(r0, n[m], r).transpose(1, 0, 2)
        SV = s[:r, None] * Vt[:r, :]                              # r x r1
        G[m + 1] = np.einsum("cb,ibd->icd", SV, G[m + 1])
    return G, svals, norm


def tt_combine(terms, eps):
    """round(sum_t c_t X_t, eps) for terms [(c_t, cores_t)]."""
    return tt_round(tt_add(terms), eps)[0]


def ssprk3_stage(stage, dt, Un, Uk, Lk, eps):
    """One stage of Eq. (tt-ssprk3) given L(U^k) as a TT: the forward Euler step
    F = round(U^k + dt L(U^k)) (Eq. tt-forward-euler), then, for stages 1 and 2,
    round(a U^n + b F) with (a, b) = (3/4, 1/4) and (1/3, 2/3)."""
    F = tt_combine([(1.0, Uk), (dt, Lk)], eps)
    if stage == 0:
        return F
    a, b = ((0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))[stage - 1]
    return tt_combine([(a, Un), (b, F)], eps)
