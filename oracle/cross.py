"""Oracle for the cross-index selection of TT-cross (Sec. 3 "TT-cross
Interpolation": skeleton/CUR decompositions whose rows and columns are chosen
by the maximum-volume principle): the maxvol algorithm and an alternating
fixed-rank TT-cross sweep over a 3D tensor whose last core also carries the
five Euler components (the layout of the LF-cross method, Sec. 4.2, cores
(1 x N1 x r1)(r1 x N2 x r2)(r2 x N3 x 5)).  FP64 numpy.  TEST INFRASTRUCTURE
ONLY (tests, the smoke check and the benchmark's CPU legs may call it).

maxvol (Goreinov, Oseledets, Savostyanov, Tyrtyshnikov, Zamarashkin, 2010)
for an n x r matrix A of rank r:
  1. start from the r pivot rows of Gaussian elimination with partial
     pivoting (column by column, the largest remaining entry of the column);
  2. B = A A[I]^{-1}, so that B[I] = identity;
  3. while the largest |B[i, j]| exceeds 1 + delta: row i replaces I[j] (the
     volume of A[I] grows by that factor), and B is updated by the rank-one
     formula B -= B[:, j] (B[i, :] - e_j) / B[i, j].
Ties in the argmax take the first entry in row-major order.

The TT-cross sweep (fixed ranks; AMEn's rank adaptation is not part of it)
keeps right index sets J1 (over (j, k, f)) and J2 (over (k, f)) and left sets
I1 (over i) and I2 (over (i, j)):
  left-to-right:  C0 = A(:, J1) -> QR -> maxvol -> I1, core 1 = Q Q[I1]^{-1};
                  C1 = A(I1, :, J2) unfolded (r1 n2) x r2 -> QR -> maxvol -> I2,
                  core 2 = Q Q[I2]^{-1};  core 3 = A(I2, :, :) (all five f);
  right-to-left:  A(I2, :, :) as (n3 5) x r2 -> QR -> maxvol -> J2;
                  A(I1, :, J2) as (n2 r2) x r1 -> QR -> maxvol -> J1.
The TT interpolates A on the cross: it equals A at every (I1, :, J1),
(I2, :, J2)-type sample of the last left-to-right pass.
"""
import numpy as np


def maxvol(A, delta=1e-2, max_iters=200):
    """Row indices (length r) of a dominant r x r submatrix of A (n x r, n >= r),
    the matrix B = A A[I]^{-1}, and the number of swaps taken."""
    A = np.asarray(A, dtype=np.float64)
    n, r = A.shape
    W = A.copy()
    chosen = np.zeros(n, dtype=bool)
    I = np.zeros(r, dtype=np.int64)
    for j in range(r):  # partial pivoting, column by column
        col = np.where(chosen, -1.0, np.abs(W[:, j]))
        p = int(np.argmax(col))
        I[j] = p
        chosen[p] = True
        if W[p, j] != 0.0:
            f = W[:, j] / W[p, j]
            f[chosen] = 0.0
            W -= np.outer(f, W[p, :])
    B = np.linalg.solve(A[I].T, A.T).T
    swaps = 0
    for _ in range(max_iters):
        flat = int(np.argmax(np.abs(B)))
        i, j = divmod(flat, r)
        if abs(B[i, j]) <= 1.0 + delta:
            break
        piv = B[i, j]
        row = B[i, :].copy()
        row[j] -= 1.0
        B -= np.outer(B[:, j], row) / piv
        I[j] = i
        swaps += 1
    return I, B, swaps


def _qr_q(C):
    Q, _ = np.linalg.qr(C)
    return Q


def cross_sweeps(fun, n, r, J1, J2, sweeps=1, delta=1e-2):
    """Alternating TT-cross of A(i, j, k, f) (f = 0..4 in the last core).

    fun(mode, left, right) returns the fibers [5][n_left][n_mode][n_right] with
    left multi-indices over the modes before `mode` and right ones over the
    spatial modes after it (the shape of a weno_fiber_set's output).
    J1: [r1][3] (j, k, f); J2: [r2][2] (k, f) -- initial right index sets.
    Runs `sweeps` right-to-left updates, each preceded by a left-to-right pass,
    and ends with a left-to-right pass.  Returns (cores, I1, I2, J1, J2)."""
    n1, n2, n3 = n
    r1, r2 = r
    J1 = np.array(J1, dtype=np.int64).reshape(r1, 3)
    J2 = np.array(J2, dtype=np.int64).reshape(r2, 2)
    for it in range(sweeps + 1):
        # left-to-right
        F0 = fun(0, np.zeros((1, 0), np.int32), J1[:, :2].astype(np.int32))        # [5][1][n1][r1]
        C0 = F0[J1[:, 2], 0, :, np.arange(r1)].T                                    # n1 x r1
        I1, B1, _ = maxvol(_qr_q(C0), delta)                                        # core 1 = Q Q[I1]^{-1}
        F1 = fun(1, I1[:, None].astype(np.int32), J2[:, :1].astype(np.int32))      # [5][r1][n2][r2]
        C1 = np.stack([F1[J2[b, 1], :, :, b] for b in range(r2)], axis=-1)          # r1 x n2 x r2
        sel, B2, _ = maxvol(_qr_q(C1.reshape(r1 * n2, r2)), delta)                  # rows (a, j)
        I2 = np.stack([I1[sel // n2], sel % n2], axis=1)
        F2 = fun(2, I2.astype(np.int32), np.zeros((1, 0), np.int32))               # [5][r2][n3][1]
        G3 = F2[:, :, :, 0].transpose(2, 1, 0)                                      # n3 x r2 x 5
        cores = [B1[:, None, :], B2.reshape(r1, n2, r2).transpose(1, 0, 2), np.ascontiguousarray(G3)]
        if it == sweeps:
            return cores, I1, I2, J1, J2
        # right-to-left
        R2 = F2[:, :, :, 0].transpose(2, 0, 1).reshape(n3 * 5, r2)                  # rows (k, f)
        sel, _, _ = maxvol(_qr_q(R2), delta)
        J2 = np.stack([sel // 5, sel % 5], axis=1)
        F1 = fun(1, I1[:, None].astype(np.int32), J2[:, :1].astype(np.int32))
        R1 = np.stack([F1[J2[b, 1], :, :, b] for b in range(r2)], axis=-1)         # r1 x n2 x r2
        R1t = R1.transpose(1, 2, 0).reshape(n2 * r2, r1)                            # rows (j, b)
        sel, _, _ = maxvol(_qr_q(R1t), delta)
        jj, bb = sel // r2, sel % r2
        J1 = np.stack([jj, J2[bb, 0], J2[bb, 1]], axis=1)


def tt4_full(cores):
    """Full A[i, j, k, f] of the cross TT (last core [n3][r2][5])."""
    G1, G2, G3 = cores
    return np.einsum("ia,jab,kbf->ijkf", G1[:, 0, :], G2, G3)
