// tt_internal.h -- declarations shared by the TT-algebra kernels (k_tt.cu,
// k_maxvol.cu, k_cross_drv.cu) and the C ABI in api_tt.cu: descriptors of
// the batched Householder QR, Q apply and Jacobi SVD of TT-rounding, of
// maxvol, and of the TT-cross sweep's bookkeeping kernels.
#pragma once
#include <cstddef>

#include <cuda_runtime.h>

namespace wg {

// ---- batched TT-rounding (k_tt.cu)
constexpr int TT_KMAX = 96;  // largest rank of a TT sum the rounding takes

// Householder QR of a tall-skinny m x k row-major matrix, in chunks of rows.
struct QRDesc {
    double *A;             // m x k (row stride lda); reflectors on exit
    long long m;
    int k, lda;
    int b;                 // sub-block rows (>= k)
    int chunks;
    long long chunk_rows;
    int sub_per_chunk;
    double *tau;           // [chunks][sub_per_chunk][k]
    double *Rout;          // [chunks][k][k] row-major R of each chunk
};

// out = Q [X; 0] for the reflectors left by one QRDesc level.
struct QApplyDesc {
    const double *A;
    const double *tau;
    long long m;
    int k, lda, b, chunks;
    long long chunk_rows;
    int sub_per_chunk;
    const double *X;           // per chunk: rows of X (min(chunk rows, k) x p), row stride ldx
    long long x_chunk_stride;  // between chunks' X blocks
    int ldx, p;
    double *out;               // out(row, col) = out[(row % P) sP + (row / P) sQ + col sC]
    long long P, sP, sQ, sC;
};

// One-sided Jacobi SVD of T^T (T: pk x q row-major, stride ldt) and truncation.
struct SvdDesc {
    const double *T;
    int ldt, pk, q;
    double eps;
    int set_delta;       // 1: delta[0] = eps / sqrt(2) ||T||_F, delta[1] = ||T||_F; 0: read delta[0]
    double *delta;
    int *rank;
    int rmax;
    double *sv;          // pk singular values, descending
    double *Vsel;        // pk x rank, left singular vectors of T (stride ld_out)
    double *Wt;          // q x rank, columns sigma_t u_t (stride ld_out)
    int ld_out;
};

// The TT sum sum_t coef_t X_t of one problem and its first unfoldings.
struct TTSumDesc {
    int nt;
    int n[3];
    int R1, R2, k3;
    int a0[4], b0[4], r1[4], r2[4];
    double coef[4];
    const double *core[4][3];
    double *C1;          // [n1][R1]
    double *MA;          // [n3][R2]
    double *MB;          // [(n2 k3)][R1]
    const double *TA;    // [R2][R2] row-major triangular factor of MA
};

struct GemmDesc {  // out[rows][cols] = L[rows][ka] Rt[cols][ka]^T
    const double *L, *Rt;
    double *out;
    long long rows;
    int cols, ka;
};

size_t qr_factor_smem(int k, int b);
size_t qr_apply_smem(int k, int b, int p);
size_t svd_smem(int pk, int q);
cudaError_t launch_qr_factor(const QRDesc *d, int n, int max_chunks, size_t smem, cudaStream_t s);
cudaError_t launch_qr_apply(const QApplyDesc *d, int n, int max_chunks, size_t smem, cudaStream_t s);
cudaError_t launch_svd_jacobi(const SvdDesc *d, int n, size_t smem, cudaStream_t s);
cudaError_t launch_tt_build(const TTSumDesc *d, int n, cudaStream_t s);
cudaError_t launch_tt_contract(const TTSumDesc *d, int n, cudaStream_t s);
cudaError_t launch_tt_gemm_tr(const GemmDesc *d, int n, cudaStream_t s);


// ---- batched maxvol (k_maxvol.cu)
constexpr int MV_RMAX = 64;
constexpr int MV_NMAX = 1 << 16;  // rows of a maxvol matrix
struct MaxvolDesc {
    const double *A;   // n x r row-major
    double *B;         // n x r: A A[I]^{-1} on exit
    double *W;         // n x r scratch (column-major working copy, then the multipliers L)
    double *Linv;      // r x r scratch: the inverse of the unit lower triangular L[I]
    int *idx;          // r selected rows
    int *status;       // 0 ok, 1 A[I] singular after pivoting
    int *swaps;
    int n, r;
};
size_t maxvol_smem(int r);
constexpr int MV_LAUNCHES = 3;  // kernels of one launch_maxvol
// Orders a batch largest first (n r^2), so the biggest matrices start first.
void maxvol_order(MaxvolDesc *d, int n);
cudaError_t launch_maxvol(const MaxvolDesc *d, int n, int max_r, double delta, int max_iters, cudaStream_t s);


// ---- TT-cross sweep bookkeeping (k_cross_drv.cu)
enum XdKind {
    XD_PREP_L0, XD_PREP_L1, XD_PREP_L2,
    XD_GATHER_L0, XD_GATHER_L1, XD_GATHER_L2, XD_GATHER_R1,
    XD_UPDATE_L0, XD_UPDATE_L1, XD_UPDATE_R2, XD_UPDATE_R1
};
struct CrossDrvDesc {
    int n[3];
    int r1, r2;
    int fp64;            // fiber values are double (else float)
    const void *out;     // fiber-set output [5][n_left][n_mode][n_right]
    double *M;           // gathered matrix
    double *core;        // output core written by a gather / update
    const int *idx;      // rows maxvol selected
    const double *B;     // maxvol's A A[I]^{-1}
    int *I1, *I2, *J1, *J2;
    int *left, *right;   // fiber-set index arrays
};
cudaError_t launch_cross_drv(const CrossDrvDesc *d, int n, int kind, cudaStream_t s);

}  // namespace wg
