// k_cross_drv.cu -- the bookkeeping kernels of the fixed-rank TT-cross sweep
// (weno_tt_cross): fiber-set index arrays from the current index sets,
// gathers of the fiber values into FP64 matrices (the component f of a right
// index picks one of the five outputs), and the index-set / core updates from
// the rows maxvol selected.  The tensor is A(i, j, k, f) with f the Euler
// component, carried by the last core as in the LF-cross layout (Sec. 4.2).
#include "weno_dev.cuh"
#include "weno_internal.h"
#include "tt_internal.h"

namespace wg {

template <class T>
__device__ __forceinline__ double fiber(const CrossDrvDesc &d, int f, int a, int t, int b, int nl, int nm, int nr)
{
    return (double)static_cast<const T *>(d.out)[(((long long)f * nl + a) * nm + t) * nr + b];
}

template <class T>
__device__ void drv_body(const CrossDrvDesc &d, int kind)
{
    const int n1 = d.n[0], n2 = d.n[1], n3 = d.n[2], r1 = d.r1, r2 = d.r2;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long step = (long long)gridDim.x * blockDim.x;
    switch (kind) {
    case XD_PREP_L0:  // right (j, k) of J1
        for (long long e = tid; e < r1; e += step) {
            d.right[2 * e] = d.J1[3 * e];
            d.right[2 * e + 1] = d.J1[3 * e + 1];
        }
        break;
    case XD_PREP_L1:  // left I1, right k of J2
        for (long long e = tid; e < r1 || e < r2; e += step) {
            if (e < r1) d.left[e] = d.I1[e];
            if (e < r2) d.right[e] = d.J2[2 * e];
        }
        break;
    case XD_PREP_L2:  // left (i, j) of I2
        for (long long e = tid; e < 2 * r2; e += step) d.left[e] = d.I2[e];
        break;
    case XD_GATHER_L0:  // M[i][b] = A(i, J1[b])
        for (long long e = tid; e < (long long)n1 * r1; e += step) {
            const int i = (int)(e / r1), b = (int)(e - (long long)i * r1);
            d.M[e] = fiber<T>(d, d.J1[3 * b + 2], 0, i, b, 1, n1, r1);
        }
        break;
    case XD_GATHER_L1:  // M[(a n2 + j)][b] = A(I1[a], j, J2[b])
    case XD_GATHER_R1:  // M[(j r2 + b)][a] = A(I1[a], j, J2[b])
        for (long long e = tid; e < (long long)r1 * n2 * r2; e += step) {
            const int b = (int)(e % r2);
            const long long aj = e / r2;
            const int j = (int)(aj % n2), a = (int)(aj / n2);
            const double v = fiber<T>(d, d.J2[2 * b + 1], a, j, b, r1, n2, r2);
            if (kind == XD_GATHER_L1) d.M[e] = v;
            else d.M[((long long)j * r2 + b) * r1 + a] = v;
        }
        break;
    case XD_GATHER_L2:  // core 3 [k][b][f] = A(I2[b], k, f); M[(k 5 + f)][b] the same values
        for (long long e = tid; e < 5LL * r2 * n3; e += step) {
            const int k = (int)(e % n3);
            const long long fb = e / n3;
            const int b = (int)(fb % r2), f = (int)(fb / r2);
            const double v = fiber<T>(d, f, b, k, 0, r2, n3, 1);
            d.core[((long long)k * r2 + b) * 5 + f] = v;
            d.M[((long long)k * 5 + f) * r2 + b] = v;
        }
        break;
    case XD_UPDATE_L0:  // I1 = selected rows (core 1 is maxvol's B itself)
        for (long long e = tid; e < r1; e += step) d.I1[e] = d.idx[e];
        break;
    case XD_UPDATE_L1:  // I2 = (I1[a], j) of the selected rows a n2 + j; core 2 [j][a][b] = B[(a n2 + j)][b]
        for (long long e = tid; e < r2; e += step) {
            const int s = d.idx[e];
            d.I2[2 * e] = d.I1[s / n2];
            d.I2[2 * e + 1] = s % n2;
        }
        for (long long e = tid; e < (long long)r1 * n2 * r2; e += step) {
            const int b = (int)(e % r2);
            const long long aj = e / r2;
            const int j = (int)(aj % n2), a = (int)(aj / n2);
            d.core[((long long)j * r1 + a) * r2 + b] = d.B[e];
        }
        break;
    case XD_UPDATE_R2:  // J2 = (k, f) of the selected rows k 5 + f
        for (long long e = tid; e < r2; e += step) {
            d.J2[2 * e] = d.idx[e] / 5;
            d.J2[2 * e + 1] = d.idx[e] % 5;
        }
        break;
    case XD_UPDATE_R1:  // J1 = (j, J2[b]) of the selected rows j r2 + b (J2 already updated)
        for (long long e = tid; e < r1; e += step) {
            const int s = d.idx[e], j = s / r2, b = s % r2;
            d.J1[3 * e] = j;
            d.J1[3 * e + 1] = d.J2[2 * b];
            d.J1[3 * e + 2] = d.J2[2 * b + 1];
        }
        break;
    default:
        break;
    }
}

__global__ void k_cross_drv(const CrossDrvDesc *descs, int kind)
{
    const CrossDrvDesc &d = descs[blockIdx.y];
    if (d.fp64) drv_body<double>(d, kind);
    else drv_body<float>(d, kind);
}

cudaError_t launch_cross_drv(const CrossDrvDesc *d, int n, int kind, cudaStream_t s)
{
    k_cross_drv<<<dim3(32, n), 256, 0, s>>>(d, kind);
    return cudaGetLastError();
}

}  // namespace wg
