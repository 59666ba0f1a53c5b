// weno_internal.h -- interface between the C ABI layer and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wg {

struct Ctl;

// Epilogue of a sweep kernel (what it does with the direction's residual).
enum Epi { EPI_STORE = 0, EPI_ADD = 1, EPI_RHS = 2, EPI_STAGE = 3 };
// Conservation law: Euler (nf = dim + 2), scalar advection or Burgers (nf = 1).
enum Model { MODEL_EULER = 0, MODEL_ADVECT = 1, MODEL_BURGERS = 2 };

struct SweepArgs {
    const double *U;     // stencil state U^(k) (device, FP64 SoA)
    const double *Un;    // U^n, read by the stage-2/3 combination
    double *Uout;        // U^(k+1)
    void *acc;           // residual accumulator: float (FP32-bulk) or double (FP64)
    double *Rout;        // output of EPI_RHS
    // 2D FP32-bulk stage state (k_xy2): the FP32 hi/lo split of U^n, written
    // by stage 1, and the FP32 increments Delta_k = U^(k) - U^n
    // 2D: planes H, L of float4 [N] each; 3D: planes H4, L4 (float4 [N]: rho, m_x,
    // m_y, m_z) then H1, L1 (float [N]: E)
    float2 *hl;
    const float *din;    // Delta_k read by stages 2 and 3 (3D: the float4 [N] plane of the first four fields)
    float *dout;         // Delta_{k+1} written by stages 1 and 2 (3D: as din)
    const float *din1;   // 3D: Delta_k of E (float [N])
    float *dout1;        // 3D: Delta_{k+1} of E
    Ctl *ctl;
    long long N;         // cells per field (field stride)
    int n[3];
    long long stride[3]; // 1, nx, nx * ny
    int bc[3][2];
    double bc_state[3][2][5];  // conserved state held by the ghosts of an inflow side
    const double *bcs;   // the same in device memory ([3][2][5]), for out-of-line boundary loads
    double inv_h[3];
    double gamma;
    double eps;
    float gamma_f, gm1_f, eps_f;  // the same constants in FP32, rounded on the host
    float inv_h_f[3];
    float2 ih23[3];      // -(2/3) / h_d as FP32 pairs hi + lo (the 2D FP32-bulk residual factor)
    int stage;           // 0, 1, 2
    int slot_in;         // alpha slot used for the splitting
    int slot_out;        // alpha slot the EPI_STAGE epilogue publishes to
    int check_dt;        // skip all work when ctl->dt == 0
    int per_dir;         // LF alpha per direction (alpha_dir slots) instead of one global alpha
};

// Launches the sweep of direction dir for a dim-dimensional grid.
cudaError_t launch_sweep(int model, int dim, int dir, bool bulk, int epi, const SweepArgs &a, cudaStream_t s);
cudaError_t sweep_set_attributes();
// Fused x+y residual of a 2D grid (EPI_RHS / EPI_STAGE) or of the z-planes of a 3D grid (EPI_STORE).
cudaError_t launch_xy(int dim, bool bulk, int epi, const SweepArgs &a, cudaStream_t s);
// 2D FP32-bulk residual / stage in pair-difference form (EPI_RHS / EPI_STAGE).
cudaError_t launch_xy2(int epi, const SweepArgs &a, cudaStream_t s);
// z direction of a 3D grid, adding the accumulator and ending the residual (EPI_RHS / EPI_STAGE).
cudaError_t launch_z(bool bulk, int epi, const SweepArgs &a, cudaStream_t s);
// z direction of a 3D FP32-bulk grid in pair-difference form (EPI_RHS / EPI_STAGE).
cudaError_t launch_z2(int epi, const SweepArgs &a, cudaStream_t s);

cudaError_t launch_alpha(int model, int dim, bool bulk, const double *U, long long N, double gamma, Ctl *ctl, int slot,
                         int per_dir, cudaStream_t s);
cudaError_t launch_reset_slot(Ctl *ctl, int slot, cudaStream_t s);
cudaError_t launch_step_begin(Ctl *ctl, cudaStream_t s);
cudaError_t launch_step_end(Ctl *ctl, cudaStream_t s);
cudaError_t launch_copy_alpha(const Ctl *ctl, int slot, double *out, cudaStream_t s);
cudaError_t launch_sums(const double *U, int nf, long long N, double *partials, int nblocks, double *out,
                        cudaStream_t s);
int sums_blocks(long long N);
// Number of SMs of the current device (queried once per device; persistent and
// grid-stride launches are sized from it).
int sm_count();

}  // namespace wg
