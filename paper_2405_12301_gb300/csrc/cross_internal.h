// cross_internal.h -- descriptors of the pointwise residual at TT-cross
// sample points (k_cross.cu), shared with the C ABI in api_cross.cu.
#pragma once
#include <cuda_runtime.h>

namespace wg {

// ---------------------------------------------------------------- cross eval
struct CrossInst {
    int n[3];
    int r[2];
    const float *core[5][3];
    double h[3];
    double alpha;
    int bc[3][2];
};

struct CrossSet {
    int inst, mode, fd;
    int n_mode;
    long long n_left, n_right;
    const int *left;
    const int *right;
    void *out;
    long long work_begin;  // first work item of this set (prefix sum)
    int nsl, nsr;          // shifted copies stored per left / right vector (7 or 1)
    long long lvec_off, rvec_off;  // element offsets of the set's vectors in CrossArgs::vecs
};

struct CrossArgs {
    const CrossInst *inst;
    const CrossSet *sets;
    int n_sets;
    long long n_work;      // total work items
    double gamma, eps;
    unsigned long long *counter;
    int *status;           // ST_BADINDEX is latched here
    int *bad;              // per set: an index set held an out-of-range index
    void *vecs;            // contracted left/right vectors (float or double)
    int fp64;
};

// variant: one of the compiled (threads per CTA, samples per chunk) pairs of
// k_cross; ctas_per_sm: persistent grid of (SM count) x ctas_per_sm CTAs.
cudaError_t launch_cross(const CrossArgs &a, int variant, int ctas_per_sm, cudaStream_t s);
int cross_max_rank();
int cross_vec_len();
int cross_num_variants();
// The configuration used until the autotuner has timed a workload class.
void cross_default(int *variant, int *ctas_per_sm);
void cross_variant(int v, int *threads, int *chunk);
cudaError_t cross_set_attributes();

}  // namespace wg
