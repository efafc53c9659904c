// Host launchers whose shapes the C ABI tunes, and the sticky device status.
#pragma once

#include <cuda_runtime.h>

#include "emo_internal.cuh"

namespace emo {

// The association kernels of every problem; grid = sms x blocks_per_sm.
cudaError_t launch_assoc(Plan* plan, int nprob, const int* m_of, int sms, int blocks_per_sm, cudaStream_t s);
// Sticky device status: the first failure any call on this device reported
// since the last read (k_finish sets it); read after the stream's prior work.
cudaError_t sticky_status(cudaStream_t s, int32_t* out, bool clear);
// Folds a call's device status word into the sticky status (stream order).
cudaError_t sticky_merge(const int32_t* status, cudaStream_t s);

// TensorMOEA/D selection (Algorithm S.8): caller arrays and the workspace
// regions (status word, z_min keys, per-subproblem best marked value and
// its lowest offspring index, per-pair marked value).
struct MoeadArgs {
    const float* X;
    const float* F1;
    const float* O;
    const float* F2;
    const float* W;
    const int32_t* I_nb;
    float* z;
    float* X_next;
    float* F_next;
    int32_t* winner;
    int32_t* status_out;
    int64_t n, d;
    int32_t m, T;
    double theta;
    int32_t* status;
    uint32_t* zkey;
    unsigned long long* gmin;
    int32_t* tie;
    double* gpair;
    double* sub;  // [n][m + 2]: ||w_j||, the subproblem's own PBI value, w_j / ||w_j||
};
// Workspace bytes of one TensorMOEA/D selection (regions 256-byte aligned);
// fills the region pointers of `a` when `ws` is given.
int64_t moead_layout(int64_t n, int32_t m, int32_t T, char* ws, MoeadArgs* a);
cudaError_t launch_moead_select(const MoeadArgs& a, int sms, cudaStream_t s);

// One generation's offspring (random mating, SBX, PM; Appendix S.I).
struct VariationArgs {
    const float* X;
    const float* lo;
    const float* hi;
    float* Xoff;
    int32_t* parents;
    int64_t n, d, n_off;
    uint64_t seed, gen;
    double eta_c, eta_m, p_c, p_m;
};
cudaError_t launch_variation(const VariationArgs& a, int sms, cudaStream_t s);
cudaError_t launch_standin(const float* X, int64_t n, int64_t d, int m, int shape, float* F, int sms, cudaStream_t s);
cudaError_t launch_gather_rows(const float* src, const int32_t* idx, int64_t rows, int64_t width, float* dst, int sms,
                               cudaStream_t s);
cudaError_t launch_igd(const float* F, int64_t n, int m, const float* Ref, int64_t n_ref, double* dist, double* out,
                       int sms, cudaStream_t s);

}  // namespace emo
