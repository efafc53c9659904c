// TensorMOEA/D environmental selection (Algorithm S.8) with the PBI
// aggregation of Section IV-B.
//
// The paper materialises I_new (n x n) and takes one argmin per column. Only
// the n*T (offspring, neighbour) pairs can be marked, so here every pair is
// one thread: it computes both PBI values, marks the pair when the
// offspring's value does not exceed the neighbour's own (H(0) = 1), and
// lowers the neighbour's best marked value with a 64-bit atomicMin on the
// bits of the (non-negative) double. A second pass finds the lowest
// offspring index at that value. The column argmin of the paper then
// resolves per subproblem j without the n x n tensor:
//   * no marked pair               -> j keeps its solution;
//   * best marked value <  g_old_j -> the lowest offspring at that value;
//   * best marked value == g_old_j -> every marked value equals g_old_j, the
//     first position holding g_old_j is 0 (unmarked unless offspring 0 is
//     marked), so offspring 0 wins exactly when it is the lowest marked one.
// Each PBI value is computed in FP64 from the float32 inputs with k
// ascending and explicitly rounded operations (no contraction), so every
// decision equals that of the same arithmetic done on a CPU. What depends
// only on the subproblem -- ||w||, the unit weights w / ||w|| and the
// subproblem's own value g_old -- is computed once per subproblem (same
// operations, so the same bits) and read by every pair of that subproblem;
// a pair then needs one division and one square root.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "emo_internal.cuh"
#include "emo_launch.cuh"

namespace emo {
namespace {

constexpr int kMoeadThreads = 256;
constexpr unsigned long long kNoMark = 0x7FF0000000000000ull;  // +inf: above every PBI value

// Order-preserving map of a float to uint32 (-0 and +0 map alike).
__device__ __forceinline__ uint32_t fkey(float v)
{
    uint32_t b = __float_as_uint(v);
    if (b == 0x80000000u) b = 0u;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__device__ __forceinline__ void set_status(int32_t* st, int32_t code) { atomicCAS(st, 0, code); }

// d1 = |(f - z).w| / ||w||, d2 = ||(f - z) - d1 w / ||w||||, g = d1 + theta d2.
__device__ double pbi(const float* __restrict__ f, const float* __restrict__ w, const float* z, int m, double theta)
{
    double ww = 0.0, fw = 0.0, dd = 0.0;
    for (int k = 0; k < m; ++k) {
        const double wk = (double)__ldg(w + k);
        ww = __dadd_rn(ww, __dmul_rn(wk, wk));
    }
    const double nw = __dsqrt_rn(ww);
    for (int k = 0; k < m; ++k)
        fw = __dadd_rn(fw, __dmul_rn(__dsub_rn((double)__ldg(f + k), (double)z[k]), (double)__ldg(w + k)));
    const double d1 = __ddiv_rn(fabs(fw), nw);
    for (int k = 0; k < m; ++k) {
        const double r = __dsub_rn(__dsub_rn((double)__ldg(f + k), (double)z[k]),
                                   __dmul_rn(d1, __ddiv_rn((double)__ldg(w + k), nw)));
        dd = __dadd_rn(dd, __dmul_rn(r, r));
    }
    return __dadd_rn(d1, __dmul_rn(theta, __dsqrt_rn(dd)));
}

// pbi() of an offspring with the subproblem's ||w|| and unit weights taken
// from `sub` (computed by the same operations in k_moead_prep).
__device__ double pbi_pre(const float* __restrict__ f, const float* __restrict__ w, const double* __restrict__ sub,
                          const float* z, int m, double theta)
{
    const double nw = __ldg(sub);
    double fw = 0.0, dd = 0.0;
    for (int k = 0; k < m; ++k)
        fw = __dadd_rn(fw, __dmul_rn(__dsub_rn((double)__ldg(f + k), (double)z[k]), (double)__ldg(w + k)));
    const double d1 = __ddiv_rn(fabs(fw), nw);
    for (int k = 0; k < m; ++k) {
        const double r = __dsub_rn(__dsub_rn((double)__ldg(f + k), (double)z[k]), __dmul_rn(d1, __ldg(sub + 2 + k)));
        dd = __dadd_rn(dd, __dmul_rn(r, r));
    }
    return __dadd_rn(d1, __dmul_rn(theta, __dsqrt_rn(dd)));
}

__device__ __forceinline__ void load_zmin(const uint32_t* zkey, int m, float* z)
{
    for (int k = 0; k < m; ++k) z[k] = fkey_inv(zkey[k]);
}

__global__ void __launch_bounds__(kMoeadThreads) k_moead_init(MoeadArgs a)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = tid; j < a.n; j += stride) {
        a.gmin[j] = kNoMark;
        a.tie[j] = INT32_MAX;
    }
    if (tid == 0) *a.status = 0;
    if (tid < a.m) {
        const float zk = a.z[tid];
        if (!isfinite(zk)) set_status(a.status, EMO_ERR_NONFINITE);
        a.zkey[tid] = fkey(zk);
    }
}

// z_min = min(z, column minima of F2); F2 must be finite.
__global__ void __launch_bounds__(kMoeadThreads) k_moead_zmin(MoeadArgs a)
{
    uint32_t lk[kMaxM];
    for (int k = 0; k < kMaxM; ++k) lk[k] = 0xFFFFFFFFu;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
        for (int k = 0; k < a.m; ++k) {
            const float v = __ldg(a.F2 + i * a.m + k);
            bad |= !isfinite(v);
            lk[k] = min(lk[k], fkey(v));
        }
    if (bad) set_status(a.status, EMO_ERR_NONFINITE);
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < a.m; ++k) {
        const uint32_t v = __reduce_min_sync(0xFFFFFFFFu, lk[k]);
        if (lane == 0 && v != 0xFFFFFFFFu) atomicMin(a.zkey + k, v);
    }
}

// Per subproblem j: sub[j] = (||w_j||, g_old_j = PBI(F1_j | w_j, z_min),
// w_j0 / ||w_j||, ..., w_j,m-1 / ||w_j||), in the operation order of pbi().
__global__ void __launch_bounds__(kMoeadThreads) k_moead_prep(MoeadArgs a)
{
    float z[kMaxM];
    load_zmin(a.zkey, a.m, z);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.n; j += stride) {
        const float* w = a.W + j * a.m;
        double* sub = a.sub + j * (a.m + 2);
        double ww = 0.0;
        for (int k = 0; k < a.m; ++k) {
            const double wk = (double)__ldg(w + k);
            ww = __dadd_rn(ww, __dmul_rn(wk, wk));
        }
        const double nw = __dsqrt_rn(ww);
        sub[0] = nw;
        for (int k = 0; k < a.m; ++k) sub[2 + k] = __ddiv_rn((double)__ldg(w + k), nw);
        sub[1] = pbi(a.F1 + j * a.m, w, z, a.m, a.theta);
    }
}

// One thread per (offspring i, neighbour slot t): mark and lower gmin[j].
__global__ void __launch_bounds__(kMoeadThreads) k_moead_compare(MoeadArgs a)
{
    float z[kMaxM];
    load_zmin(a.zkey, a.m, z);
    const int64_t pairs = a.n * (int64_t)a.T;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pairs; p += stride) {
        const int64_t i = p / a.T;
        const int32_t t = (int32_t)(p - i * a.T);
        const int32_t j = __ldg(a.I_nb + p);
        double g = -1.0;
        bool dup = false;
        if (j < 0 || j >= a.n) {
            set_status(a.status, EMO_ERR_INVALID_ARG);
            dup = true;
        }
        for (int32_t u = 0; u < t && !dup; ++u) dup = __ldg(a.I_nb + i * a.T + u) == j;  // count a neighbour once
        if (!dup) {
            const double* sub = a.sub + (int64_t)j * (a.m + 2);
            const double g_old = __ldg(sub + 1);
            const double g_new = pbi_pre(a.F2 + i * a.m, a.W + (int64_t)j * a.m, sub, z, a.m, a.theta);
            if (__dsub_rn(g_old, g_new) >= 0.0) {
                g = g_new;
                atomicMin(a.gmin + j, (unsigned long long)__double_as_longlong(g_new));
            }
        }
        a.gpair[p] = g;
    }
}

// The lowest offspring index whose marked value equals gmin[j].
__global__ void __launch_bounds__(kMoeadThreads) k_moead_tie(MoeadArgs a)
{
    const int64_t pairs = a.n * (int64_t)a.T;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pairs; p += stride) {
        const double g = a.gpair[p];
        if (!(g >= 0.0)) continue;
        const int32_t j = __ldg(a.I_nb + p);
        if ((unsigned long long)__double_as_longlong(g) == a.gmin[j]) atomicMin(a.tie + j, (int32_t)(p / a.T));
    }
}

// One warp per subproblem: resolve the winner, copy its row of X / O and F.
__global__ void __launch_bounds__(kMoeadThreads) k_moead_gather(MoeadArgs a)
{
    float z[kMaxM];
    load_zmin(a.zkey, a.m, z);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < a.n; j += warps) {
        int32_t win = -1;
        if (lane == 0) {
            const float* f1 = a.F1 + j * a.m;
            const float* w = a.W + j * a.m;
            bool bad = false;
            double ww = 0.0;
            for (int k = 0; k < a.m; ++k) {
                const float fv = __ldg(f1 + k), wv = __ldg(w + k);
                bad |= !isfinite(fv) || !isfinite(wv);
                ww += (double)wv * (double)wv;
            }
            if (bad || !(ww > 0.0)) set_status(a.status, EMO_ERR_NONFINITE);
            const unsigned long long gm = a.gmin[j];
            if (gm != kNoMark) {
                const double g_old = a.sub[j * (a.m + 2) + 1];
                const double best = __longlong_as_double((long long)gm);
                const int32_t tie = a.tie[j];
                win = best < g_old ? tie : (tie == 0 ? 0 : -1);
            }
        }
        win = __shfl_sync(0xFFFFFFFFu, win, 0);
        const float* xs = win >= 0 ? a.O + (int64_t)win * a.d : a.X + j * a.d;
        const float* fs = win >= 0 ? a.F2 + (int64_t)win * a.m : a.F1 + j * a.m;
        // read the source rows before writing: X_next may be X and F_next may be F1
        const float fv = lane < a.m ? __ldg(fs + lane) : 0.0f;
        __syncwarp();
        float* xd = a.X_next + j * a.d;
        for (int64_t k = lane; k < a.d; k += 32) xd[k] = xs[k];
        if (lane < a.m) a.F_next[j * a.m + lane] = fv;
        if (lane == 0 && a.winner) a.winner[j] = win;
    }
}

__global__ void k_moead_finish(MoeadArgs a)
{
    const int k = threadIdx.x;
    if (k < a.m) a.z[k] = fkey_inv(a.zkey[k]);
    if (k == 0 && a.status_out) *a.status_out = *a.status;
}

}  // namespace

int64_t moead_layout(int64_t n, int32_t m, int32_t T, char* ws, MoeadArgs* a)
{
    auto up = [](int64_t b) { return (b + 255) / 256 * 256; };
    const int64_t off_gmin = 256;                       // status word at 0, z_min keys at 64
    const int64_t off_tie = up(off_gmin + 8 * n);
    const int64_t off_pair = up(off_tie + 4 * n);
    const int64_t off_sub = up(off_pair + 8 * n * (int64_t)T);
    const int64_t total = up(off_sub + 8 * n * (int64_t)(m + 2));
    if (ws && a) {
        a->status = (int32_t*)ws;
        a->zkey = (uint32_t*)(ws + 64);
        a->gmin = (unsigned long long*)(ws + off_gmin);
        a->tie = (int32_t*)(ws + off_tie);
        a->gpair = (double*)(ws + off_pair);
        a->sub = (double*)(ws + off_sub);
    }
    return total;
}

cudaError_t launch_moead_select(const MoeadArgs& a, int sms, cudaStream_t s)
{
    auto grid_for = [&](int64_t work, int per_block, int max_per_sm) {
        const int64_t need = (work + per_block - 1) / per_block;
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * max_per_sm));
    };
    const int64_t pairs = a.n * (int64_t)a.T;
    k_moead_init<<<grid_for(a.n, kMoeadThreads, 8), kMoeadThreads, 0, s>>>(a);
    k_moead_zmin<<<grid_for(a.n, kMoeadThreads, 4), kMoeadThreads, 0, s>>>(a);
    k_moead_prep<<<grid_for(a.n, kMoeadThreads, 8), kMoeadThreads, 0, s>>>(a);
    k_moead_compare<<<grid_for(pairs, kMoeadThreads, 16), kMoeadThreads, 0, s>>>(a);
    k_moead_tie<<<grid_for(pairs, kMoeadThreads, 16), kMoeadThreads, 0, s>>>(a);
    k_moead_gather<<<grid_for(a.n, kMoeadThreads / 32, 16), kMoeadThreads, 0, s>>>(a);
    k_moead_finish<<<1, 32, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = sticky_merge(a.status, s);
    return e;
}

}  // namespace emo
