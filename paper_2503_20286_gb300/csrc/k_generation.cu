// One generation around the selection: random mating, simulated binary
// crossover and polynomial mutation (Appendix S.I), the stand-in objective
// evaluation, the row gather that forms the next population, and IGD.
//
// Random numbers: Philox-4x32-10 keyed by the seed, counter (row,
// 0x80000000 | tag << 24 | slot, generation lo, generation hi); tag 1 the
// two parents of a pair (slot 0 / 1; word 1 of slot 0 decides crossover),
// tag 2 the SBX spread of a variable, tag 3 the mutation of a child's
// variable (word 0 decides, word 1 is mu). A word x is the uniform x 2^-32
// and the index (x n) >> 32.
// Arithmetic is FP64 with explicitly rounded operations in the order of the
// operator definitions; pow is CUDA's, so children can differ from another
// implementation's in the last bit of the FP64 value.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "emo_internal.cuh"
#include "emo_launch.cuh"

namespace emo {
namespace {

constexpr int kGenThreads = 256;
constexpr int kIgdTile = 2048;  // population points per shared-memory tile

__device__ __forceinline__ uint4 gen_random(uint64_t seed, uint64_t gen, int64_t row, uint32_t tag, int64_t slot)
{
    const uint4 c = make_uint4((uint32_t)row, 0x80000000u | (tag << 24) | ((uint32_t)slot & 0x00FFFFFFu),
                               (uint32_t)gen, (uint32_t)(gen >> 32));
    return philox4x32_10(c, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}
__device__ __forceinline__ double unit_of(uint32_t x) { return (double)x * 2.3283064365386962890625e-10; }
__device__ __forceinline__ int64_t index_of(uint32_t x, int64_t n)
{
    return (int64_t)(((unsigned long long)x * (unsigned long long)n) >> 32);
}
__device__ __forceinline__ bool hit(uint32_t x, double p)
{
    if (p >= 1.0) return true;
    if (!(p > 0.0)) return false;
    return (double)x < p * 4294967296.0;
}
__device__ __forceinline__ double clip(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

// SBX of one variable: beta from mu, children 0.5[(1 +- beta) x1 + (1 -+ beta) x2].
__device__ void sbx(double x1, double x2, double mu, double eta_c, double& c1, double& c2)
{
    const double e = __ddiv_rn(1.0, __dadd_rn(eta_c, 1.0));
    const double beta = mu <= 0.5 ? pow(__dmul_rn(2.0, mu), e)
                                  : pow(__ddiv_rn(1.0, __dsub_rn(2.0, __dmul_rn(2.0, mu))), e);
    const double bp = __dadd_rn(1.0, beta), bm = __dsub_rn(1.0, beta);
    c1 = __dmul_rn(0.5, __dadd_rn(__dmul_rn(bp, x1), __dmul_rn(bm, x2)));
    c2 = __dmul_rn(0.5, __dadd_rn(__dmul_rn(bm, x1), __dmul_rn(bp, x2)));
}

// Polynomial mutation of one variable (original form, eta = eta_m + 1).
__device__ double pm(double x, double lo, double hi, double mu, double eta_m)
{
    const double eta = __dadd_rn(eta_m, 1.0);
    const double width = __dsub_rn(hi, lo);
    const double inv = __ddiv_rn(1.0, eta);
    double step;
    if (mu <= 0.5) {
        const double delta1 = __ddiv_rn(__dsub_rn(x, lo), width);
        const double t = __dadd_rn(__dmul_rn(2.0, mu),
                                   __dmul_rn(__dsub_rn(1.0, __dmul_rn(2.0, mu)), pow(__dsub_rn(1.0, delta1), eta)));
        step = __dsub_rn(pow(t, inv), 1.0);
    } else {
        const double delta2 = __ddiv_rn(__dsub_rn(hi, x), width);
        const double t = __dadd_rn(__dsub_rn(2.0, __dmul_rn(2.0, mu)),
                                   __dmul_rn(__dsub_rn(__dmul_rn(2.0, mu), 1.0), pow(__dsub_rn(1.0, delta2), eta)));
        step = __dsub_rn(1.0, pow(t, inv));
    }
    return __dadd_rn(x, __dmul_rn(step, width));
}

// One thread per (pair, variable): both children of that variable.
__global__ void __launch_bounds__(kGenThreads) k_variation(VariationArgs a)
{
    const int64_t pairs = (a.n_off + 1) / 2;
    const int64_t work = pairs * a.d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < work; e += stride) {
        const int64_t p = e / a.d, k = e - p * a.d;
        const uint4 r0 = gen_random(a.seed, a.gen, p, 1u, 0), r1 = gen_random(a.seed, a.gen, p, 1u, 1);
        const int64_t pa = index_of(r0.x, a.n), pb = index_of(r1.x, a.n);
        if (k == 0 && a.parents) {
            a.parents[2 * p] = (int32_t)pa;
            a.parents[2 * p + 1] = (int32_t)pb;
        }
        const double x1 = (double)a.X[pa * a.d + k], x2 = (double)a.X[pb * a.d + k];
        const double lo = a.lo ? (double)a.lo[k] : 0.0, hi = a.hi ? (double)a.hi[k] : 1.0;
        double c[2] = {x1, x2};
        if (hit(r0.y, a.p_c)) {
            const uint4 rs = gen_random(a.seed, a.gen, p, 2u, k);
            sbx(x1, x2, unit_of(rs.x), a.eta_c, c[0], c[1]);
        }
        for (int child = 0; child < 2; ++child) {
            const int64_t row = child == 0 ? p : pairs + p;
            if (row >= a.n_off) continue;
            double v = clip(c[child], lo, hi);
            const uint4 rm = gen_random(a.seed, a.gen, row, 3u, k);
            // PM is defined over (x - lo) / (hi - lo): a variable without a
            // positive width (outside the contract) is left unmutated.
            if (hit(rm.x, a.p_m) && hi > lo) v = clip(pm(v, lo, hi, unit_of(rm.y), a.eta_m), lo, hi);
            a.Xoff[row * a.d + k] = (float)v;
        }
    }
}

// Stand-in objectives: g = sum_{i >= m-1} (x_i - 0.5)^2; sphere: (1 + g)
// times the unit vector of angles x_i pi/2; linear: 0.5 (1 + 100 g) times
// the stick-breaking simplex point of x_0 .. x_{m-2}.
__global__ void __launch_bounds__(kGenThreads) k_standin(const float* __restrict__ X, int64_t n, int64_t d, int m,
                                                          int shape, float* __restrict__ F)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float* x = X + i * d;
        double g = 0.0;
        for (int64_t v = m - 1; v < d; ++v) {
            const double t = __dsub_rn((double)x[v], 0.5);
            g = __dadd_rn(g, __dmul_rn(t, t));
        }
        double s[kMaxM];
        if (shape == EMO_SHAPE_SPHERE) {
            double prod = 1.0;
            for (int k = 0; k < m - 1; ++k) {
                const double ang = (double)x[k] * 1.5707963267948966;
                s[m - 1 - k] = __dmul_rn(prod, sin(ang));
                prod = __dmul_rn(prod, cos(ang));
            }
            s[0] = prod;
            for (int k = 0; k < m; ++k) F[i * m + k] = (float)__dmul_rn(__dadd_rn(1.0, g), s[k]);
        } else {
            double rest = 1.0;
            for (int k = 0; k < m - 1; ++k) {
                s[k] = __dmul_rn(rest, (double)x[k]);
                rest = __dmul_rn(rest, __dsub_rn(1.0, (double)x[k]));
            }
            s[m - 1] = rest;
            const double scale = __dmul_rn(0.5, __dadd_rn(1.0, __dmul_rn(100.0, g)));
            for (int k = 0; k < m; ++k) F[i * m + k] = (float)__dmul_rn(scale, s[k]);
        }
    }
}

// dst[j] = src[idx[j]] for rows of `width` floats, one warp per row.
__global__ void __launch_bounds__(kGenThreads) k_gather_rows(const float* __restrict__ src, const int32_t* idx,
                                                              int64_t rows, int64_t width, float* __restrict__ dst)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < rows; j += warps) {
        const int64_t s = idx[j];
        for (int64_t k = lane; k < width; k += 32) dst[j * width + k] = src[s * width + k];
    }
}

// Distance of every reference point to its nearest population point
// (FP32 squared distances, square root in FP64): one thread per reference
// point, population points staged through shared memory in tiles.
__global__ void __launch_bounds__(kGenThreads) k_igd_nearest(const float* __restrict__ F, int64_t n, int m,
                                                              const float* __restrict__ Ref, int64_t n_ref,
                                                              double* __restrict__ dist)
{
    __shared__ float tile[kIgdTile * 4];
    const int per_tile = kIgdTile * 4 / m;  // points per tile
    for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x; r0 < n_ref; r0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = r0 + threadIdx.x;
        float q[kMaxM];
        for (int k = 0; k < m; ++k) q[k] = r < n_ref ? Ref[r * m + k] : 0.0f;
        float best = INFINITY;
        for (int64_t base = 0; base < n; base += per_tile) {
            const int64_t cnt = min((int64_t)per_tile, n - base);
            __syncthreads();
            for (int64_t e = threadIdx.x; e < cnt * m; e += blockDim.x) tile[e] = F[base * m + e];
            __syncthreads();
            for (int64_t i = 0; i < cnt; ++i) {
                float s = 0.0f;
                for (int k = 0; k < m; ++k) {
                    const float t = q[k] - tile[i * m + k];
                    s = fmaf(t, t, s);
                }
                best = fminf(best, s);
            }
        }
        if (r < n_ref) dist[r] = sqrt((double)best);
    }
}

// Sum of the distances in index order (one block; deterministic), / n_ref.
__global__ void k_igd_sum(const double* __restrict__ dist, int64_t n_ref, double* out)
{
    __shared__ double part[kGenThreads];
    double s = 0.0;
    const int64_t chunk = (n_ref + blockDim.x - 1) / blockDim.x;
    const int64_t lo = threadIdx.x * chunk, hi = min(n_ref, lo + chunk);
    for (int64_t r = lo; r < hi; ++r) s += dist[r];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) t += part[i];
        *out = t / (double)n_ref;
    }
}

unsigned grid_for(int64_t work, int per_block, int sms, int max_per_sm)
{
    const int64_t need = (work + per_block - 1) / per_block;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * max_per_sm));
}

}  // namespace

cudaError_t launch_variation(const VariationArgs& a, int sms, cudaStream_t s)
{
    const int64_t work = (a.n_off + 1) / 2 * a.d;
    k_variation<<<grid_for(work, kGenThreads, sms, 16), kGenThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_standin(const float* X, int64_t n, int64_t d, int m, int shape, float* F, int sms, cudaStream_t s)
{
    k_standin<<<grid_for(n, kGenThreads, sms, 8), kGenThreads, 0, s>>>(X, n, d, m, shape, F);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const float* src, const int32_t* idx, int64_t rows, int64_t width, float* dst, int sms,
                               cudaStream_t s)
{
    k_gather_rows<<<grid_for(rows, kGenThreads / 32, sms, 16), kGenThreads, 0, s>>>(src, idx, rows, width, dst);
    return cudaGetLastError();
}

cudaError_t launch_igd(const float* F, int64_t n, int m, const float* Ref, int64_t n_ref, double* dist, double* out,
                       int sms, cudaStream_t s)
{
    k_igd_nearest<<<grid_for(n_ref, kGenThreads, sms, 4), kGenThreads, 0, s>>>(F, n, m, Ref, n_ref, dist);
    k_igd_sum<<<1, kGenThreads, 0, s>>>(dist, n_ref, out);
    return cudaGetLastError();
}

}  // namespace emo
