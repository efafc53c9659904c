// Group-wide stable LSD radix pass shared by the ordering and CSR stages.
#pragma once

#include "emo_kernels.cuh"

namespace emo {

// ------------------------------------------------ group-wide stable radix sort
// One LSD pass over idx_src[0..n) -> idx_dst, digit = (key(v) >> shift) & 255.
// Returns false when the group failed. Sets `skipped` when every element has
// the same digit (the pass would not move anything).
// Shared-memory scratch of radix_pass; declared once by the calling kernel
// (a function-scope __shared__ array in a template would be duplicated per
// key function).
struct RadixSmem {
    int hist[kRadix];
    int off[kRadix];
    int wc[kCoopThreads / 32][kRadix];
    int tot[kRadix];
    int skip;
};

template <typename KeyFn>
__device__ bool radix_pass(const ProbDev& d, const Group& g, int gs, long long budget, int64_t n,
                           const int32_t* src, int32_t* dst, int shift, KeyFn key, bool& skipped, RadixSmem& rsm)
{
    int* s_hist = rsm.hist;
    int* s_off = rsm.off;
    int (*s_wc)[kRadix] = rsm.wc;
    int* s_tot = rsm.tot;
    int& s_skip = rsm.skip;
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool active = g.rank < gs;
    const int64_t chunk = cdiv(n, gs);
    const int64_t lo = active ? min(n, chunk * g.rank) : n, hi = active ? min(n, lo + chunk) : n;

    for (int i = tid; i < kRadix; i += blockDim.x) s_hist[i] = 0;
    __syncthreads();
    for (int64_t i = lo + tid; i < hi; i += blockDim.x)
        atomicAdd(&s_hist[(key(__ldcg(&src[i])) >> shift) & (kRadix - 1)], 1);
    __syncthreads();
    if (active)
        for (int i = tid; i < kRadix; i += blockDim.x) d.hist[g.rank * kRadix + i] = s_hist[i];
    if (!group_sync(d.sc, g.size, budget)) return false;

    // digit offsets of this CTA: all earlier digits + same digit of earlier CTAs
    if (tid == 0) s_skip = 0;
    __syncthreads();
    for (int dg = tid; dg < kRadix; dg += blockDim.x) {
        int col = 0, pre = 0;
        for (int c = 0; c < gs; ++c) {
            int v = __ldcg(&d.hist[c * kRadix + dg]);
            col += v;
            if (c < g.rank) pre += v;
        }
        s_tot[dg] = col;
        s_off[dg] = pre;
        if ((int64_t)col == n) s_skip = 1;
    }
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int dg = 0; dg < kRadix; ++dg) { int c = s_tot[dg]; s_tot[dg] = run; run += c; }
    }
    __syncthreads();
    skipped = s_skip != 0;
    if (!skipped) {
        for (int dg = tid; dg < kRadix; dg += blockDim.x) s_off[dg] += s_tot[dg];
        for (int i = tid; i < (kCoopThreads / 32) * kRadix; i += blockDim.x) (&s_wc[0][0])[i] = 0;
        __syncthreads();
        // stable scatter, one tile of blockDim elements at a time
        for (int64_t base = lo; base < hi; base += blockDim.x) {
            int64_t i = base + tid;
            bool valid = i < hi;
            int32_t v = valid ? __ldcg(&src[i]) : 0;
            int dg = valid ? (int)((key(v) >> shift) & (kRadix - 1)) : kRadix;
            unsigned peers = __match_any_sync(0xffffffffu, dg);
            int r = __popc(peers & lanemask_lt());
            if (valid && r == 0) s_wc[warp][dg] = __popc(peers);
            __syncthreads();
            for (int dd = tid; dd < kRadix; dd += blockDim.x) {
                int run = 0;
                for (int w = 0; w < kCoopThreads / 32; ++w) { int c = s_wc[w][dd]; s_wc[w][dd] = run; run += c; }
                s_hist[dd] = run;  // tile count of digit dd
            }
            __syncthreads();
            if (valid) dst[s_off[dg] + s_wc[warp][dg] + r] = v;
            __syncthreads();
            for (int dd = tid; dd < kRadix; dd += blockDim.x) {
                s_off[dd] += s_hist[dd];
                for (int w = 0; w < kCoopThreads / 32; ++w) s_wc[w][dd] = 0;
            }
            __syncthreads();
        }
    }
    return group_sync(d.sc, g.size, budget);
}

}  // namespace emo
